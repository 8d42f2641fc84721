"""CPU: the seeded input recipes (lra_inputs) produce what the design states.

  * batch_shapes: rows in [64, 2048], columns in [32, 1024], both ranges covered;
  * batch_matrix: FP32, column-major, sigma_i = i^-2 on the first min(64, m, n)
    singular values up to the noise (Frobenius norm 1e-3 ||sigma||_2);
  * stability_matrix (Sec. 5.5): singular values exactly 1/i^2, and A^T A =
    V_A Sigma^2 V_A^T block diagonal with d blocks (zero outside them);
  * device_low_rank: exact rank, sigma_i = 10^(-i/100);
  * the same seed gives the same matrix.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from lra_inputs import batch_matrix, batch_shapes, device_low_rank, stability_matrix  # noqa: E402


def test_batch_shapes():
    sh = batch_shapes(4096, 11)
    ms = np.array([m for m, _ in sh])
    ns = np.array([n for _, n in sh])
    assert ms.min() >= 64 and ms.max() <= 2048 and ns.min() >= 32 and ns.max() <= 1024
    assert ms.min() < 100 and ms.max() > 2000 and ns.min() < 50 and ns.max() > 1000
    assert np.mean(ms < ns) > 0.05           # m < n occurs
    assert batch_shapes(10, 3) == batch_shapes(10, 3)


def test_batch_matrix_spectrum():
    A = batch_matrix(300, 120, 5, device="cpu")
    assert A.dtype == torch.float32 and A.stride() == (1, 300)
    s = np.linalg.svd(A.double().numpy(), compute_uv=False)
    sig = 1.0 / np.arange(1, 65) ** 2
    noise = 1e-3 * np.linalg.norm(sig)
    # the signal part: Weyl, |s_i - sigma_i| <= ||noise||_2 <= its Frobenius norm
    assert np.all(np.abs(s[:64] - sig) <= 1.5 * noise)
    # the rest is noise only
    assert np.sum(s[64:] ** 2) <= (1.5 * noise) ** 2
    assert torch.equal(A, batch_matrix(300, 120, 5, device="cpu"))


@pytest.mark.parametrize("d", [1, 4, 40])
def test_stability_matrix(d):
    n = 40
    A = stability_matrix(n, d, 7, device="cpu").numpy()
    s = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(s, 1.0 / np.arange(1, n + 1) ** 2, rtol=1e-10, atol=1e-15)
    G = A.T @ A
    h = n // d
    mask = np.kron(np.eye(d), np.ones((h, h))) > 0
    if d > 1:
        assert np.abs(G[~mask]).max() <= 1e-15
    if d < n:
        assert np.abs(G[mask]).max() > 1e-6


def test_device_low_rank():
    A = device_low_rank(200, 100, 30, 9, dtype=torch.float64, device="cpu").numpy()
    s = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(s[:30], 10.0 ** (-np.arange(1, 31) / 100.0), rtol=1e-10)
    assert s[30] < 1e-12


@pytest.mark.parametrize("spectrum", ["exp100", "matrix1", "matrix2", "poly1.5"])
def test_low_rank_matrix_spectrum(spectrum):
    """The Sec. 5 recipe: A = U diag(sigma) V^T with orthonormal U, V, so its
    singular values are the named spectrum's first `rank` values, the rest zero;
    column-major; the same seed gives the same matrix; noise adds N(0, noise^2)."""
    from lra_inputs import low_rank_matrix, singular_values
    m, n, r = 300, 200, 120
    A = low_rank_matrix(m, n, spectrum, 4, rank=r)
    assert A.flags["F_CONTIGUOUS"] and A.dtype == np.float64
    s = np.linalg.svd(A, compute_uv=False)
    sig = singular_values(spectrum, r)
    assert np.allclose(s[:r], sig, rtol=1e-10, atol=1e-14 * sig[0])
    assert s[r] <= 1e-13 * sig[0]
    assert np.array_equal(A, low_rank_matrix(m, n, spectrum, 4, rank=r))
    N = low_rank_matrix(m, n, spectrum, 4, rank=r, noise=1e-3) - A
    assert abs(np.linalg.norm(N) / np.sqrt(m * n) - 1e-3) < 1e-4
