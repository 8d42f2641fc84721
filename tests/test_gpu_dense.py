"""GPU: one full pass over A (lra_apply), the contraction of Alg. 1's A G_j and
A^T Y_j, against numpy FP64.

Bound (derived from the arithmetic): numpy's FP64 product carries at most
gamma_K = K u / (1 - K u) times (|op(A)| |Y|) per entry; the tensor-core path
truncates each operand to 56 bits relative to its row / column maximum, drops
slice pairs of weight >= 7 and sums in double-float (48 bits), so its error is at
most ~2^-52 (rowmax_A |Y|^T 1 + |op(A)| 1 colmax_Y) per entry.  The test allows
the sum of both, times 4.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2506_03859_gb300 import lra  # noqa: E402
from paper_2506_03859_gb300.build import build  # noqa: E402

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def library():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build()
    lra.load()


def colmajor(X):
    return lra.column_major(torch.from_numpy(np.ascontiguousarray(X)).cuda())


def bound(opA, Y):
    K = opA.shape[1]
    aa, ay = np.abs(opA), np.abs(Y)
    gam = K * U / (1 - K * U)
    rowmax = aa.max(axis=1, keepdims=True)
    colmax = ay.max(axis=0, keepdims=True)
    ours = 2.0 ** -52 * (rowmax * ay.sum(axis=0, keepdims=True) + aa.sum(axis=1, keepdims=True) * colmax)
    return 4.0 * (gam * (aa @ ay) + ours)


def make(m, n, N, seed, spread=20):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    A *= 2.0 ** rng.integers(-spread, spread + 1, size=(m, 1))
    A *= 2.0 ** rng.integers(-spread, spread + 1, size=(1, n))
    A[rng.random((m, n)) < 0.05] = 0.0
    A[m // 3, :] = 0.0
    A[:, n // 2] = 0.0
    return A


@pytest.mark.parametrize("m,n", [(1000, 700), (333, 1111), (128, 64), (4097, 515), (20, 3000)])
@pytest.mark.parametrize("N", [1, 7, 50, 64])
@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("engine", ["tensor", "fp64_simt"])
def test_apply_fp64_bound(m, n, N, trans, engine):
    A = make(m, n, N, seed=m * 7 + n + N)
    rng = np.random.default_rng(N)
    Y = rng.standard_normal((m if trans else n, N)) * 2.0 ** rng.integers(-30, 31, size=(1, N))
    f = lra.Farpca(m, n, eps=1e-2, b=min(8, m, n), P=1, kind=lra.SPARSE_SIGN, zeta=1,
                   fp64_simt=(engine == "fp64_simt"))
    C = f.apply(colmajor(A), colmajor(Y), trans=trans).cpu().numpy()
    opA = A.T if trans else A
    ref = opA @ Y
    err = np.abs(C - ref)
    assert np.all(err <= bound(opA, Y)), float((err / np.maximum(bound(opA, Y), 1e-300)).max())
    nrm = np.linalg.norm(ref)
    if nrm > 0:
        assert np.linalg.norm(C - ref) <= 1e-14 * nrm
    f.close()


def test_apply_large_ragged_and_padded_lda():
    m, n, N = 20001, 10003, 50
    rng = np.random.default_rng(3)
    A = rng.standard_normal((m, n))
    Ad = torch.empty_strided((m, n), (1, m + 5), dtype=torch.float64, device="cuda")
    Ad.copy_(torch.from_numpy(A))
    f = lra.Farpca(m, n, eps=1e-2, b=50, P=1, kind=lra.SPARSE_SIGN, zeta=8)
    for trans in (False, True):
        Y = rng.standard_normal((m if trans else n, N))
        C = f.apply(Ad, colmajor(Y), trans=trans).cpu().numpy()
        opA = A.T if trans else A
        ref = opA @ Y
        assert np.all(np.abs(C - ref) <= bound(opA, Y))
    f.close()
