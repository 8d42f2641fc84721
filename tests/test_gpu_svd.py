"""GPU parity for lra_svd: the SVD the method returns and its truncation.

Compared with oracle.svd (numpy's LAPACK eigendecomposition of B B^T, then
U = Q Vt, V = B^T Vt sigma^{-1}) on the same Q and B -- the device's own, copied
to the host -- so that only the extraction differs.  Bars, from the arithmetic
of an eigendecomposition of the Gram C = B B^T in FP64 (both sides):
  * the Gram on each side carries an error of order u ||C|| (u = 2^-53), and
    both eigensolvers are backward stable with errors of order l u ||C||, so
    |d lambda_i| <= c l u lambda_1: |d sigma_i| <= 8 l u sigma_1^2 / sigma_i;
  * an eigenvector moves by at most ||dC|| / gap_i (gap_i = distance of lambda_i
    to the other eigenvalues), so U's column i by 8 l u lambda_1 / gap_i and V's
    (V = B^T Vt sigma^{-1}) by that times sigma_1 / sigma_i, plus the rounding
    of that product; columns whose bound exceeds 0.05 (near-degenerate
    eigenvalues, where the vectors are not determined) are checked through the
    products only;
  * U^T U = I, V^T V = I and U diag(sigma) V^T = Q B, which hold for any valid
    SVD, within 10x the oracle's own deviation plus 1e-13;
  * the truncated rank r equal (a threshold within 1e-9 ||A||^2 of E_r or
    E_{r-1} may fall either way), E_r within 1e-12 ||A||_F^2.
And against the oracle's whole pipeline (the oracle's own loop, then its
SVD): singular values within ||B_gpu - B_oracle||_2 (Weyl) plus the bound above.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from lra_inputs import low_rank_matrix, workload_matrix  # noqa: E402
from oracle import farpca as F  # noqa: E402
from oracle import omega as om  # noqa: E402
from oracle import svd as S  # noqa: E402
from paper_2506_03859_gb300 import lra  # noqa: E402
from paper_2506_03859_gb300.build import build  # noqa: E402

pytestmark = pytest.mark.gpu
U_EPS = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def library():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build()
    lra.load()


def dev(A):
    m, n = A.shape
    buf = torch.empty_strided((m, n), (1, m), dtype=torch.float64, device="cuda")
    buf.copy_(torch.from_numpy(np.ascontiguousarray(A)))
    return buf


def _align(X, Y):
    s = np.sign(np.sum(X * Y, axis=0))
    s[s == 0] = 1.0
    return X * s[None, :]


def check_svd(sv, Q, B, normA2, eps, k=0):
    """sv: the device result; Q, B: the run's factors on the host."""
    l = B.shape[0]
    U, s, V = sv["U"].cpu().numpy(), sv["sigma"].cpu().numpy(), sv["V"].cpu().numpy()
    Uo, so, Vo = S.svd_qb(Q, B)
    assert sv["l"] == l and U.shape == Uo.shape and V.shape == Vo.shape
    assert np.all(np.diff(s) <= 0)
    tol_s = 8 * l * U_EPS * so[0] ** 2 / np.maximum(so, 1e-300)
    assert np.all(np.abs(s - so) <= tol_s), float(np.max(np.abs(s - so) / tol_s))
    lam = so ** 2
    gap = np.array([np.min(np.abs(np.delete(lam, i) - lam[i])) if l > 1 else np.inf for i in range(l)])
    tu = 8 * l * U_EPS * lam[0] / np.maximum(gap, 1e-300)
    tv = tu * so[0] / np.maximum(so, 1e-300) + 8 * l * U_EPS * so[0] / np.maximum(so, 1e-300)
    cu = np.abs(_align(U, Uo) - Uo).max(axis=0)
    cv = np.abs(_align(V, Vo) - Vo).max(axis=0)
    okc = tv < 0.05
    assert np.all(cu[okc] <= tu[okc]), float(np.max(cu[okc] / tu[okc]))
    assert np.all(cv[okc] <= tv[okc]), float(np.max(cv[okc] / tv[okc]))
    # invariants of any SVD of Q B
    I = np.eye(l)
    assert np.abs(U.T @ U - I).max() <= 10 * np.abs(Uo.T @ Uo - I).max() + 1e-13
    assert np.abs(V.T @ V - I).max() <= 10 * np.abs(Vo.T @ Vo - I).max() + 1e-13
    QB = Q @ B
    ro = np.abs((Uo * so[None, :]) @ Vo.T - QB).max()
    assert np.abs((U * s[None, :]) @ V.T - QB).max() <= 10 * ro + 1e-13 * np.abs(QB).max()
    # truncation
    r_o, E_o = S.truncation_rank(so, normA2, eps, k)
    thr = eps * eps * normA2
    if k == 0 and r_o > 0:
        Es = normA2 - np.cumsum(so.astype(np.float64) ** 2)
        near = abs(Es[r_o - 1] - thr) <= 1e-9 * normA2 or (r_o >= 2 and abs(Es[r_o - 2] - thr) <= 1e-9 * normA2)
    else:
        near = False
    if near:
        assert abs(sv["r"] - r_o) <= 1
    else:
        assert sv["r"] == r_o
        assert abs(sv["E_r"] - E_o) <= 1e-12 * normA2
    return s, so


def _run(A, eps, P, b, kind, p, zeta, seed, k=0, fp64_simt=False, max_blocks=0):
    m, n = A.shape
    f = lra.Farpca(m, n, eps=eps, k=k, b=b, P=P, kind=kind, zeta=zeta, p=p, seed=seed,
                   fp64_simt=fp64_simt, max_blocks=max_blocks)
    st = f.run(dev(A))
    r = f.result()
    return f, st, r


CASES = [
    # (m, n, spectrum, eps, P, b, kind, p, zeta)
    (2000, 1000, "poly1.5", 1e-2, 1, 20, om.SPARSE_SIGN, 0.0, 8),
    (1500, 900, "matrix2", 1e-4, 0, 16, om.GAUSSIAN, 0.0, 0),
    (1200, 1300, "matrix1", 1e-3, 2, 10, om.STD_BERNOULLI, 0.5, 0),
    (900, 700, "poly1", 3e-2, 1, 5, om.SPARSE_GAUSSIAN, 0.0, 0),      # l = 350: long Jacobi sweeps
]


@pytest.mark.parametrize("case", CASES, ids=["ss8", "gauss_p0", "sb_p2", "sg_b5"])
@pytest.mark.parametrize("engine", ["tensor", "fp64_simt"])
def test_svd_parity(case, engine):
    m, n, spec, eps, P, b, kind, p, zeta = case
    A = low_rank_matrix(m, n, spec, 11) + 1e-7 * np.random.default_rng(2).standard_normal((m, n))
    f, st, r = _run(A, eps, P, b, kind, p, zeta, 3, fp64_simt=engine == "fp64_simt")
    assert r["rank"] > 0
    sv = f.svd()
    assert sv["status"] == lra.OK and 1 <= sv["sweeps"] <= 40
    Q, B = r["Q"].cpu().numpy(), r["B"].cpu().numpy()
    s, so = check_svd(sv, Q, B, r["normA2"], eps)
    # against the oracle's own loop: Weyl's bound for the change of B
    ref = F.farpca(A, eps, P=P, b=b, kind=kind, seed=3, zeta=zeta, p=p)
    assert ref["rank"] == r["rank"]
    _, sr, _ = S.svd_qb(ref["Q"], ref["B"])
    dB = np.linalg.norm(B - ref["B"], 2)
    assert np.all(np.abs(s - sr) <= dB + 8 * B.shape[0] * U_EPS * sr[0] ** 2 / sr)
    if r["status"] == lra.OK:
        assert sv["E_r"] < eps * eps * r["normA2"] and sv["r"] <= r["rank"]
    f.close()


def test_svd_full_size_bench_config():
    """20000 x 10000 (sigma_i = 10^(-i/100) + 1e-6 noise), sparse sign zeta = 8, b = 50,
    P = 1, eps = 1e-2: the configuration bench.py times."""
    A = workload_matrix("dense20000x10000_exp100")
    m, n = A.shape
    f = lra.Farpca(m, n, eps=1e-2, b=50, P=1, kind=lra.SPARSE_SIGN, zeta=8, seed=1)
    assert f.run(dev(A)) == lra.OK
    r = f.result()
    sv = f.svd()
    assert sv["status"] == lra.OK
    Q, B = r["Q"].cpu().numpy(), r["B"].cpu().numpy()
    check_svd(sv, Q, B, r["normA2"], 1e-2)
    # the truncated approximation meets eps against A itself (sampled rows)
    rows = np.random.default_rng(0).choice(m, 400, replace=False)
    U, s, V = sv["U"].cpu().numpy(), sv["sigma"].cpu().numpy(), sv["V"].cpu().numpy()
    q = sv["r"]
    approx = (U[rows, :q] * s[None, :q]) @ V[:, :q].T
    est = float(np.sum((A[rows] - approx) ** 2)) * m / 400
    assert est < 1.2 * 1e-4 * r["normA2"]
    f.close()


def test_svd_edge_cases():
    # before any run
    f = lra.Farpca(300, 200, eps=1e-2, b=10)
    with pytest.raises(lra.LraError):
        f.svd()
    # zero matrix: rank 0
    assert f.run(dev(np.zeros((300, 200)))) == lra.OK
    sv = f.svd()
    assert sv["l"] == 0 and sv["r"] == 0 and sv["E_r"] == 0.0 and "U" not in sv
    # a larger rank on the same context grows the workspace
    A = low_rank_matrix(300, 200, "poly1", 4)
    f.run(dev(A))
    r1 = f.result()
    check_svd(f.svd(), r1["Q"].cpu().numpy(), r1["B"].cpu().numpy(), r1["normA2"], 1e-2)
    f.close()
    # l = 1 (one block of one column)
    A = low_rank_matrix(200, 150, "matrix2", 6)
    f, st, r = _run(A, 0.99, 1, 1, om.SPARSE_SIGN, 0.0, 4, 1)
    assert r["rank"] == 1
    sv = f.svd()
    check_svd(sv, r["Q"].cpu().numpy(), r["B"].cpu().numpy(), r["normA2"], 0.99)
    f.close()
    # fixed rank: r = min(k, l)
    A = low_rank_matrix(400, 300, "poly1.5", 8)
    f, st, r = _run(A, 0.0, 1, 10, om.SPARSE_SIGN, 0.0, 8, 2, k=37)
    assert r["rank"] == 40
    sv = f.svd()
    assert sv["r"] == 37
    check_svd(sv, r["Q"].cpu().numpy(), r["B"].cpu().numpy(), r["normA2"], 0.0, k=37)
    f.close()
    # odd l = 35 (the round-robin ordering pads one index)
    f, st, r = _run(A, 0.0, 1, 5, om.SPARSE_SIGN, 0.0, 8, 4, k=35)
    assert r["rank"] == 35
    sv = f.svd()
    assert sv["r"] == 35
    check_svd(sv, r["Q"].cpu().numpy(), r["B"].cpu().numpy(), r["normA2"], 0.0, k=35)
    f.close()
    # a run that stops at its block cap: no r passes, r = l
    A = low_rank_matrix(400, 300, "poly1", 9)
    f, st, r = _run(A, 1e-6, 1, 10, om.SPARSE_SIGN, 0.0, 8, 2, max_blocks=3)
    assert st == lra.NOT_CONVERGED and r["rank"] == 30
    sv = f.svd()
    assert sv["r"] == 30
    check_svd(sv, r["Q"].cpu().numpy(), r["B"].cpu().numpy(), r["normA2"], 1e-6)
    f.close()
