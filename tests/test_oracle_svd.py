"""Pins for oracle.svd: the final SVD of farPCA and the post-processing truncation.

What fixes each part, independently of oracle.svd's own code:
  * the extraction: the paper-literal form of Alg. 1's last three steps
    (oracle.farpca_paper.svd_from_yw, from Y, W, Z, T through two
    eigendecompositions) gives the same singular triplets; on exact-rank inputs
    the result is the SVD of A itself (LAPACK's SVD of A);
  * invariants: U^T U = I, V^T V = I, U diag(sigma) V^T = Q B, sigma descending;
  * the truncation: the residual A - U_r diag(sigma_r) V_r^T formed explicitly
    for every r gives the same rank and the same squared error;
  * planted mistakes (ascending order, a missing sigma^{-1}) make a pin fail.
"""
import math
import types

import numpy as np
import pytest

from lra_inputs import exact_rank_matrix, low_rank_matrix
from oracle import farpca as F
from oracle import farpca_paper as FP
from oracle import omega as om
from oracle import svd as S


def _align(X, Y):
    """Flip the sign of each column of X to match the column of Y."""
    s = np.sign(np.sum(X * Y, axis=0))
    s[s == 0] = 1.0
    return X * s[None, :]


@pytest.mark.parametrize("kind,p", [(om.SPARSE_SIGN, 0.0), (om.GAUSSIAN, 0.0), (om.STD_BERNOULLI, 0.5)])
def test_matches_paper_literal_extraction(kind, p):
    A = low_rank_matrix(300, 200, "poly1.5", 5)
    a = FP.farpca_paper(A, 1e-2, P=1, b=10, kind=kind, seed=3, zeta=4, p=p)
    Up, sp, Vp = FP.svd_from_yw(a["Y"], a["W"], a["Z"], a["T"])
    Up, sp, Vp = Up[:, ::-1], sp[::-1], Vp[:, ::-1]          # Alg. 1 returns ascending order
    r = F.farpca(A, 1e-2, P=1, b=10, kind=kind, seed=3, zeta=4, p=p)
    assert r["rank"] == a["rank"]
    U, s, V = S.svd_qb(r["Q"], r["B"])
    assert np.abs(s - sp).max() < 1e-12 * s[0]
    # singular vectors: perturbation theory bounds their difference by (change of
    # the operator) / (gap to the neighbouring singular values)
    gap = np.minimum(np.r_[np.inf, -np.diff(s)], np.r_[-np.diff(s), np.inf]) / s[0]
    assert np.all(np.abs(_align(U, Up) - Up).max(axis=0) * gap < 1e-12)
    assert np.all(np.abs(_align(V, Vp) - Vp).max(axis=0) * gap < 1e-12)


def test_exact_rank_gives_the_svd_of_A():
    b = 8
    A = exact_rank_matrix(200, 150, 2 * b, 3)
    r = F.farpca(A, 1e-6, P=1, b=b, kind=om.SPARSE_SIGN, seed=1, zeta=4)
    assert r["rank"] == 2 * b
    U, s, V = S.svd_qb(r["Q"], r["B"])
    Ua, sa, Vta = np.linalg.svd(A, full_matrices=False)
    l = r["rank"]
    assert np.allclose(s, sa[:l], rtol=1e-12, atol=0)
    assert np.abs(_align(U, Ua[:, :l]) - Ua[:, :l]).max() < 1e-10
    assert np.abs(_align(V, Vta[:l].T) - Vta[:l].T).max() < 1e-10


@pytest.mark.parametrize("P", [0, 1, 2])
def test_invariants(P):
    A = low_rank_matrix(400, 250, "matrix2", 7)
    r = F.farpca(A, 1e-4, P=P, b=10, kind=om.SPARSE_SIGN, seed=2, zeta=8)
    U, s, V = S.svd_qb(r["Q"], r["B"])
    l = r["rank"]
    assert np.all(np.diff(s) <= 0)
    assert np.abs(U.T @ U - np.eye(l)).max() < 1e-12 * math.sqrt(l)
    assert np.abs(V.T @ V - np.eye(l)).max() < 1e-11 * math.sqrt(l)
    QB = r["Q"] @ r["B"]
    assert np.abs((U * s[None, :]) @ V.T - QB).max() < 1e-13 * np.abs(QB).max() * l
    # sum sigma^2 = ||B||_F^2, so the last truncation error is the loop's indicator
    assert abs(float(np.sum(s ** 2)) - float(np.sum(r["B"] ** 2))) < 1e-13 * r["normA2"]


@pytest.mark.parametrize("eps", [1e-1, 3e-2, 1e-2, 1e-3])
def test_truncation_against_explicit_residuals(eps):
    A = low_rank_matrix(300, 200, "poly1", 9) + 1e-4 * np.random.default_rng(4).standard_normal((300, 200))
    r = F.farpca(A, eps, P=1, b=10, kind=om.SPARSE_SIGN, seed=5, zeta=4)
    U, s, V = S.svd_qb(r["Q"], r["B"])
    normA2 = r["normA2"]
    rank, E_r = S.truncation_rank(s, normA2, eps)
    direct = [float(np.sum((A - (U[:, :q] * s[None, :q]) @ V[:, :q].T) ** 2)) for q in range(0, s.size + 1)]
    passing = [q for q in range(s.size + 1) if direct[q] < eps * eps * normA2]
    want = passing[0] if passing else s.size
    # a value within rounding of the threshold may fall either way (tie rule)
    if passing and abs(direct[want] - eps * eps * normA2) > 1e-9 * normA2 \
            and abs(direct[want - 1] - eps * eps * normA2) > 1e-9 * normA2:
        assert rank == want
    else:
        assert abs(rank - want) <= 1
    assert abs(E_r - direct[rank]) < 1e-10 * normA2
    assert rank <= r["rank"]
    if r["status"] == F.OK:
        assert E_r < eps * eps * normA2


def test_truncation_edge_cases():
    s = np.array([3.0, 2.0, 1.0])
    normA2 = 14.0
    assert S.truncation_rank(s, normA2, 0.5) == (2, 1.0)          # 14-9-4 = 1 < 3.5
    assert S.truncation_rank(s, normA2, 1e-9) == (3, 0.0)
    assert S.truncation_rank(s, normA2, 0.0, k=2) == (2, 1.0)
    assert S.truncation_rank(s, normA2, 0.0, k=7) == (3, 0.0)
    assert S.truncation_rank(np.zeros(0), 0.0, 0.1) == (0, 0.0)
    # strict test: E_r equal to the threshold does not pass
    assert S.truncation_rank(np.array([2.0, 1.0, 1.0, 1.0]), 8.0, 0.5) == (4, 1.0)   # E_3 = 2 = thr
    # zero singular value: a zero column of V
    Q = np.eye(4)[:, :2]
    B = np.array([[1.0, 0, 0], [0, 0, 0]])
    U, sg, V = S.svd_qb(Q, B)
    assert sg.tolist() == [1.0, 0.0] and np.all(V[:, 1] == 0.0)


def _planted(replacements):
    src = open(S.__file__).read()
    for a, b_ in replacements:
        assert a in src
        src = src.replace(a, b_)
    mod = types.ModuleType("oracle.planted_svd")
    mod.__package__ = "oracle"
    exec(compile(src, "planted_svd", "exec"), mod.__dict__)
    return mod


def test_planted_mistakes_are_caught():
    A = low_rank_matrix(300, 200, "poly1.5", 5)
    r = F.farpca(A, 1e-2, P=1, b=10, kind=om.SPARSE_SIGN, seed=3, zeta=4)
    eps = 3e-2
    # ascending order: the truncation keeps the wrong end of the spectrum
    bad = _planted([("order = np.argsort(-lam, kind=\"stable\")", "order = np.argsort(lam, kind=\"stable\")")])
    U, s, V = bad.svd_qb(r["Q"], r["B"])
    q, _ = bad.truncation_rank(s, r["normA2"], eps)
    direct = float(np.sum((A - (U[:, :q] * s[None, :q]) @ V[:, :q].T) ** 2))
    assert not direct < eps * eps * r["normA2"] or q == s.size
    # V without sigma^{-1}: V is no longer orthonormal
    bad = _planted([("V[:, nz] /= sigma[nz][None, :]", "pass")])
    U, s, V = bad.svd_qb(r["Q"], r["B"])
    assert np.abs(V.T @ V - np.eye(s.size)).max() > 1e-3
