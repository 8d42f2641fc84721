"""Pins for oracle.omega: the test matrices of arxiv 2506.03859 Sec. 2.2."""
import math

import numpy as np
import pytest
from scipy import stats

from lra_inputs import haar_columns, low_rank_matrix
from oracle import omega as om
from oracle.farpca import sketch


@pytest.mark.parametrize("n,b,zeta", [(1000, 20, 8), (37, 5, 37), (200, 50, 16), (10, 3, 1)])
def test_fixed_zeta_distinct_rows(n, b, zeta):
    rows, signs = om.sparse_sign_fixed(3, n, b, zeta, seed=11)
    assert rows.shape == (b, zeta)
    for c in range(b):
        assert len(set(rows[c].tolist())) == zeta
        assert rows[c].min() >= 0 and rows[c].max() < n
    assert set(np.unique(signs).tolist()) <= {-1.0, 1.0}
    dense = om.omega_dense(om.SPARSE_SIGN, 3, n, b, 11, zeta=zeta)
    assert np.all(np.count_nonzero(dense, axis=0) == zeta)
    assert np.all(np.abs(dense[dense != 0]) == 1.0 / math.sqrt(zeta))


def test_reproducible_and_block_dependent():
    a = om.omega_dense(om.SPARSE_GAUSSIAN, 4, 500, 10, 99, p=0.05)
    b_ = om.omega_dense(om.SPARSE_GAUSSIAN, 4, 500, 10, 99, p=0.05)
    c = om.omega_dense(om.SPARSE_GAUSSIAN, 5, 500, 10, 99, p=0.05)
    d = om.omega_dense(om.SPARSE_GAUSSIAN, 4, 500, 10, 98, p=0.05)
    assert np.array_equal(a, b_)
    assert not np.array_equal(a, c) and not np.array_equal(a, d)


def _moments_ok(x, var_target=1.0, k=5.0):
    x = np.asarray(x, dtype=np.float64).ravel()
    N = x.size
    m4 = float(np.mean(x ** 4))
    assert abs(float(x.mean())) < k * math.sqrt(var_target / N)
    # sample variance = E x^2 - mean^2; the mean^2 term is O(1/N) (exactly so for +-1 entries)
    assert abs(float(x.var()) - var_target) < k * math.sqrt(max(m4 - var_target ** 2, 0.0) / N) + k * k / N


@pytest.mark.parametrize("kind,p", [(om.GAUSSIAN, 0.0), (om.STD_BERNOULLI, 0.5), (om.STD_BERNOULLI, 0.05),
                                    (om.SPARSE_SIGN_IID, 0.05), (om.SPARSE_GAUSSIAN, 0.05)])
def test_entry_mean0_var1(kind, p):
    # Standardized entries have mean 0 and variance 1 (Thm. 3.2 proof; Def. 2.2-2.4).
    n, b = 4000, 50
    x = np.concatenate([om.omega_dense(kind, j, n, b, 5, p=p).ravel() for j in range(3)])
    _moments_ok(x)


def test_fixed_zeta_scaled_moments():
    # +-1/sqrt(zeta) on zeta of n rows: sqrt(n) * omega has mean 0, variance 1.
    n, b, zeta = 1000, 50, 8
    x = np.concatenate([om.omega_dense(om.SPARSE_SIGN, j, n, b, 5, zeta=zeta).ravel() for j in range(4)])
    _moments_ok(math.sqrt(n) * x)


def test_bernoulli_mean_p():
    p = 0.2
    x = np.concatenate([om.bernoulli_matrix(j, 3000, 40, p, 17).ravel() for j in range(2)])
    assert abs(float(x.mean()) - p) < 5 * math.sqrt(p * (1 - p) / x.size)
    assert set(np.unique(x).tolist()) == {0.0, 1.0}


@pytest.mark.parametrize("kind", [om.BERNOULLI, om.SPARSE_SIGN_IID, om.SPARSE_GAUSSIAN])
def test_hoeffding_nnz(kind):
    # P(|nnz - n l p| >= t) <= exp(-2 t^2 / (n l)) (Sec. 3.1 / 3.2); t for failure prob 1e-9.
    n, b, p = 5000, 50, 0.002
    t = math.sqrt(-math.log(1e-9) * n * b / 2.0)
    for j in range(3):
        nnz = int(np.count_nonzero(om.omega_dense(kind, j, n, b, 3, p=p)))
        assert abs(nnz - n * b * p) < t


def test_gaussian_ks():
    g = np.concatenate([om.gaussian(j, 2000, 20, 8).ravel() for j in range(2)])
    assert stats.kstest(g, "norm").pvalue > 1e-4


@pytest.mark.parametrize("kind,p,zeta", [(om.STD_BERNOULLI, 0.1, 0), (om.SPARSE_SIGN_IID, 0.1, 0),
                                         (om.SPARSE_GAUSSIAN, 0.1, 0), (om.GAUSSIAN, 0.0, 0)])
def test_theorem32_rotated_entries_near_gaussian(kind, p, zeta):
    # Thm. 3.2 / Prop. 3.5-3.6: V^T Omega -> N(0,1) entrywise for Haar V (max |v_ij| -> 0),
    # Kolmogorov distance O(sum_k |v_ik|^3) = O(n^-1/2).
    n, b = 2000, 10
    V = haar_columns(n, n, np.random.default_rng(42))
    x = np.concatenate([(V.T @ om.omega_dense(kind, j, n, b, 1, p=p, zeta=zeta)).ravel() for j in range(2)])
    d = stats.kstest(x, "norm").statistic
    assert d < 0.03


def test_theorem32_fails_for_localised_v():
    # Condition (3.1) violated (V = I, i.e. d = n in Sec. 5.5): entries stay Bernoulli-like.
    n, b = 2000, 10
    x = np.concatenate([om.omega_dense(om.STD_BERNOULLI, j, n, b, 1, p=0.1).ravel() for j in range(2)])
    assert stats.kstest(x, "norm").statistic > 0.2


def test_standardized_bernoulli_identity():
    # Sec. 3.1: sqrt(p(1-p)) A Omega_j = A B_j - p A 1.
    A = low_rank_matrix(60, 40, "poly1", 3)
    for p in (0.5, 0.1):
        Om = om.omega_dense(om.STD_BERNOULLI, 2, 40, 6, 13, p=p)
        lhs = math.sqrt(p * (1 - p)) * (A @ Om)
        rhs = sketch(A, om.STD_BERNOULLI, 2, 1, 6, 13, p=p)
        assert np.allclose(lhs, rhs, rtol=0, atol=1e-13 * np.abs(A).sum())


def test_entries_match_dense():
    n, b = 300, 7
    for kind, kw in [(om.SPARSE_SIGN, dict(zeta=5)), (om.SPARSE_SIGN_IID, dict(p=0.05)),
                     (om.SPARSE_GAUSSIAN, dict(p=0.05)), (om.BERNOULLI, dict(p=0.05)),
                     (om.GAUSSIAN, {})]:
        dense = om.omega_dense(kind, 1, n, b, 21, **kw)
        ent = om.omega_entries(kind, 1, n, b, 21, **kw)
        rebuilt = np.zeros((n, b))
        for c, (r, v) in enumerate(ent):
            rebuilt[r, c] = v
        assert np.array_equal(rebuilt, dense)
    ent = om.omega_entries(om.STD_BERNOULLI, 1, n, b, 21, p=0.05)
    bm = om.bernoulli_matrix(1, n, b, 0.05, 21)
    for c, (r, v) in enumerate(ent):
        assert np.array_equal(np.nonzero(bm[:, c])[0], r) and np.all(v == 1.0)


def test_default_p():
    # Sec. 5.1: p1 = max(1e-3, ln n / n) (SB), p2 = max(1e-3, 10/n) (others).
    assert om.default_p(om.STD_BERNOULLI, 5000) == pytest.approx(math.log(5000) / 5000)
    assert om.default_p(om.SPARSE_SIGN_IID, 5000) == pytest.approx(0.002)
    assert om.default_p(om.SPARSE_SIGN_IID, 30000) == pytest.approx(1e-3)
    assert om.default_p(om.SPARSE_GAUSSIAN, 10000, zeta=8) == pytest.approx(8e-4)
    assert om.mask_threshold(0.5) == 2 ** 31
