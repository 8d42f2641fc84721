"""farPCA, QB form: the plain FP64 statement of the steps the CUDA path runs.

Paper: arxiv 2506.03859.  Sec. 2.1 states that farPCA (Alg. 1) is, for
P = 0, 1, 2, the randQB_EI scheme (a blocked orthonormal basis Q with
C = B = Q^T A and the indicator ||A - QB||_F^2 = ||A||_F^2 - ||B||_F^2) followed
by a direct SVD.  This module writes that QB form out, block by block:

  a1  Omega_j from Philox (oracle.omega); for the standardized Bernoulli kind
      Alg. 2's form: the Bernoulli matrix B_j and the shift w = p 1, z = A w.
  a2  S0 = A Omega_j   (Alg. 2: A B_j - z).
  a3  P >= 1: W = A^T S0 - B^T (B Omega_j)   -- the deflation W Z^{-1} W^T G_j
      of Alg. 1, since W Z^{-1} W^T = A^T Q Q^T A = B^T B;
      G = orth(W); then P-1 times W = A^T (A G) - B^T (B G), G = orth(W);
      Y_j = A G.   P = 0: Y_j = S0.
  a4/a5  Y' = (I - Q Q^T) Y_j applied twice (classical Gram-Schmidt, twice);
      Q_j = orth(Y'); B_j = Q_j^T A; append.  Z = Y^T Y of Alg. 1 is kept
      implicitly as Q's block Cholesky factor.
  a6  E <- E - ||B_j||_F^2 from E = ||A||_F^2 (the increment of tr(T Z^{-1}));
      stop when E < eps^2 ||A||_F^2 (relative tolerance, Sec. 5.2), or after
      ceil(min(m, n) / (2b)) blocks (Sec. 5.2's cap), or, in fixed-rank mode,
      after ceil(k/b) blocks.

orth(X) is the Q factor of the QR factorisation of X with positive diagonal R
(unique for full-rank X), computed as X R^{-1} with R = chol(X^T X), twice
(CholQR2).  The paper's eigSVD gives another basis of the same span; for
P <= 2 the attained rank and E are the same.  A Cholesky pivot d_c (the
diagonal before the square root) that is not > 1e-13 * S_cc, or not finite,
marks column c numerically dependent.  In a power-step panel W the run goes on:
orth_panel replaces the dependent columns by fixed random directions, as the
near-null columns of the paper's eigSVD are noise directions.  In the block
Y' that is appended to Q it ends the run with status BREAKDOWN; results stay
those of block j-1.

Pins (tests/test_oracle_farpca.py): Q^T Q = I; E = ||A - QB||_F^2 computed
directly; the Eckart-Young lower bound and the bound of eq. (4.9) against a
full SVD; exact-rank matrices end in ceil(r/b) blocks with E ~ 0 (this fails if
the deflation term is dropped or has the wrong sign); P = 0 span equals the
span of [A Omega_1 ... A Omega_j]; orth equals numpy's Householder QR with the
sign of diag(R) fixed; agreement with oracle.farpca_paper (Alg. 1 / 2 as
printed); the ranks of Table 1 (n = 5000) for every kind.

Test infrastructure only: see oracle/__init__.py.
"""
import math

import numpy as np
from scipy.linalg import solve_triangular

from . import omega as om

OK = 0
NOT_CONVERGED = 1
BREAKDOWN = 2
PIVOT_TAU = 1e-13


def default_max_blocks(m, n, b):
    """Sec. 5.2: at most ceil(n / (2b)) blocks (m >= n there); min(m, n) here."""
    return -(-min(m, n) // (2 * b))


def cholesky_upper(S, tau=PIVOT_TAU):
    """Upper R with R^T R = S, column by column; None on a failed pivot."""
    b = S.shape[0]
    R = np.zeros_like(S)
    for c in range(b):
        d = S[c, c] - R[:c, c] @ R[:c, c]
        if not (np.isfinite(d) and d > tau * S[c, c]):
            return None
        R[c, c] = math.sqrt(d)
        R[c, c + 1:] = (S[c, c + 1:] - R[:c, c] @ R[:c, c + 1:]) / R[c, c]
    return R


def cholesky_upper_skip(S, tau=PIVOT_TAU):
    """cholesky_upper that passes over a failed pivot instead of stopping: column c
    is then marked dependent, its row of R is e_c (it takes no part in the later
    columns' updates), and the factor of the remaining columns is that of S with
    the dependent rows and columns left out.  Returns (R, dead)."""
    b = S.shape[0]
    R = np.zeros_like(S)
    dead = np.zeros(b, dtype=bool)
    for c in range(b):
        d = S[c, c] - R[:c, c] @ R[:c, c]
        if not (np.isfinite(d) and d > tau * S[c, c]):
            dead[c] = True
            R[c, c] = 1.0
            continue
        R[c, c] = math.sqrt(d)
        R[c, c + 1:] = (S[c, c + 1:] - R[:c, c] @ R[:c, c + 1:]) / R[c, c]
    return R, dead


def orth_panel(X, j, step, seed, tau=PIVOT_TAU):
    """Orthonormal basis G of a power-step panel (Alg. 1's eigSVD step) that keeps
    going when the panel is numerically rank deficient.

    The paper's eigSVD returns, for the near-null directions of X^T X, columns made
    of rounding noise; this reading replaces them by fixed random directions: the
    first CholQR pass skips the failed pivots (cholesky_upper_skip), the columns it
    marks dependent are replaced by +-1/sqrt(n) columns of the TAG_FILL stream
    (column counter c + 64 step), and a second, plain CholQR pass orthonormalises the
    completed panel.  With no failed pivot this is orth(X) exactly.  Returns None
    only if the second pass fails."""
    R1, dead = cholesky_upper_skip(X.T @ X, tau)
    X1 = solve_triangular(R1, X.T, trans='T', lower=False).T
    if dead.any():
        for c in np.nonzero(dead)[0]:
            X1[:, c] = om.fill_column(X.shape[0], j, int(c) + 64 * step, seed)
    R2 = cholesky_upper(X1.T @ X1, tau)
    if R2 is None:
        return None
    return solve_triangular(R2, X1.T, trans='T', lower=False).T


def orth(X, tau=PIVOT_TAU):
    """Q factor of X = QR with diag(R) > 0, via Gram + Cholesky, twice (CholQR2)."""
    R1 = cholesky_upper(X.T @ X, tau)
    if R1 is None:
        return None
    X1 = solve_triangular(R1, X.T, trans='T', lower=False).T
    R2 = cholesky_upper(X1.T @ X1, tau)
    if R2 is None:
        return None
    return solve_triangular(R2, X1.T, trans='T', lower=False).T


def check_args(m, n, eps, P, b, kind, zeta, p, k, max_blocks):
    if m < 1 or n < 1:
        raise ValueError("empty matrix")
    if not (1 <= b <= min(m, n)):
        raise ValueError("block size b must lie in [1, min(m, n)]")
    if P < 0:
        raise ValueError("P must be >= 0")
    if k < 0 or k > min(m, n):
        raise ValueError("k must lie in [0, min(m, n)]")
    if k == 0 and not (eps > 0.0):
        raise ValueError("eps must be > 0 in fixed-precision mode")
    if k > 0 and -(-k // b) * b > min(m, n):
        raise ValueError("ceil(k/b) b exceeds min(m, n)")
    if kind not in om.KINDS:
        raise ValueError("unknown Omega kind")
    if kind == om.SPARSE_SIGN and not (1 <= zeta <= n):
        raise ValueError("zeta must lie in [1, n]")
    if not (0.0 <= p < 1.0):
        raise ValueError("p must lie in (0, 1) (0 selects the default)")
    if max_blocks < 0:
        raise ValueError("max_blocks must be >= 0")
    if max_blocks * b > min(m, n):
        raise ValueError("max_blocks * b exceeds min(m, n)")


def farpca(A, eps=0.0, P=1, b=20, kind=om.SPARSE_SIGN, seed=0, zeta=8, p=0.0,
           k=0, max_blocks=0, keep_y=False):
    """Run the QB-form farPCA loop on A (m x n, float64) and return a dict.

    Keys: status, rank, blocks, E, normA2, Q (m x rank), B (rank x n),
    E_trace (E after each block), Y (the pre-projection Y_j of each block,
    side by side, when keep_y).
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    check_args(m, n, eps, P, b, kind, zeta, p, k, max_blocks)
    if kind in (om.STD_BERNOULLI, om.SPARSE_SIGN_IID, om.SPARSE_GAUSSIAN, om.BERNOULLI):
        p = p if p > 0.0 else om.default_p(kind, n, zeta)
    normA2 = float(np.sum(A * A))
    out = dict(status=OK, rank=0, blocks=0, E=normA2, normA2=normA2,
               Q=np.zeros((m, 0)), B=np.zeros((0, n)), E_trace=[], Y=np.zeros((m, 0)))
    if not math.isfinite(normA2):
        raise ValueError("A has non-finite entries")
    if normA2 == 0.0:
        out["E"] = 0.0
        return out
    nblk = -(-k // b) if k > 0 else (max_blocks or default_max_blocks(m, n, b))
    Q = np.zeros((m, 0))
    B = np.zeros((0, n))
    E = normA2
    thr = eps * eps * normA2
    Ys, E_trace = [], []
    status = OK if k > 0 else NOT_CONVERGED
    if kind == om.STD_BERNOULLI:
        w = p * np.ones(n)
        z = A @ w
    for j in range(nblk):
        # a1 + a2: the sketch (and the same Omega applied to B for deflation)
        if kind == om.STD_BERNOULLI:
            Bj = om.bernoulli_matrix(j, n, b, p, seed)
            S0 = A @ Bj - z[:, None]
            BOm = B @ Bj - (B @ w)[:, None]
        else:
            Om = om.omega_dense(kind, j, n, b, seed, zeta, p)
            S0 = A @ Om
            BOm = B @ Om
        # a3 + a4: deflated power steps
        if P >= 1:
            W = A.T @ S0 - B.T @ BOm
            G = orth_panel(W, j, 0, seed)
            for s in range(1, P):
                if G is None:
                    break
                W = A.T @ (A @ G) - B.T @ (B @ G)
                G = orth_panel(W, j, s, seed)
            if G is None:
                status = BREAKDOWN
                break
            Y = A @ G
        else:
            Y = S0
        # a5: project against Q twice, orthonormalise, B_j = Q_j^T A
        F = Q.T @ Y
        Yp = Y - Q @ F
        F = Q.T @ Yp
        Yp = Yp - Q @ F
        Qj = orth(Yp)
        if Qj is None:
            status = BREAKDOWN
            break
        Bj_rows = (A.T @ Qj).T
        Q = np.hstack([Q, Qj])
        B = np.vstack([B, Bj_rows])
        # a6: indicator and stop test
        E = E - float(np.sum(Bj_rows * Bj_rows))
        E_trace.append(E)
        if keep_y:
            Ys.append(Y)
        if k == 0 and E < thr:
            status = OK
            break
    out.update(status=status, rank=Q.shape[1], blocks=Q.shape[1] // b, E=E, Q=Q, B=B,
               E_trace=E_trace, Y=np.hstack(Ys) if Ys else np.zeros((m, 0)))
    return out


def sketch(A, kind, j0, nblk, b, seed, zeta=8, p=0.0):
    """Y = A [Omega_j0 ... Omega_{j0+nblk-1}] (Alg. 2 form A B_j - z for SB)."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    if kind in (om.STD_BERNOULLI, om.SPARSE_SIGN_IID, om.SPARSE_GAUSSIAN, om.BERNOULLI):
        p = p if p > 0.0 else om.default_p(kind, n, zeta)
    cols = []
    for j in range(j0, j0 + nblk):
        if kind == om.STD_BERNOULLI:
            z = A @ (p * np.ones(n))
            cols.append(A @ om.bernoulli_matrix(j, n, b, p, seed) - z[:, None])
        else:
            cols.append(A @ om.omega_dense(kind, j, n, b, seed, zeta, p))
    return np.hstack(cols) if cols else np.zeros((m, 0))
