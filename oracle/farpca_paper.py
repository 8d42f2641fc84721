"""farPCA as Alg. 1 and Alg. 2 of arxiv 2506.03859 print it.

Keeps the paper's cumulative Y, W (sketches and their A^T images), Z = Y^T Y,
T = W^T W, and the deflation W (Z^{-1} (W^T G_j)) literally; the basis of each
power step comes from eigSVD (the economic SVD through the eigendecomposition
of the Gram matrix, the routine Alg. 1 cites).  Readings:
  * Alg. 1 / 2 update the indicator by subtracting tr(T Z^{-1}) of the
    cumulative T and Z; here the indicator after block j is
    E_j = ||A||_F^2 - tr(T_j Z_j^{-1}) (tr(T_j Z_j^{-1}) already holds every block
    so far, so subtracting it from the previous E would count earlier blocks
    again);
  * the stop test is relative, E < eps^2 ||A||_F^2 (Sec. 5.2);
  * the shift alpha only acts from the third power step on (Alg. 1 updates it
    after step k > 1 and uses it at step k + 1), so it is omitted for P <= 2.

This form is numerically fragile when Z is ill conditioned (P = 0 with a steep
spectrum); tests compare it with oracle.farpca on well-conditioned cases.

The SVD extraction after the loop (the two eigendecompositions that follow the
loop in Alg. 1 / Alg. 2) is ``svd_from_yw``.

Pins: tests/test_oracle_farpca.py (same rank and E as oracle.farpca; the
extracted SVD reproduces Q Q^T A and its singular values match those of B).

Test infrastructure only: see oracle/__init__.py.
"""
import numpy as np

from . import omega as om
from .farpca import check_args, default_max_blocks, OK, NOT_CONVERGED


def eig_svd(W):
    """Economic SVD of tall W from W^T W = V D V^T: S = sqrt(D), U = W V S^{-1}."""
    D, V = np.linalg.eigh(W.T @ W)
    S = np.sqrt(D)
    U = (W @ V) / S[None, :]
    return U, S, V


def farpca_paper(A, eps, P=1, b=20, kind=om.SPARSE_SIGN, seed=0, zeta=8, p=0.0,
                 max_blocks=0):
    """Fixed-precision farPCA (Alg. 1, or Alg. 2 for the standardized Bernoulli kind)."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    check_args(m, n, eps, P, b, kind, zeta, p, 0, max_blocks)
    if kind in (om.STD_BERNOULLI, om.SPARSE_SIGN_IID, om.SPARSE_GAUSSIAN, om.BERNOULLI):
        p = p if p > 0.0 else om.default_p(kind, n, zeta)
    normA2 = float(np.sum(A * A))
    E = normA2
    Y = np.zeros((m, 0))
    W = np.zeros((n, 0))
    Z = T = np.zeros((0, 0))
    status = NOT_CONVERGED
    nblk = max_blocks or default_max_blocks(m, n, b)
    if kind == om.STD_BERNOULLI:
        w = p * np.ones(n)
        z = A @ w

    def deflate(X, shift=None):
        if W.shape[1] == 0:
            return 0.0
        WtX = W.T @ X if shift is None else W.T @ X - shift[:, None]
        return W @ np.linalg.solve(Z, WtX)

    for j in range(nblk):
        if kind == om.STD_BERNOULLI:
            Bj = om.bernoulli_matrix(j, n, b, p, seed)
            if P == 0:
                Yj = A @ Bj - z[:, None]
            else:
                Wj = A.T @ (A @ Bj - z[:, None]) - deflate(Bj, W.T @ w)
                G = eig_svd(Wj)[0]
                for _ in range(2, P + 1):
                    Wj = A.T @ (A @ G) - deflate(G)
                    G = eig_svd(Wj)[0]
                Yj = A @ G
        else:
            G = om.omega_dense(kind, j, n, b, seed, zeta, p)
            for _ in range(P):
                Wj = A.T @ (A @ G) - deflate(G)
                G = eig_svd(Wj)[0]
            Yj = A @ G
        Wj = A.T @ Yj
        Y = np.hstack([Y, Yj])
        W = np.hstack([W, Wj])
        Z = Y.T @ Y
        T = W.T @ W
        E = normA2 - float(np.trace(np.linalg.solve(Z, T)))
        if E < eps * eps * normA2:
            status = OK
            break
    return dict(status=status, rank=Y.shape[1], blocks=Y.shape[1] // b, E=E,
                normA2=normA2, Y=Y, W=W, Z=Z, T=T)


def svd_from_yw(Y, W, Z, T):
    """The SVD A ~ U diag(s) V^T that Alg. 1 / Alg. 2 extract after the loop.

    eig(Z) = (Vh, Sh), D = Vh Sh^{-1/2}; eig(D^T T D) = (Vt, St), s = St^{1/2};
    U = Y D Vt, V = W D Vt diag(s)^{-1}.  Singular values come out ascending.
    """
    Sh, Vh = np.linalg.eigh(Z)
    D = Vh / np.sqrt(Sh)[None, :]
    St, Vt = np.linalg.eigh(D.T @ T @ D)
    s = np.sqrt(np.maximum(St, 0.0))
    U = Y @ D @ Vt
    V = (W @ D @ Vt) / s[None, :]
    return U, s, V
