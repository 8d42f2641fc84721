"""The SVD that farPCA returns, extracted from its QB form, and the truncation.

Paper: arxiv 2506.03859.  Alg. 1 / Alg. 2 end with two eigendecompositions that
turn the loop's Y, W, Z = Y^T Y, T = W^T W into A ~ U diag(sigma) V^T
(oracle.farpca_paper.svd_from_yw writes them out as printed).  In the QB form of
the loop (Sec. 2.1: farPCA = randQB_EI + a direct SVD for P <= 2) the same SVD
is the SVD of the l x n matrix B = Q^T A, lifted by Q:

    B B^T = Vt diag(lambda) Vt^T         (eigendecomposition of an l x l Gram)
    sigma = sqrt(lambda),  U = Q Vt,  V = B^T Vt diag(sigma)^{-1}

because Y D (D = Vh Sh^{-1/2} from eig(Z)) and Q are orthonormal bases of one
span, so D^T T D and B B^T are the same operator written in two bases.  Readings:
  * order: descending sigma (the direct SVD's order; Sec. 2.1 notes that Alg. 1
    itself returns them ascending) so that a truncation keeps a prefix;
  * a zero singular value gets a zero column of V (V = B^T Vt sigma^{-1} is
    undefined there; U's column still spans the null direction of B).

Post-processing truncation (Sec. 5.3, after Hallman's block method): the lowest
rank r whose truncated SVD meets the threshold.  With P_r the projector
Q Vt_r Vt_r^T Q^T, ||A - U_r S_r V_r^T||_F^2 = ||A||_F^2 - sum_{i<=r} sigma_i^2,
accumulated in this order, and r is the first r with that value
< eps^2 ||A||_F^2 (the loop's strict, relative test).  If no r <= l passes
(a run that hit its block cap), r = l.  Fixed-rank mode (k > 0): r = min(k, l).

Pins (tests/test_oracle_svd.py): the paper-literal extraction from Y, W, Z, T
(separate code, two eigendecompositions); the exact SVD of exact-rank inputs
(numpy's LAPACK SVD of A itself); orthonormal U and V and U S V^T = Q B; the
truncation rank and its error against the residual A - U_r S_r V_r^T formed
explicitly for every r.

Test infrastructure only: see oracle/__init__.py.
"""
import numpy as np


def svd_qb(Q, B):
    """U (m x l), sigma (l, descending), V (n x l) with Q B = U diag(sigma) V^T."""
    Q = np.asarray(Q, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    lam, Vt = np.linalg.eigh(B @ B.T)
    order = np.argsort(-lam, kind="stable")
    lam, Vt = lam[order], Vt[:, order]
    sigma = np.sqrt(np.maximum(lam, 0.0))
    U = Q @ Vt
    V = B.T @ Vt
    nz = sigma > 0.0
    V[:, nz] /= sigma[nz][None, :]
    V[:, ~nz] = 0.0
    return U, sigma, V


def truncation_rank(sigma, normA2, eps, k=0):
    """(r, E_r): the post-processing rank and ||A||^2 - sum_{i<=r} sigma_i^2."""
    sigma = np.asarray(sigma, dtype=np.float64)
    l = sigma.shape[0]
    E = float(normA2)
    if k > 0:
        r = min(int(k), l)
        for i in range(r):
            E -= float(sigma[i]) * float(sigma[i])
        return r, E
    thr = eps * eps * float(normA2)
    for i in range(l):
        E -= float(sigma[i]) * float(sigma[i])
        if E < thr:
            return i + 1, E
    return l, E
