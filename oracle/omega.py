"""Test matrices Omega (n x b, one per block j) drawn from Philox counters.

Definitions (arxiv 2506.03859, Sec. 2.2):
  * Gaussian (farPCA, Alg. 1): i.i.d. N(0, 1) entries.
  * Bernoulli matrix (Def. 2.1): i.i.d. entries, 1 with probability p, else 0.
  * Sparse sign, i.i.d. form (Def. 2.2): +-1/sqrt(p) each with probability
    p/2, else 0.
  * Sparse sign, fixed-nonzeros form (the variant the paper mentions right after
    Def. 2.2): exactly zeta distinct nonzero rows per column, value
    +-1/sqrt(zeta).
  * Standardized Bernoulli (Def. 2.3): (b_ij - p)/sqrt(p(1-p)) for a Bernoulli
    matrix B; Alg. 2 works with B itself and the rank-one shift p*1 (Sec. 3.1,
    the scale 1/sqrt(p(1-p)) dropped).
  * Sparse Gaussian (Def. 2.4): B o G / sqrt(p).

Recommended p when the caller gives none (Sec. 5.1): p1 = max(1e-3, ln n / n)
for the standardized Bernoulli kind, p2 = max(1e-3, 10/n) for the others.

Nonzero values are sign * (1.0 / sqrt(x)) with x = zeta or p, and g * (1.0 /
sqrt(p)) for the sparse Gaussian: one IEEE square root, one IEEE division, one
product, so both implementations round identically.

Counter layout (this library's convention; the paper only says "generate"):
Philox4x32-10 with key = (seed_lo, seed_hi) and counter (x, j, c, tag), where
j is the 0-based block, c the column within the block, x the draw index (fixed
zeta) or the row r (i.i.d. kinds), and tag names the stream:
  TAG_SPARSE_SIGN  draws of the fixed-zeta kind: row = floor(u0 * n / 2^32),
                   sign = + if bit 0 of u1 is 0 else -; a row already taken in
                   the column is rejected and the next draw used.
  TAG_MASK         Bernoulli mask: nonzero iff u0 < floor(p * 2^32); for the
                   i.i.d. sparse sign kind the sign is bit 0 of u1.
  TAG_GAUSS        Box-Muller from two 53-bit uniforms: a = (k(u0,u1) + 1) 2^-53
                   in (0, 1], c = k(u2,u3) 2^-53 in [0, 1), with
                   k(x, y) = (x >> 5) 2^26 + (y >> 6); value sqrt(-2 ln a) cos(2 pi c).
  TAG_FILL         the direction that replaces a dependent column of a power-step
                   panel (oracle.farpca.orth_panel): entry r of column c is
                   +-1/sqrt(n), + if bit 0 of u0 is 0, with counter (r, j, c', TAG_FILL),
                   c' = c + 64 s for power step s.

Pins (tests/test_oracle_omega.py): exactly zeta distinct rows per column;
entry mean 0 / variance 1 after standardisation; Hoeffding's nnz bound
(Sec. 3.1); Thm. 3.2 / Prop. 3.5-3.6 (V^T Omega close to N(0,1) for Haar V,
Kolmogorov distance test); the standardized-Bernoulli identity of Sec. 3.1.

Test infrastructure only: see oracle/__init__.py.
"""
import math

import numpy as np

from .philox import philox4x32_10, seed_key

GAUSSIAN = 0
STD_BERNOULLI = 1
SPARSE_SIGN = 2
SPARSE_SIGN_IID = 3
SPARSE_GAUSSIAN = 4
BERNOULLI = 5
KINDS = (GAUSSIAN, STD_BERNOULLI, SPARSE_SIGN, SPARSE_SIGN_IID, SPARSE_GAUSSIAN, BERNOULLI)
KIND_NAMES = {GAUSSIAN: "farPCA", STD_BERNOULLI: "farPCASB", SPARSE_SIGN: "farPCASS",
              SPARSE_SIGN_IID: "farPCASS-iid", SPARSE_GAUSSIAN: "farPCASG", BERNOULLI: "farPCAB"}

TAG_SPARSE_SIGN = 1
TAG_MASK = 2
TAG_GAUSS = 3
TAG_FILL = 4

TWO32 = 4294967296.0
TWO_M53 = 2.0 ** -53


def max_draws(zeta):
    """Cap on draws per column for the fixed-zeta kind (both sides use it)."""
    return 64 * zeta + 1024


def default_p(kind, n, zeta=0):
    """Bernoulli probability used when the caller passes p <= 0 (Sec. 5.1)."""
    if kind == SPARSE_GAUSSIAN and zeta > 0:
        return zeta / n
    if kind == STD_BERNOULLI:
        return max(1e-3, math.log(n) / n)
    return max(1e-3, 10.0 / n)


def mask_threshold(p):
    """Integer threshold t = floor(p 2^32): an entry is nonzero iff u0 < t."""
    return int(math.floor(p * TWO32))


def _draw(x, j, c, tag, seed):
    k0, k1 = seed_key(seed)
    return philox4x32_10(x, j, c, tag, k0, k1)


def sparse_sign_fixed(j, n, b, zeta, seed):
    """Rows and signs of the fixed-zeta sparse sign block j, in acceptance order.

    Returns (rows int64 [b, zeta], signs float64 [b, zeta] of +-1).
    """
    if not (1 <= zeta <= n):
        raise ValueError("zeta must lie in [1, n]")
    rows = np.empty((b, zeta), dtype=np.int64)
    signs = np.empty((b, zeta), dtype=np.float64)
    cap = max_draws(zeta)
    for c in range(b):
        t_all = np.arange(cap, dtype=np.uint64)
        u0, u1, _, _ = _draw(t_all, j, c, TAG_SPARSE_SIGN, seed)
        cand = ((u0 * np.uint64(n)) >> np.uint64(32)).astype(np.int64)
        sgn = np.where((u1 & np.uint64(1)) == 0, 1.0, -1.0)
        taken = []
        for t in range(cap):
            r = int(cand[t])
            if r in taken:
                continue
            taken.append(r)
            signs[c, len(taken) - 1] = sgn[t]
            if len(taken) == zeta:
                break
        if len(taken) < zeta:
            raise RuntimeError("fixed-zeta draw cap exceeded")
        rows[c] = taken
    return rows, signs


def mask_and_u1(j, n, b, p, seed):
    """Bernoulli(p) mask [n, b] (bool) and the u1 word of the same draws."""
    r = np.arange(n, dtype=np.uint64)[:, None]
    c = np.arange(b, dtype=np.uint64)[None, :]
    u0, u1, _, _ = _draw(r, j, c, TAG_MASK, seed)
    return u0 < np.uint64(mask_threshold(p)), u1


def fill_column(n, j, c, seed):
    """A +-1/sqrt(n) column from the TAG_FILL stream: the direction that replaces a
    numerically dependent column of a power-step panel."""
    r = np.arange(n, dtype=np.uint64)
    u0, _, _, _ = _draw(r, j, c, TAG_FILL, seed)
    v = 1.0 / math.sqrt(n)
    return np.where((u0 & np.uint64(1)) == 0, v, -v)


def gaussian(j, n, b, seed):
    """Standard normal block [n, b] by Box-Muller on Philox uniforms."""
    r = np.arange(n, dtype=np.uint64)[:, None]
    c = np.arange(b, dtype=np.uint64)[None, :]
    u0, u1, u2, u3 = _draw(r, j, c, TAG_GAUSS, seed)
    k_a = (u0 >> np.uint64(5)) * np.uint64(1 << 26) + (u1 >> np.uint64(6))
    k_c = (u2 >> np.uint64(5)) * np.uint64(1 << 26) + (u3 >> np.uint64(6))
    a = (k_a.astype(np.float64) + 1.0) * TWO_M53
    cc = k_c.astype(np.float64) * TWO_M53
    return np.sqrt(-2.0 * np.log(a)) * np.cos(2.0 * np.pi * cc)


def bernoulli_matrix(j, n, b, p, seed):
    """The Bernoulli matrix B_j of Def. 2.1 (float64 0/1), as Alg. 2 uses it."""
    mask, _ = mask_and_u1(j, n, b, p, seed)
    return mask.astype(np.float64)


def omega_dense(kind, j, n, b, seed, zeta=0, p=0.0):
    """Omega_j as an explicit n x b matrix, exactly as its definition states.

    For STD_BERNOULLI this is the standardized matrix of Def. 2.3
    (entries (b_ij - p)/sqrt(p(1-p))); the farPCA oracle itself follows
    Alg. 2 and multiplies by the Bernoulli matrix and the shift instead.
    """
    if kind == GAUSSIAN:
        return gaussian(j, n, b, seed)
    if kind == SPARSE_SIGN:
        rows, signs = sparse_sign_fixed(j, n, b, zeta, seed)
        om = np.zeros((n, b))
        for c in range(b):
            om[rows[c], c] = signs[c] * (1.0 / math.sqrt(zeta))
        return om
    if p <= 0.0:
        p = default_p(kind, n, zeta)
    if kind == STD_BERNOULLI:
        bm = bernoulli_matrix(j, n, b, p, seed)
        return (bm - p) / math.sqrt(p * (1.0 - p))
    if kind == BERNOULLI:
        return bernoulli_matrix(j, n, b, p, seed)
    if kind == SPARSE_SIGN_IID:
        mask, u1 = mask_and_u1(j, n, b, p, seed)
        sgn = np.where((u1 & np.uint64(1)) == 0, 1.0, -1.0)
        return np.where(mask, sgn * (1.0 / math.sqrt(p)), 0.0)
    if kind == SPARSE_GAUSSIAN:
        mask, _ = mask_and_u1(j, n, b, p, seed)
        return np.where(mask, gaussian(j, n, b, seed) * (1.0 / math.sqrt(p)), 0.0)
    raise ValueError("unknown kind %r" % (kind,))


def omega_entries(kind, j, n, b, seed, zeta=0, p=0.0):
    """Per-column nonzero structure of the matrix the sketch multiplies by.

    Returns a list of b pairs (rows int64, vals float64).  Order: acceptance
    order for the fixed-zeta kind, increasing row for the others.  For
    STD_BERNOULLI the entries are those of the Bernoulli matrix B_j (value 1),
    the matrix Alg. 2 stores as sparse(B_j); dense kinds list every row.
    """
    if kind == SPARSE_SIGN:
        rows, signs = sparse_sign_fixed(j, n, b, zeta, seed)
        s = 1.0 / math.sqrt(zeta)
        return [(rows[c].copy(), signs[c] * s) for c in range(b)]
    if p <= 0.0:
        p = default_p(kind, n, zeta)
    all_rows = np.arange(n, dtype=np.int64)
    if kind == GAUSSIAN:
        g = gaussian(j, n, b, seed)
        return [(all_rows.copy(), g[:, c].copy()) for c in range(b)]
    mask, _ = mask_and_u1(j, n, b, p, seed)
    vals = bernoulli_matrix(j, n, b, p, seed) if kind == STD_BERNOULLI \
        else omega_dense(kind, j, n, b, seed, zeta, p)
    out = []
    for c in range(b):
        nz = np.nonzero(mask[:, c])[0].astype(np.int64)
        out.append((nz, vals[nz, c].copy()))
    return out
