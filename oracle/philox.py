"""Philox4x32-10, written from its published definition.

Source: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11, Sec. 3 (the Philox S-box: two 32x32->64
multiplications per round, a Weyl sequence on the key, 10 rounds for the
recommended 4x32 variant).

Pinned by tests/test_oracle_philox.py against the known-answer vectors that
accompany that paper's reference implementation (tests/golden/).

Test infrastructure only: see oracle/__init__.py.
"""
import numpy as np

MASK32 = np.uint64(0xFFFFFFFF)
# Round multipliers and key increments of Philox4x32 (SC'11, Table 2 / Sec. 3.3).
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint64(0x9E3779B9)
PHILOX_W1 = np.uint64(0xBB67AE85)
ROUNDS = 10


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Apply the 10-round Philox4x32 bijection to counters (c0..c3) under key (k0, k1).

    All arguments are array-likes of unsigned 32-bit values (broadcastable);
    returns four uint64 arrays holding the 32-bit outputs.  One round maps
    (c0, c1, c2, c3) to (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1,
    lo(M0*c0)); between rounds the key advances by (W0, W1) mod 2^32.
    """
    c0, c1, c2, c3, k0, k1 = (np.asarray(x, dtype=np.uint64) & MASK32
                              for x in (c0, c1, c2, c3, k0, k1))
    c0, c1, c2, c3, k0, k1 = np.broadcast_arrays(c0, c1, c2, c3, k0, k1)
    for r in range(ROUNDS):
        if r > 0:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * c0          # < 2^64, exact in uint64
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def seed_key(seed):
    """Split a 64-bit seed into the Philox key words (low word first)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32
