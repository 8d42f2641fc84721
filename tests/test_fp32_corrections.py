"""Host checks of the arithmetic behind the two FP32 corrections of the solve.

The second X R^{-1} of CholQR2 (when the Cholesky finds its Gram within 2^-40
of the identity) and the second update of CGS2 (when F = Q^T Y is small against
Y's column scale) take their correction term in FP32 instead of the
FP64-accurate product.  The device truncates FP64 to FP32 by integer operations
and sums FP32 products.  These tests emulate that arithmetic in numpy (the
truncation bit for bit, the products and sums in float32 with a rounding after
each operation, which errs at least as much as the device's fused
multiply-adds) and check the bounds the design rests on:

* the truncation: relative error below 2^-23, toward zero, magnitudes below
  2^-126 to zero; the widening back to FP64 exact;
* CholQR2 near the identity: R^{-1} = I - Phi(S - I) (Phi: strict upper
  triangle plus half the diagonal), and X + X (R^{-1} - I) with the correction
  in FP32 errs by less than 2^-55 of each row's norm when every entry of S - I
  is within 2^-40 (b <= 64);
* the CGS2 gate: when every |F[k, c]| <= 2^-29 / ((l + 4) sqrt(l)) 2^(e_c - 1022)
  (e_c the biased exponent of column c's largest entry of Y), Y - Q F in FP32
  errs by at most 2^-53 2^(e_c - 1022).

No GPU: these pin the bounds, the GPU parity tests the kernels.
"""
import numpy as np


def trunc_f32(v):
    """FP64 -> FP32 by the device's integer steps: sign, exponent rebiased, the
    top 23 fraction bits kept; below 2^-126 to zero, above the range to inf."""
    v = np.asarray(v, dtype=np.float64)
    u = v.view(np.uint64)
    hi = (u >> np.uint64(32)).astype(np.uint64)
    lo = (u & np.uint64(0xFFFFFFFF)).astype(np.uint64)
    sign = hi & np.uint64(0x80000000)
    e = ((hi >> np.uint64(20)) & np.uint64(0x7FF)).astype(np.int64) - 1023 + 127
    frac = ((hi & np.uint64(0xFFFFF)) << np.uint64(3)) | (lo >> np.uint64(29))
    ec = np.clip(e, 0, 254).astype(np.uint64)
    bits = np.where(e <= 0, sign,
                    np.where(e >= 255, sign | np.uint64(0x7F800000),
                             sign | (ec << np.uint64(23)) | frac))
    return bits.astype(np.uint32).view(np.float32)


def widen_f64(f):
    """FP32 -> FP64 by the device's integer steps (subnormals to zero)."""
    u = np.asarray(f, dtype=np.float32).view(np.uint32).astype(np.uint64)
    sign = u & np.uint64(0x80000000)
    ef = (u >> np.uint64(23)) & np.uint64(0xFF)
    m = u & np.uint64(0x7FFFFF)
    ed = np.where(ef == 255, np.uint64(2047), ef - np.uint64(127) + np.uint64(1023))
    hi = np.where(ef == 0, sign, sign | (ed << np.uint64(20)) | (m >> np.uint64(3)))
    lo = np.where(ef == 0, np.uint64(0), (m << np.uint64(29)) & np.uint64(0xFFFFFFFF))
    return ((hi << np.uint64(32)) | lo).view(np.float64)


def fp32_matmul(X32, D32):
    """sum_k X32[:, k] D32[k, :] in float32, one rounding per product and per sum,
    k in order (the device's order)."""
    acc = np.zeros((X32.shape[0], D32.shape[1]), dtype=np.float32)
    for k in range(X32.shape[1]):
        acc = (acc + (X32[:, k:k + 1] * D32[k:k + 1, :]).astype(np.float32)).astype(np.float32)
    return acc


def exact_matmul(X, D):
    """The reference product: per entry, math.fsum (an exactly rounded sum) of the
    FP64 products.  Each product is rounded once (2^-53 of itself); the terms
    here are ~2^-40 of X's entries or smaller, so the reference errs far below
    the 2^-53 to 2^-55 bounds checked against it."""
    import math
    out = np.empty((X.shape[0], D.shape[1]))
    for i in range(X.shape[0]):
        for c in range(D.shape[1]):
            out[i, c] = math.fsum(float(X[i, k]) * float(D[k, c]) for k in range(X.shape[1]))
    return out


def test_truncation_and_widening():
    rng = np.random.default_rng(7)
    v = rng.standard_normal(200000) * 10.0 ** rng.integers(-37, 37, 200000)
    f = trunc_f32(v)
    back = f.astype(np.float64)
    normal = (np.abs(v) >= 2.0 ** -126) & (np.abs(v) < 2.0 ** 128)
    rel = np.abs(back[normal] - v[normal]) / np.abs(v[normal])
    assert normal.sum() > 150000 and rel.max() < 2.0 ** -23
    assert np.all(np.abs(back) <= np.abs(v))          # toward zero
    assert np.all(np.sign(back[normal]) == np.sign(v[normal]))
    assert np.all(back[np.abs(v) < 2.0 ** -126] == 0.0)
    # below the normal range to zero, above it to infinity
    assert np.all(trunc_f32(np.array([2.0 ** -127, -2.0 ** -130, 0.0])) == 0.0)
    assert np.all(np.isinf(trunc_f32(np.array([2.0 ** 128, -2.0 ** 200]))))
    # widening is exact for every normal FP32 value
    assert np.array_equal(widen_f64(f), f.astype(np.float64))


def phi(E):
    """Strict upper triangle plus half the diagonal."""
    return np.triu(E, 1) + np.diag(np.diag(E)) / 2


def test_cholqr2_near_identity_correction_bound():
    rng = np.random.default_rng(11)
    for b, rows, mag in ((50, 300, 2.0 ** -40), (64, 200, 2.0 ** -40), (16, 400, 2.0 ** -44)):
        X = np.linalg.qr(rng.standard_normal((rows, b)))[0]
        E = rng.uniform(-mag, mag, (b, b))
        E = (E + E.T) / 2
        assert np.abs(E).max() <= 2.0 ** -40
        Rinv = np.eye(b) - phi(E)
        D = Rinv - np.eye(b)
        corr32 = widen_f64(fp32_matmul(trunc_f32(X), trunc_f32(D)))
        corr = exact_matmul(X, D)
        err = np.abs(corr32 - corr)
        row_norm = np.linalg.norm(X, axis=1)
        assert np.all(err.max(axis=1) < 2.0 ** -55 * row_norm), (b, (err.max(axis=1) / row_norm).max())
        # and the closed form is R^{-1} to 2 b max|E|^2 per entry
        R = np.linalg.cholesky(np.eye(b) + E).T
        assert np.abs(Rinv - np.linalg.inv(R)).max() <= 2 * b * np.abs(E).max() ** 2 + 1e-15


def test_cgs2_gate_bound():
    rng = np.random.default_rng(13)
    for m, l, b in ((2000, 50, 50), (1500, 200, 50), (800, 300, 16)):
        Q = np.linalg.qr(rng.standard_normal((m, l)))[0]
        Y = rng.standard_normal((m, b)) * 10.0 ** rng.integers(-3, 3, b)
        ecol = np.array([(np.abs(Y[:, c]).max().view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)
                         for c in range(b)]).astype(np.int64)
        scale = np.ldexp(1.0, (ecol - 1022).astype(int))
        assert np.all(np.abs(Y).max(axis=0) < scale)
        g = 2.0 ** -29 / ((l + 4) * np.sqrt(l))
        # F at the gate (the worst case the test admits), and far below it as after
        # a first projection
        for level in (1.0, 2.0 ** -20):
            F = rng.uniform(-1, 1, (l, b)) * (g * level) * scale[None, :]
            assert np.all(np.abs(F) <= g * scale[None, :])
            upd32 = widen_f64(fp32_matmul(trunc_f32(Q), trunc_f32(F)))
            upd = exact_matmul(Q, F)
            err = np.abs(upd32 - upd).max(axis=0)
            assert np.all(err <= 2.0 ** -53 * scale), (m, l, b, level, (err / scale).max())
