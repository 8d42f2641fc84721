"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Every comparison prints its measured worst deviation beside its bar
(``PARITY <case> <quantity> measured=... bar=...``; run with ``-s`` to see them).

Bars (FP64 on both sides):
  * Omega: row indices bit-exact; values bit-exact except the Gaussian ones
    (Box-Muller through the device's log/cospi vs the host libm's log/cos: the
    angle 2 pi c is rounded differently, |diff| <= 1e-13 in units of the N(0,1)
    draw, times the 1/sqrt(p) scale);
  * sketch: max |diff| <= 1e-12 max |ref|;
  * ||A||_F^2: both sides sum exact or once-rounded squares with short
    summation chains (relative error of each a few units of 2^-53), so
    |diff| <= 1e-14 ||A||_F^2;
  * the indicator E = ||A||_F^2 - sum_j ||B_j||_F^2: |diff| <= 5e-14 ||A||_F^2,
    the resolution of the FP64 indicator (Sec. 2.1: the indicator is reliable
    for eps > 2.1e-7, i.e. E resolved to (2.1e-7)^2 ~ 4.4e-14 ||A||_F^2);
  * the final relative error sqrt(E / ||A||_F^2): within 1e-10 of the oracle's,
    relative (the stated FP64 tolerance of the method's result), or within
    8 * 2^-53 / rel^2 where that is larger: E itself is resolved only to a few
    units of 2^-53 ||A||_F^2, which at rel ~ 1e-3 is ~1e-10 of rel;
  * pre-projection Y_j: P = 0 (raw sketches) ||diff||_F <= 1e-12 ||ref||_F; P >= 1
    <= 1e-9: the deflated power step A^T (A G) - B^T (B G) cancels by about
    (sigma_1 / sigma_l)^2, so Y_j is ill conditioned; a change of the oracle's
    own summation order alone moves it by up to ~4e-10
    (tests/test_oracle_farpca.py::test_y_sensitivity_to_summation_order);
  * attained rank and status equal; Q within 1e-10 absolute (entries are
    O(m^-1/2)); B within 1e-10 of max |B|.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from lra_inputs import low_rank_matrix, workload_matrix  # noqa: E402
from oracle import farpca as F  # noqa: E402
from oracle import omega as om  # noqa: E402
from paper_2506_03859_gb300 import lra  # noqa: E402
from paper_2506_03859_gb300.build import build  # noqa: E402

pytestmark = pytest.mark.gpu

KIND_CASES = [(om.GAUSSIAN, 0.0, 0), (om.STD_BERNOULLI, 0.5, 0), (om.STD_BERNOULLI, 0.0, 0),
              (om.SPARSE_SIGN, 0.0, 8), (om.SPARSE_SIGN_IID, 0.0, 0), (om.SPARSE_GAUSSIAN, 0.0, 0),
              (om.BERNOULLI, 0.0, 0)]
IDS = ["gauss", "sb_half", "sb_p1", "ss8", "ss_iid", "sg", "bern"]


@pytest.fixture(scope="module", autouse=True)
def library():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build()
    lra.load()


def dev(A, pad=0):
    m, n = A.shape
    buf = torch.empty_strided((m + pad, n), (1, m + pad), dtype=torch.float64, device="cuda")
    view = buf[:m]
    view.copy_(torch.from_numpy(np.ascontiguousarray(A)))
    return view


def maxrel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def frorel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# bars, one per compared quantity (see the module docstring)
BAR_NORMA2 = 1e-14   # |diff| / ||A||_F^2
BAR_E = 5e-14        # |diff| / ||A||_F^2
BAR_REL_ERR = 1e-10  # relative deviation of the final error sqrt(E / ||A||_F^2) ...
U64 = 2.0 ** -53     # ... but not below what the FP64 indicator resolves at that error


def rel_err_bar(rel):
    """The bar on the final error's relative deviation: 1e-10, or, for a final error
    rel so small that E = rel^2 ||A||_F^2 is resolved only to a few units of
    2^-53 ||A||_F^2 (the cancellation in ||A||_F^2 - sum_j ||B_j||_F^2, Sec. 2.1),
    8 such units over rel^2 (a relative error d on E is d/2 on rel)."""
    return max(BAR_REL_ERR, 8 * U64 / max(rel, 1e-300) ** 2)
BAR_Y_RAW = 1e-12    # Frobenius-relative, P = 0
BAR_Y_POWER = 1e-9   # Frobenius-relative, P >= 1
BAR_Q = 1e-10        # max absolute
BAR_B = 1e-10        # max |diff| / max |B|


def check(case, quantity, measured, bar):
    """Print one measured deviation beside its bar, then hold it to the bar."""
    print("PARITY %s %s measured=%.3e bar=%.1e" % (case, quantity, measured, bar))
    assert measured <= bar, (case, quantity, measured, bar)


def rel_err_dev(r, ref):
    """Relative deviation of the final relative Frobenius error sqrt(E / ||A||^2)."""
    e = math.sqrt(max(r["E"], 0.0) / r["normA2"])
    e_ref = math.sqrt(max(ref["E"], 0.0) / ref["normA2"])
    return abs(e - e_ref) / max(e_ref, 1e-300)


def check_run(case, r, ref, Y=None, P=1):
    """The comparisons shared by every full run: normA2, E, Q, B (and Y_j)."""
    nA = ref["normA2"]
    check(case, "normA2", abs(r["normA2"] - nA) / nA, BAR_NORMA2)
    if ref["rank"] > 0:
        check(case, "E", abs(r["E"] - ref["E"]) / nA, BAR_E)
        check(case, "rel_err", rel_err_dev(r, ref), rel_err_bar(math.sqrt(max(ref["E"], 0.0) / nA)))
        if Y is not None:
            check(case, "Y_P%d" % P, frorel(Y, ref["Y"]), BAR_Y_RAW if P == 0 else BAR_Y_POWER)
        check(case, "Q", float(np.abs(r["Q"].cpu().numpy() - ref["Q"]).max()), BAR_Q)
        check(case, "B", maxrel(r["B"].cpu().numpy(), ref["B"]), BAR_B)


def test_kind_numbers_agree():
    assert (lra.GAUSSIAN, lra.STD_BERNOULLI, lra.SPARSE_SIGN, lra.SPARSE_SIGN_IID, lra.SPARSE_GAUSSIAN,
            lra.BERNOULLI) == (om.GAUSSIAN, om.STD_BERNOULLI, om.SPARSE_SIGN, om.SPARSE_SIGN_IID,
                               om.SPARSE_GAUSSIAN, om.BERNOULLI)


@pytest.mark.parametrize("kind,p,zeta", KIND_CASES + [(om.SPARSE_SIGN, 0.0, 1), (om.SPARSE_SIGN, 0.0, 16),
                                                      (om.SPARSE_SIGN, 0.0, 256)], ids=IDS + ["ss1", "ss16", "ss256"])
@pytest.mark.parametrize("n", [1000, 777])
def test_omega_bit_exact(kind, p, zeta, n):
    b, seed = 20, 12345678901
    f = lra.Farpca(50, n, eps=1e-2, b=b, P=1, kind=kind, zeta=zeta, p=p, seed=seed)
    for j in (0, 3, 1000):
        counts, rows, vals = f.copy_omega(j)
        ref = om.omega_entries(kind, j, n, b, seed, zeta=zeta, p=p)
        for c in range(b):
            r_ref, v_ref = ref[c]
            k = int(counts[c])
            assert k == len(r_ref)
            assert np.array_equal(rows[c, :k].astype(np.int64), r_ref)
            if kind in (om.GAUSSIAN, om.SPARSE_GAUSSIAN):
                scale = 1.0 if kind == om.GAUSSIAN else 1.0 / math.sqrt(
                    p if p > 0 else om.default_p(kind, n, zeta))
                assert np.all(np.abs(vals[c, :k] - v_ref) <= 1e-13 * scale)
            else:
                assert np.array_equal(vals[c, :k], v_ref)
    f.close()


@pytest.mark.parametrize("kind,p,zeta", KIND_CASES, ids=IDS)
@pytest.mark.parametrize("m,n,pad", [(1001, 700, 0), (640, 513, 3)])
def test_sketch_parity(kind, p, zeta, m, n, pad):
    b, seed = 12, 99
    A = low_rank_matrix(m, n, "poly1", 5) + 1e-3 * np.random.default_rng(0).standard_normal((m, n))
    f = lra.Farpca(m, n, eps=1e-2, b=b, P=1, kind=kind, zeta=zeta, p=p, seed=seed)
    Y = f.sketch(dev(A, pad), 2, 3).cpu().numpy()
    ref = F.sketch(A, kind, 2, 3, b, seed, zeta=zeta, p=p)
    assert Y.shape == ref.shape
    check("sketch_%dx%d_k%d" % (m, n, kind), "S0", maxrel(Y, ref), 1e-12)
    f.close()


def _compare(A, eps, P, b, kind, p, zeta, seed, k=0, max_blocks=0, pad=0, fp64_simt=False):
    m, n = A.shape
    f = lra.Farpca(m, n, eps=eps, k=k, b=b, P=P, kind=kind, zeta=zeta, p=p, seed=seed,
                   max_blocks=max_blocks, keep_y=True, fp64_simt=fp64_simt)
    status = f.run(dev(A, pad))
    r = f.result()
    ref = F.farpca(A, eps, P=P, b=b, kind=kind, seed=seed, zeta=zeta, p=p, k=k, max_blocks=max_blocks,
                   keep_y=True)
    assert status == ref["status"] == r["status"]
    assert r["rank"] == ref["rank"] and r["blocks"] == ref["blocks"]
    case = "%dx%d_k%d_P%d_b%d_%s" % (m, n, kind, P, b, "simt" if fp64_simt else "tc")
    check_run(case, r, ref, Y=r["Y"].cpu().numpy() if ref["rank"] > 0 else None, P=P)
    f.close()
    return r, ref


@pytest.mark.parametrize("kind,p,zeta", KIND_CASES, ids=IDS)
@pytest.mark.parametrize("P", [0, 1, 2])
@pytest.mark.parametrize("engine", ["tensor", "fp64_simt"])
def test_farpca_parity(kind, p, zeta, P, engine):
    A = low_rank_matrix(700, 450, "poly1.5", 77)
    _compare(A, 2e-2, P, 16, kind, p, zeta, seed=9, fp64_simt=(engine == "fp64_simt"))


@pytest.mark.parametrize("kind,p,zeta", KIND_CASES, ids=IDS)
def test_farpca_parity_2000x1000(kind, p, zeta):
    # sigma_i = i^-1.5, b = 20, P = 1, eps = 1e-2, zeta = 8 (the 2000 x 1000 workload)
    A = workload_matrix("dense2000x1000_poly1.5")
    r, ref = _compare(A, 1e-2, 1, 20, kind, p, zeta, seed=2024)
    assert r["status"] == 0 and r["rel_err"] < 1e-2


def test_edge_cases():
    m, n = 300, 200
    # zero matrix: rank 0, OK
    Z = np.zeros((m, n))
    f = lra.Farpca(m, n, eps=1e-2, b=8, P=1, kind=lra.SPARSE_SIGN, zeta=4)
    assert f.run(dev(Z)) == lra.OK
    r = f.result()
    assert r["rank"] == 0 and r["E"] == 0.0
    # one nonzero column: the first block is rank deficient -> BREAKDOWN, rank 0
    Z[:, 7] = np.arange(m) + 1.0
    f2 = lra.Farpca(m, n, eps=1e-3, b=4, P=0, kind=lra.SPARSE_SIGN, zeta=1)
    assert f2.run(dev(Z)) == lra.BREAKDOWN
    assert f2.result()["rank"] == 0
    # non-finite input is an error
    Z[3, 3] = np.nan
    with pytest.raises(lra.LraError):
        f.run(dev(Z))
    # wrong shape is an error
    with pytest.raises(lra.LraError):
        f.run(dev(np.ones((m + 1, n))))
    A = low_rank_matrix(m, n, "poly1", 3)
    # fixed rank, cap, b = 1, b = 64, padded lda, wide matrix
    _compare(A, 0.0, 1, 7, lra.SPARSE_GAUSSIAN, 0.1, 0, seed=5, k=30)
    r, _ = _compare(A, 1e-12, 0, 7, lra.SPARSE_SIGN, 0.0, 3, seed=5)
    assert r["status"] == lra.NOT_CONVERGED and r["blocks"] == F.default_max_blocks(m, n, 7)
    _compare(A, 5e-2, 1, 1, lra.SPARSE_SIGN, 0.0, 2, seed=1)
    _compare(A, 1e-3, 1, 64, lra.GAUSSIAN, 0.0, 0, seed=1, pad=5)
    _compare(np.asfortranarray(A.T), 2e-2, 2, 10, lra.SPARSE_SIGN, 0.0, 4, seed=3)


def test_deterministic_and_host_path():
    m, n = 900, 500
    A = low_rank_matrix(m, n, "poly1.5", 8)
    f = lra.Farpca(m, n, eps=1e-2, b=20, P=1, kind=lra.SPARSE_SIGN, zeta=8, seed=4)
    Ad = dev(A)
    f.run(Ad)
    r1 = f.result()
    Q1, B1 = r1["Q"].cpu().numpy().copy(), r1["B"].cpu().numpy().copy()
    f.run(Ad)
    r2 = f.result()
    assert r2["E"] == r1["E"] and np.array_equal(r2["Q"].cpu().numpy(), Q1)
    cap = f.capacity
    Qh = np.zeros((m, cap), order="F")
    Bh = np.zeros((cap, n), order="F")
    rh = f.run_host(np.asfortranarray(A), Qh, Bh)
    assert rh["rank"] == r1["rank"] and rh["E"] == r1["E"]
    assert np.array_equal(Qh[:, :rh["rank"]], Q1) and np.array_equal(Bh[:rh["rank"]], B1)


def test_full_size_bench_config():
    """20000 x 10000, sigma_i = 10^(-i/100) + 1e-6 noise, sparse sign zeta = 8, b = 50,
    P = 1, eps = 1e-2: the configuration bench.py times, against the oracle at full size."""
    A = workload_matrix("dense20000x10000_exp100")
    m, n = A.shape
    Ad = dev(A)
    r, ref = None, None
    f = lra.Farpca(m, n, eps=1e-2, b=50, P=1, kind=lra.SPARSE_SIGN, zeta=8, seed=1, keep_y=True)
    assert f.run(Ad) == lra.OK
    r = f.result()
    ref = F.farpca(A, 1e-2, P=1, b=50, kind=om.SPARSE_SIGN, seed=1, zeta=8, keep_y=True)
    assert r["rank"] == ref["rank"] and r["status"] == ref["status"] == 0
    check_run("full_ss8_P1", r, ref, Y=r["Y"].cpu().numpy(), P=1)
    # many-block sketch pass (the sketch bandwidth measurement), sampled blocks
    Y = f.sketch(Ad, 0, 64)
    for j in (0, 17, 63):
        cols = Y[:, j * 50:(j + 1) * 50].cpu().numpy()
        refc = A @ om.omega_dense(om.SPARSE_SIGN, j, n, 50, 1, zeta=8)
        check("full_sketch64", "block%d" % j, maxrel(cols, refc), 1e-12)
    f.close()


@pytest.fixture(scope="module")
def big():
    """The 20000 x 10000 benchmark matrix, on the host and on the device (built once)."""
    A = workload_matrix("dense20000x10000_exp100")
    return A, dev(A)


# The other variants of the 20000 x 10000 configuration: every Omega kind, zeta in
# {4, 16}, P in {0, 2}, eps in {1e-1, 1e-2}
# (seed 2 of the sparse Gaussian kind draws an empty Omega column in block 0: that
# column of the first power-step panel is zero, the panel completion replaces it by
# a fixed random direction, and the run goes on, on both sides)
BIG_CASES = [(om.GAUSSIAN, 0.0, 0, 1, 1e-2, 2), (om.STD_BERNOULLI, 0.5, 0, 1, 1e-2, 2),
             (om.SPARSE_SIGN, 0.0, 4, 0, 1e-1, 2), (om.SPARSE_SIGN, 0.0, 16, 2, 1e-2, 2),
             (om.SPARSE_GAUSSIAN, 0.0, 8, 1, 1e-2, 3), (om.SPARSE_GAUSSIAN, 0.0, 8, 1, 1e-2, 2)]


@pytest.mark.parametrize("kind,p,zeta,P,eps,seed", BIG_CASES,
                         ids=["gauss_P1", "sb_half_P1", "ss4_P0_eps1e-1", "ss16_P2", "sg8_P1",
                              "sg8_empty_omega_column"])
def test_full_size_variants(big, kind, p, zeta, P, eps, seed):
    """Full-size parity for the other Omega kinds and settings of the benchmark's
    matrix family: attained rank and status equal, E, Q and B within the bars."""
    A, Ad = big
    m, n = A.shape
    f = lra.Farpca(m, n, eps=eps, b=50, P=P, kind=kind, zeta=zeta, p=p, seed=seed)
    f.run(Ad)
    r = f.result()
    ref = F.farpca(A, eps, P=P, b=50, kind=kind, seed=seed, zeta=zeta, p=p)
    assert r["rank"] == ref["rank"] and r["status"] == ref["status"]
    check_run("full_k%d_z%d_P%d_eps%g_s%d" % (kind, zeta, P, eps, seed), r, ref)
    f.close()


@pytest.mark.parametrize("kind,p,zeta,P", [(om.SPARSE_SIGN, 0.0, 8, 0), (om.SPARSE_SIGN, 0.0, 8, 1),
                                           (om.SPARSE_SIGN, 0.0, 8, 2), (om.GAUSSIAN, 0.0, 0, 1)],
                         ids=["ss8_P0", "ss8_P1", "ss8_P2", "gauss_P1"])
def test_full_passes_per_block(kind, p, zeta, P):
    """Sec. 3 (cost model, Remark 3.4): past the sketch, a block streams A 2P + 1 times
    (P power steps of two passes, then B_j); the sketch adds one more full pass only
    for a dense Omega.  The phase profile counts the dense passes."""
    A = low_rank_matrix(600, 400, "poly1.5", seed=31)
    f = lra.Farpca(600, 400, eps=1e-2, b=16, P=P, kind=kind, zeta=zeta, p=p, seed=3, profile=True)
    f.run(dev(A))
    r = f.result()
    ph = f.phase_times(reset=True)
    assert r["blocks"] >= 2
    assert ph["dense"][1] == r["blocks"] * (2 * P + 1)
    assert ph["sketch"][1] == r["blocks"]
    f.close()


@pytest.mark.parametrize("kind,p,zeta,P", [(om.SPARSE_SIGN, 0.0, 8, 1), (om.GAUSSIAN, 0.0, 0, 2),
                                           (om.STD_BERNOULLI, 0.0, 0, 1)],
                         ids=["ss8_P1", "gauss_P2", "sb_p1_P1"])
def test_digit_images_change_nothing(kind, p, zeta, P):
    """A cut once into its digit images (the default) and A cut on every pass
    (LRA_FLAG_NO_A_DIGITS) feed the tensor cores the same digits in the same order:
    the runs agree bit for bit.  Ragged sizes: neither m nor n is a multiple of the
    128-row tile or the 32-deep stage."""
    m, n = 1001, 643
    A = low_rank_matrix(m, n, "poly1.5", seed=41)
    Ad = dev(A)
    out = []
    for digits in (True, False):
        f = lra.Farpca(m, n, eps=1e-2, b=24, P=P, kind=kind, zeta=zeta, p=p, seed=5, a_digits=digits)
        f.run(Ad)
        r = f.result()
        out.append((r["status"], r["rank"], r["E"], r["Q"].cpu().numpy().copy(), r["B"].cpu().numpy().copy()))
        f.close()
    (s0, k0, e0, q0, b0), (s1, k1, e1, q1, b1) = out
    assert (s0, k0) == (s1, k1) and k0 > 0
    assert e0 == e1
    assert np.array_equal(q0, q1) and np.array_equal(b0, b1)


@pytest.mark.parametrize("kind,p,zeta,P", [(om.SPARSE_SIGN, 0.0, 8, 1), (om.STD_BERNOULLI, 0.0, 0, 2)],
                         ids=["ss8_P1", "sb_p1_P2"])
def test_graphs_change_nothing(kind, p, zeta, P):
    """Each block's kernels replayed from a captured CUDA graph (the default) and
    launched one by one (LRA_FLAG_NO_GRAPHS) agree bit for bit, on the first run
    (capture) and on a second run (replay), and count the same launches."""
    m, n = 1201, 757
    A = low_rank_matrix(m, n, "poly1.5", seed=43)
    Ad = dev(A)
    runs = []
    for graphs in (True, False):
        f = lra.Farpca(m, n, eps=1e-2, b=24, P=P, kind=kind, zeta=zeta, p=p, seed=9, graphs=graphs)
        for _ in range(2):
            k0 = lra.kernel_launches()
            f.run(Ad)
            r = f.result()
            runs.append((r["status"], r["rank"], r["E"], lra.kernel_launches() - k0,
                         r["Q"].cpu().numpy().copy(), r["B"].cpu().numpy().copy()))
        f.close()
    ref = runs[-1]  # no graphs, second run
    assert ref[1] > 0
    for got in runs:
        assert got[:4] == ref[:4]
        assert np.array_equal(got[4], ref[4]) and np.array_equal(got[5], ref[5])


@pytest.mark.parametrize("kind,p,zeta,P,size", [(om.SPARSE_SIGN, 0.0, 8, 1, "small"),
                                                (om.GAUSSIAN, 0.0, 0, 1, "small"),
                                                (om.STD_BERNOULLI, 0.5, 0, 2, "small"),
                                                (om.SPARSE_SIGN, 0.0, 8, 1, "full")],
                         ids=["ss8_P1", "gauss_P1", "sb_half_P2", "ss8_P1_full"])
def test_mixed_precision_form(request, kind, p, zeta, P, size):
    """LRA_FLAG_MIXED: the sketch and power passes from the top 4 of the 7 digits,
    B_j = Q_j^T A, projections, Gram, Cholesky and indicator FP64-accurate.  Against
    the FP64 oracle: the same attained rank and status, the final relative error
    within 1% of the oracle's; and for the basis it found: Q^T Q = I, B = Q^T A and
    E = ||A - Q B||_F^2 to FP64 accuracy."""
    if size == "full":
        A, Ad = request.getfixturevalue("big")
        b, eps, seed = 50, 1e-2, 1
    else:
        A = workload_matrix("dense2000x1000_poly1.5")
        Ad = dev(A)
        b, eps, seed = 20, 1e-2, 4
    m, n = A.shape
    f = lra.Farpca(m, n, eps=eps, b=b, P=P, kind=kind, zeta=zeta, p=p, seed=seed, mixed=True)
    f.run(Ad)
    r = f.result()
    ref = F.farpca(A, eps, P=P, b=b, kind=kind, seed=seed, zeta=zeta, p=p)
    assert r["rank"] == ref["rank"] and r["status"] == ref["status"] == 0
    rel, rel_ref = math.sqrt(max(r["E"], 0.0) / r["normA2"]), math.sqrt(max(ref["E"], 0.0) / ref["normA2"])
    assert abs(rel - rel_ref) <= 0.01 * rel_ref
    Q = r["Q"].cpu().numpy()
    B = r["B"].cpu().numpy()
    assert float(np.abs(Q.T @ Q - np.eye(Q.shape[1])).max()) <= 1e-12
    assert maxrel(B, Q.T @ A) <= 1e-10
    if size == "small":  # E against the residual, computed directly (Sec. 2.1)
        E_direct = float(np.linalg.norm(A - Q @ B) ** 2)
        assert abs(r["E"] - E_direct) <= 1e-10 * r["normA2"]
    f.close()


def dev32(A, pad=0):
    m, n = A.shape
    buf = torch.empty_strided((m + pad, n), (1, m + pad), dtype=torch.float32, device="cuda")
    view = buf[:m]
    view.copy_(torch.from_numpy(np.ascontiguousarray(A.astype(np.float32))))
    return view


def _same_run(f32, f64):
    """Two contexts' results: identical bits (rank, status, E, Q, B)."""
    a, b_ = f32.result(), f64.result()
    assert (a["status"], a["rank"], a["blocks"]) == (b_["status"], b_["rank"], b_["blocks"])
    assert a["E"] == b_["E"] and a["normA2"] == b_["normA2"]
    if a["rank"] > 0:
        assert torch.equal(a["Q"], b_["Q"]) and torch.equal(a["B"], b_["B"])
    return a


# FP32 input: entries are converted exactly where A is read, so the run on FP32
# data and the run on its FP64 conversion must agree bit for bit (the FP64 run is
# itself pinned to the oracle above).
@pytest.mark.parametrize("kind,p,zeta", [KIND_CASES[0], KIND_CASES[1], KIND_CASES[3], KIND_CASES[5]],
                         ids=["gauss", "sb_half", "ss8", "sg"])
@pytest.mark.parametrize("P", [0, 1])
@pytest.mark.parametrize("shape,pad", [((1000, 700), 0), ((1037, 611), 1), ((600, 900), 3)],
                         ids=["aligned", "ragged", "wide"])
def test_fp32_input_matches_its_fp64_conversion(kind, p, zeta, P, shape, pad):
    m, n = shape
    A = low_rank_matrix(m, n, "poly1.5", 21).astype(np.float32).astype(np.float64)
    kw = dict(eps=1e-2, b=16, P=P, kind=kind, zeta=zeta, p=p, seed=5)
    f32, f64 = lra.Farpca(m, n, **kw), lra.Farpca(m, n, **kw)
    s32, s64 = f32.run(dev32(A, pad)), f64.run(dev(A, pad))
    assert s32 == s64
    r = _same_run(f32, f64)
    assert r["rank"] > 0
    mixed32, mixed64 = lra.Farpca(m, n, mixed=True, **kw), lra.Farpca(m, n, mixed=True, **kw)
    mixed32.run(dev32(A, pad))
    mixed64.run(dev(A, pad))
    _same_run(mixed32, mixed64)
    if kind in (lra.SPARSE_SIGN, lra.SPARSE_GAUSSIAN):
        Y32 = f32.sketch(dev32(A, pad), 0, 3)
        Y64 = f64.sketch(dev(A, pad), 0, 3)
        assert torch.equal(Y32, Y64)
    for f in (f32, f64, mixed32, mixed64):
        f.close()


def test_fp32_host_path_and_unsupported_forms():
    m, n = 800, 500
    A = low_rank_matrix(m, n, "poly1.5", 22).astype(np.float32)
    kw = dict(eps=1e-2, b=10, P=1, kind=lra.SPARSE_SIGN, zeta=8, seed=2)
    f32, f64 = lra.Farpca(m, n, **kw), lra.Farpca(m, n, **kw)
    Qh = np.zeros((m, f32.capacity), order="F")
    r32 = f32.run_host(np.asfortranarray(A), Q_host=Qh)
    f64.run(dev(A.astype(np.float64)))
    r64 = f64.result()
    assert (r32["rank"], r32["E"]) == (r64["rank"], r64["E"])
    assert np.array_equal(Qh[:, :r32["rank"]], r64["Q"].cpu().numpy())
    # the allocation-free sketch on FP32 data
    Y32 = lra.sketch_noalloc(dev32(A.astype(np.float64)), 0, 2, 10, lra.SPARSE_SIGN, zeta=8, seed=2)
    Y64 = lra.sketch_noalloc(dev(A.astype(np.float64)), 0, 2, 10, lra.SPARSE_SIGN, zeta=8, seed=2)
    assert torch.equal(Y32, Y64)
    # forms that read A as FP64 refuse FP32 data
    simt = lra.Farpca(m, n, fp64_simt=True, **kw)
    with pytest.raises(lra.LraError) as e:
        simt.run(dev32(A.astype(np.float64)))
    assert e.value.status == lra.ERR_UNSUPPORTED
    with pytest.raises(lra.LraError) as e:
        f32.apply(dev32(A.astype(np.float64)), torch.zeros((n, 4), dtype=torch.float64, device="cuda").t().contiguous().t())
    assert e.value.status == lra.ERR_UNSUPPORTED
    for f in (f32, f64, simt):
        f.close()


def test_fp32_full_size(big):
    """20000 x 10000 in FP32 (the FP32 form of the same workload): the run on the
    FP32 data equals the run on its FP64 conversion bit for bit."""
    A, _ = big
    A32 = A.astype(np.float32)
    m, n = A.shape
    kw = dict(eps=1e-2, b=50, P=1, kind=lra.SPARSE_SIGN, zeta=8, seed=1)
    f32 = lra.Farpca(m, n, **kw)
    assert f32.run(dev32(A32.astype(np.float64))) == lra.OK
    r32 = f32.result()
    Q32, B32 = r32["Q"].clone(), r32["B"].clone()
    f32.close()
    f64 = lra.Farpca(m, n, **kw)
    assert f64.run(dev(A32.astype(np.float64))) == lra.OK
    r64 = f64.result()
    assert (r32["rank"], r32["E"]) == (r64["rank"], r64["E"])
    assert torch.equal(Q32, r64["Q"]) and torch.equal(B32, r64["B"])
    f64.close()


@pytest.mark.parametrize("kind,p,zeta", [(om.STD_BERNOULLI, 0.5, 0), (om.SPARSE_SIGN, 0.0, 8)],
                         ids=["sb_pm1", "ss8"])
def test_precision_workload_family(kind, p, zeta):
    """The precision workload's family (sigma_i = i^-1, b = 64, P = 1, eps = 1e-3) at a
    reduced size: 6000 x 2000 of rank 1200, so that eps stays out of reach within the
    block cap ceil(2000 / 128) = 16 blocks (rank 1024) and every form ends
    NOT_CONVERGED at the cap.  FP64 form: against the oracle at the parity bars.
    Mixed form: the same rank and status, the final error within 1% of the oracle's."""
    A = low_rank_matrix(6000, 2000, "poly1", 61, rank=1200)
    m, n = A.shape
    Ad = dev(A)
    ref = F.farpca(A, 1e-3, P=1, b=64, kind=kind, seed=3, zeta=zeta, p=p)
    assert ref["status"] == F.NOT_CONVERGED and ref["rank"] == 1024
    for mixed in (False, True):
        f = lra.Farpca(m, n, eps=1e-3, b=64, P=1, kind=kind, zeta=zeta, p=p, seed=3, mixed=mixed)
        f.run(Ad)
        r = f.result()
        assert (r["status"], r["rank"]) == (ref["status"], ref["rank"])
        if mixed:
            check("poly1_6000x2000_k%d_mixed" % kind, "rel_err_1pct", rel_err_dev(r, ref), 0.01)
        else:
            check_run("poly1_6000x2000_k%d" % kind, r, ref)
        f.close()


@pytest.mark.parametrize("kind,p", [(om.STD_BERNOULLI, 0.0), (om.SPARSE_SIGN_IID, 2e-3), (om.BERNOULLI, 1e-2)],
                         ids=["sb_lnn", "ss_iid_2e-3", "bern_1e-2"])
def test_dependent_power_panel_completion(kind, p):
    """Sec. 5.5's hard case at n = 1000: Matrix 1's spectrum with V_A = diag(+-1)
    (d = n blocks), where A^T A is diagonal and the power-step panels are
    numerically rank deficient.  The panel completion (dependent columns replaced
    by fixed random directions) runs on both sides."""
    n = 1000
    rng = np.random.default_rng(55)
    U, R = np.linalg.qr(rng.standard_normal((n, n)))
    U *= np.sign(np.diag(R))[None, :]
    A = np.asfortranarray((U * (1.0 / np.arange(1, n + 1) ** 2)[None, :]) * rng.choice([-1.0, 1.0], n)[None, :])
    f = lra.Farpca(n, n, eps=1e-4, b=20, P=1, kind=kind, p=p, seed=8)
    f.run(dev(A))
    r = f.result()
    ref = F.farpca(A, 1e-4, P=1, b=20, kind=kind, seed=8, p=p)
    assert ref["status"] != F.BREAKDOWN and ref["rank"] > 0
    assert (r["status"], r["rank"]) == (ref["status"], ref["rank"])
    # The completed panels are ill conditioned by nature (pivots next to the
    # threshold decide which columns are replaced; the kept ones are fixed inside
    # their nearly dependent span only to 2^-53 cond^2), so the two sides' bases
    # agree at the method's level: the same rank and status, the final error
    # within 1%, and a valid QB on the device (Q^T Q = I, B = Q^T A,
    # E = ||A - Q B||_F^2).
    check("dnn_completion_k%d" % kind, "rel_err_1pct", rel_err_dev(r, ref), 0.01)
    Q, B = r["Q"].cpu().numpy(), r["B"].cpu().numpy()
    check("dnn_completion_k%d" % kind, "QtQ-I", float(np.abs(Q.T @ Q - np.eye(Q.shape[1])).max()), 1e-12)
    check("dnn_completion_k%d" % kind, "B-QtA", maxrel(B, Q.T @ A), 1e-10)
    check("dnn_completion_k%d" % kind, "E-direct", abs(r["E"] - np.linalg.norm(A - Q @ B) ** 2) / r["normA2"],
          1e-12)
    f.close()


def test_host_prefetch_stream():
    """lra_farpca_host_prefetch: a stream of host matrices, each copied to the device
    while the previous one is solved (two device buffers, one graph set each), gives
    the same bits as solving each matrix from device memory; a prefetch that the
    next call does not use is waited for and skipped; a plain lra_farpca_host call
    on the prefetched matrix uses the copy."""
    m, n = 1200, 700
    mats = [np.asfortranarray(low_rank_matrix(m, n, "poly1.5", 50 + i)) for i in range(3)]
    f = lra.Farpca(m, n, eps=1e-2, b=20, P=1, kind=lra.SPARSE_SIGN, zeta=8, seed=4)
    ref = []
    for A in mats:
        f.run(dev(A))
        r = f.result()
        ref.append((r["rank"], r["E"], r["Q"].cpu().numpy().copy(), r["B"].cpu().numpy().copy()))
    cap = f.capacity
    Qh = np.zeros((m, cap), order="F")
    Bh = np.zeros((cap, n), order="F")

    def check(i, r):
        rank, E, Q, B = ref[i]
        assert (r["rank"], r["E"]) == (rank, E)
        assert np.array_equal(Qh[:, :rank], Q) and np.array_equal(Bh[:rank], B)

    order = [(0, 1), (1, 2), (2, 0), (0, 1), (2, None), (1, 0), (0, None)]
    for i, nxt in order:  # (2, None) after prefetching 1: the unused prefetch is skipped
        r = f.run_host(mats[i], Qh, Bh, next_A=mats[nxt] if nxt is not None else None)
        check(i, r)
    f.close()
