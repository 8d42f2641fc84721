"""GPU: the batched form (lra_batch_*) against the FP64 oracle, problem by problem.

Each problem's FP32 matrix is converted exactly to FP64 and run through
oracle.farpca with the same Omega (fixed-zeta sparse sign, same seed, b, P).
The batched path computes in FP32 (Gram sums, Cholesky and indicator in FP64),
so the bars come from FP32 accumulation: every FP32 sum has at most 64 terms per
lane plus a 5-level shuffle tree, a relative error of about (64 + 5) 2^-24 ~ 4e-6
of the sum of |terms|, on ||A||_F^2 and on each ||B_j||_F^2:
  * status and rank equal, except where the oracle's E after some block lies
    within 1e-4 ||A||_F^2 of the threshold (the decision may then move by a block);
  * |E - E_oracle| <= 3e-5 ||A||_F^2 when the ranks agree;
  * Q^T Q = I within 1e-4 (CGS2 and shifted Cholesky QR3 in FP32 keep a few
    hundred units of 2^-24);
  * E against the residual ||A - Q B||_F^2 formed in FP64 from the device's
    factors: within (2 ||Q^T Q - I||_2 + 3e-5) ||A||_F^2, the gap the identity
    E = ||A||^2 - ||B||^2 has when Q is orthonormal only to that level.
A problem's result is the same bits in any batch (its Omega depends on its seed
alone and every reduction has a fixed order).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from lra_inputs import batch_matrix, batch_shapes  # noqa: E402
from oracle import farpca as F  # noqa: E402
from oracle import omega as om  # noqa: E402
from paper_2506_03859_gb300 import lra  # noqa: E402
from paper_2506_03859_gb300.build import build  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def library():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build()
    lra.load()


def check_problem(res, A32, eps, b, P, zeta, seed):
    A = A32.double().cpu().numpy()
    ref = F.farpca(A, eps, P=P, b=b, kind=om.SPARSE_SIGN, seed=seed, zeta=zeta)
    normA2 = ref["normA2"]
    assert abs(res["normA2"] - normA2) <= 1e-5 * normA2 + 1e-300
    thr = eps * eps * normA2
    near = any(abs(e - thr) <= 1e-4 * normA2 for e in ref["E_trace"])
    if near:
        assert abs(res["rank"] - ref["rank"]) <= b
    else:
        assert (res["status"], res["rank"]) == (ref["status"], ref["rank"])
    if res["rank"] == 0:
        return ref
    Q = res["Q"].double().cpu().numpy()
    B = res["Bt"].double().cpu().numpy().T
    l = res["rank"]
    orth = np.linalg.norm(Q.T @ Q - np.eye(l), 2)
    assert orth <= 1e-4, orth
    if res["rank"] == ref["rank"]:
        assert abs(res["E"] - ref["E"]) <= 3e-5 * normA2, (res["E"], ref["E"], normA2)
    direct = float(np.sum((A - Q @ B) ** 2))
    assert abs(res["E"] - direct) <= (2 * orth + 3e-5) * normA2
    if res["status"] == lra.OK:
        assert res["E"] < thr
    return ref


def make(shapes, seed0):
    mats = [batch_matrix(m, n, seed0 + k) for k, (m, n) in enumerate(shapes)]
    eps = [1e-1 if k % 2 else 1e-2 for k in range(len(shapes))]
    seeds = [7000 + seed0 + k for k in range(len(shapes))]
    return mats, eps, seeds


EDGE = [(64, 32), (2048, 1024), (100, 700), (1000, 32), (2048, 33), (65, 1024), (513, 257)]


@pytest.mark.parametrize("b,P", [(16, 1), (16, 0), (8, 1), (32, 1)])
def test_batch_parity(b, P):
    shapes = EDGE + batch_shapes(17, 3)
    mats, eps, seeds = make(shapes, 100)
    bt = lra.Batch(mats, eps, seeds, b=b, P=P, zeta=4)
    bt.run()
    assert 1 <= bt.steps() <= max((min(m, n) + 2 * b - 1) // (2 * b) for m, n in shapes)
    for k in range(len(shapes)):
        check_problem(bt.result(k), mats[k], eps[k], b, P, 4, seeds[k])
    bt.close()


def test_batch_independence_and_edge_states():
    shapes = [(300, 200), (1500, 900), (64, 32), (2000, 1000)]
    mats, eps, seeds = make(shapes, 200)
    zero = torch.zeros((500, 300), dtype=torch.float32, device="cuda").t().contiguous().t()
    alone = lra.Batch([mats[1]], [eps[1]], [seeds[1]], b=16, P=1, zeta=4)
    alone.run()
    mixed = lra.Batch(mats + [zero], eps + [1e-2], seeds + [1], b=16, P=1, zeta=4)
    mixed.run()
    a, m = alone.result(0), mixed.result(1)
    assert (a["status"], a["rank"], a["E"], a["normA2"]) == (m["status"], m["rank"], m["E"], m["normA2"])
    assert torch.equal(a["Q"], m["Q"]) and torch.equal(a["Bt"], m["Bt"])
    z = mixed.result(4)
    assert (z["status"], z["rank"], z["E"], z["normA2"]) == (lra.OK, 0, 0.0, 0.0)
    # a second run of the same batch gives the same bits, and so does the
    # host-driven form (each step launched from the host instead of the graph)
    q0 = m["Q"].clone()
    mixed.run()
    assert torch.equal(mixed.result(1)["Q"], q0)
    host = lra.Batch(mats + [zero], eps + [1e-2], seeds + [1], b=16, P=1, zeta=4, graph=False)
    host.run()
    for k in range(5):
        a, h = mixed.result(k), host.result(k)
        assert (a["status"], a["rank"], a["E"]) == (h["status"], h["rank"], h["E"])
        if a["rank"]:
            assert torch.equal(a["Q"], h["Q"]) and torch.equal(a["Bt"], h["Bt"])
    host.close()
    alone.close()
    mixed.close()


def test_batch_arguments():
    A = batch_matrix(100, 50, 1)
    with pytest.raises(lra.LraError):
        lra.Batch([A], [1e-2], [0], b=12)          # b not in {8, 16, 32}
    with pytest.raises(lra.LraError):
        lra.Batch([A], [0.0], [0], b=16)           # eps must be > 0
    with pytest.raises(lra.LraError):
        lra.Batch([A], [1e-2], [0], b=16, P=2)     # P in {0, 1}
    with pytest.raises(lra.LraError):
        lra.Batch([batch_matrix(100, 12, 2)], [1e-2], [0], b=16)   # b > min(m, n)


def test_batch_full_size_sampled():
    """4096 problems, rows uniform 64..2048, columns uniform 32..1024, eps in
    {1e-1, 1e-2}, zeta = 4, b = 16, P = 1: every problem ends in a valid state;
    16 sampled problems against the oracle."""
    shapes = batch_shapes(4096, 11)
    mats, eps, seeds = make(shapes, 1000)
    bt = lra.Batch(mats, eps, seeds, b=16, P=1, zeta=4)
    bt.run()
    states = [bt.result(k) for k in range(len(shapes))]
    assert all(s["status"] in (lra.OK, lra.NOT_CONVERGED) for s in states)
    assert all(s["E"] < e * e * s["normA2"] for s, e in zip(states, eps) if s["status"] == lra.OK)
    for k in np.random.default_rng(0).choice(len(shapes), 16, replace=False):
        check_problem(states[int(k)], mats[int(k)], eps[int(k)], 16, 1, 4, seeds[int(k)])
    bt.close()


def _snapshot(bt, count):
    out = []
    for k in range(count):
        r = bt.result(k)
        out.append((r["status"], r["rank"], r["E"], r["normA2"],
                    r["Q"].clone() if r["rank"] else None, r["Bt"].clone() if r["rank"] else None))
    return out


@pytest.mark.parametrize("b", [8, 16, 32])
def test_tilings_give_the_same_bits(b):
    """The tile shape of each class (columns / rows per thread of the products)
    changes how the work is cut, not what a thread sums or in which order: every
    tiling gives the same bits, and a run after the autotuner too."""
    shapes = EDGE + [(300, 200), (1500, 900), (700, 400), (2000, 1000), (200, 600)]
    mats, eps, seeds = make(shapes, 300)
    bt = lra.Batch(mats, eps, seeds, b=b, P=1, zeta=4)
    assert bt.tiling() == {"tn": [2, 2, 2], "nn": [2, 2, 2]}
    bt.run()
    ref = _snapshot(bt, len(shapes))
    for tn, nn in [([1, 1, 1], [1, 1, 1]), ([4, 4, 4], [4, 4, 4]), ([1, 4, 2], [4, 1, 2])]:
        bt.set_tiling(tn, nn)
        assert bt.tiling() == {"tn": tn, "nn": nn}
        bt.run()
        for got, want in zip(_snapshot(bt, len(shapes)), ref):
            assert got[:4] == want[:4]
            if want[1]:
                assert torch.equal(got[4], want[4]) and torch.equal(got[5], want[5])
    t = bt.tune(reps=1)
    assert all(v in (1, 2, 4) for v in t["tn"] + t["nn"]) and t["ms"] > 0 and t["ms"] <= t["base_ms"] * 1.5
    assert bt.tiling() == {"tn": t["tn"], "nn": t["nn"]}
    bt.run()
    for got, want in zip(_snapshot(bt, len(shapes)), ref):
        assert got[:4] == want[:4]
    with pytest.raises(lra.LraError):
        bt.set_tiling([3, 2, 2], [2, 2, 2])
    bt.close()
