"""GPU: the serving runtime (lra_server_*).

Each request's Omega comes from its own Philox key and every kernel of the path
is deterministic, so a request's result must be the same bits whether it runs
alone or beside others; served results also match the FP64 CPU oracle at the
parity bars of tests/test_gpu_parity.py (the mixed precision served form at its
own bar: the same rank and status, the final error within 1%); the admission
rules (budget, slots, arrival order) are checked against the completions' own
start and finish times.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from lra_inputs import low_rank_matrix  # noqa: E402
from oracle import farpca as F  # noqa: E402
from paper_2506_03859_gb300 import lra  # noqa: E402
from paper_2506_03859_gb300.build import build  # noqa: E402

pytestmark = pytest.mark.gpu

KINDS = [(lra.GAUSSIAN, 0.0, 0), (lra.STD_BERNOULLI, 0.5, 0), (lra.SPARSE_SIGN, 0.0, 8),
         (lra.SPARSE_GAUSSIAN, 0.0, 0)]


@pytest.fixture(scope="module", autouse=True)
def library():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build()
    lra.load()


def dev(A, dtype=torch.float64):
    m, n = A.shape
    buf = torch.empty_strided((m, n), (1, m), dtype=dtype, device="cuda")
    buf.copy_(torch.from_numpy(np.ascontiguousarray(A)))
    return buf


def _requests(count, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        m = int(rng.integers(400, 3000))
        n = int(rng.integers(200, m + 1))
        kind, p, zeta = KINDS[i % len(KINDS)]
        eps = [1e-1, 1e-2, 1e-3][i % 3]
        A = low_rank_matrix(m, n, "exp100", 100 + i, rank=min(m, n, 300))
        dtype = torch.float32 if i % 2 else torch.float64
        if dtype == torch.float32:
            A = A.astype(np.float32).astype(np.float64)
        reqs.append(dict(id=i, A=dev(A, dtype), prm=lra.params(eps=eps, b=16, P=1, kind=kind, zeta=zeta,
                                                               p=p, seed=1000 + i)))
    return reqs


def test_results_equal_alone_and_in_the_mix():
    reqs = _requests(12, 0)
    srv = lra.Server(slots=4, flags=lra.FLAG_NO_GRAPHS)
    for r in reqs:
        srv.submit(r["A"], r["prm"], r["id"], keep=True)
    got = {}
    while len(got) < len(reqs):
        for c in srv.poll(wait=True):
            got[c["id"]] = c
    for r in reqs:
        c = got[r["id"]]
        assert c["status"] >= 0 and c["t_submit"] <= c["t_admit"] <= c["t_start"] <= c["t_done"]
        mix = c["run"].result()
        m, n = r["A"].shape
        pr = r["prm"]
        f = lra.Farpca(m, n, eps=pr.eps, b=pr.b, P=pr.P, kind=pr.kind, zeta=pr.zeta, p=pr.p, seed=pr.seed)
        f.run(r["A"])
        alone = f.result()
        assert (mix["status"], mix["rank"], mix["E"]) == (alone["status"], alone["rank"], alone["E"])
        assert c["rank"] == alone["rank"]
        if alone["rank"] > 0:
            assert torch.equal(mix["Q"], alone["Q"]) and torch.equal(mix["B"], alone["B"])
        f.close()
        c["run"].release()
    assert srv.pending() == 0
    srv.close()


def test_admission_limits_and_order():
    reqs = _requests(16, 1)
    need = [lra.workspace_bytes(r["A"].shape[0], r["A"].shape[1], r["prm"]) for r in reqs]
    budget = int(2.2 * max(need))
    srv = lra.Server(hbm_budget=budget, slots=3, flags=lra.FLAG_NO_GRAPHS)
    for r in reqs:
        srv.submit(r["A"], r["prm"], r["id"])
    done = []
    while len(done) < len(reqs):
        done += srv.poll(wait=True)
    srv.close()
    by_id = {c["id"]: c for c in done}
    assert all(c["status"] >= 0 for c in done)
    # arrival order: a request is never admitted before an earlier one
    admits = [by_id[i]["t_admit"] for i in range(len(reqs))]
    assert all(a <= b for a, b in zip(admits, admits[1:]))
    assert all(by_id[i]["t_submit"] <= by_id[i]["t_admit"] <= by_id[i]["t_start"] <= by_id[i]["t_done"]
               for i in range(len(reqs)))
    # at every admission, the requests then running fit the budget and the slots
    for i in range(len(reqs)):
        t = by_id[i]["t_admit"]
        live = [j for j in range(len(reqs)) if by_id[j]["t_admit"] <= t < by_id[j]["t_done"]]
        assert len(live) <= 3
        assert sum(need[j] for j in live) <= budget


def test_refusals():
    A = dev(low_rank_matrix(600, 400, "exp100", 5, rank=100))
    prm = lra.params(eps=1e-2, b=16, P=1, kind=lra.SPARSE_SIGN, zeta=8, seed=1)
    srv = lra.Server(hbm_budget=lra.workspace_bytes(600, 400, prm) - 1, slots=1)
    with pytest.raises(lra.LraError) as e:
        srv.submit(A, prm, 0)
    assert e.value.status == lra.ERR_UNSUPPORTED
    with pytest.raises(lra.LraError) as e:
        srv.submit(A, lra.params(eps=0.0, b=16), 1)      # eps = 0 without k
    assert e.value.status == lra.ERR_INVALID_ARG
    assert srv.pending() == 0
    srv.close()
    # the footprint estimate is what a context actually allocates
    f = lra.Farpca(600, 400, eps=1e-2, b=16, P=1, kind=lra.SPARSE_SIGN, zeta=8, seed=1)
    assert f.device_bytes() + 64 >= lra.workspace_bytes(600, 400, prm) >= f.device_bytes()
    f.close()


def _served(reqs, flags):
    """Serve every request (kept), return {id: completion with its result}."""
    srv = lra.Server(slots=4, flags=flags)
    for r in reqs:
        srv.submit(r["A"], r["prm"], r["id"], keep=True)
    got = {}
    while len(got) < len(reqs):
        for c in srv.poll(wait=True):
            got[c["id"]] = c
    for c in got.values():
        c["result"] = c["run"].result()
    return srv, got


def _oracle_requests():
    """One small request per hot-path kind (FP64 and FP32 data, eps 1e-2 and 1e-3).
    The rank (500) exceeds what eps = 1e-3 needs (~300 singular values of
    10^(-i/100)) and the block cap (ceil(n / 32) blocks of 16) leaves room for it, so
    no run ends at the edge of the exact rank, where a breakdown would hinge on
    rounding noise that the mixed form does not share."""
    out = []
    for i, (kind, p, zeta) in enumerate(KINDS):
        m, n = 1400 + 37 * i, 900 - 41 * i
        A = low_rank_matrix(m, n, "exp100", 300 + i, rank=500)
        dtype = torch.float32 if i % 2 else torch.float64
        if dtype == torch.float32:
            A = A.astype(np.float32).astype(np.float64)
        eps = 1e-2 if i < 2 else 1e-3
        out.append(dict(id=i, host=A, A=dev(A, dtype), kind=kind, p=p, zeta=zeta, eps=eps,
                        prm=lra.params(eps=eps, b=16, P=1, kind=kind, zeta=zeta, p=p, seed=700 + i)))
    return out


def test_served_results_match_the_oracle():
    """FP64 served form: rank and status equal; E within 5e-14 ||A||_F^2, the final
    relative error within 1e-10 (or the FP64 indicator's resolution at eps = 1e-3),
    Q within 1e-10, B within 1e-10 of max |B|."""
    reqs = _oracle_requests()
    srv, got = _served(reqs, lra.FLAG_NO_GRAPHS)
    for r in reqs:
        res = got[r["id"]]["result"]
        ref = F.farpca(r["host"], r["eps"], P=1, b=16, kind=r["kind"], seed=700 + r["id"], zeta=r["zeta"],
                       p=r["p"])
        assert (res["status"], res["rank"]) == (ref["status"], ref["rank"]) and ref["rank"] > 0
        nA = ref["normA2"]
        dE = abs(res["E"] - ref["E"]) / nA
        rel, rel_ref = (math.sqrt(max(x, 0.0) / nA) for x in (res["E"], ref["E"]))
        dQ = float(np.abs(res["Q"].cpu().numpy() - ref["Q"]).max())
        dB = float(np.abs(res["B"].cpu().numpy() - ref["B"]).max() / np.abs(ref["B"]).max())
        # final error: 1e-10 relative, or the FP64 indicator's resolution 8 * 2^-53 / rel^2
        rel_bar = max(1e-10, 8 * 2.0 ** -53 / rel_ref ** 2)
        print("PARITY served_%d E=%.3e rel_err=%.3e (bar %.1e) Q=%.3e B=%.3e"
              % (r["id"], dE, abs(rel - rel_ref) / rel_ref, rel_bar, dQ, dB))
        assert dE <= 5e-14 and abs(rel - rel_ref) <= rel_bar * rel_ref and dQ <= 1e-10 and dB <= 1e-10
        got[r["id"]]["run"].release()
    srv.close()


def test_mixed_served_form_against_the_oracle():
    """The mixed precision served form (LRA_FLAG_MIXED for every request): against
    the FP64 oracle the same rank and status and the final relative error within 1%;
    for the basis it found, Q^T Q = I and B = Q^T A to FP64 accuracy."""
    reqs = _oracle_requests()
    srv, got = _served(reqs, lra.FLAG_NO_GRAPHS | lra.FLAG_MIXED)
    for r in reqs:
        res = got[r["id"]]["result"]
        ref = F.farpca(r["host"], r["eps"], P=1, b=16, kind=r["kind"], seed=700 + r["id"], zeta=r["zeta"],
                       p=r["p"])
        assert (res["status"], res["rank"]) == (ref["status"], ref["rank"])
        rel, rel_ref = (math.sqrt(max(x, 0.0) / ref["normA2"]) for x in (res["E"], ref["E"]))
        assert abs(rel - rel_ref) <= 0.01 * rel_ref
        Q, B = res["Q"].cpu().numpy(), res["B"].cpu().numpy()
        assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() <= 1e-12
        assert np.abs(B - Q.T @ r["host"]).max() <= 1e-10 * np.abs(B).max()
        got[r["id"]]["run"].release()
    srv.close()
