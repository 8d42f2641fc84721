"""GPU: the serving runtime (lra_server_*).

Each request's Omega comes from its own Philox key and every kernel of the path
is deterministic, so a request's result must be the same bits whether it runs
alone or beside others; the admission rules (budget, slots, arrival order) are
checked against the completions' own start and finish times.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from lra_inputs import low_rank_matrix  # noqa: E402
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
