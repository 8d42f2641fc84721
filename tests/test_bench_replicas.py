"""CPU, world size 2 over gloo: bench.py's multi-rank logic.

With N GPUs each rank solves its own replica (one matrix per step, no collective
on the data path); the job's time is the slowest rank's and its throughput the
solves of all ranks over that time.  The reference arm runs on rank 0 only.
These ranks exchange nothing but the timing reduction, so two CPU processes over
gloo exercise exactly the code the GPU ranks run.
"""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_env()
        ms = 10.0 * (rank + 1)            # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms, w, "cpu")
        value = bench.whole_job_value(ms_max, w, steps=5)
        # the reference arm: only rank 0 works and prints
        buf = io.StringIO()
        args = type("A", (), {"warmup": 0, "steps": 0, "gpus": w, "workload": "tiny"})()
        if r != 0:
            with redirect_stdout(buf):
                bench.run_reference(args, cfg=None)
        dist.barrier()
        out.put((r, w, local, ms_max, value, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_all_solves():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    for r, w, local, ms_max, value, printed in got:
        assert (w, local) == (world, r)
        assert ms_max == 20.0                      # max over ranks, on every rank
        assert value == pytest.approx(2 * 5 / 0.020)  # 2 ranks x 5 solves in 20 ms
        assert printed == ""                       # non-zero ranks print nothing


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.whole_job_value(12.5, 1, 5) == pytest.approx(400.0)


def test_reference_line_carries_the_same_config_keys(monkeypatch):
    """The reference arm's JSON line: same metric, unit, direction and config as ours (run
    results such as the attained rank sit under "result", outside the config)."""
    import bench
    import numpy as np
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    cfg = dict(bench.WORKLOADS["farpcass_2000x1000_poly1.5_zeta8_b20_P1_eps1e-2"])
    rng = np.random.default_rng(0)
    small = rng.standard_normal((120, 80)) @ np.diag(0.5 ** np.arange(80)) @ rng.standard_normal((80, 80))
    monkeypatch.setattr("lra_inputs.workload_matrix", lambda name: small)
    args = type("A", (), {"warmup": 0, "steps": 1, "gpus": 1,
                          "workload": "farpcass_2000x1000_poly1.5_zeta8_b20_P1_eps1e-2"})()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args, cfg)
    line = json.loads(buf.getvalue())
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == "solves/s" and line["higher_is_better"]
    ours = bench.workload_config(args, cfg, 120, 80, 1)
    assert line["config"] == ours  # the same workload description in both arms
    assert set(line["result"]) == {"rank", "blocks", "rel_err", "status"}
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_solve_bytes_pass_count():
    """The time-to-eps roofline counts the full passes over A of Sec. 3's cost model
    (Remark 3.4): one for ||A||_F^2, then 2P + 1 per block for a gathered sketch and
    2P + 2 for a dense one; each full pass moves A once plus its skinny operands."""
    import bench
    m, n, b = 2000, 1000, 20
    for P in (0, 1, 2):
        for blocks in (1, 5):
            _, sparse = bench.solve_bytes(m, n, b, P, blocks, 2, 8)
            _, dense = bench.solve_bytes(m, n, b, P, blocks, 0, 0)
            assert sparse == 1 + blocks * (2 * P + 1)
            assert dense == 1 + blocks * (2 * P + 2)
    total, passes = bench.solve_bytes(20000, 10000, 50, 1, 5, 2, 8)
    assert passes == 16
    # the full passes dominate: 16 x 8 m n bytes of A, plus everything else
    assert 16 * 8.0 * 20000 * 10000 < total < 1.2 * 16 * 8.0 * 20000 * 10000
    rl = bench.solve_roofline(20000, 10000, 50, 1, 5, 2, 8, 15.6, {"hbm_gbs": 6700.0, "bf16_tflops": 1900.0},
                              "test")
    assert rl["roofline_ms"] == pytest.approx(total / 6.7e12 * 1e3)
    assert rl["roofline_ms"] < rl["design_floor_ms"] < 15.6
