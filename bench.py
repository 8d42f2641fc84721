#!/usr/bin/env python3
"""Time-to-eps of the fixed-precision farPCA loop on GB300 (arxiv 2506.03859).

One step = one lra_farpca_run on a device-resident A: Omega generation, the
sketch, the deflated power steps, the projections and CholQR2, and the error
indicator, block by block until E < eps^2 ||A||_F^2.  Inputs are synthetic
(seeded Haar U, V and the stated spectrum; lra_inputs), larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Prints one JSON line (rank 0).  With N > 1 (torchrun) each rank solves its own
replica (no collective on the data path); value = solves of all ranks / max time.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SPARSE_SIGN = 2
WORKLOADS = {
    # 20000 x 10000 FP64, sigma_i = 10^(-i/100) + 1e-6 N(0,1) noise; farPCASS zeta = 8, b = 50, P = 1
    "farpcass_20000x10000_exp100_zeta8_b50_P1_eps1e-2": dict(
        matrix="dense20000x10000_exp100", kind=SPARSE_SIGN, zeta=8, p=0.0, b=50, P=1, eps=1e-2, seed=1),
    # 10000 x 5000 FP64, the 20000 x 10000 family at a quarter of the size (profiling)
    "farpcass_10000x5000_exp100_zeta8_b50_P1_eps1e-2": dict(
        matrix="dense10000x5000_exp100", kind=SPARSE_SIGN, zeta=8, p=0.0, b=50, P=1, eps=1e-2, seed=1),
    # 5000 x 5000 FP64, Matrix 1 of Sec. 5 (sigma_j = 1/j^2); farPCASS zeta = 8, b = 50, P = 1;
    # Table 1's eps = 1e-4 (rank 350).  A (200 MB) is larger than L2 yet small enough for
    # full ncu captures.
    "farpcass_5000x5000_matrix1_zeta8_b50_P1_eps1e-4": dict(
        matrix="matrix1_5000", kind=SPARSE_SIGN, zeta=8, p=0.0, b=50, P=1, eps=1e-4, seed=1),
    # 2000 x 1000 FP64, sigma_i = i^-1.5; farPCASS zeta = 8, b = 20, P = 1
    "farpcass_2000x1000_poly1.5_zeta8_b20_P1_eps1e-2": dict(
        matrix="dense2000x1000_poly1.5", kind=SPARSE_SIGN, zeta=8, p=0.0, b=20, P=1, eps=1e-2, seed=1),
}
DEFAULT_WORKLOAD = "farpcass_20000x10000_exp100_zeta8_b50_P1_eps1e-2"
METRIC = "time-to-eps per matrix (fixed-precision farPCA), as solves/s"
FP64_PEAK_TFLOPS = 1.25   # nominal GB300 FP64 (152 SMs x ~2 FP64 FMA/clk x 2 flop x 2.07 GHz)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--sketch-blocks", type=int, default=100,
                    help="blocks of the sketch-only pass (one launch over all of them)")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the timed farPCA steps (for launch-list profiling)")
    ap.add_argument("--engine", choices=("tensor", "fp64_simt"), default="tensor",
                    help="dense passes on the tensor cores (FP64-accurate slicing) or FP64 CUDA cores")
    ap.add_argument("--serve-slots", type=int, default=8,
                    help="with --only serve: requests run at once")
    ap.add_argument("--batch-count", type=int, default=4096,
                    help="with --only batch: number of problems (4096 is the benchmark batch)")
    ap.add_argument("--no-graphs", action="store_true",
                    help="with --only batch: launch the batch's steps from the host (for profiling)")
    ap.add_argument("--only", choices=("sketch", "dense", "serve", "batch", "fixedrank", "stability", "svd",
                                       "runlist", "precision"),
                    default=None,
                    help="run only the sketch pass (lra_sketch over --sketch-blocks blocks) or only "
                         "the two dense passes A Y and A^T Y (lra_apply), for profiling")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def oracle_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n and n[0]:
            return int(n[0])
    except Exception:
        pass
    return os.cpu_count() or 1


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while timing."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(ms, world, device):
    """The timed duration of the slowest rank (all ranks call this after the timed region)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(ms_max, world, steps):
    """Solves per second of the whole job: every rank solves `steps` matrices."""
    return world * steps / (ms_max / 1e3)


def workload_config(args, cfg, m, n, world):
    return {"workload": args.workload, "m": m, "n": n, "b": cfg["b"], "P": cfg["P"], "eps": cfg["eps"],
            "omega": "sparse sign, zeta=%d" % cfg["zeta"],
            "l2": "inputs larger than L2 (A = %.2f GB)" % (8.0 * m * n / 1e9),
            "parallelism": "replicas" if world > 1 else "single GPU"}


def source_digest(names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2506_03859_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_for(kernel, digest, workload):
    """DRAM bytes per launch from the committed ncu summary, if the kernel is unchanged
    and the figure is for this workload."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f).get(kernel)
    except (OSError, ValueError):
        return None
    if not t or t.get("source_digest") != digest or t.get("workload") != workload:
        return None
    return t.get("dram_bytes_per_launch")


def run_reference(args, cfg):
    """The FP64 CPU oracle, as it stands, on the host cores: one full solve per step."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np  # noqa: F401
    from lra_inputs import workload_matrix
    from oracle import farpca as F
    A = workload_matrix(cfg["matrix"])
    kw = dict(P=cfg["P"], b=cfg["b"], kind=cfg["kind"], seed=cfg["seed"], zeta=cfg["zeta"], p=cfg["p"])
    for _ in range(args.warmup):
        F.farpca(A, cfg["eps"], **kw)
    times = []
    r = None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = F.farpca(A, cfg["eps"], **kw)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps / total
    cores = oracle_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(args, cfg, A.shape[0], A.shape[1], 1),
        "result": {"rank": r["rank"], "blocks": r["blocks"], "rel_err": (max(r["E"], 0) / r["normA2"]) ** 0.5,
                   "status": ["LRA_OK", "LRA_NOT_CONVERGED", "LRA_BREAKDOWN"][r["status"]]},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": "one full fixed-precision solve of the workload per step "
                                   "(numpy/OpenBLAS FP64, QB form)"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    cfg = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, cfg)
        return
    import numpy as np
    import torch
    import torch.distributed as dist
    from lra_inputs import workload_matrix
    from paper_2506_03859_gb300 import lra
    from paper_2506_03859_gb300.build import build

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    if local == 0:
        build()
    if world > 1:
        dist.barrier()
    lra.load()
    peaks, peak_src = measured_peaks()

    A = workload_matrix(cfg["matrix"])
    m, n = A.shape
    Ad = lra.column_major(torch.from_numpy(A).cuda())
    stream = torch.cuda.current_stream()
    f = lra.Farpca(m, n, eps=cfg["eps"], b=cfg["b"], P=cfg["P"], kind=cfg["kind"], zeta=cfg["zeta"],
                   p=cfg["p"], seed=cfg["seed"] + rank, profile=True, stream=stream,
                   fp64_simt=(args.engine == "fp64_simt"))
    if args.only in ("sketch", "dense", "serve", "batch", "fixedrank", "stability", "svd", "runlist",
                     "precision"):
        if args.only == "precision":
            out = {"precision_cfg3": precision_workload(lra, torch, np, stream)}
        elif args.only == "runlist":
            out = {"run_list": run_list(lra, torch, np, Ad, peaks, peak_src, stream)}
        elif args.only == "serve":
            out = {"serving": serving(lra, torch, np, slots=args.serve_slots)}
        elif args.only == "svd":
            f.run(Ad)
            out = {"svd": svd_extraction(torch, f, args.steps, stream)}
        elif args.only == "stability":
            out = {"stability": stability(lra, torch)}
        elif args.only == "fixedrank":
            out = {"fixed_rank_sweep": fixed_rank_sweep(lra, torch)}

        elif args.only == "batch":
            out = {"batched": batched(lra, torch, np, peaks, peak_src, count=args.batch_count,
                                      graph=not args.no_graphs)}
        elif args.only == "sketch":
            out = {"sketch_pass": sketch_pass(lra, torch, f, Ad, cfg, args.sketch_blocks, peaks, peak_src)}
        else:
            out = {"dense_pass": dense_pass(lra, torch, f, Ad, cfg, args.steps, args.warmup, peaks, peak_src)}
        if rank == 0:
            print(json.dumps(out), flush=True)
        f.close()
        return
    for _ in range(max(args.warmup, 0)):
        f.run(Ad)
    torch.cuda.synchronize()
    f.phase_times(reset=True)

    sampler = ClockSampler(torch.cuda.current_device())
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    launches0 = lra.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        f.run(Ad)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = lra.kernel_launches() - launches0
    ms = e0.elapsed_time(e1)
    clocks = sampler.stop()
    ms = max_over_ranks(ms, world, "cuda")
    if world > 1:
        dist.barrier()
    res = f.result()
    phases = f.phase_times(reset=True)
    value = whole_job_value(ms, world, args.steps)

    # roofline of the dominant phase: the full passes over A (one lra dense pass = one
    # k_ozgemm launch plus its small prep / fixup kernels)
    dense_ms, dense_calls = phases["dense"]
    dense_avg_ms = dense_ms / max(dense_calls, 1)
    b = cfg["b"]
    algo_bytes = 8.0 * (m * n + (m + n) * b)       # A once, the skinny operand and result
    algo_flops = 2.0 * m * n * b
    if args.engine == "fp64_simt":
        achieved = algo_flops / (dense_avg_ms * 1e-3) / 1e12 if dense_calls else 0.0
        roofline = {"kernel": "k_dgemm (FP64 FMA on the CUDA cores)", "bound": "alu",
                    "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                    "peak_source": "nominal FP64 of the profiling recipe (no measured FP64 peak)"}
    else:
        achieved = algo_bytes / (dense_avg_ms * 1e-3) / 1e9 if dense_calls else 0.0
        pair_flops = 28 * 2.0 * m * n * 64           # bf16 MMA work of the 28 digit pairs (N padded to 64)
        tflops = pair_flops / (dense_avg_ms * 1e-3) / 1e12 if dense_calls else 0.0
        roofline = {"kernel": "k_ozgemm_img (FP64-accurate GEMM on tcgen05 from the f16 digit images of A)",
                    "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"],
                    "traffic": traffic_for("k_ozgemm_img", source_digest(["ozgemm.cu"]), args.workload),
                    "peak_source": peak_src + " HBM copy bandwidth",
                    "tensor_pipe": {"bf16_tflops": tflops, "peak": peaks["bf16_tflops"],
                                    "frac": tflops / peaks["bf16_tflops"],
                                    "note": "28 f16 digit-pair products per FP64 product, N padded to 64"}}
    roofline.update({"algorithmic_per_launch": {"bytes": algo_bytes, "flops_fp64": algo_flops},
                     "avg_launch_ms": dense_avg_ms, "launches": dense_calls,
                     "time_to_eps": solve_roofline(m, n, cfg["b"], cfg["P"], res["blocks"], cfg["kind"],
                                                   cfg["zeta"], ms / args.steps, peaks, peak_src)})
    total_phase = sum(v[0] for v in phases.values()) or 1.0

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, cfg, m, n, world),
        "result": {"rank": res["rank"], "blocks": res["blocks"], "rel_err": res["rel_err"],
                   "status": lra.status_string(res["status"])},
        "roofline": roofline,
        "phase_share": {k: round(v[0] / total_phase, 4) for k, v in phases.items()},
        "phase_ms_per_step": {k: v[0] / args.steps for k, v in phases.items()},
        "gpu_launches": launches,
        "clocks": clocks,
    }

    if not args.no_extras:
        # the headline's own measurements first, before the other workloads use
        # host and device memory
        line["e2e"] = e2e(lra, torch, np, f, A, args.steps)
        line["sketch_pass"] = sketch_pass(lra, torch, f, Ad, cfg, args.sketch_blocks, peaks, peak_src)
        line["run_list"] = run_list(lra, torch, np, Ad, peaks, peak_src, stream)
        line["mixed"] = mixed_form(lra, torch, Ad, cfg, m, n, args.steps, res["rel_err"], stream)
        line["precision_cfg3"] = precision_workload(lra, torch, np, stream)
        line["svd"] = svd_extraction(torch, f, args.steps, stream)
        line["fp32_input"] = fp32_form(lra, torch, Ad, cfg, m, n, args.steps, stream)
        if rank == 0 and world == 1:
            line["cpu_baseline"] = cpu_baseline(A, cfg)
        line["serving"] = serving(lra, torch, np)
        line["batched"] = batched(lra, torch, np, peaks, peak_src)
        line["fixed_rank_sweep"] = fixed_rank_sweep(lra, torch)
    else:
        line["e2e"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)
    f.close()
    if world > 1:
        dist.destroy_process_group()


def solve_bytes(m, n, b, P, blocks, kind, zeta):
    """Algorithmic bytes of one fixed-precision solve (what an FP64 implementation of
    the steps must move through HBM), and the number of full passes over A.

    ||A||_F^2: one pass (8 m n).  Per block j (l = j b columns of Q and rows of B so far):
    the sketch (a gather of the distinct columns of A for the sparse kinds, a full pass
    for the dense ones); with P >= 1 the power step A^T S0 and P - 1 more pairs A G /
    A^T T, each deflated with B (B Omega_j or B G, then B^T F: B read twice) and
    orthonormalised (CholQR2 of an n x b panel: two Grams and two X R^-1); Y_j = A G;
    two projections against Q (Q^T Y and Y - Q F); CholQR2 of the m x b block;
    B_j = Q_j^T A (a full pass); ||B_j||_F^2 and the append of B_j."""
    e = 8.0
    dense_kind = kind in (0, 1)  # Gaussian and standardized Bernoulli: a dense sketch pass
    pass_bytes = e * (m * n + (m + n) * b)
    total, passes = e * m * n, 1
    for j in range(blocks):
        l = j * b
        if dense_kind:
            total += pass_bytes
            passes += 1
        else:
            total += e * m * (min(zeta * b if zeta > 0 else n, n) + b)
        if P >= 1:
            for _ in range(P):
                total += 2 * pass_bytes if _ > 0 else pass_bytes
                passes += 2 if _ > 0 else 1
                if l > 0:
                    total += e * 2 * (l * n + l * b + n * b)
                total += e * 6 * n * b
            total += pass_bytes  # Y_j = A G
            passes += 1
        if l > 0:
            total += 2 * e * ((m * l + m * b + l * b) + (m * l + l * b + 2 * m * b))
        total += e * 6 * m * b
        total += pass_bytes  # B_j = Q_j^T A
        passes += 1
        total += e * 2 * n * b
    return total, passes


def solve_roofline(m, n, b, P, blocks, kind, zeta, ms, peaks, peak_src):
    """Time-to-eps roofline of one solve: its algorithmic bytes (solve_bytes) over the HBM
    copy bandwidth, against the measured time per solve.  The FP64 flops are not a bound
    here: the dense passes run FP64-accurate on the tensor cores (28 bf16 digit-pair
    products per FP64 product, N padded to 64), whose own floor is given beside it."""
    total, passes = solve_bytes(m, n, b, P, blocks, kind, zeta)
    hbm_ms = total / (peaks["hbm_gbs"] * 1e9) * 1e3
    # the full passes of this design: max(image-free HBM time, 28-pair tensor time) each
    pass_hbm = 8.0 * (m * n + (m + n) * b) / (peaks["hbm_gbs"] * 1e9) * 1e3
    pass_tc = 28 * 2.0 * m * n * 64 / (peaks["bf16_tflops"] * 1e12) * 1e3
    design_ms = hbm_ms + (passes - 1) * max(0.0, pass_tc - pass_hbm)
    return {"bound": "hbm", "algorithmic_bytes": total, "full_passes": passes,
            "roofline_ms": hbm_ms, "measured_ms": ms, "frac": hbm_ms / ms,
            "design_floor_ms": design_ms, "frac_of_design_floor": design_ms / ms,
            "peak": peaks["hbm_gbs"], "peak_source": peak_src + " HBM copy bandwidth",
            "note": "design floor: each full pass over A at max(its HBM time, the tensor time of "
                    "its 28 digit-pair products at the bf16 peak)"}


def run_list(lra, torch, np, Ad, peaks, peak_src, stream, reps=3):
    """The measurement runs beside the headline: the 2000 x 1000 workload (sigma_i =
    i^-1.5, b = 20, P = 1, eps = 1e-2) with the four hot-path kinds, and the variants of
    the 20000 x 10000 workload (P in {0, 2}, zeta in {4, 16}, eps in {1e-1, 1e-3} -- the
    latter ends NOT_CONVERGED at the block cap, the noise floor being ~3e-3 -- and the
    Gaussian, standardized Bernoulli +-1 and sparse Gaussian kinds).  Per run: rank,
    blocks, status, final relative error, ms per solve and the time-to-eps roofline."""
    from lra_inputs import workload_matrix
    kinds = {"ss8": (lra.SPARSE_SIGN, 0.0, 8), "gauss": (lra.GAUSSIAN, 0.0, 0),
             "sb_pm1": (lra.STD_BERNOULLI, 0.5, 0), "sg8": (lra.SPARSE_GAUSSIAN, 0.0, 8)}

    def timed(A, m, n, b, P, eps, kind, p, zeta, k_reps):
        f = lra.Farpca(m, n, eps=eps, b=b, P=P, kind=kind, zeta=zeta, p=p, seed=1, stream=stream)
        f.run(A)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k_reps):
            f.run(A)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k_reps
        r = f.result()
        f.close()
        rl = solve_roofline(m, n, b, P, r["blocks"], kind, zeta, ms, peaks, peak_src)
        return {"rank": r["rank"], "blocks": r["blocks"], "status": lra.status_string(r["status"]),
                "rel_err": r["rel_err"], "ms": ms, "solves_per_s": 1e3 / ms,
                "time_to_eps_frac": rl["frac"], "frac_of_design_floor": rl["frac_of_design_floor"]}

    out = {}
    A1 = lra.column_major(torch.from_numpy(workload_matrix("dense2000x1000_poly1.5")).cuda())
    for name, (kind, p, zeta) in kinds.items():
        out["C1_2000x1000_%s_P1_eps1e-2" % name] = timed(A1, 2000, 1000, 20, 1, 1e-2, kind, p, zeta, 10)
    del A1
    m, n = Ad.shape
    c2 = [("ss8_P0_eps1e-2", "ss8", 0, 1e-2), ("ss8_P2_eps1e-2", "ss8", 2, 1e-2),
          ("ss4_P1_eps1e-2", (lra.SPARSE_SIGN, 0.0, 4), 1, 1e-2),
          ("ss16_P1_eps1e-2", (lra.SPARSE_SIGN, 0.0, 16), 1, 1e-2),
          ("ss8_P1_eps1e-1", "ss8", 1, 1e-1), ("gauss_P1_eps1e-2", "gauss", 1, 1e-2),
          ("sb_pm1_P1_eps1e-2", "sb_pm1", 1, 1e-2), ("sg8_P1_eps1e-2", "sg8", 1, 1e-2),
          ("ss8_P1_eps1e-3_capped", "ss8", 1, 1e-3)]
    for name, kd, P, eps in c2:
        kind, p, zeta = kinds[kd] if isinstance(kd, str) else kd
        out["C2_20000x10000_%s" % name] = timed(Ad, m, n, 50, P, eps, kind, p, zeta,
                                               1 if eps < 1e-2 else reps)
    return out


def precision_workload(lra, torch, np, stream, m=60000, n=20000, rank=11000, oracle_blocks=2):
    """The precision workload: 60000 x 20000 FP64, sigma_i = i^-1 on rank 11000 (built in
    FP32 on the device), b = 64, P = 1, eps = 1e-3, the standardized Bernoulli +-1 sketch
    (and the sparse sign sketch, zeta = 8, beside it).  eps is out of reach within the cap
    ceil(n / 2b) = 157 blocks (rank 10048), so every run ends NOT_CONVERGED at the cap:
    reported are the time to the cap and the final error of the FP64-accurate form and of
    the mixed precision form (LRA_FLAG_MIXED), and, against the FP64 CPU oracle at an equal
    block count (`oracle_blocks` blocks, the oracle's cost bound), the indicator and final
    error of both forms."""
    import math
    from lra_inputs import device_low_rank
    from oracle import farpca as F
    A = device_low_rank(m, n, rank, 4242, dtype=torch.float64, spectrum="poly1", build_dtype=torch.float32)
    torch.cuda.synchronize()
    out = {"workload": "precision_%dx%d_poly1_rank%d_b64_P1_eps1e-3" % (m, n, rank)}
    kinds = {"sb_pm1": (lra.STD_BERNOULLI, 0.5, 0), "ss8": (lra.SPARSE_SIGN, 0.0, 8)}
    for kname, (kind, p, zeta) in kinds.items():
        for mixed in (False, True):
            f = lra.Farpca(m, n, eps=1e-3, b=64, P=1, kind=kind, zeta=zeta, p=p, seed=5, mixed=mixed,
                           stream=stream)
            f.run(A)   # warm-up (captures the block graphs)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = f.run(A)
            e1.record(stream)
            torch.cuda.synchronize()
            r = f.result()
            out["%s_%s" % (kname, "mixed" if mixed else "fp64")] = {
                "ms_to_cap": e0.elapsed_time(e1), "status": lra.status_string(st), "rank": r["rank"],
                "blocks": r["blocks"], "rel_err": r["rel_err"]}
            f.close()
    # against the oracle at an equal block count (standardized Bernoulli +-1)
    Ah = A.cpu().numpy()
    t0 = time.perf_counter()
    ref = F.farpca(Ah, 1e-3, P=1, b=64, kind=lra.STD_BERNOULLI, seed=5, p=0.5, max_blocks=oracle_blocks)
    t_oracle = time.perf_counter() - t0
    cmp = {}
    for mixed in (False, True):
        f = lra.Farpca(m, n, eps=1e-3, b=64, P=1, kind=lra.STD_BERNOULLI, p=0.5, seed=5, mixed=mixed,
                       max_blocks=oracle_blocks, stream=stream)
        f.run(A)
        r = f.result()
        rel, rel_ref = (math.sqrt(max(x, 0.0) / ref["normA2"]) for x in (r["E"], ref["E"]))
        cmp["mixed" if mixed else "fp64"] = {
            "rank": r["rank"], "rank_oracle": ref["rank"], "dE_over_normA2": abs(r["E"] - ref["E"]) / ref["normA2"],
            "rel_err": rel, "rel_err_oracle": rel_ref, "rel_err_dev": abs(rel - rel_ref) / rel_ref}
        f.close()
    out["vs_oracle"] = dict(cmp, blocks=oracle_blocks, oracle_seconds=t_oracle, cores=oracle_threads())
    del A, Ah
    return out


def sketch_pass(lra, torch, f, Ad, cfg, nblk, peaks, peak_src):
    """lra_sketch over nblk consecutive blocks (one launch of the gather kernel)."""
    m, n, b = f.m, f.n, f.b
    Y = torch.empty_strided((m, nblk * b), (1, m), dtype=torch.float64, device="cuda")
    distinct = 0
    for j in range(nblk):
        counts, rows, _ = f.copy_omega(j)
        distinct += len(set(rows[:, :cfg["zeta"]].ravel().tolist()))
    algo_bytes = 8.0 * m * (distinct + nblk * b)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        f.sketch(Ad, 0, nblk, Y)
    torch.cuda.synchronize()
    reps = 5
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for r in range(reps):
        f.sketch(Ad, r * nblk, nblk, Y)   # a different Omega each repetition
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    gbs = algo_bytes / (ms * 1e-3) / 1e9
    return {"kernel": "k_gather_staged (sparse-sign sketch, Omega generated in the same call)",
            "blocks": nblk, "ms": ms, "algorithmic_bytes": algo_bytes, "gbs": gbs,
            "bound": "hbm", "peak": peaks["hbm_gbs"], "frac": gbs / peaks["hbm_gbs"],
            "frac_of_nominal_7900": gbs / 7900.0, "peak_source": peak_src}


def mixed_form(lra, torch, Ad, cfg, m, n, steps, rel_err_fp64, stream):
    """The mixed precision form (LRA_FLAG_MIXED) on the same workload: time-to-eps as
    solves/s and its final relative error beside the FP64 form's."""
    f = lra.Farpca(m, n, eps=cfg["eps"], b=cfg["b"], P=cfg["P"], kind=cfg["kind"], zeta=cfg["zeta"],
                   p=cfg["p"], seed=cfg["seed"], mixed=True, stream=stream)
    for _ in range(2):
        f.run(Ad)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        f.run(Ad)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    r = f.result()
    f.close()
    return {"value": 1e3 / ms, "unit": "solves/s", "ms_per_step": ms, "rank": r["rank"],
            "rel_err": r["rel_err"], "rel_err_fp64_form": rel_err_fp64,
            "note": "sketch and power passes from 4 of the 7 digits; B_j, projections, "
                    "Gram, Cholesky and indicator FP64-accurate"}


SERVE_KINDS = ((0, 0.0, 0), (1, 0.5, 0), (2, 0.0, 8), (4, 0.0, 8))   # Gaussian, SB +-1, SS zeta=8, SG 8/n


def serve_block(m, n):
    """Sec. 5.4's block size rule: b = min(max(20, floor(min(m, n) / 100)), 50)."""
    return min(max(20, min(m, n) // 100), 50)


def serving(lra, torch, np, duration_s=3.0, rate=200.0, slots=8, seed=11, pool_size=24):
    """Served solves/s and p50/p99 latency: a Poisson stream (mean `rate` req/s) of
    FP32 requests, sizes log-uniform 1000x500 .. 40000x20000 (a pool of `pool_size`
    device-resident matrices of seeded log-uniform sizes, n = m/2, exact rank 400,
    sigma_i = 10^(-i/100)), mixed Omega kinds and eps in {1e-1, 1e-2, 1e-3}.

    Three arms on the same trace, every latency measured (completion time minus
    arrival time on the host clock):
      * served, mixed precision form (LRA_FLAG_MIXED): lra_server, `slots` at once;
      * served, FP64-accurate form: the same server without the flag;
      * plain FP64 one at a time: the trace replayed in real time by one host loop
        that waits for each arrival, then runs the request alone (a context from the
        same stream-ordered pool as the server's, LRA_FLAG_POOL) and waits for it."""
    from lra_inputs import device_low_rank
    rng = np.random.default_rng(seed)
    sizes = sorted(int(round(v)) for v in np.exp(rng.uniform(np.log(1000), np.log(40000), pool_size)))
    sizes[0], sizes[-1] = 1000, 40000   # both ends of the range are in the pool
    pool = [device_low_rank(mm, mm // 2, min(400, mm // 2), 500 + i) for i, mm in enumerate(sizes)]
    trace, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration_s:
            break
        k = int(rng.integers(len(sizes)))
        kind, p, zeta = SERVE_KINDS[int(rng.integers(len(SERVE_KINDS)))]
        eps = [1e-1, 1e-2, 1e-3][int(rng.integers(3))]
        mm, nn = pool[k].shape
        prm = lra.params(eps=eps, b=serve_block(mm, nn), P=1, kind=kind, zeta=zeta, p=p,
                         seed=int(rng.integers(1 << 62)))
        trace.append((t, k, prm))

    def served(flags):
        torch.cuda.synchronize()
        srv = lra.Server(slots=slots, flags=flags)
        t0 = srv.clock()
        done = []
        for i, (ta, k, prm) in enumerate(trace):
            while srv.clock() - t0 < ta:
                done += srv.poll()
                time.sleep(0.0002)
            srv.submit(pool[k], prm, i)
        while len(done) < len(trace):
            done += srv.poll(wait=True)
        srv.close()
        lat = np.array([c["t_done"] - c["t_submit"] for c in done])
        span = max(c["t_done"] for c in done) - min(c["t_submit"] for c in done)
        ok = sum(1 for c in done if c["status"] >= 0)
        return {"solves_per_s": len(trace) / span, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)), "completed_ok": ok,
                "mean_rel_err": float(np.mean([c["rel_err"] for c in done]))}

    mixed = served(lra.FLAG_NO_GRAPHS | lra.FLAG_MIXED)
    fp64_served = served(lra.FLAG_NO_GRAPHS)
    # the same trace, plain FP64, one request at a time, replayed in real time
    pool64 = []
    for A in pool:
        B = torch.empty_strided(A.shape, (1, A.shape[0]), dtype=torch.float64, device="cuda")
        B.copy_(A)
        pool64.append(B)
    torch.cuda.synchronize()
    lat1 = []
    t0 = time.perf_counter()
    for ta, k, prm in trace:
        now = time.perf_counter() - t0
        if now < ta:
            time.sleep(ta - now)
        mm, nn = pool64[k].shape
        f = lra.Farpca(mm, nn, eps=prm.eps, b=prm.b, P=prm.P, kind=prm.kind, zeta=prm.zeta, p=prm.p,
                       seed=prm.seed, pool=True, graphs=False)
        f.run(pool64[k])
        f.close()
        torch.cuda.synchronize()
        lat1.append(time.perf_counter() - t0 - ta)
    span1 = time.perf_counter() - t0 - trace[0][0]
    lat1 = np.array(lat1)
    del pool64, pool
    return {"requests": len(trace), "rate_req_s": rate, "slots": slots,
            "solves_per_s": mixed["solves_per_s"], "p50_ms": mixed["p50_ms"], "p99_ms": mixed["p99_ms"],
            "form": "mixed precision (LRA_FLAG_MIXED)", "completed_ok": mixed["completed_ok"],
            "served_mixed": mixed, "served_fp64": fp64_served,
            "one_at_a_time_fp64": {"solves_per_s": len(trace) / span1,
                                   "p50_ms": 1e3 * float(np.percentile(lat1, 50)),
                                   "p99_ms": 1e3 * float(np.percentile(lat1, 99)),
                                   "allocation": "stream-ordered pool (LRA_FLAG_POOL)",
                                   "latency": "measured (real-time replay of the trace)"},
            "sizes": "log-uniform %dx%d .. %dx%d (%d matrices)" % (sizes[0], sizes[0] // 2, sizes[-1],
                                                                 sizes[-1] // 2, len(sizes))}


def batched(lra, torch, np, peaks, peak_src, count=4096, reps=3, graph=True):
    """The batched form: `count` FP32 problems, rows uniform 64..2048, columns
    uniform 32..1024 (sigma_i = i^-2, rank <= 64, plus noise 1e-3), eps alternating
    1e-1 / 1e-2, fixed-zeta sparse sign zeta = 4, b = 16, P = 1, run by one graph
    launch.  Roofline: the bytes of A each problem's passes must read (one pass for
    ||A||^2, then per block A^T X, A G, Q_j^T A, and the gathered columns of the
    sketch), over the batch time, against the HBM copy bandwidth."""
    from lra_inputs import batch_matrix, batch_shapes
    shapes = batch_shapes(count, 11)
    mats = [batch_matrix(m, n, 1000 + k) for k, (m, n) in enumerate(shapes)]
    eps = [1e-1 if k % 2 else 1e-2 for k in range(count)]
    seeds = [8000 + k for k in range(count)]
    bt = lra.Batch(mats, eps, seeds, b=16, P=1, zeta=4, graph=graph)
    bt.run()
    torch.cuda.synchronize()
    # the autotuner picks the tile shape of each shape class on this batch
    tuned = bt.tune(reps=2) if graph else None
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        bt.run()
        times.append(time.perf_counter() - t0)
    t = min(times)
    res = [bt.result(k) for k in range(count)]
    blocks = [r["rank"] // 16 for r in res]
    algo = sum(4.0 * m * n * (1 + 3 * nb) + 4.0 * m * 16 * 4 * nb for (m, n), nb in zip(shapes, blocks))
    gbs = algo / t / 1e9
    ok = sum(1 for r in res if r["status"] == lra.OK)
    out = {"problems": count, "ms": 1e3 * t, "problems_per_s": count / t, "steps": bt.steps(),
           "converged": ok, "mean_rank": float(np.mean([r["rank"] for r in res])),
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": gbs / peaks["hbm_gbs"], "algorithmic_bytes": algo,
                        "peak_source": peak_src},
           "device_bytes": bt.device_bytes(), "timing": "wall clock of lra_batch_run (min of %d)" % reps,
           "tiling": {"chosen": tuned and {"tn": tuned["tn"], "nn": tuned["nn"]},
                      "tuned_ms": tuned and tuned["ms"], "default_ms": tuned and tuned["base_ms"],
                      "classes": "tn by n: <256, <640, rest; nn by m: <384, <1200, rest (columns / rows "
                                 "per thread, 64 threads per tile)"}}
    bt.close()
    del mats
    return out


def fixed_rank_sweep(lra, torch, reps=3):
    """Sec. 5.1's fixed-rank comparison on the 5000 x 5000 Matrix 1 (sigma_i = i^-2):
    k = 10 b with b = 20 (ten blocks), P in {0, 1}, every Omega kind with the
    paper's p (p1 for the standardized Bernoulli kind, p2 for the others; fixed
    zeta = 8 for the sparse sign kind); ms per solve and the ratio to the Gaussian
    kind (Remark 3.4 expects (2P + 1) / (2P + 2) passes over A: 0.5 at P = 0, 0.75
    at P = 1, for the kinds whose sketch is a gather)."""
    from lra_inputs import workload_matrix
    A = workload_matrix("matrix1_5000")
    m, n = A.shape
    Ad = lra.column_major(torch.from_numpy(A).cuda())
    kinds = {"gaussian": (lra.GAUSSIAN, 0.0, 0), "std_bernoulli": (lra.STD_BERNOULLI, 0.0, 0),
             "sparse_sign_zeta8": (lra.SPARSE_SIGN, 0.0, 8), "sparse_gaussian": (lra.SPARSE_GAUSSIAN, 0.0, 0),
             "bernoulli": (lra.BERNOULLI, 0.0, 0)}
    out = {}
    for P in (0, 1):
        row = {}
        for name, (kind, p, zeta) in kinds.items():
            f = lra.Farpca(m, n, k=200, b=20, P=P, kind=kind, zeta=zeta, p=p, seed=3)
            f.run(Ad)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                f.run(Ad)
            torch.cuda.synchronize()
            row[name] = 1e3 * (time.perf_counter() - t0) / reps
            f.close()
        g = row["gaussian"]
        out["P%d" % P] = {k: {"ms": v, "ratio_to_gaussian": v / g} for k, v in row.items()}
    del Ad
    return out


def table4():
    """Table 4 (Sec. 5.5) as printed: algorithm -> p -> (d1, d2, d3) success counts."""
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", "table4_n5000.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                alg, p, d1, d2, d3 = line.split()
                out.setdefault(alg, {})[p] = (int(d1), int(d2), int(d3))
    return out


def stability(lra, torch, sims=100, n=5000):
    """Sec. 5.5: Matrix 1 with a block-diagonal V_A of d in {1, 500, 5000} blocks;
    the standardized Bernoulli, i.i.d. sparse sign, sparse Gaussian and Bernoulli
    kinds at p in {ln(n)/n, 2e-3, 1e-2}; eps = 1e-4, b = 50, P = 1, the cap
    ceil(n / (2b)) blocks; a simulation succeeds when the run ends with LRA_OK.
    Success rates in `sims` simulations (seeds) beside the paper's Table 4."""
    import math
    from lra_inputs import stability_matrix
    kinds = {"farPCASB": lra.STD_BERNOULLI, "farPCASS": lra.SPARSE_SIGN_IID,
             "farPCASG": lra.SPARSE_GAUSSIAN, "farPCAB": lra.BERNOULLI}
    ps = {"ln(n)/n": math.log(n) / n, "2e-3": 2e-3, "1e-2": 1e-2}
    paper = table4()
    out = {}
    t0 = time.perf_counter()
    for di, d in enumerate((1, 500, 5000)):
        A = stability_matrix(n, d, 77 + d)
        for kname, kind in kinds.items():
            for pname, p in ps.items():
                ok = 0
                for s in range(sims):
                    f = lra.Farpca(n, n, eps=1e-4, b=50, P=1, kind=kind, p=p, seed=10000 + s)
                    ok += f.run(A) == lra.OK
                    f.close()
                out.setdefault(kname, {}).setdefault(pname, {})["d%d" % (di + 1)] = {
                    "success": ok, "paper": paper[kname][pname][di]}
        del A
    return {"simulations": sims, "n": n, "rates": out, "seconds": time.perf_counter() - t0}


def fp32_form(lra, torch, Ad, cfg, m, n, steps, stream):
    """Time-to-eps on the FP32 rounding of the same matrix (FP32 input A: the cut,
    the statistics pass and the gather read 4-byte entries; every sum is FP64)."""
    A32 = torch.empty_strided((m, n), (1, m), dtype=torch.float32, device="cuda")
    A32.copy_(Ad)
    f = lra.Farpca(m, n, eps=cfg["eps"], b=cfg["b"], P=cfg["P"], kind=cfg["kind"], zeta=cfg["zeta"],
                   p=cfg["p"], seed=cfg["seed"], stream=stream)
    for _ in range(2):
        f.run(A32)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        f.run(A32)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    r = f.result()
    f.close()
    del A32
    return {"value": 1e3 / ms, "unit": "solves/s", "ms_per_step": ms, "rank": r["rank"],
            "rel_err": r["rel_err"], "bytes_of_A": 4 * m * n}


def svd_extraction(torch, f, steps, stream):
    """lra_svd after the timed runs: the SVD the method returns (Gram B B^T, Jacobi
    eigendecomposition, U = Q Vt, V = B^T Vt sigma^-1) and the truncated rank."""
    sv = f.svd()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(steps, 1)
    e0.record(stream)
    for _ in range(reps):
        sv = f.svd()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return {"ms": ms, "l": sv["l"], "r": sv["r"], "sweeps": sv["sweeps"],
            "rel_err_r": (max(sv["E_r"], 0.0) / sv["normA2"]) ** 0.5 if sv["normA2"] > 0 else 0.0,
            "note": "includes two host synchronisations (sweep count, sigma for the truncation)"}


def dense_pass(lra, torch, f, Ad, cfg, steps, warmup, peaks, peak_src):
    """lra_apply with N = b: C = A Y and C = A^T Y, each timed alone (row exponents of A,
    the cut of Y, the tensor-core pass and its fixup)."""
    m, n, b = f.m, f.n, f.b
    g = torch.Generator(device="cuda").manual_seed(7)
    out = {}
    for trans in (False, True):
        rows_y = m if trans else n
        Y = torch.randn((b, rows_y), generator=g, dtype=torch.float64, device="cuda").t()
        for _ in range(max(warmup, 1)):
            C = f.apply(Ad, Y, trans=trans)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(steps, 1)
        e0.record(stream)
        for _ in range(reps):
            f.apply(Ad, Y, trans=trans, C=C)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        algo_bytes = 8.0 * (m * n + (m + n) * b)
        out["AT_Y" if trans else "A_Y"] = {"ms": ms, "gbs": algo_bytes / (ms * 1e-3) / 1e9,
                                           "frac": algo_bytes / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"]}
    out.update({"peak_gbs": peaks["hbm_gbs"], "peak_source": peak_src,
                "note": "each includes one exponent pass over A (lra_apply recomputes them)"})
    return out


def e2e(lra, torch, np, f, A, steps):
    """Through host buffers: every step copies its A (1.6 GB) from pinned host memory
    and reads Q and B back into pinned host memory.  The headline form solves a
    stream of matrices with lra_farpca_host_prefetch (two distinct pinned host
    matrices of the workload, alternating): each step's copy to the device runs
    while the previous step is solved, all copies inside the timed region.  Beside
    it, lra_farpca_host one call at a time (copy, solve, read back, in turn)."""
    m, n = A.shape
    cap = f.capacity
    hosts = []
    for _ in range(2):
        Ah = torch.empty((n, m), dtype=torch.float64, pin_memory=True).numpy().T
        Ah[...] = A
        hosts.append(Ah)
    Qh = torch.empty((cap, m), dtype=torch.float64, pin_memory=True).numpy().T
    Bh = torch.empty((n, cap), dtype=torch.float64, pin_memory=True).numpy().T
    k = max(3, min(steps, 5))
    # one call at a time
    f.run_host(hosts[0], Qh, Bh)
    t0 = time.perf_counter()
    r = None
    for _ in range(k):
        r = f.run_host(hosts[0], Qh, Bh)
    serial = (time.perf_counter() - t0) / k
    # a stream: the first call copies its own A and prefetches the next one
    f.run_host(hosts[0], Qh, Bh, next_A=hosts[1])
    f.run_host(hosts[1], Qh, Bh, next_A=hosts[0])
    t0 = time.perf_counter()
    for i in range(k):
        r = f.run_host(hosts[i % 2], Qh, Bh, next_A=hosts[(i + 1) % 2])
    dt = (time.perf_counter() - t0) / k
    rank = r["rank"]
    return {"value": 1.0 / dt, "unit": "solves/s", "h2d_bytes_per_step": 8 * m * n,
            "d2h_bytes_per_step": 8 * (m * rank + rank * n), "ms_per_step": 1e3 * dt,
            "api": "lra_farpca_host_prefetch (a stream of two pinned host matrices; each step's "
                   "copy overlaps the previous step's solve)",
            "serial": {"value": 1.0 / serial, "ms_per_step": 1e3 * serial, "api": "lra_farpca_host"}}


def cpu_baseline(A, cfg):
    from oracle import farpca as F
    t0 = time.perf_counter()
    r = F.farpca(A, cfg["eps"], P=cfg["P"], b=cfg["b"], kind=cfg["kind"], seed=cfg["seed"],
                 zeta=cfg["zeta"], p=cfg["p"])
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": "solves/s", "cores": oracle_threads(), "kind": "oracle",
            "sample": "one full fixed-precision solve of the same workload (rank %d, numpy/OpenBLAS "
                      "FP64, QB form)" % r["rank"], "seconds": dt}


if __name__ == "__main__":
    main()
