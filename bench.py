"""Benchmark: LM bundle-adjustment iterations/s on the 1M-observation scene.

Workload: 200 cameras, 100k points, ~1M observations (track length 3-20,
truncated geometric, mean 10), FP32 hot path with the cost in double-float
arithmetic (FP32 pairs; 1e-12 relative to FP64), the gain ratio in FP64 and the
PCG dots in FP64 (implicit system) or compensated double-float sums of FP64-level
accuracy (explicit system); 2% outliers, depth priors on 50% of observations.  A step is one
full LM iteration (extraction, residuals/Jacobians, normal equations and
Schur terms, PCG + back-substitution, candidate evaluation and accept/reject).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --workload dense --solver dense|implicit   (other scenes, same line)
  python bench.py --dense-kernels                            (tensor-core GEMM and Cholesky)

Prints one JSON line.  With N > 1 (torchrun) every rank solves its own replica
on its own GPU ("replicas only": the solve does not shard across GPUs) and the
time is the maximum over ranks.  --impl reference times the CPU oracle on the
same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2510_13310_b300 import scenes  # noqa: E402

METRIC = "BA LM iters/s & Jacobian+Schur Gobs/s at 1M obs; time-to-RMSE vs FP64 GPU"

# DRAM bytes (read + write) of one launch of a roofline kernel on a workload, from
# ncu captures (profiles/k_spcg_medium_1M_obs.md,
# profiles/k_form_S_runs_medium_1M_obs.md,
# profiles/k_form_S_cam_dense_mid_1M_obs.md); absent once the kernel has changed
# since the counters were taken, or for workloads not captured.
NCU_TRAFFIC = {("medium", "k_spcg"): 13154816 + 26368, ("medium", "k_form_S_runs"): 302387200 + 8206336,
               ("medium", "k_form_S_rec"): 170823424 + 7443968,
               ("dense_mid", "k_form_S_cam"): 367535616 + 51516160}
# the measured limiter of a kernel whose roofline bound (ALU) is not what stops it:
# ncu counters of one launch on the workload (profiles/<kernel>_<workload>...md)
NCU_LIMITER = {("medium", "k_spcg"): {
    "counter": "gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed", "value_pct": 0.72,
    "issue_active_pct": 40.4, "l1tex_throughput_pct": 39.3, "warps_active_pct": 25.1,
    "reading": "latency-bound: S^ is read from HBM once per launch and then from shared memory; each PCG "
               "iteration is a shared-memory matvec of 12-13 rows per block and one all-gather of q through "
               "tagged words in L2 (about a third of the iteration waiting for the slowest block's words)",
    "source": "profiles/k_spcg_medium_1M_obs.md"},
    ("medium", "k_form_S_runs"): {
    "counter": "l1tex__throughput.avg.pct_of_peak_sustained_active", "value_pct": 93.9,
    "long_scoreboard_cycles_per_issue": 8.0, "warp_cycles_per_issue": 9.92,
    "reading": "the L1TEX pipe moving the scattered 112-byte Y^ row gathers (two per co-visible pair) is "
               "the limiter, not the FP32 pipe",
    "source": "profiles/k_form_S_runs_medium_1M_obs.md"},
    ("medium", "k_form_S_rec"): {
    "counter": "smsp__average_warps_issue_stalled_long_scoreboard_per_issue_active.ratio", "value": 4.53,
    "warp_cycles_per_issue": 7.20, "issue_active_pct": 40.6, "fma_pipe_pct": 32.8, "l1tex_throughput_pct": 76.1,
    "reading": "the warps wait on the scattered record gathers (three 32-byte-aligned records per pair, 12 "
               "resident warps per SM at 168 registers); the FP32 pipe is a third busy. Staging the gathers "
               "through shared memory (cp.async or per-record cp.async.bulk rings) measured slower",
    "source": "profiles/k_form_S_rec_medium_1M_obs.md"}}
WORKLOAD = "medium"
LM_ITERS = 30
E2E_RUNS = 3


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def build_scene(workload=WORKLOAD):
    return scenes.make_scene(workload)


def max_over_ranks(x, dist, device):
    """The largest of the ranks' values (the slowest replica's time); x itself
    without a process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, steps, max_ms):
    """Whole-job LM iterations per second: every replica runs `steps` iterations, the
    job takes as long as the slowest replica."""
    return world * steps / (max_ms / 1e3)


def _covis_pairs(scene):
    """Flags over the C x C camera pairs (i < j) that share at least one point."""
    C = scene.spec.n_cams
    order = np.argsort(scene.obs_pt, kind="stable")
    cams, pts = scene.obs_cam[order].astype(np.int64), scene.obs_pt[order]
    off = np.searchsorted(pts, np.arange(scene.spec.n_pts + 1))
    flags = np.zeros(C * C, bool)
    lens = np.diff(off)
    for L in np.unique(lens):
        rows = np.flatnonzero(lens == L)
        if L < 2:
            continue
        tr = cams[(off[rows][:, None] + np.arange(L)[None, :])]
        iu, ju = np.triu_indices(L, 1)
        a, b = np.minimum(tr[:, iu], tr[:, ju]), np.maximum(tr[:, iu], tr[:, ju])
        flags[(a * C + b).ravel()] = True
    return flags


def _workload_name(scene):
    sp = scene.spec
    return "%s scene: %d cams, %d pts, %d obs" % (sp.name, sp.n_cams, sp.n_pts, scene.n_obs)


def _tf32_peak():
    """Dense TF32 tensor peak: the measured BF16 burst peak times the nominal
    TF32/BF16 ratio (1.1 / 2.25 PFLOP/s)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]) * 1.1 / 2.25, "measured bf16 x nominal tf32/bf16"
    return 1800.0 * 1.1 / 2.25, "fallback bf16 x nominal tf32/bf16"


def run_dense_kernels():
    """Times the tensor-core kernels on their own: C -= A B^T (TF32, FP32
    accumulation) and the blocked Cholesky of an SPD matrix of the dense
    workload's order (17,991), with CUDA events after warm-up."""
    import torch
    from paper_2510_13310_b300 import ba
    dev = torch.device("cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timeit(f, reps):
        f()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0.record()
            f()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    peak, src = _tf32_peak()
    g = torch.Generator(device="cpu").manual_seed(0)
    out = {"metric": "tensor-core dense kernels", "peak_tf32_tflops": peak, "peak_source": src, "gemm": []}
    for (M, N, K) in [(8192, 8192, 8192), (16384, 16384, 1024)]:
        A = torch.randn(M, K, generator=g).to(dev)
        B = torch.randn(N, K, generator=g).to(dev)
        C = torch.zeros(M, N, device=dev)
        ms = timeit(lambda: ba.tc_gemm_nt(A, B, C, alpha=-1.0, beta=1.0), 10)
        tf = 2.0 * M * N * K / (ms * 1e-3) / 1e12
        out["gemm"].append({"M": M, "N": N, "K": K, "ms": ms, "tflops": tf, "frac": tf / peak})
        del A, B, C
    n = 17991
    X = torch.randn(n, n + 64, generator=g).to(dev) / (n ** 0.5)
    S = X @ X.T + 0.1 * torch.eye(n, device=dev)
    d = S.diagonal().sqrt()
    S = S / d[:, None] / d[None, :]
    del X
    ms = timeit(lambda: ba.dense_cholesky(S), 3)
    out["cholesky"] = {"n": n, "ms_incl_copies": ms, "tflops": n ** 3 / 3.0 / (ms * 1e-3) / 1e12}
    print(json.dumps(out), flush=True)
    return 0


def gp_oracle_cpu_baseline(sc, max_seconds=10.0, max_iters=8):
    """The FP64 CPU oracle of global positioning (test infrastructure) on a bounded
    sample of the same scene: LM iterations until max_seconds of work or max_iters
    (at least one), one iteration per call with the state carried over."""
    import oracle
    ob = oracle.OracleGP.from_scene(sc)
    t, X, s = sc.centres0.copy(), sc.pts0.copy(), sc.scales0.copy()
    done, t_tot = 0, 0.0
    while done < max_iters and t_tot < max_seconds:
        t0 = time.perf_counter()
        t, X, s, _ = ob.lm(t, X, s, 1)
        t_tot += time.perf_counter() - t0
        done += 1
    return {"value": done / t_tot, "unit": "LM iters/s", "cores": oracle.get_threads(), "kind": "oracle",
            "sample": f"{done} LM iteration(s) of the global-positioning scene (FP64, dense Cholesky of the "
                      f"centre system), {t_tot:.1f} s"}


def run_gp_measure(torch, ba, dev, stream, steps=8, warmup=3, cpu=True):
    """Depth-constrained global positioning on the same geometry (200 cameras, 100k
    points, ~1M observations, rays with 0.5 px angular noise, 2% outliers, metric
    range priors on 50%): LM iterations/s over `steps` timed iterations (CUDA
    events, L2 flushed between steps) and per-phase device times.  The dominant
    phase's roofline: the point-side linearisation streams per observation the ray
    (16 B), the camera centre (16 B, L2), the scale (4 B) and writes its 80 B
    record and 48 B Schur factor; per point 16 B in and 64 B out."""
    sc = scenes.make_gp_scene(WORKLOAD)
    prob = ba.GPProblem.from_scene(sc, stream=stream.cuda_stream)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    for _ in range(warmup):
        prob.lm_step()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms, infos = [], []
    for _ in range(steps):
        flush.zero_()
        ev0.record(stream)
        infos.append(prob.lm_step())
        ev1.record(stream)
        ev1.synchronize()
        ms.append(ev0.elapsed_time(ev1))
    N, P = sc.n_obs, sc.spec.n_pts
    lin_ms = statistics.median(i["ms"][0] for i in infos)
    hbm, kind = _peaks()
    lin_bytes = N * (16 + 16 + 4 + 80 + 48) + P * (16 + 64)
    out = {"metric": "GP LM iters/s", "value": steps / (sum(ms) / 1e3), "unit": "LM iters/s",
           "ms_per_step": statistics.mean(ms), "workload": _workload_name(sc) + " (global positioning)",
           "n_free_scales": int(infos[0]["n_obs_act"]), "cg_iters": [i["pcg_iters"] for i in infos],
           "phase_ms_median": {"linearize (point pass + camera chunks)": lin_ms,
                               "Schur diagonal + S formation": statistics.median(i["ms"][1] for i in infos),
                               "centre-system solve (block-Jacobi PCG)": statistics.median(i["ms"][2] for i in infos),
                               "back-substitution + candidate + cost": statistics.median(i["ms"][3] for i in infos)},
           "final_cost": infos[-1]["cost"], "gpu_launches": prob.kernel_launches,
           "roofline_linearize": {"bound": "hbm", "achieved": lin_bytes / (lin_ms * 1e-3) / 1e9, "peak": hbm,
                                  "unit": "GB/s", "frac": lin_bytes / (lin_ms * 1e-3) / 1e9 / hbm,
                                  "peak_source": kind + " (burst copy)",
                                  "formula": "164 B x obs + 80 B x points"}}
    prob.close()
    if cpu:
        out["cpu_baseline"] = gp_oracle_cpu_baseline(sc)
    return out


def _oracle_for(scene):
    """The oracle as it stands: its dense Cholesky of the Schur system, or, above
    500 cameras (an order of 4,500 and more, where one FP64 factorisation on the
    host takes minutes), its block-Jacobi PCG with the library's stopping rule."""
    import oracle
    big = scene.spec.n_cams > 500
    return oracle.OracleBA.from_scene(scene, oracle.OracleOptions(solver=1) if big else None), \
        ("PCG of the Schur system" if big else "dense Cholesky of the Schur system")


def oracle_cpu_baseline(scene, max_seconds=20.0, max_iters=30):
    """The FP64 CPU oracle (test infrastructure) on a bounded sample: LM iterations
    of the same scene until max_seconds of work or max_iters (at least one)."""
    import oracle
    ob, how = _oracle_for(scene)
    cams, pts = scene.cams0.copy(), scene.pts0.copy()
    done, t_tot = 0, 0.0
    alive = np.ones(scene.n_obs, np.uint8)
    # one iteration per call keeps the loop bounded; the state carries over
    lam_state = None
    while done < max_iters and t_tot < max_seconds:
        t0 = time.perf_counter()
        cams, pts, rows = ob.lm(cams, pts, 1, alive=alive)
        t_tot += time.perf_counter() - t0
        done += 1
        lam_state = rows[-1]["lam"] if rows else lam_state
    # the same oracle on one host thread: one iteration (bounded)
    cores = oracle.get_threads()
    oracle.set_threads(1)
    t0 = time.perf_counter()
    ob.lm(cams, pts, 1, alive=alive)
    t1 = time.perf_counter() - t0
    oracle.set_threads(cores)
    return {"value": done / t_tot, "unit": "LM iters/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{done} LM iteration(s) of the {_workload_name(scene)} (FP64, {how}), {t_tot:.1f} s",
            "one_thread": {"value": 1.0 / t1, "unit": "LM iters/s", "sample": "1 LM iteration, 1 thread"}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    scene = build_scene(args.workload)
    import oracle
    ob, how = _oracle_for(scene)
    cams, pts = scene.cams0.copy(), scene.pts0.copy()
    alive = np.ones(scene.n_obs, np.uint8)
    # W warm-up iterations, then K timed iterations, one oracle LM iteration per step
    for _ in range(args.warmup):
        cams, pts, _ = ob.lm(cams, pts, 1, alive=alive)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        cams, pts, _ = ob.lm(cams, pts, 1, alive=alive)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "LM iters/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": _workload_name(scene),
                       "n_cams": scene.spec.n_cams, "n_pts": scene.spec.n_pts,
                       "n_obs": scene.n_obs},
            "cpu_baseline": {"value": value, "unit": "LM iters/s", "cores": oracle.get_threads(),
                             "kind": "oracle",
                             "sample": f"{args.steps} timed LM iterations of the full scene after "
                                       f"{args.warmup} warm-up iterations (FP64, {how})"},
            "e2e": {"value": value, "unit": "LM iters/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=27)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ttr", action="store_true", help="skip the time-to-RMSE comparison")
    ap.add_argument("--no-gp", action="store_true", help="skip the global-positioning measurement")
    ap.add_argument("--gp-only", action="store_true", help="only the global-positioning measurement")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(scenes.SPECS),
                    help="scene (default: the 1M-observation scene)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"],
                    help="working precision of the timed path (the configured workload is FP32)")
    ap.add_argument("--solver", default="auto", choices=["auto", "implicit", "explicit", "dense", "sparse"])
    ap.add_argument("--dense-kernels", action="store_true", help="time the tensor-core kernels only")
    args = ap.parse_args()
    if args.dense_kernels:
        return run_dense_kernels()
    if args.impl == "reference":
        return run_reference(args)
    if args.gp_only:
        import torch
        from paper_2510_13310_b300 import ba
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        print(json.dumps(run_gp_measure(torch, ba, dev, torch.cuda.current_stream(dev), steps=args.steps,
                                        warmup=args.warmup, cpu=not args.no_cpu_baseline)), flush=True)
        return 0

    import torch
    from paper_2510_13310_b300 import ba

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)

    scene = build_scene(args.workload)
    N = scene.n_obs
    solver = {"auto": ba.BA_SOLVER_AUTO, "implicit": ba.BA_SOLVER_IMPLICIT, "explicit": ba.BA_SOLVER_EXPLICIT,
              "dense": ba.BA_SOLVER_DENSE, "sparse": ba.BA_SOLVER_SPARSE}[args.solver]
    fp64 = args.precision == "fp64"
    opts = ba.Options(precision=ba.BA_FP64 if fp64 else ba.BA_FP32, solver=solver)
    prob = ba.Problem.from_scene(scene, opts, stream=stream.cuda_stream)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 126 MB L2

    infos = []
    for _ in range(args.warmup):
        prob.lm_step()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    launches0 = prob.kernel_launches
    step_ms = []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            ev0.record(stream)
            infos.append(prob.lm_step())
            ev1.record(stream)
            ev1.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
    torch.cuda.synchronize(dev)
    launches = prob.kernel_launches - launches0
    tot_ms = max_over_ranks(sum(step_ms), dist, dev)
    value = job_throughput(world, args.steps, tot_ms)

    # Jacobian+Schur throughput: observations through steps (a)+(b) per second
    lin = [i for i in infos if i["ms"][1] > 0]
    ab_ms = statistics.median([i["ms"][1] + i["ms"][2] for i in lin]) if lin else None
    schur_ms = statistics.median([i["ms"][2] for i in infos])
    gobs = N / (ab_ms * 1e-3) / 1e9 if ab_ms else None
    # (a)+(b) against HBM: per observation 16 B in (uv 8, prior 4, point index 4) and
    # the W row (108 B) or, for the formation from records, the 64-byte record
    # written; per point 12 B read and 36 B written
    rec_out = 64 if prob.formation_kernel == "k_form_S_rec" else 108
    ab_bytes = (16 + rec_out) * N + 48 * scene.spec.n_pts
    ab_roof = {"bytes_algorithmic": ab_bytes, "ms": ab_ms,
               "achieved_gbs": ab_bytes / (ab_ms * 1e-3) / 1e9 if ab_ms else None,
               "frac_of_hbm": ab_bytes / (ab_ms * 1e-3) / 1e9 / _peaks()[0] if ab_ms else None}
    # step (c) alone (ba_extract: validity bits, peel, ranks, one host readback),
    # against its bytes: per observation bits, alive, valid, two masks (5 B) and the
    # camera and point indices of the peel (8 B); per camera and point ~16 B
    ext_ms = []
    for _ in range(5):
        flush.zero_()
        ev0.record(stream)
        prob.extract()
        ev1.record(stream)
        ev1.synchronize()
        ext_ms.append(ev0.elapsed_time(ev1))
    ext_ms = statistics.median(ext_ms)
    ext_bytes = 13 * N + 16 * (scene.spec.n_cams + scene.spec.n_pts)
    ext_roof = {"bytes_algorithmic": ext_bytes, "ms": ext_ms,
                "achieved_gbs": ext_bytes / (ext_ms * 1e-3) / 1e9,
                "frac_of_hbm": ext_bytes / (ext_ms * 1e-3) / 1e9 / _peaks()[0],
                "note": "one CUDA graph replay (the first pass: ~16 kernels and 7 memsets) and one blocking "
                        "readback of the counts: latency-bound"}

    # roofline of the dominant kernel: of the PCG launch (ms[4]) and the co-visibility
    # product that forms the explicit system (ms[7]), the one with the larger mean
    # CUDA-event time over the timed steps (events recorded by the library on its stream)
    hbm, peak_kind = _peaks()
    solved = [i for i in infos if i["pcg_iters"] > 0 and i["ms"][4] > 0]
    P = scene.spec.n_pts
    n_fixed = 1
    Cf = int(solved[0]["n_cam_act"]) - n_fixed if solved else 0
    n = 9 * Cf
    esz = 8 if fp64 else 4  # bytes per element of the working precision
    mean_it = statistics.mean(i["pcg_iters"] for i in solved) if solved else 0.0
    kern_ms = statistics.mean(i["ms"][4] for i in solved) if solved else None
    kind = prob.solver_kind
    form_kernel = prob.formation_kernel
    solver_name = {ba.BA_SOLVER_DENSE: "dense", ba.BA_SOLVER_EXPLICIT: "explicit",
                   ba.BA_SOLVER_SPARSE: "sparse"}.get(kind, "implicit")
    if kind == ba.BA_SOLVER_DENSE:
        # the launch covers factorisation + CG; report the factorisation's flops
        per_launch = n ** 3 / 3.0
        kname = "dense solve: tensor-core blocked Cholesky (tcgen05 kind::tf32) + preconditioned CG"
        unit_txt = "n^3/3 flops of the factorisation, n = 9 Cf (timed launch includes the CG)"
    elif kind == ba.BA_SOLVER_SPARSE:
        # the stored blocks (2 per co-visible camera pair + the diagonal, 84 floats
        # each) read by every matvec, plus the set-up reads
        n_runs = int(np.count_nonzero(_covis_pairs(scene)))
        per_launch = ((2 * n_runs + Cf) * 84 * esz * mean_it + 81 * esz * Cf + 5 * esz * n)
        kname = "k_spcg (block-sparse explicit Schur matrix, block-row matvec)"
        unit_txt = f"(2 co-visible pairs + Cf) x 84 x {esz} B x iters + 81 x {esz} Cf + 5 x {esz} n bytes"
    elif prob.explicit_solver and prob.explicit_layout["rows_in_smem"]:
        # the explicit-S PCG iteration's algorithmic bytes: its matvec reads all of
        # S^ (4 n^2) once per iteration; plus the set-up reads (preconditioner
        # blocks 324 Cf; b, D, 1/D and x 20 n).  The rows stay in shared memory after
        # the first read, so the DRAM traffic (ncu) is about one read of S^.
        per_launch = esz * (n * n * mean_it + 81 * Cf + 5 * n)
        kname = "k_spcg (persistent block-Jacobi PCG on the explicit scaled Schur matrix, rows in shared memory)"
        unit_txt = f"{esz} (n^2 x iters + 81 Cf + 5 n) bytes, n = 9 Cf (S^ rows held in shared memory)"
    elif prob.explicit_solver:
        # rows of S^ streamed from device memory by every matvec: 4 n^2 per iteration
        # (S^ does not fit in L2 at these orders), plus the set-up reads
        per_launch = esz * (n * n * mean_it + 81 * Cf + 5 * n)
        kname = "k_spcg (persistent block-Jacobi PCG on the explicit scaled Schur matrix, rows streamed)"
        unit_txt = f"{esz} (n^2 x iters + 81 Cf + 5 n) bytes, n = 9 Cf"
    else:
        # per matvec, FP32 (W recomputed from a signed IRLS weight): the weight (4 B)
        # and the tile record (~13 B) per observation; point coordinates (16 B) and
        # V*^-1 (24 B) per point
        per_launch = mean_it * (N * 17 + P * 40)
        kname = "k_pcg (persistent block-Jacobi PCG, implicit Schur matvec, W recomputed)"
        unit_txt = "(17 B x obs + 40 B x points) x iters"
    if kind == ba.BA_SOLVER_DENSE:
        tpeak, tsrc = _tf32_peak()
        achieved = per_launch / (kern_ms * 1e-3) / 1e12 if kern_ms else 0.0
        bound, peak, unit, psrc = "tensor", tpeak, "TFLOP/s", tsrc
    else:
        achieved = per_launch / (kern_ms * 1e-3) / 1e9 if kern_ms else 0.0
        bound, peak, unit, psrc = "hbm", hbm, "GB/s", peak_kind + " (burst copy)"
    roof_pcg = {"kernel": kname, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "peak_source": psrc,
                "traffic": NCU_TRAFFIC.get((args.workload, "k_spcg" if prob.explicit_solver else "k_pcg"))
                if kind != ba.BA_SOLVER_DENSE and args.precision == "fp32" else None,
                "algorithmic_per_launch": per_launch,
                "formula": unit_txt, "launch_ms_mean": kern_ms,
                "mean_pcg_iters": mean_it, "us_per_pcg_iter": (kern_ms * 1e3 / mean_it) if mean_it else None,
                "solver": solver_name,
                "measured_limiter": NCU_LIMITER.get((args.workload, "k_spcg"))
                if kind == ba.BA_SOLVER_EXPLICIT and args.precision == "fp32" else None}
    roof_form = None
    form = [i["ms"][7] for i in infos if i["ms"][7] > 0]
    if form:
        # 9x9 block products Y^_k Y^_k2^T over co-visible observation pairs whose
        # cameras are both free: 243 FMA = 486 flops per pair, on the FP32 pipes
        free = np.ones(scene.spec.n_cams, bool)
        free[np.asarray(scene.fixed_cams, int)] = False
        t = np.bincount(scene.obs_pt[free[scene.obs_cam]], minlength=P).astype(np.int64)
        npairs = int((t * (t - 1) // 2).sum())
        form_ms = statistics.mean(form)
        flops = 486.0 * npairs
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        fp32_peak = sms * 128 * 2 * 2032e6 / 1e12
        # the kernel the library picked at creation
        fname = form_kernel or "k_form_S_runs"
        if fname == "k_form_S_rec":
            # pair list (8 B) and its point (4 B); one 64-byte record per observation,
            # one 32-byte record (V*^-1) per point; the dense S^ written once
            form_bytes = 12 * npairs + 64 * N + 32 * P + 4 * n * n
            form_bytes_txt = "12 B x pairs + 64 B x observations + 32 B x points + 4 n^2"
        else:
            form_bytes = 8 * npairs + 108 * N + 4 * n * n
            form_bytes_txt = "8 B x pairs + 108 B x observations + 4 n^2"
        roof_form = {"kernel": fname
                     + " (co-visibility block products forming the explicit system)",
                     "bound": "alu", "achieved": flops / (form_ms * 1e-3) / 1e12, "peak": fp32_peak,
                     "unit": "TFLOP/s", "frac": flops / (form_ms * 1e-3) / 1e12 / fp32_peak,
                     "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 flops x 2032 MHz",
                     "traffic": NCU_TRAFFIC.get((args.workload, fname)) if args.precision == "fp32" else None,
                     "measured_limiter": NCU_LIMITER.get((args.workload, fname)) if args.precision == "fp32" else None,
                     "algorithmic_per_launch": flops,
                     "formula": "486 flops x co-visible pairs of free cameras", "pairs": npairs,
                     "hbm_bytes_algorithmic": form_bytes,
                     "hbm_bytes_formula": form_bytes_txt,
                     "hbm_frac_of_measured": form_bytes / (form_ms * 1e-3) / 1e9 / hbm,
                     "launch_ms_mean": form_ms}
    if roof_form is not None and roof_form["launch_ms_mean"] > (kern_ms or 0.0):
        roofline, roofline_next = roof_form, roof_pcg
    else:
        roofline, roofline_next = roof_pcg, roof_form

    # end to end through the public API from pinned host buffers: one full solve
    # (create from pinned host arrays, LM_ITERS iterations, parameters back, destroy),
    # one untimed warm-up pass, then the median of E2E_RUNS timed passes
    prob.close()
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_in = [pin(scene.cams0), pin(scene.pts0), pin(scene.obs_cam), pin(scene.obs_pt),
            pin(scene.obs_uv), pin(scene.depth)]
    h_cams = torch.empty((scene.spec.n_cams, 9), dtype=torch.float64).pin_memory()
    h_pts = torch.empty((P, 3), dtype=torch.float64).pin_memory()
    e2e_runs = []
    for rep in range(1 + E2E_RUNS):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        p2 = ba.Problem(*h_in, options=opts, stream=stream.cuda_stream)
        p2.solve(LM_ITERS)
        p2.get_params(h_cams, h_pts)
        torch.cuda.synchronize(dev)
        if rep:
            e2e_runs.append(time.perf_counter() - t0)
        p2.close()
    e2e_s = statistics.median(e2e_runs)
    h2d = sum(t.numel() * t.element_size() for t in h_in)
    d2h = (h_cams.numel() + h_pts.numel()) * 8
    e2e = {"value": LM_ITERS / e2e_s, "unit": "LM iters/s",
           "h2d_bytes_per_step": h2d / LM_ITERS, "d2h_bytes_per_step": d2h / LM_ITERS,
           "what": f"ba_create from pinned host arrays + {LM_ITERS} LM iterations + "
                   f"parameters back to pinned host memory, wall clock; median of {E2E_RUNS} "
                   "runs after one untimed warm-up run",
           "runs_s": e2e_runs}

    # time to the FP64 GPU path's final RMSE
    ttr = None
    if not args.no_ttr:
        def trajectory(prec, solver=ba.BA_SOLVER_AUTO):
            try:
                p = ba.Problem.from_scene(scene, ba.Options(precision=prec, solver=solver),
                                          stream=stream.cuda_stream)
            except ba.BAError:
                # the FP64 implicit PCG keeps each block's cameras in shared memory and
                # does not fit 2,000 FP64 cameras: the FP64 reference runs the explicit PCG
                p = ba.Problem.from_scene(scene, ba.Options(precision=prec, solver=ba.BA_SOLVER_EXPLICIT),
                                          stream=stream.cuda_stream)
            rows, t = [], 0.0
            for _ in range(LM_ITERS):
                ev0.record(stream)
                r = p.lm_step()
                ev1.record(stream)
                ev1.synchronize()
                t += ev0.elapsed_time(ev1) / 1e3
                rows.append((t, r))
            F, rm = p.eval_cost()
            p.close()
            return rows, F, rm
        rows64, F64, rmse64 = trajectory(ba.BA_FP64)
        rows32, F32, rmse32 = trajectory(ba.BA_FP32, solver)

        def reach(rows, target_rmse):
            # the end time of the first iteration whose accepted result is within
            # 1e-5 (relative) of the target RMSE, or None
            for i, (t, r) in enumerate(rows):
                nxt = rows[i + 1][1]["rmse_px"] if i + 1 < len(rows) else None
                if nxt is not None and abs(nxt - target_rmse) <= 1e-5 * target_rmse:
                    return t
            return None
        t64 = reach(rows64, rmse64)
        t32 = reach(rows32, rmse64)
        ttr = {"target_rmse_px": rmse64, "fp64_final_cost": F64, "fp32_final_rmse_px": rmse32,
               "fp32_final_cost": F32, "fp64_s": t64, "fp32_s": t32,
               "speedup": (t64 / t32) if (t64 and t32) else None,
               "fp64_total_s": rows64[-1][0], "fp32_total_s": rows32[-1][0],
               "rule": "first iteration whose result RMSE is within 1e-5 of the FP64 final RMSE"}

    gp = None
    if not args.no_gp and args.workload == WORKLOAD:
        gp = run_gp_measure(torch, ba, dev, stream, cpu=rank == 0 and not args.no_cpu_baseline)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = oracle_cpu_baseline(scene)

    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": value, "unit": "LM iters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64" if fp64 else "f32",
            "data": "synthetic",
            "config": {"workload": _workload_name(scene) + (", FP64 throughout" if fp64 else
                                                            ", FP32 with double-float cost, FP64-accurate PCG "
                                                            "dots (double-float) and FP64 gain ratio"),
                       "n_cams": scene.spec.n_cams, "n_pts": P, "n_obs": N,
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "flushed between steps (256 MB write)"},
            "jacobian_schur_gobs_s": gobs, "jacobian_schur_ms": ab_ms, "schur_terms_ms": schur_ms,
            "jacobian_schur_hbm": ab_roof, "extraction_hbm": ext_roof, "gp": gp,
            "roofline": roofline, "roofline_next": roofline_next, "cpu_baseline": cpu, "e2e": e2e,
            "time_to_rmse": ttr,
            "gpu_launches": launches, "clocks": clk.summary(),
            "lm_trace": [{"cost": i["cost"], "rmse_px": i["rmse_px"], "accepted": i["accepted"],
                          "pcg_iters": i["pcg_iters"], "ms": [round(m, 3) for m in i["ms"]]}
                         for i in infos[:5]]}
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
