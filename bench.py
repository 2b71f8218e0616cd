"""Benchmark: time to a 1e-10 relative residual per block solve (block MINRES, band Lanczos version).

Workload (the configuration the metric is quoted on): 3D 7-point Laplacian on a 128^3 grid
(n = 2,097,152, 14,581,760 nonzeros) shifted by sigma at 10% of its spectrum (indefinite), p = 8
right-hand sides of which column 6 = 0.5 col0 - 1.2 col3 + 1e-12 noise and column 7 = col1 + col2
(two dependences at set-up), tol 1e-10, synthetic data (seeded).

One step = one complete solve from X0 = 0 until the FP64 TRUE relative residual ||b_i - A x_i|| /
||b_i|| of every column is <= 1e-10.  Modes (--mode, comma-separated; the first is the headline):
  fp64_refined  the paper's FP64 method, restarted inside FP64 iterative refinement until the true
                residual meets tol (the default headline: on this workload plain FP64 stops when its
                recursive residual meets tol with a true residual near 7e-8, which misses the metric)
  mixed_dw      double-word (FP32 pair) inner solves in the same refinement loop (default second)
  mixed         FP32 inner solves in the same loop (does not converge at 128^3)
  fp64          the plain method, stopped by the recursive residual (reported with its true residual)

Each timed step calls the public C ABI with B and X in pinned host memory: `value` is the CUDA-event
time of the device part of that call (recorded on the solve's stream after B and X0 have landed in
HBM, until the FP64 true residual is known), `e2e` is the host wall time of the whole call
(host->device copy of B and X0, solve, device->host copy of X).  The inputs (134 MB per block) and
the per-solve traffic (hundreds of GB) exceed L2, so no flush is needed.

Full solves take minutes.  Each mode gets its warm-up and one timed solve; further headline solves run
while the wall budget (--budget-s, counted from the start of the process) allows, so `steps` is the
number of headline solves actually timed and `steps_requested` the --steps asked for.  A guard prints
the line from the solves finished so far and exits if the process reaches --deadline-s.

`--impl reference` times the CPU oracle (plain C, FP64, OpenMP over every host core) on the same
workload: each step is the oracle's set-up plus a bounded number of band iterations, scaled to the
band iterations a solve of this workload to a true 1e-10 needs (`extrapolated: true`).  Under torchrun
every rank runs its own replica of the solve (the method does not shard across GPUs here); rank 0
prints the JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

T_START = time.time()
ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time-to-1e-10 rel. residual per block solve (FP64 vs mixed), % of HBM roofline"
TOL = 1e-10
MAXIT = 4_000_000
# Band iterations a solve of the 128^3 workload needs to reach a TRUE relative residual of 1e-10
# (FP64 inner solves in FP64 refinement, two restarts to an inner 1e-6, measured on GB300; the oracle
# follows the same iteration within the parity bar).  Used to scale the reference arm's sampled
# oracle time per band iteration to a full solve; the repo arm uses its own measured count.
REF_ITERS_128 = 1_555_397
REF_OUTER_128 = 2


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured copy (MEASURED_PEAKS.json)"
    except Exception:
        return 6800.0, "fallback"


def workload(N: int):
    from paper_1301_2102_gb300 import workloads

    A = workloads.laplacian(N, 3, workloads.shift_at_fraction(N, 3, 0.10))
    B = workloads.dependent_rhs_p8(A.n, seed=0)
    return A, B


def config(args, A, p):
    return {"workload": f"3D 7-point Laplacian {args.grid}^3 shifted at 10% of the spectrum, p={p} with two "
                        "dependent columns, time to a true relative residual of 1e-10 per column",
            "n": A.n, "nnz": A.nnz, "p": p, "tol": TOL, "x0": "zero",
            "l2": "inputs and per-solve traffic larger than L2 (no flush needed)"}


def pass_bytes(n: int, nnz: int, p: int, nb: int, s: int, sx: int):
    """Algorithmic bytes per band iteration of each streaming pass as this design moves them, each
    vector element read or written once per pass (element size s, iterate element size sx):
    fused window pass (w', p window vectors, W_{t+1}, p-1 known vectors, nb bench in; w, W_{t+1} out;
    the last iteration of a cycle has no A step), block product once per cycle (CSR, 2p vectors in,
    p out) and the direction/iterate pass once per cycle (2p old directions, p Lanczos vectors, the
    iterate and nb bench vectors in; p directions, the iterate and nb bench vectors out)."""
    ba = ((p - 1) * (2 * p + 3 + nb) + (p + 2 + nb)) / p * n * s
    sp = (4 * (n + 1) + nnz * (4 + s) + 3 * p * n * s) / p
    dr = (4 * p * n * s + 2 * n * p * sx + 2 * nb * n * s) / p
    return {"fused": ba, "block_product": sp, "directions": dr}


def algorithmic(n: int, nnz: int, p: int, nb: int, s: int):
    """Algorithmic FLOPs and bytes of one band iteration.

    flops: block product 2 nnz (2 nnz p per cycle), orthogonalisation (6p + 4) n (known part, p
    inner products, update, norm, ||A u_j||), bench maintenance 4 nb n, directions and iterate
    (6p + 1) n.  bytes (element size s): the minimum the method must move per band iteration with
    the orthogonalisation in block-Gram form, B_min = CSR and the p-vector block product amortised
    over the cycle + 7 n s (orthogonalisation) + 4 n s + 2 n 8 (directions and iterate) + bench
    (3 nb / p + 2) n s."""
    flops = 2.0 * nnz + (6 * p + 4) * n + 4 * nb * n + (6 * p + 1) * n
    spmm = (nnz * (s + 4) + 4 * (n + 1)) / p + 2 * n * s
    bytes_ = spmm + 7 * n * s + 4 * n * s + 2 * n * 8 + (3.0 * nb / p + 2) * n * s
    return flops, bytes_


# DRAM bytes of bminres_solve_kernel<double,8> on this workload from ncu (dram__bytes_read.sum +
# dram__bytes_write.sum of launches of 160 and 320 band iterations: 90.971 GB and 180.217 GB), per band
# iteration and for the set-up of one launch.  None: the kernel has changed since the counters were taken.
TRAFFIC_PER_ITER_F64 = 557.8e6
TRAFFIC_SETUP_F64 = 1.73e9


def passes_report(info, n, nnz, p, s, sx, hbm):
    """Per-pass time per band iteration (block 0's device timeline) and algorithmic HBM rate."""
    it = max(info["iters"], 1)
    t = {"fused": (info["stream_ms"] - info["spmm_ms"] - info["dir_ms"]) / it,
         "block_product": info["spmm_ms"] / it, "directions": info["dir_ms"] / it}
    b = pass_bytes(n, nnz, p, 2, s, sx)
    out = {}
    for k in t:
        gbs = b[k] / (t[k] * 1e-3) / 1e9 if t[k] > 0 else None
        out[k] = {"us_per_iter": 1e3 * t[k], "bytes_per_iter": b[k], "gbs": gbs,
                  "hbm_frac": gbs / hbm if gbs else None}
    out["reduce_us_per_iter"] = 1e3 * info["reduce_ms"] / it
    out["scalar_us_per_iter"] = 1e3 * info["scalar_ms"] / it
    return out


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in list(self.lines):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as td

        backend = "nccl" if os.environ.get("BMINRES_BENCH_BACKEND", "") != "gloo" else "gloo"
        td.init_process_group(backend)
        return td, td.get_rank(), ws
    return None, 0, 1


def barrier(td):
    if td is not None:
        td.barrier()


def max_over_ranks(td, x: float) -> float:
    if td is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if td.get_backend() == "nccl" else "cpu")
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def host_cores() -> int:
    try:
        n = len(os.sched_getaffinity(0))
    except Exception:
        n = os.cpu_count() or 1
    env = os.environ.get("OMP_NUM_THREADS")
    return min(n, int(env)) if env and env.isdigit() and int(env) > 0 else n


def oracle_sample(A, B, variant: str, target_s: float, max_iters: int = 2000):
    """Set-up time and seconds per band iteration of the oracle build `variant` on the workload:
    set-up alone, then set-up + K band iterations with K sized to take about target_s."""
    from oracle import oracle

    oracle.build(variant=variant)
    t0 = time.perf_counter()
    oracle.bminres(A, B, tol=TOL, maxit=0, variant=variant)
    t_setup = time.perf_counter() - t0
    k = 8
    t0 = time.perf_counter()
    r = oracle.bminres(A, B, tol=TOL, maxit=k, variant=variant)
    per_it = max(time.perf_counter() - t0 - t_setup, 1e-9) / max(r.iters, 1)
    k2 = int(min(max_iters, max(k, target_s / per_it)))
    if k2 > k:
        t0 = time.perf_counter()
        r = oracle.bminres(A, B, tol=TOL, maxit=k2, variant=variant)
        per_it = max(time.perf_counter() - t0 - t_setup, 1e-9) / max(r.iters, 1)
    return t_setup, per_it, r.iters


def cpu_sample(A, B, target_s: float):
    """The oracle as it stands, on the host cores: a bounded sample of the all-core OpenMP build (the
    reported baseline) and of the single-threaded parity build beside it."""
    ts, pi, k = oracle_sample(A, B, "omp", target_s)
    ts1, pi1, k1 = oracle_sample(A, B, "fp64", max(2.0, target_s / 4), max_iters=200)
    return {"cores": host_cores(), "setup_s": ts, "s_per_iter": pi, "iters": k,
            "setup_s_1core": ts1, "s_per_iter_1core": pi1, "iters_1core": k1}


def cpu_baseline(cs, iters: int, outer: int):
    """`cpu_baseline` object: the sample scaled to `iters` band iterations and `outer` set-ups."""
    return {"value": outer * cs["setup_s"] + cs["s_per_iter"] * iters, "unit": "s", "cores": cs["cores"],
            "kind": "oracle",
            "sample": (f"oracle (OpenMP build, {cs['cores']} threads) on the full workload: set-up "
                       f"({cs['setup_s']:.2f} s) + {cs['iters']} band iterations ({cs['s_per_iter'] * 1e3:.2f} ms "
                       f"each), scaled to the {iters} band iterations and {outer} set-up(s) of the headline solve"),
            "extrapolated": True, "s_per_band_iteration": cs["s_per_iter"], "setup_s": cs["setup_s"],
            "single_core": {"value": outer * cs["setup_s_1core"] + cs["s_per_iter_1core"] * iters,
                            "s_per_band_iteration": cs["s_per_iter_1core"], "setup_s": cs["setup_s_1core"],
                            "sample_iters": cs["iters_1core"], "build": "single-threaded parity oracle"}}


def fp64_peak():
    from paper_1301_2102_gb300 import _lib

    best = 0.0
    for _ in range(2):
        g, _ms = _lib.fp64_peak_gflops(100000)
        best = max(best, g)
    return best


def run_reference(args):
    td, rank, ws = dist()
    if rank != 0:
        return 0
    A, B = workload(args.grid)
    p = B.shape[1]
    from oracle import oracle

    oracle.build(variant="omp")
    iters = REF_ITERS_128 if args.grid == 128 else None
    if iters is None:  # other grid sizes (host tests): the oracle's own count on the small problem
        iters = oracle.bminres(A, B, tol=TOL, maxit=MAXIT, variant="omp").iters
    cores = host_cores()
    t0 = time.perf_counter()
    oracle.bminres(A, B, tol=TOL, maxit=0, variant="omp")
    t_setup = time.perf_counter() - t0
    for _ in range(args.warmup):
        oracle.bminres(A, B, tol=TOL, maxit=2, variant="omp")
    k = args.ref_sample_iters
    steps, per = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.bminres(A, B, tol=TOL, maxit=k, variant="omp")
        t = time.perf_counter() - t0
        pi = max(t - t_setup, 1e-9) / max(r.iters, 1)
        per.append(pi)
        steps.append(REF_OUTER_128 * t_setup + pi * iters)
    value = statistics.median(steps)
    sample = (f"each step: oracle (OpenMP build, {cores} threads) set-up + {k} band iterations on the full "
              f"workload ({statistics.median(per) * 1e3:.2f} ms per band iteration, set-up {t_setup:.2f} s), scaled "
              f"to {iters} band iterations and {REF_OUTER_128} set-ups")
    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * value, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config(args, A, p),
            "extrapolated": True, "iters_used": iters,
            "iters_source": "band iterations of the FP64-refined solve of this workload on GB300",
            "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.time() - T_START}
    print(json.dumps(line), flush=True)
    return 0


def one_solve(solver, Bh, Xh, maxit, stream):
    import torch

    Xh.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X, info, rel = solver.solve(Bh, Xh, tol=TOL, maxit=maxit, stream=stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    return info, rel, wall


DTYPE = {"fp64": "f64", "fp64_refined": "f64", "mixed": "f32+f64", "mixed_dw": "f32x2+f64"}
ELEM = {"fp64": 8, "fp64_refined": 8, "mixed": 4, "mixed_dw": 8}
KERNEL = {"fp64": "bminres_solve_kernel<double,8,256>", "fp64_refined": "bminres_solve_kernel<double,8,256>",
          "mixed": "bminres_solve_kernel<float,8,256>", "mixed_dw": "bminres_solve_kernel<dw,8,256>"}


def mode_summary(mode, steps, n, nnz, p, hbm, peak64):
    """Figures of one mode from its timed solves (median time; per-iteration rates of the last)."""
    info = steps[-1][0]
    se = ELEM[mode]
    fl, by = algorithmic(n, nnz, p, 2, se)
    it = max(info["iters"], 1)
    ks = info["kernel_ms"] * 1e-3
    d = {"value": statistics.median([s[0]["device_ms"] * 1e-3 for s in steps]), "unit": "s",
         "solves_timed": len(steps), "e2e_s": statistics.median([s[2] for s in steps]),
         "band_iterations": info["iters"], "cycles": info["cycles"], "outer": info["outer"],
         "setup_deflations": info["setup_deflations"], "relres_true_max": info["relres_true_max"],
         "status": info["status_name"], "us_per_band_iteration": 1e6 * ks / it,
         "kernel": KERNEL[mode], "gflops": fl * it / ks / 1e9, "hbm_gbs_bmin": by * it / ks / 1e9}
    d["hbm_frac_bmin"] = d["hbm_gbs_bmin"] / hbm
    if mode in ("fp64", "fp64_refined"):
        d["fp64_frac"] = d["gflops"] / peak64 if peak64 else None
    d["passes"] = passes_report(info, n, nnz, p, se, 8 if mode in ("fp64", "fp64_refined") else se, hbm)
    return d


def run_ours(args):
    import torch

    td, rank, ws = dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_1301_2102_gb300 import Solver

    A, B = workload(args.grid)
    n, p = B.shape
    modes = args.mode.split(",")
    head = modes[0]
    hbm, hbm_src = hbm_peak()
    # CPU leg first (rank 0 at N=1): a bounded sample, scaled to the solve once its count is known
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_sample(A, B, args.cpu_target_s)
    peak64 = fp64_peak()
    Bh = torch.from_numpy(B).pin_memory()
    Xh = torch.zeros_like(Bh).pin_memory()
    stream = torch.cuda.current_stream().cuda_stream
    results = {m: [] for m in modes}
    lock = threading.Lock()
    printed = threading.Event()

    def compose(clocks, collective):
        if not results[head]:
            return {"metric": METRIC, "value": None, "unit": "s", "n_gpus": ws, "steps": 0,
                    "steps_requested": args.steps, "warmup": args.warmup, "higher_is_better": False,
                    "impl": "ours", "error": "no headline solve finished within the wall budget",
                    "config": dict(config(args, A, p), mode=head)}
        hs = mode_summary(head, results[head], n, A.nnz, p, hbm, peak64)
        value = max_over_ranks(td, hs["value"]) if collective else hs["value"]
        info = results[head][-1][0]
        it = max(info["iters"], 1)
        ks = info["kernel_ms"] * 1e-3
        fl, by = algorithmic(n, A.nnz, p, 2, ELEM[head])
        if head in ("fp64", "fp64_refined"):
            roof = {"bound": "alu", "achieved": fl * it / ks / 1e9, "peak": peak64, "unit": "GFLOP/s",
                    "peak_source": "FP64 FMA throughput measured in this run (bminres_fp64_peak)"}
        else:
            roof = {"bound": "hbm", "achieved": by * it / ks / 1e9, "peak": hbm, "unit": "GB/s",
                    "peak_source": hbm_src}
        roof["frac"] = roof["achieved"] / roof["peak"]
        roof["kernel"] = KERNEL[head]
        # per launch of the persistent kernel (one launch per refinement step), like `achieved`
        launches = max(info["outer"], 1)
        roof["traffic"] = (TRAFFIC_SETUP_F64 + TRAFFIC_PER_ITER_F64 * it / launches
                           if head in ("fp64", "fp64_refined") and TRAFFIC_PER_ITER_F64 else None)
        roof["kernel_launches"] = launches
        roof["algorithmic_bytes_per_launch"] = by * it / launches
        roof["hbm_gbs_bmin"] = by * it / ks / 1e9
        roof["hbm_frac_bmin"] = roof["hbm_gbs_bmin"] / hbm
        roof["bmin_bytes_per_iter"] = by
        roof["flops_per_iter"] = fl
        roof["passes"] = hs["passes"]
        line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": ws, "steps": len(results[head]),
                "steps_requested": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3,
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[head],
                "data": "synthetic", "impl": "ours", "config": dict(config(args, A, p), mode=head),
                "headline": hs, "roofline": roof,
                "e2e": {"value": hs["e2e_s"], "unit": "s", "h2d_bytes_per_step": 2 * n * p * 8,
                        "d2h_bytes_per_step": n * p * 8},
                "gpu_launches": sum(s[0]["launches"] for s in results[head]),
                "clocks": clocks, "fp64_peak_gflops": peak64,
                "parallelism": f"{ws} independent replica(s)", "wall_s": time.time() - T_START}
        for m in modes[1:]:
            if results[m]:
                line[m] = mode_summary(m, results[m], n, A.nnz, p, hbm, peak64)
        if cpu is not None:
            line["cpu_baseline"] = cpu_baseline(cpu, info["iters"], info["outer"])
        return line

    clk = ClockSampler(local)

    def emit(reason=None):
        with lock:
            if printed.is_set():
                return
            line = compose(clk.summary(), collective=reason is None and td is not None)
            if reason:
                line["ended_by"] = reason
            if rank == 0:
                print(json.dumps(line), flush=True)
            printed.set()

    def guard():
        emit("deadline: printed from the solves finished so far")
        os._exit(0)

    timer = None
    if args.deadline_s > 0:
        timer = threading.Timer(max(1.0, args.deadline_s - (time.time() - T_START)), guard)
        timer.daemon = True
        timer.start()
    solvers = {}
    try:
        for m in modes:
            kw = {"tol_inner": args.tol_inner} if m != "fp64" else {}
            solvers[m] = Solver(A, precision=m, bench=4, **kw)
            for _ in range(args.warmup):  # short solves: module load, allocation, clocks
                one_solve(solvers[m], Bh, Xh, args.warmup_maxit, stream)
        barrier(td)
        with clk:
            last = {}
            for m in modes:  # one timed solve per mode
                barrier(td)
                t0 = time.time()
                results[m].append(one_solve(solvers[m], Bh, Xh, MAXIT, stream))
                last[m] = time.time() - t0
                barrier(td)
            # more headline solves while the budget allows
            while len(results[head]) < args.steps:
                # the same decision on every rank: stop when any rank would overrun the budget
                over = float(time.time() - T_START + 1.1 * last[head] > args.budget_s)
                if max_over_ranks(td, over) > 0:
                    break
                barrier(td)
                t0 = time.time()
                results[head].append(one_solve(solvers[head], Bh, Xh, MAXIT, stream))
                last[head] = time.time() - t0
                barrier(td)
    finally:
        for s in solvers.values():
            s.close()
    if timer is not None:
        timer.cancel()
    emit()
    if td is not None:
        td.destroy_process_group()
    return 0


def run_profile_case(args):
    """Profiling aid (not a benchmark result): one solve of the workload capped at
    --profile-iters band iterations, for ncu captures of the persistent kernel."""
    import torch

    from paper_1301_2102_gb300 import Solver

    A, B = workload(args.grid)
    Bd = torch.from_numpy(B).cuda()
    mode = args.mode.split(",")[0]
    with Solver(A, precision=mode, bench=4, max_outer=1) as s:
        X, info, rel = s.solve(Bd, tol=TOL, maxit=args.profile_iters)
        torch.cuda.synchronize()
    print(json.dumps({"profile_case": True, "grid": args.grid, "mode": mode, **info}), flush=True)
    return 0


def run_paper_e1(args):
    """The paper's first experiment on its own operator (Sec. 8), unpreconditioned here: one block
    solve with p = 10 N(0,1) right-hand sides against 10 single-vector solves, tol 1e-8."""
    import torch

    from paper_1301_2102_gb300 import Solver, workloads

    A = workloads.paper_e1_operator(200)
    B = workloads.randn_rhs(A.n, 10, 0)
    tol, maxit = 1e-8, 2_000_000
    out = {"experiment": "paper E1 operator, -L - 200 I on 200 x 200, p = 10, tol 1e-8, no preconditioner",
           "n": A.n, "nnz": A.nnz}
    with Solver(A) as s:
        Bd = torch.from_numpy(B).cuda()
        s.solve(Bd, tol=tol, maxit=100)
        X, info, rel = s.solve(Bd, tol=tol, maxit=maxit)
        out.update(block_iters=info["iters"], block_s=info["device_ms"] * 1e-3, block_relres_true=float(rel.max()))
        its, t = 0, 0.0
        for c in range(10):
            Xc, ic, rc = s.solve(Bd[:, c:c + 1].contiguous(), tol=tol, maxit=maxit)
            its += ic["iters"]
            t += ic["device_ms"] * 1e-3
        out.update(sequential_iters=its, sequential_s=t)
    out["paper_context"] = ("paper (ichol-preconditioned, Matlab on a 2.3 GHz Core i5): block 1048 iterations / "
                            "16.8 s, sequential 3787 iterations / 23.5 s")
    print(json.dumps(out), flush=True)
    return 0


def run_paper_e2(args):
    """The paper's second experiment on its operator (Sec. 8), unpreconditioned here: for each p, the
    band iterations of one block solve with right-hand sides [ones, e_1 .. e_{p-1}] against the total
    of the p single-vector solves, tol 1e-8."""
    import torch

    from paper_1301_2102_gb300 import Solver, workloads

    A = workloads.paper_e1_operator(200)
    tol, maxit = 1e-8, 2_000_000
    ps = [1, 2, 3, 4, 6, 8, 10, 12, 16, 20, 24, 32]
    Bfull = workloads.ones_identity_rhs(A.n, max(ps))
    rows = []
    with Solver(A) as s:
        Bd = torch.from_numpy(Bfull).cuda()
        single = []
        for c in range(max(ps)):
            _, ic, rc = s.solve(Bd[:, c:c + 1].contiguous(), tol=tol, maxit=maxit)
            single.append((ic["iters"], ic["device_ms"]))
        for p in ps:
            X, info, rel = s.solve(Bd[:, :p].contiguous(), tol=tol, maxit=maxit)
            seq_it = sum(x[0] for x in single[:p])
            seq_ms = sum(x[1] for x in single[:p])
            rows.append({"p": p, "block_iters": info["iters"], "sequential_iters": seq_it,
                         "iteration_ratio": info["iters"] / seq_it, "block_ms": info["device_ms"],
                         "sequential_ms": seq_ms, "status": info["status_name"],
                         "relres_true_max": float(rel.max()), "deflations": info["deflations"],
                         "setup_deflations": info["setup_deflations"]})
    print(json.dumps({"experiment": "paper E2 operator, -L - 200 I on 200 x 200, right-hand sides [ones, e_1 .. "
                                    "e_{p-1}], tol 1e-8, no preconditioner", "n": A.n, "rows": rows}), flush=True)
    return 0


def run_c1_latency(args):
    """The 32 x 32 singular operator (latency-bound: n = 1024): microseconds per band iteration of the
    range-projected solve to 1e-10, median of 50 timed solves after 5 warm-up solves, and of the
    literal run (2000 band iterations, stalls at the least-squares floor)."""
    import torch

    from paper_1301_2102_gb300 import Solver, workloads

    A, B = workloads.config_c1()
    Q = workloads.laplacian_null_modes_2d(32, 4.0)
    out = {"experiment": "config 1: 2D 5-point Laplacian 32x32, sigma = 4 (singular), p = 4, tol 1e-10"}
    with Solver(A) as s:
        for name, rhs, maxit in (("projected", workloads.project_out(B, Q), 4000), ("literal", B, 2000)):
            Bd = torch.from_numpy(rhs).cuda()
            for _ in range(5):
                s.solve(Bd, tol=1e-10, maxit=maxit)
            us, ms = [], []
            for _ in range(50):
                X, info, rel = s.solve(Bd, tol=1e-10, maxit=maxit)
                us.append(1e3 * info["kernel_ms"] / max(info["iters"], 1))
                ms.append(info["device_ms"])
            out[name] = {"us_per_band_iteration_median": statistics.median(us), "solve_ms_median": statistics.median(ms),
                         "band_iterations": info["iters"], "status": info["status_name"],
                         "relres_true_max": float(rel.max()), "grid_blocks": info["grid_blocks"], "solves_timed": 50}
    print(json.dumps(out), flush=True)
    return 0


def run_c3_sweep(args):
    """Block-size scaling on the 128^3 operator (p N(0,1) right-hand sides): microseconds per band
    iteration of capped solves (--sweep-iters band iterations, after one warm-up) per precision, and
    per right-hand side."""
    import torch

    from paper_1301_2102_gb300 import Solver, workloads

    N = args.grid
    A = workloads.laplacian(N, 3, workloads.shift_at_fraction(N, 3, 0.10))
    rows = []
    for p in (1, 4, 8, 16):
        B = torch.from_numpy(workloads.randn_rhs(A.n, p, 0)).cuda()
        for mode in ("fp64", "mixed_dw", "mixed"):
            with Solver(A, precision=mode, max_outer=1, tol_inner=1e-12) as s:
                s.solve(B, tol=1e-12, maxit=200)
                X, info, rel = s.solve(B, tol=1e-12, maxit=args.sweep_iters)
            it = max(info["iters"], 1)
            us = 1e3 * info["kernel_ms"] / it
            rows.append({"p": p, "mode": mode, "band_iterations": info["iters"], "us_per_band_iteration": us,
                         "us_per_band_iteration_per_rhs": us / p,
                         "block_product_us": 1e3 * info["spmm_ms"] / it, "directions_us": 1e3 * info["dir_ms"] / it,
                         "fused_us": 1e3 * (info["stream_ms"] - info["spmm_ms"] - info["dir_ms"]) / it})
    print(json.dumps({"experiment": f"config 3 block-size sweep, {N}^3, capped at {args.sweep_iters} band iterations",
                      "rows": rows}), flush=True)
    return 0


def run_c5(args):
    """Config 5 (192^3, sigma at 5 % of the spectrum, p = 32 N(0,1) right-hand sides): per band
    iteration times of the FP64 and FP32-inner forward solves and of the FP64 adjoint solve for
    L = sum(X^2) (G = 2X), capped at --sweep-iters band iterations, and the device memory in use."""
    import torch

    from paper_1301_2102_gb300 import Solver, workloads

    A, B0 = workloads.config_c5()
    B = torch.from_numpy(B0).cuda()
    out = {"experiment": "config 5: 3D 7-point Laplacian 192^3 shifted at 5%, p = 32, capped solves",
           "n": A.n, "nnz": A.nnz, "p": 32, "iters_cap": args.sweep_iters}
    for mode in ("fp64", "mixed"):
        free0 = torch.cuda.mem_get_info()[0]
        with Solver(A, precision=mode, max_outer=1, tol_inner=1e-12) as s:
            s.solve(B, tol=1e-12, maxit=100)
            X, info, rel = s.solve(B, tol=1e-12, maxit=args.sweep_iters)
            free1 = torch.cuda.mem_get_info()[0]
            it = max(info["iters"], 1)
            d = {"us_per_band_iteration": 1e3 * info["kernel_ms"] / it, "band_iterations": info["iters"],
                 "relres_true_max": float(rel.max()), "device_bytes_in_use": free0 - free1,
                 "block_product_us": 1e3 * info["spmm_ms"] / it, "directions_us": 1e3 * info["dir_ms"] / it}
            if mode == "fp64":
                dB, dA, binfo = s.backward((2.0 * X).contiguous(), X, tol=1e-12, maxit=args.sweep_iters)
                d["adjoint_us_per_band_iteration"] = 1e3 * binfo["kernel_ms"] / max(binfo["iters"], 1)
                d["adjoint_band_iterations"] = binfo["iters"]
            out[mode] = d
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--warmup-maxit", type=int, default=2000)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", default="fp64_refined,mixed_dw",
                    help="comma-separated modes (fp64_refined, mixed_dw, mixed, fp64); the first is the headline")
    ap.add_argument("--tol-inner", type=float, default=1e-6, help="inner tolerance of the refined forms")
    ap.add_argument("--grid", type=int, default=128)
    ap.add_argument("--budget-s", type=float, default=1300.0,
                    help="no further headline solve starts if it would end after this many seconds of wall time")
    ap.add_argument("--deadline-s", type=float, default=1650.0,
                    help="print the line from the solves finished so far and exit at this wall time (0: off)")
    ap.add_argument("--cpu-target-s", type=float, default=12.0, help="seconds of the oracle's timed sample")
    ap.add_argument("--ref-sample-iters", type=int, default=40, help="band iterations per reference-arm step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-iters", type=int, default=0,
                    help="profiling aid: run one solve capped at this many band iterations and print its info")
    ap.add_argument("--paper-e1", action="store_true",
                    help="run the paper's first experiment on its operator (block vs sequential) and exit")
    ap.add_argument("--paper-e2", action="store_true",
                    help="run the paper's second experiment (iteration ratio over p) on its operator and exit")
    ap.add_argument("--c1-latency", action="store_true", help="config 1 microseconds per band iteration and exit")
    ap.add_argument("--c3-sweep", action="store_true", help="config 3 block-size sweep (capped solves) and exit")
    ap.add_argument("--c5", action="store_true", help="config 5 capped forward and adjoint solves and exit")
    ap.add_argument("--sweep-iters", type=int, default=1500, help="band iterations of the capped solves")
    args = ap.parse_args()
    if args.paper_e1:
        return run_paper_e1(args)
    if args.paper_e2:
        return run_paper_e2(args)
    if args.c1_latency:
        return run_c1_latency(args)
    if args.c3_sweep:
        return run_c3_sweep(args)
    if args.c5:
        return run_c5(args)
    if args.profile_iters > 0:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
