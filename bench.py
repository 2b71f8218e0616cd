"""Benchmark: time to a 1e-10 relative residual per block solve (block MINRES, band Lanczos version).

Workload (the configuration the metric is quoted on): 3D 7-point Laplacian on a 128^3 grid
(n = 2,097,152, 14,581,760 nonzeros) shifted by sigma at 10% of its spectrum (indefinite), p = 8
right-hand sides of which column 6 = 0.5 col0 - 1.2 col3 + 1e-12 noise and column 7 = col1 + col2
(two dependences at set-up), FP64, tol 1e-10, synthetic data (seeded).

One step = one complete solve from X0 = 0 to the tolerance.  Each timed step calls the public C ABI
with B and X in pinned host memory: `value` is the CUDA-event time of the device part of that call
(recorded on the solve's stream after B and X0 have landed in HBM, until the FP64 true residual
is known), `e2e` is the host wall time of the whole call (host->device copy of B and X0, solve,
device->host copy of X).  The inputs (134 MB per block) and the per-solve traffic (GBs) exceed L2.

`--mode` adds the refined forms (fp64_refined, mixed_dw, mixed: FP64 iterative refinement around
FP64, double-word or FP32 inner solves, each to an FP64 true residual below tol) as extra objects of
the same line; the first mode listed is the headline.

`--impl reference` times the CPU oracle (plain C, FP64, one core) on the same workload: set-up plus
a bounded number of band iterations, scaled to a full solve.  Under torchrun every rank runs its own
replica of the solve (the method does not shard across GPUs here); rank 0 prints the JSON line.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time-to-1e-10 rel. residual per block solve (FP64 vs mixed), % of HBM roofline"
TOL = 1e-10
MAXIT = 3_000_000
# oracle band-iteration counts measured on the same operator family (10% shift, p = 8 random
# right-hand sides, tol 1e-10) at N = 16, 24, 32, 40: used only to scale the reference arm's
# sampled per-iteration time to a full solve when no GPU count is at hand
ORACLE_ITERS_N40 = 24596


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    except Exception:
        return 6800.0, "fallback"


FP64_PEAK_GFLOPS = 1250.0  # nominal dense FP64 of GB300 (1.25 TFLOP/s)


def workload(N: int):
    from paper_1301_2102_gb300 import workloads

    A = workloads.laplacian(N, 3, workloads.shift_at_fraction(N, 3, 0.10))
    B = workloads.dependent_rhs_p8(A.n, seed=0)
    return A, B


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
    """Algorithmic FLOPs and bytes of one band iteration ('Measurement').

    flops: block product 2 nnz (2 nnz p per cycle), orthogonalisation (6p + 4) n (known part, p
    inner products, update, norm, ||A u_j||), bench maintenance 4 nb n, directions and iterate
    (6p + 1) n.  bytes (element size s): CSR and the p-vector block product amortised over the
    cycle, the fused window pass (2p + 3) n s, the direction/iterate pass 6 n s, bench 3 nb/p n s."""
    flops = 2.0 * nnz + (6 * p + 4) * n + 4 * nb * n + (6 * p + 1) * n
    bytes_ = (nnz * (s + 4) + 4 * (n + 1)) / p + 2 * n * s + (2 * p + 3) * n * s + 6 * n * s + 3.0 * nb / p * n * s
    return flops, bytes_


# DRAM bytes of bminres_solve_kernel<double,8> on this workload, from ncu (dram__bytes_read.sum +
# dram__bytes_write.sum of launches of 160 and 320 band iterations: 90.981 GB and 180.249 GB, i.e.
# 557.9 MB per band iteration plus 1.71 GB of set-up); None when the kernel has changed since
TRAFFIC_PER_ITER_F64 = 557.9e6
TRAFFIC_SETUP_F64 = 1.71e9


def passes_report(info, n, nnz, p, s, sx, hbm_peak):
    """Per-pass time per band iteration (block 0's device timeline) and algorithmic HBM rate."""
    it = max(info["iters"], 1)
    t = {"fused": (info["stream_ms"] - info["spmm_ms"] - info["dir_ms"]) / it,
         "block_product": info["spmm_ms"] / it, "directions": info["dir_ms"] / it}
    b = pass_bytes(n, nnz, p, 2, s, sx)
    out = {}
    for k in t:
        gbs = b[k] / (t[k] * 1e-3) / 1e9 if t[k] > 0 else None
        out[k] = {"us_per_iter": 1e3 * t[k], "bytes_per_iter": b[k], "gbs": gbs,
                  "hbm_frac": gbs / hbm_peak if gbs else None}
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
        for ln in self.lines:
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


def cpu_baseline(A, B, gpu_iters: int | None, sample_iters: int):
    """Oracle (plain C, one core) on the workload: set-up, then set-up + sample_iters iterations."""
    from oracle import oracle

    oracle.build()
    t0 = time.perf_counter()
    oracle.bminres(A, B, tol=TOL, maxit=0)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    r = oracle.bminres(A, B, tol=TOL, maxit=sample_iters)
    t_run = time.perf_counter() - t0
    per_it = max(t_run - t_setup, 1e-9) / max(r.iters, 1)
    if gpu_iters is None:
        N = round(A.n ** (1.0 / 3.0))
        iters = int(ORACLE_ITERS_N40 * (N / 40.0) ** 3)
        how = f"{iters} band iterations (oracle count at 40^3 scaled by (N/40)^3)"
    else:
        iters = gpu_iters
        how = f"{iters} band iterations (the count the GPU solve needed)"
    value = t_setup + per_it * iters
    sample = (f"oracle set-up ({t_setup:.2f} s) + {r.iters} band iterations ({per_it * 1e3:.1f} ms each) on the "
              f"full workload, scaled to {how}")
    return {"value": value, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample,
            "s_per_band_iteration": per_it, "setup_s": t_setup, "sample_iters": r.iters}


def run_reference(args):
    td, rank, ws = dist()
    if rank != 0:
        return 0
    A, B = workload(args.grid)
    t0 = time.perf_counter()
    cb = cpu_baseline(A, B, None, args.cpu_sample_iters)
    steps = []
    for _ in range(args.steps):
        steps.append(cb["value"])
    line = {"metric": METRIC, "value": statistics.median(steps), "unit": "s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(steps), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"3D 7-point Laplacian {args.grid}^3 shifted at 10% of the spectrum, p=8 with two "
                                   "dependent columns, FP64, tol 1e-10", "n": A.n, "nnz": A.nnz, "p": 8},
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": statistics.median(steps), "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}
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


def run_ours(args):
    import torch

    td, rank, ws = dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_1301_2102_gb300 import Solver

    A, B = workload(args.grid)
    n, p = B.shape
    Bh = torch.from_numpy(B).pin_memory()
    Xh = torch.zeros_like(Bh).pin_memory()
    stream = torch.cuda.current_stream().cuda_stream
    hbm_peak, peak_src = peaks()
    results = {}
    modes = ["fp64", "mixed_dw"] if args.mode == "both" else args.mode.split(",")
    for mode in modes:
        kw = {"tol_inner": args.tol_inner} if mode != "fp64" else {}
        with Solver(A, precision=mode, bench=4, **kw) as s:
            for _ in range(args.warmup):  # short solves: module load, allocation, clocks
                one_solve(s, Bh, Xh, args.warmup_maxit, stream)
            barrier(td)
            steps = []
            with ClockSampler(local) as clk:
                for _ in range(args.steps):
                    barrier(td)
                    info, rel, wall = one_solve(s, Bh, Xh, MAXIT, stream)
                    barrier(td)
                    steps.append((info, rel, wall))
            results[mode] = (steps, clk.summary())
    # headline: FP64 (the configuration's mode) unless only mixed was run
    head = "fp64" if "fp64" in results else modes[0]
    steps, clocks = results[head]
    dev = [st[0]["device_ms"] * 1e-3 for st in steps]
    walls = [st[2] for st in steps]
    value = max_over_ranks(td, statistics.median(dev))
    e2e = max_over_ranks(td, statistics.median(walls))
    info = steps[-1][0]
    s_elem = 4 if head == "mixed" else 8
    fl, by = algorithmic(n, A.nnz, p, 2, s_elem)
    iters = info["iters"]
    kern_s = info["kernel_ms"] * 1e-3
    if head in ("fp64", "fp64_refined"):
        roof = {"bound": "alu", "achieved": fl * iters / kern_s / 1e9, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                "peak_source": "nominal FP64 of GB300 (1.25 TFLOP/s; 1.19 measured by an FMA probe)",
                "traffic": None, "kernel": "bminres_solve_kernel<double,8>"}
    else:
        roof = {"bound": "hbm", "achieved": by * iters / kern_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                "peak_source": peak_src, "traffic": None,
                "kernel": "bminres_solve_kernel<float,8>" if head == "mixed" else "bminres_solve_kernel<dw,8>"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["hbm_gbs"] = by * iters / kern_s / 1e9
    roof["hbm_frac"] = roof["hbm_gbs"] / hbm_peak
    if head == "fp64" and TRAFFIC_PER_ITER_F64:
        roof["traffic"] = TRAFFIC_SETUP_F64 + TRAFFIC_PER_ITER_F64 * iters
    roof["passes"] = passes_report(info, n, A.nnz, p, s_elem, 8 if head == "fp64" else s_elem, hbm_peak)
    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp64_refined": "f64", "mixed": "f32+f64", "mixed_dw": "f32x2+f64"}[head],
            "data": "synthetic",
            "config": {"workload": f"3D 7-point Laplacian {args.grid}^3 shifted at 10% of the spectrum, p=8 with two "
                                   "dependent columns, tol 1e-10", "mode": head, "n": n, "nnz": A.nnz, "p": p,
                       "band_iterations": iters, "cycles": info["cycles"], "setup_deflations": info["setup_deflations"],
                       "relres_true_max": info["relres_true_max"], "status": info["status_name"],
                       "grid_blocks": info["grid_blocks"], "us_per_band_iteration": 1e6 * kern_s / max(iters, 1),
                       "l2": "inputs and per-solve traffic larger than L2 (no flush needed)",
                       "warmup": f"{args.warmup} solves capped at {args.warmup_maxit} band iterations",
                       "parallelism": f"{ws} independent replica(s)", "timeline_ms": {
                           k: info[k] for k in ("kernel_ms", "stream_ms", "spmm_ms", "dir_ms", "reduce_ms", "scalar_ms",
                                                "qr_ms")}},
            "roofline": roof,
            "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": 2 * n * p * 8, "d2h_bytes_per_step": n * p * 8},
            "gpu_launches": info["launches"], "clocks": clocks}
    for mode, (st, ck) in results.items():
        if mode == head:
            continue
        inf = st[-1][0]
        se = 4 if mode == "mixed" else 8
        flm, bym = algorithmic(n, A.nnz, p, 2, se)
        line[mode] = {"value": statistics.median([x[0]["device_ms"] * 1e-3 for x in st]), "unit": "s",
                      "band_iterations": inf["iters"], "outer": inf["outer"], "relres_true_max": inf["relres_true_max"],
                      "status": inf["status_name"], "e2e_s": statistics.median([x[2] for x in st]),
                      "hbm_gbs": bym * inf["iters"] / (inf["kernel_ms"] * 1e-3) / 1e9,
                      "us_per_band_iteration": 1e3 * inf["kernel_ms"] / max(inf["iters"], 1),
                      "tol_inner": args.tol_inner, "passes": passes_report(inf, n, A.nnz, p, se, se, hbm_peak)}
        line[mode]["hbm_frac"] = line[mode]["hbm_gbs"] / hbm_peak
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(A, B, iters, args.cpu_sample_iters)
        line["cpu_baseline"] = {k: line["cpu_baseline"][k] for k in ("value", "unit", "cores", "kind", "sample")}
    if rank == 0:
        print(json.dumps(line), flush=True)
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
    with Solver(A, precision="fp64" if args.mode == "both" else args.mode, bench=4) as s:
        X, info, rel = s.solve(Bd, tol=TOL, maxit=args.profile_iters)
        torch.cuda.synchronize()
    print(json.dumps({"profile_case": True, "grid": args.grid, "mode": args.mode, **info}), flush=True)
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


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--warmup-maxit", type=int, default=2000)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", default="fp64",
                    help="fp64 (default), fp64_refined, mixed, mixed_dw, a comma-separated list, or both (= fp64,mixed_dw)")
    ap.add_argument("--tol-inner", type=float, default=1e-6, help="inner tolerance of the mixed forms")
    ap.add_argument("--grid", type=int, default=128)
    ap.add_argument("--cpu-sample-iters", type=int, default=24)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-iters", type=int, default=0,
                    help="profiling aid: run one solve capped at this many band iterations and print its info")
    ap.add_argument("--paper-e1", action="store_true",
                    help="run the paper's first experiment on its operator (block vs sequential) and exit")
    args = ap.parse_args()
    if args.paper_e1:
        return run_paper_e1(args)
    if args.profile_iters > 0:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
