"""Host-side logic of bench.py without a GPU: the per-pass byte model, the max-over-ranks
reduction of a replica run (2 gloo ranks), and the reference arm under torchrun (rank 0 alone
prints one JSON line, the other rank exits 0 without work)."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_pass_bytes_headline():
    import bench

    n, nnz, p = 128 ** 3, 14581760, 8
    b = bench.pass_bytes(n, nnz, p, 2, 8, 8)
    # fused pass: 7 iterations move 2p + 3 + b = 21 vectors, the cycle's last one p + 2 + b = 12
    assert b["fused"] == (7 * 21 + 12) / 8 * n * 8
    # block product per cycle: CSR (int32 + FP64) and 3p vectors, amortised over p iterations
    assert b["block_product"] == (4 * (n + 1) + nnz * 12 + 3 * p * n * 8) / 8
    # directions per cycle: 4p vectors, the iterate twice, 2 bench vectors twice
    assert b["directions"] == (4 * p * n * 8 + 2 * n * p * 8 + 2 * 2 * n * 8) / 8
    fl, by = bench.algorithmic(n, nnz, p, 2, 8)
    assert abs(fl - 259e6) < 2e6


def _rank_main(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                      LOCAL_RANK=str(rank), BMINRES_BENCH_BACKEND="gloo")
    import bench

    td, r, ws = bench.dist()
    v = bench.max_over_ranks(td, 1.0 + rank)
    bench.barrier(td)
    out.put((r, ws, v))
    td.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert res == [(0, 2, 2.0), (1, 2, 2.0)]


@pytest.mark.slow
def test_reference_arm_under_torchrun_prints_one_line():
    env = dict(os.environ, BMINRES_BENCH_BACKEND="gloo")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--grid", "10", "--ref-sample-iters", "2", "--steps", "2", "--warmup", "1"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["extrapolated"] is True and d["steps"] == 2 and d["cpu_baseline"]["cores"] >= 1


def test_paper_e1_operator():
    from paper_1301_2102_gb300 import workloads

    A = workloads.paper_e1_operator(20)
    h = 1.0 / 19
    D = A.to_dense()
    assert A.n == 400 and np.allclose(np.diag(D), 4.0 - 200.0 * h * h)
    assert np.allclose(D, D.T) and set(np.unique(D[D != np.diag(D)[0]]).tolist()) <= {-1.0, 0.0}
