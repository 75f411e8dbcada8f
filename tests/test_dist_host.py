"""Multi-process paths of bench.py on the CPU (gloo, world size 2): the replica aggregation (sum of
iterations over ranks, slowest rank's time) and the reference arm printing one line from rank 0."""

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_init(None)
    bench.barrier(w)
    total = bench.reduce(w, 10.0 * (r + 1), "sum")      # iterations of every rank
    slowest = bench.reduce(w, 1.0 + r, "max")           # each rank's milliseconds
    out.put((r, w, total, slowest))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for r, w, total, slowest in res:
        assert w == 2
        assert total == 30.0          # 10 + 20 iterations
        assert slowest == 2.0         # the slower rank's time


def test_reference_arm_prints_once_under_torchrun():
    pytest.importorskip("torch")
    env = dict(os.environ, BENCH_REF_ITERS="2", OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    res = subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_kernel_model_covers_every_phase():
    """Every phase name the library reports gets a nonzero algorithmic-work model in bench.py (a
    missing name would put a zero into the roofline line)."""
    import bench
    sizes = dict(s_list=[30] * 100, p=100, nEL=25710, SL=46500, m=200, nnz=1542600, n_cone=1000)
    names = ["project_dual", "project_primal", "project_cones", "scatter_dual", "scatter_primal",
             "scatter_primal+finalize", "spmv_rows", "solve_y", "spmv_cols", "update_dual",
             "update_dual+finalize"]
    for name in names:
        bound, amount, unit = bench.kernel_model(name, sizes, {}, "fp32")
        assert amount > 0, name
        assert (bound, unit) in (("alu", "flop"), ("hbm", "byte")), name
    assert bench.kernel_model("project_cones", sizes, {}, "fp32")[0] == "hbm"
