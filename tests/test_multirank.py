"""The N > 1 launch of bench.py (one process per GPU, replicas of the workload, weak
scaling) exercised on CPU with the gloo backend, two ranks: the reductions behind the JSON
line's value (the maximum of the ranks' times, the sum of their particle-steps) and the
reference arm under torch.distributed.run (rank 0 alone prints one line, every rank exits 0)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    ws_, rank_, _ = bench.dist_init()
    bench.barrier(ws_)
    tmax = bench.allreduce_max(ws_, 1.5 + rank_, "cpu")     # per-rank times
    units = bench.allreduce_sum(ws_, 1000.0 * (rank_ + 1), "cpu")  # per-rank particle-steps
    bench.barrier(ws_)
    q.put((rank_, ws_, dist.get_backend(), tmax, units))
    dist.destroy_process_group()


def test_rank_reductions_over_gloo():
    torch = pytest.importorskip("torch")
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    for _, ws, backend, tmax, units in res:
        assert ws == 2 and backend == "gloo"
        assert tmax == 2.5           # the slowest rank's time
        assert units == 3000.0       # both ranks' particle-steps: value = units / tmax


def test_reference_arm_under_torchrun_two_ranks():
    pytest.importorskip("torch")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--ref-frac", "0.05", "--workload", "wald64"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
