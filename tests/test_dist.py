"""The multi-process path of bench.py on CPU: gloo ranks for the reductions
and the replica throughput, and a torchrun launch of the reference arm
(rank 0 alone measures and prints)."""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    w, r, _ = bench._dist_setup()
    slowest = bench._max_over_ranks(10.0 * (rank + 1), w)  # per-rank total ms
    total = bench._sum_over_ranks(1.0 + rank, w)
    value = bench.replica_throughput(w, 5, 1000, slowest)
    q.put((r, w, dist.get_backend(), slowest, total, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_scale():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1]
    for r, w, backend, slowest, total, value in got:
        assert w == 2 and backend == "gloo"
        assert slowest == 20.0  # the job takes the slowest rank's time
        assert total == 3.0
        # two replicas, 5 steps of 1000 units each, in 20 ms
        assert value == pytest.approx(2 * 5 * 1000 / 0.020)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(7.5, 1) == 7.5
    assert bench.replica_throughput(1, 20, 100, 2.0) == pytest.approx(1e6)


def test_torchrun_reference_arm_prints_once():
    """Under torchrun with two ranks, `--impl reference` runs on rank 0 only:
    one JSON line, both ranks exit 0."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--workload", "er10k", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
