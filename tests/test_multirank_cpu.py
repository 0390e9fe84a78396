"""The N > 1 launch path of bench.py on CPU: the timing maximum over two gloo
ranks, the per-rank seeds of the uneven-batch workload (independent populations
there; the DE batch shards one population, see test_shard_cpu.py), and the
reference arm under torchrun."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    local_ms = 100.0 + 50.0 * rank
    m = bench.max_over_ranks(local_ms, dist, "cpu")
    seeds = bench.rank_seeds(r)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ws, m, seeds, bench.throughput(ws, 64, 5, m)))


def test_two_gloo_ranks_share_only_the_timing_maximum():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ws0, m0, s0, v0), (r1, ws1, m1, s1, v1) = res
    assert ws0 == ws1 == 2
    assert m0 == m1 == 150.0
    assert s0 != s1 and s0[0] != s1[0] and s0[1] != s1[1]
    # weak scaling: 2 ranks x 64 candidates x 5 steps in the slowest rank's time
    assert abs(v0 - 2 * 64 * 5 / 0.150) < 1e-9 and v0 == v1


def test_single_process_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.dist_env()[0] >= 1


def test_reference_arm_under_torchrun_prints_one_line():
    """bench.py --impl reference launched under torchrun with two ranks: rank 0 times
    the oracle and prints one JSON line, the other rank exits 0 without work."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1",
           "--cpu-modes", "256"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
