"""The multi-rank path of bench.py on CPU (gloo, world size 2).

Every workload here is independent problems, so N GPUs run N replicas with no
data-path collective: each rank takes its own share of the work, the timing
is the slowest rank's, and the reported throughput is the node updates of all
ranks over that time.  These tests run the ranks as CPU processes over gloo:
the sharding covers every item exactly once, the reductions give the max and
the sum, per-rank lists gather in rank order, and a torchrun launch of the
reference arm prints exactly one JSON line (rank 0) with every rank exiting 0.
"""
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


def rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_env()
    dist = bench.init_dist(w, "gloo")
    out = {
        "env": (w, r),
        "max": bench.max_over_ranks(dist, 1.5 + r),
        "sum": bench.sum_over_ranks(dist, 10.0 * (r + 1)),
        "shard": bench.shard(range(7), r, w),
        "gathered": bench.gather_lists(dist, [f"r{r}a", f"r{r}b"][: r + 1]),
    }
    bench.barrier(dist)
    dist.destroy_process_group()
    q.put((rank, out))


def test_replica_helpers_over_gloo():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        assert res[r]["env"] == (2, r)
        assert res[r]["max"] == 2.5                      # slowest rank
        assert res[r]["sum"] == 30.0                     # work of all ranks
        assert res[r]["gathered"] == ["r0a", "r1a", "r1b"]
    shares = res[0]["shard"] + res[1]["shard"]
    assert sorted(shares) == list(range(7)) and not set(res[0]["shard"]) & set(res[1]["shard"])


def test_single_rank_helpers_are_identities():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 3.0) == 3.0
    assert bench.sum_over_ranks(None, 3.0) == 3.0
    assert bench.gather_lists(None, (1, 2)) == [1, 2]
    assert bench.shard([5, 6, 7], 0, 1) == [5, 6, 7]


def test_torchrun_reference_arm_prints_one_line():
    pytest.importorskip("torch")
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
