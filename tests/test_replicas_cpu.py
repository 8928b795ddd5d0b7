"""The multi-rank host logic of the replica-parallel runs, with the gloo
backend on CPU (world size 2): distinct seeds, a partition of the units, the
maximum of the ranks' times, and the reference arm printing on rank 0 only."""
import json
import os
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1704_03329_b300.replicas import barrier, max_over_ranks, rank_info, rank_seed, shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = rank_info()
    barrier(cuda=False)
    t = max_over_ranks(0.5 + r)
    lo, hi = shard(11, r, w)
    out.put((r, w, lr, rank_seed(2, r), t, lo, hi))
    barrier(cuda=False)
    dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1] and all(x[1] == 2 for x in res)
    assert res[0][3] != res[1][3]            # distinct workloads
    assert all(x[4] == 1.5 for x in res)     # the slowest rank's time everywhere
    assert res[0][5:] == (0, 6) and res[1][5:] == (6, 11)  # a partition of the 11 units


def test_shard_partitions():
    from paper_1704_03329_b300.replicas import shard
    for n in (0, 1, 7, 256):
        for w in (1, 2, 3, 8):
            blocks = [shard(n, r, w) for r in range(w)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            assert all(blocks[k][1] == blocks[k + 1][0] for k in range(w - 1))
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1


def test_reference_arm_prints_on_rank_0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--cpu-cells", "8",
                        "--cpu-steps", "1"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line_on_rank_0():
    """Rank 0 prints one JSON line: the oracle on this arm's workload, the
    requested steps and warm-up, with its cpu_baseline and e2e entries."""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--cpu-cells", "6",
                        "--steps", "3", "--warmup", "1"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 3 and d["warmup"] == 1 and d["value"] > 0
    assert d["config"]["atoms"] == 4 * 63 ** 3 and d["config"]["sample_atoms"] == 4 * 6 ** 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
