"""Host logic of the multi-GPU benchmark path, run as two gloo ranks on CPU:
the step time is the maximum over ranks, each rank draws its own query seed,
and the oracle arm prints from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = [0.25, 0.75][rank]
        tmax = bench.max_over_ranks(t, dist, torch.device("cpu"))
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.rank_seed(1, rank))
        with open(os.path.join(outdir, "rank%d.json" % rank), "w") as f:
            json.dump({"tmax": tmax, "seeds": seeds}, f)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_seeds_two_gloo_ranks(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(world)]
    for r in res:
        assert r["tmax"] == 0.75
        assert len(set(r["seeds"])) == world  # independent query sets
    assert res[0]["seeds"] == res[1]["seeds"]


def test_max_over_ranks_single_process():
    assert bench.max_over_ranks(1.5, None, None) == 1.5


def test_reference_arm_is_silent_on_other_ranks():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def _split_main(rank, world, port, outdir):
    """Each rank evaluates its contiguous, cost-balanced range of one work list
    (a deterministic stand-in for the GPU integration: value = position index
    times 1.5, so that the gathered order is checkable) and all-gathers."""
    import numpy as np

    from paper_2501_03322_gb300 import shard

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 1001
        rng = np.random.default_rng(7)
        costs = rng.integers(64, 4096, n).astype(float)  # previous run's limb samples
        out, bounds = shard.run_sharded(n, lambda lo, hi: torch.arange(lo, hi, dtype=torch.float64) * 1.5, dist,
                                        costs=costs, device=torch.device("cpu"))
        with open(os.path.join(outdir, "split%d.json" % rank), "w") as f:
            json.dump({"out": out.tolist(), "bounds": bounds.tolist()}, f)
    finally:
        dist.destroy_process_group()


def test_split_one_workload_two_gloo_ranks(tmp_path):
    """A cost-balanced contiguous partition of one work list over two ranks,
    gathered back: every rank receives the single-rank result in the
    single-rank order, and the two ranges carry equal predicted cost to within
    one position's cost."""
    import numpy as np

    from paper_2501_03322_gb300 import shard

    world = 2
    mp.spawn(_split_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / ("split%d.json" % r))) for r in range(world)]
    expect = (np.arange(1001) * 1.5).tolist()
    for r in res:
        assert r["out"] == expect
        assert r["bounds"] == res[0]["bounds"]
    costs = np.random.default_rng(7).integers(64, 4096, 1001).astype(float)
    b = res[0]["bounds"]
    loads = [costs[b[i]:b[i + 1]].sum() for i in range(world)]
    assert abs(loads[0] - loads[1]) <= costs.max()


def test_balanced_bounds_properties():
    import numpy as np

    from paper_2501_03322_gb300 import shard

    assert shard.balanced_bounds(10, 3).tolist() == [0, 3, 6, 10]
    assert shard.balanced_bounds(0, 4).tolist() == [0, 0, 0, 0, 0]
    c = np.r_[np.full(100, 1.0), np.full(10, 100.0)]  # a costly tail
    b = shard.balanced_bounds(c, 2)
    assert b[0] == 0 and b[-1] == c.size and 100 <= b[1] <= 106
    for k in (1, 2, 3, 8, 200):
        bb = shard.balanced_bounds(np.random.default_rng(k).random(150), k)
        assert bb[0] == 0 and bb[-1] == 150 and (np.diff(bb) >= 0).all() and len(bb) == k + 1
    with pytest.raises(ValueError):
        shard.balanced_bounds(np.array([1.0, -1.0]), 2)
