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
