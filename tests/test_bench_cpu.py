"""Host logic of the benchmark: launch counting, the FLOP model by precision,
and the lookup of DRAM traffic in the committed ncu summaries."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_launch_count():
    assert bench.gpu_launches({"kind": "mag", "n": 262144}, 5) == 10  # main + repair pass per step
    wl = {"kind": "surrogate", "n": 10_000_000,
          "nfb": [{"fallback": 5, "network": 0, "expansion": 1}, {"fallback": 0, "network": 0, "expansion": 1}]}
    # 10 chunks x 6 kernels, plus the contour pair only when something fell back
    assert bench.gpu_launches(wl, 2) == (60 + 2) + 60


def test_flop_model_splits_precisions():
    w = dict(samples=1000, sweeps64=2000, sweeps32=0, edges=1000, newton64=0)
    f64, f32 = bench.flops_of(w, "fp64")
    assert f64 == 1000 * bench.F_SAMPLE64 + 2000 * bench.F_SWEEP64 + 1000 * bench.F_EDGE64
    assert f32 == 1000 * bench.F_SAMPLE32 + 2000 * bench.F_SWEEP64_FP32 + 1000 * bench.F_EDGE32
    w = dict(samples=1000, sweeps64=1000, sweeps32=2000, edges=1000, newton64=0)
    f64m, f32m = bench.flops_of(w, "mixed")
    assert f64m < f64 and f32m > f32  # the FP32 sweeps move work to the FP32 side


def test_profile_summaries_parse():
    # every committed contour summary carries the fields the lookup needs;
    # the figure is used only while its source hash matches the kernel sources
    names = [f for f in os.listdir(os.path.join(ROOT, "profiles")) if f.startswith("contour_")]
    assert names
    for f in names:
        txt = open(os.path.join(ROOT, "profiles", f)).read()
        assert "dram_bytes_per_launch_scaled = `" in txt and "source_sha = `" in txt, f
    t = bench.profile_traffic("surrogate", "mixed")
    assert t is None or t > 0
    assert bench.profile_traffic("no_such_workload", "mixed") is None


def test_config_names_the_workload():
    wl = bench.workload("map_planetary")
    cfg = bench.config_of(wl, "mixed", 1)
    assert cfg["workload"] == "map_planetary_512x512" and cfg["positions_per_gpu"] == 512 * 512
    assert cfg["parallelism"] == "dp1" and "l2" in cfg
