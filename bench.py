#!/usr/bin/env python
"""Throughput benchmark: finite-source magnifications per second on GB300.

One step = one call of the C ABI over the whole workload (every position
answered to rel_tol), inputs resident in device memory.  Default workload:
surrogate + fallback on 1e7 fresh queries near caustics (log10 s ~ U[-0.5,
0.5], log10 q ~ U[-5, -1], log10 rho ~ U[-4, -2]; network trained once on 1e7
contour-integrated samples before timing), rel_tol=1e-4, mixed-precision
fallback (FP32 root iterations, FP64 polish, coefficients, residuals and
areas), with the plain contour integration of the same queries timed beside
it.  Other
workloads: the 512 x 512 planetary-caustic map, the central-caustic light
curve, 4096 batched light curves, the resonant large source.  Prints one
JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--mode fp64|mixed]
    python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Multi-GPU (torchrun, one rank per GPU): every rank integrates a workload of
the same size (the surrogate workload draws each rank's queries from its own
seed; the fixed-lens workloads are replicas), with no collective on the data
path (weak scaling); the step time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# ---------------------------------------------------------------- FLOP model
# Algorithmic FLOPs of the method per unit of work counted by the kernel
# (tw_last_launch_work), split by the precision each part runs in.  Counting
# rules: real add/mul 1, complex add 2, complex mul 6, complex multiply-add 8,
# reciprocal/division/square root 1.
#   one Aberth sweep (five roots), FP64 mode: Horner p (5 multiply-adds) and
#     p' (4) per root (5 x 72), the denominator p' - p S (5 x 8), the
#     division (5 x 12) and the update (5 x 2) in FP64: 470; the ten pair
#     reciprocals 1/(z_i - z_j) with their sums (10 x 17) and the convergence
#     magnitudes (5 x 10) in FP32: 220
#   one Aberth sweep in FP32 (mixed mode): all of it, 690
#   one limb sample outside the sweeps: limb point (8), Eq. 6 coefficients
#     (~100) and per root the two lens reciprocals, f(z) and the residual R
#     (5 x 23) in FP64: ~225; f', J, dz/dtheta, f'' and z' ^ z'' in FP32
#     (5 x 45): 225
#   one FP64 Newton pass over the five roots (kept for the work counter,
#     which stays zero): 5 x 94 = 470
#   one edge: image linking distances and 3-5 links of trapezium + parabolic
#     correction + four error terms: ~145 (FP64), ~20 (FP32)
# Feature kernel of the surrogate (point images at the query centre and at 24
# ring points, caustic sweep): per point solve outside its sweeps, Eq. 6
# coefficients (~100), their FP32 scaling (12) and per root the two lens
# reciprocals, the residual and f', J (5 x 47) in FP64: ~357, and ~30 FP32;
# per FP32 Aberth sweep 690 (as above); per FP64 Newton root step Horner p and
# p' (72), the division (12) and the update (2): 86; per Aberth iteration of
# the caustic quartic in FP32, six pair reciprocals with their sums (6 x 13)
# and four roots of Horner, division and magnitudes (4 x 85) plus the update:
# ~430.
F_FEAT_SOLVE64 = 357.0
F_FEAT_SOLVE32 = 30.0
F_FEAT_NEWTON64 = 86.0
F_CAUSTIC32 = 430.0
F_SWEEP64 = 470.0
F_SWEEP64_FP32 = 220.0
F_SWEEP32 = 690.0
F_SAMPLE64 = 225.0
F_SAMPLE32 = 225.0
F_NEWTON64 = 470.0
F_EDGE64 = 145.0
F_EDGE32 = 20.0
# Nominal peaks (FLOP/s), context only: FP64 GB300's nominal 1.25 TFLOP/s (152
# SMs x 2.07 GHz x 2 FP64 FMA per clock per SM x 2 FLOP); FP32 152 SMs x 128
# lanes x 2 FLOP x 2.07 GHz.  These unit-count peaks are the roofline's
# denominators; the FMA-chain probe (tw_peak_probe) is reported beside them
# (all SMs running FP64 FMAs draw enough power to lower the clock, to about
# 1.06 TFLOP/s).  The tensor-core GEMM uses the bf16 peak of
# MEASURED_PEAKS.json (sustained: the GEMMs run inside a seconds-long step).
NOMINAL_FP64 = 1.25e12
NOMINAL_FP32 = 152 * 128 * 2 * 2.07e9


def workload(name):
    from paper_2501_03322_gb300 import workloads as W

    if name == "map_planetary":
        c = W.MAP_PLANETARY
        y1, y2 = W.map_grid()
        return dict(kind="mag", name="map_planetary_512x512", s=c["s"], q=c["q"], rho=c["rho"], y1=y1, y2=y2,
                    rel_tol=c["rel_tol"], n=y1.size)
    if name == "lightcurve_central":
        c = W.LIGHTCURVE_CENTRAL
        t = W.lightcurve_central_times(c["n"])
        return dict(kind="lc", name="lightcurve_central_1000", times=t, n=t.size, **{k: c[k] for k in
                    ("s", "q", "rho", "u0", "alpha", "t0", "tE", "rel_tol")})
    if name == "stress_resonant":
        c = W.STRESS_RESONANT
        y1, y2 = W.stress_positions()
        return dict(kind="mag", name="stress_resonant_1e6", s=c["s"], q=c["q"], rho=c["rho"], y1=y1, y2=y2,
                    rel_tol=c["rel_tol"], n=y1.size)
    if name == "surrogate":
        return dict(kind="surrogate", name="surrogate_fallback_1e7", n=10_000_000, ntrain=10_000_000, epochs=30,
                    seed_train=0, seed_query=1, rel_tol=1e-4, kappa=3.0)
    if name == "batch_lightcurves":
        params, offsets, times = W.batch_lightcurves()
        return dict(kind="batch", name="batch_lightcurves_4096", params=params, offsets=offsets, times=times,
                    rel_tol=W.BATCH_LIGHTCURVES["rel_tol"], n=times.size)
    if name in W.FIG4:
        c = W.FIG4[name]
        y1, y2 = W.fig4_grid(name)
        return dict(kind="mag", name=name + "_480x340", s=c["s"], q=c["q"], rho=c["rho"], y1=y1, y2=y2, rel_tol=1e-4,
                    n=y1.size, golden="fig4_maps.txt", golden_map=name)
    if name == "fig6_sweep":
        a = W.fig6_sweep()
        return dict(kind="multi", name="fig6_sweep_64x900", arrays=a, rel_tol=1e-4, n=a[0].size)
    raise SystemExit("unknown workload " + name)


def config_of(wl, mode, n_gpus):
    cfg = {"workload": wl["name"], "positions_per_gpu": int(wl["n"]), "rel_tol": wl["rel_tol"], "mode": mode,
           "parallelism": "dp%d" % n_gpus, "l2": "flushed between timed steps (256 MiB write)"}
    for k in ("s", "q", "rho"):
        if k in wl:
            cfg[k] = wl[k]
    return cfg


KERNEL_SOURCES = ("cx.cuh", "lens.cuh", "contour.cuh", "kernels.cuh", "k_fp64_spl1.cu", "k_fp64_spl2.cu",
                  "k_fp64_spl4.cu", "k_mixed_spl1.cu", "k_mixed_spl2.cu", "k_mixed_spl4.cu", "k_fp64_spl2_o4.cu",
                  "k_mixed_spl2_o4.cu", "k_fp64_repair.cu", "k_mixed_repair.cu", "k_fp64_w2.cu", "k_fp64_w4.cu",
                  "k_mixed_w2.cu", "k_mixed_w4.cu")


def sources_sha():
    """Hash of the contour kernel's device sources (host runtime excluded)."""
    h = hashlib.sha256()
    cs = os.path.join(ROOT, "paper_2501_03322_gb300", "csrc")
    for fn in KERNEL_SOURCES:
        h.update(open(os.path.join(cs, fn), "rb").read())
    return h.hexdigest()[:16]


def profile_traffic(wl_name, mode):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    from the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "contour_%s_%s.md" % (mode, wl_name))
    if not os.path.exists(path):
        return None
    vals = {}
    for ln in open(path):
        if "=" in ln and ln.strip().startswith("- "):
            k, v = ln.strip()[2:].split("=", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_sha") != sources_sha():
        return None
    try:
        return float(vals["dram_bytes_per_launch_scaled"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def flops_of(work, mode):
    f64 = (F_SAMPLE64 * work["samples"] + F_SWEEP64 * work["sweeps64"] + F_EDGE64 * work["edges"]
           + F_NEWTON64 * work["newton64"])
    f32 = (F_SAMPLE32 * work["samples"] + F_SWEEP64_FP32 * work["sweeps64"] + F_SWEEP32 * work["sweeps32"]
           + F_EDGE32 * work["edges"])
    return f64, f32


GOLD = os.path.join(ROOT, "tests", "golden")


def golden_rows(name):
    """Rows of a stored oracle file (tests/golden, written by the oracle only)."""
    return [ln.split() for ln in open(os.path.join(GOLD, name)) if not ln.startswith("#") and ln.strip()]


def golden_errors(wl, prec, P, wpath=None):
    """Relative error of the GPU path against the oracle's stored values on the
    workload's golden positions, in the benchmark's call path and mode: max,
    99.9th percentile, the fraction of positions whose error estimate bounds
    the true error (contour paths), and the number of positions compared."""
    from paper_2501_03322_gb300 import workloads as W

    err_est = None
    extra = {}
    if wl["kind"] == "surrogate":
        a = np.array([[float(v) for v in r[:7]] for r in golden_rows("surrogate_queries.txt") +
                      golden_rows("surrogate_band.txt")])
        a = a[a[:, 6] == 0]
        stat = np.zeros(len(a), np.int8)
        got, _ = P.surrogate_mag(wpath, *[a[:, k].copy() for k in range(5)], rel_tol=wl["rel_tol"],
                                 kappa=wl["kappa"], precision=prec, status=stat)
        ref, name = a[:, 5], "surrogate_queries.txt+surrogate_band.txt"
        net = stat == P.POS_NETWORK
        if net.any():
            extra = {"network_answered": int(net.sum()), "network_max_rel_err": float(np.abs(got[net] / ref[net] - 1).max())}
    elif wl["kind"] == "multi":
        name = "fig6_sweep.txt"
        a = np.array([[float(v) for v in r[1:8]] for r in golden_rows(name)])
        a = a[a[:, 6] == 0]
        got, err_est, _, _ = P.mag_multi(*[a[:, k].copy() for k in range(5)], rel_tol=wl["rel_tol"], precision=prec,
                                         details=True)
        ref = a[:, 5]
    elif wl["kind"] == "mag" and wl.get("golden_map"):
        name = wl["golden"]
        rows = [r for r in golden_rows(name) if r[0] == wl["golden_map"] and int(r[5]) == 0]
        y1 = np.array([float(r[2]) for r in rows])
        y2 = np.array([float(r[3]) for r in rows])
        ref = np.array([float(r[4]) for r in rows])
        got, err_est, _, _ = P.mag(wl["s"], wl["q"], wl["rho"], y1, y2, rel_tol=wl["rel_tol"], precision=prec,
                                   details=True)
    elif wl["kind"] == "mag":
        name = "stress_resonant_1e4.txt" if wl["name"].startswith("stress") else "map_planetary.txt"
        rows = [r for r in golden_rows(name) if int(r[4]) == 0]
        y1 = np.array([float(r[1]) for r in rows])
        y2 = np.array([float(r[2]) for r in rows])
        ref = np.array([float(r[3]) for r in rows])
        got, err_est, _, _ = P.mag(wl["s"], wl["q"], wl["rho"], y1, y2, rel_tol=wl["rel_tol"], precision=prec,
                                   details=True)
    elif wl["kind"] == "lc":
        name = "lightcurve_central.txt"
        rows = [r for r in golden_rows(name) if int(r[2]) == 0]
        t = np.array([float(r[0]) for r in rows])
        ref = np.array([float(r[1]) for r in rows])
        got, err_est, _, _ = P.lightcurve(wl["s"], wl["q"], wl["rho"], wl["u0"], wl["alpha"], wl["t0"], wl["tE"], t,
                                          rel_tol=wl["rel_tol"], precision=prec, details=True)
    else:
        name = "batch_lightcurves.txt"
        rows = [r for r in golden_rows(name) if int(r[4]) == 0]
        curves = np.array([int(r[0]) for r in rows])
        t = np.array([float(r[2]) for r in rows])
        ref = np.array([float(r[3]) for r in rows])
        # the golden points as a batch of their own curves, one time each
        params = wl["params"][curves]
        offsets = np.arange(len(rows) + 1, dtype=np.int64)
        got, err_est, _, _ = P.lightcurve_batch(params, offsets, t, rel_tol=wl["rel_tol"], precision=prec,
                                                details=True)
    rel = np.abs(np.asarray(got) / ref - 1.0)
    out = {"golden": name, "positions": int(rel.size), "max_rel_err": float(rel.max()),
           "p999_rel_err": float(np.quantile(rel, 0.999)), "rel_tol": wl["rel_tol"], **extra}
    if err_est is not None:
        out["estimate_bounds_error"] = float(np.mean(np.abs(np.asarray(got) - ref) <= np.asarray(err_est)
                                                     + 1e-12 * ref))
    return out


def cpu_oracle_sample(wl, k, seed=777, cores=None):
    """Time the CPU oracle on k positions of the workload on `cores` host
    threads (all by default).  Surrogate queries are drawn on the CPU from the
    benchmark's own distribution (oracle.sample_near_caustic); every other
    workload uses a seeded subset of its own positions."""
    import concurrent.futures as cf

    import oracle as O
    from paper_2501_03322_gb300 import workloads as W

    cores = cores or os.cpu_count() or 1
    if wl["kind"] == "surrogate":
        # one lens per query: spread the queries over the cores
        a = np.array(O.sample_near_caustic(k, seed)).T
        t0 = time.perf_counter()
        with cf.ThreadPoolExecutor(max_workers=cores) as ex:
            list(ex.map(lambda r: O.mag(r[0], r[1], r[2], [r[3]], [r[4]], nthreads=1), a))
        return len(a), time.perf_counter() - t0, cores
    idx = W.sample_indices(int(wl["n"]), k, seed=seed)
    if wl["kind"] == "multi":  # per-position lens: spread the positions over the cores
        a = np.array([x[idx] for x in wl["arrays"]]).T
        t0 = time.perf_counter()
        with cf.ThreadPoolExecutor(max_workers=cores) as ex:
            list(ex.map(lambda r: O.mag(r[0], r[1], r[2], [r[3]], [r[4]], nthreads=1), a))
        return len(a), time.perf_counter() - t0, cores
    t0 = time.perf_counter()
    if wl["kind"] == "mag":
        O.mag(wl["s"], wl["q"], wl["rho"], wl["y1"][idx], wl["y2"][idx], nthreads=cores)
    elif wl["kind"] == "lc":
        O.lightcurve(wl["s"], wl["q"], wl["rho"], wl["u0"], wl["alpha"], wl["t0"], wl["tE"], wl["times"][idx],
                     nthreads=cores)
    else:
        offs = wl["offsets"]
        curve = np.searchsorted(offs, idx, side="right") - 1
        for k_c in np.unique(curve):
            s, q, rho, u0, al, t0_, tE = wl["params"][k_c]
            O.lightcurve(s, q, rho, u0, al, t0_, tE, wl["times"][idx[curve == k_c]], nthreads=cores)
    dt = time.perf_counter() - t0
    return len(idx), dt, cores


def launched_contour(wl):
    """Whether the last step launched the contour kernel (a surrogate step whose
    queries were all answered without contour integration launches none)."""
    if wl.get("gate"):
        return bool(wl["ncontour"]) and wl["ncontour"][-1] > 0
    return wl["kind"] != "surrogate" or (wl["nfb"] and wl["nfb"][-1]["fallback"] > 0)


def gpu_launches(wl, steps):
    """Kernels of this library launched in the timed steps: a contour
    integration is two launches (the main pass and the slope-repair pass over
    the positions it queued, usually none); a gated step launches the feature
    and gate kernels per chunk of 2^20 positions; a surrogate step launches, per
    chunk of 2^20 queries, the feature, input-layer, three tensor-core GEMM and
    head kernels, then contour integration of its fallbacks (when there are
    any)."""
    chunks = (wl["n"] + (1 << 20) - 1) >> 20
    if wl.get("gate"):  # feature and gate kernels per chunk, then the contour pair
        return sum(2 * chunks + (2 if nc > 0 else 0) for nc in wl["ncontour"][-steps:])
    if wl["kind"] != "surrogate":
        return 2 * steps
    return sum(6 * chunks + (2 if c["fallback"] > 0 else 0) for c in wl["nfb"][-steps:])


def load_peaks():
    """MEASURED_PEAKS.json (driver-written), or {} when absent."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except (OSError, ValueError):
        return {}


def max_over_ranks(x, dist, device):
    """Largest value of x over all ranks (x itself when dist is None)."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed(base, rank):
    """Seed of this rank's query set: ranks integrate independent queries."""
    return int(base) + 7919 * int(rank)


def run_reference(args, wl, cfg, metric, unit):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    k = args.ref_sample
    times = []
    for i in range(args.warmup + args.steps):
        n, dt, cores = cpu_oracle_sample(wl, k, seed=1000 + i)
        if i >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = k * len(times) / tot
    line = {"impl": "reference", "metric": metric, "value": value, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "binary128",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle",
                             "sample": "%d positions of the workload per step (seeded), all host cores" % k},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="surrogate",
                    choices=["map_planetary", "lightcurve_central", "stress_resonant", "batch_lightcurves",
                             "surrogate", "fig4_s05", "fig4_s1", "fig4_s3", "fig6_sweep"])
    ap.add_argument("--mode", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--cpu-sample", type=int, default=64, help="positions in the CPU oracle baseline sample")
    ap.add_argument("--ref-sample", type=int, default=24, help="positions per step of the reference arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--train-samples", type=int, default=0, help="surrogate workload: training positions")
    ap.add_argument("--queries", type=int, default=0, help="surrogate workload: query positions")
    ap.add_argument("--autotune", action="store_true", help="let the library choose the launch shape")
    ap.add_argument("--graph", action="store_true", help="replay each launch from a CUDA graph")
    ap.add_argument("--gate", action="store_true",
                    help="single-lens workloads: point-source adequacy gate (tw_mag_gated) before contour integration")
    ap.add_argument("--split", action="store_true",
                    help="single-lens workloads: split the one workload across the ranks (strong scaling)")
    ap.add_argument("--limit", type=int, default=0,
                    help="use a seeded sub-sample of this many positions (small profiling captures)")
    args = ap.parse_args()

    metric = "finite-source mags/sec at rel.err<=1e-4: surrogate+fallback vs plain, 1 GB300"
    unit = "mags/s"
    wl = workload(args.workload)
    if wl["kind"] == "surrogate":
        if args.train_samples:
            wl["ntrain"] = args.train_samples
        if args.queries:
            wl["n"] = args.queries
    if args.limit and wl["kind"] == "mag" and args.limit < wl["n"]:
        from paper_2501_03322_gb300 import workloads as W

        idx = W.sample_indices(wl["n"], args.limit, seed=4242)
        wl.update(y1=wl["y1"][idx], y2=wl["y2"][idx], n=idx.size, name=wl["name"] + "_sub%d" % idx.size)
    cfg = config_of(wl, args.mode, args.gpus)
    cfg["autotune"] = bool(args.autotune)
    cfg["graph"] = bool(args.graph)
    if args.split:
        if wl["kind"] != "mag" or args.gate:
            raise SystemExit("--split applies to the single-lens position workloads without --gate")
        cfg["split"] = "contiguous ranges balanced by the previous step's limb samples, all-gathered"
        cfg["parallelism"] = "split%d" % args.gpus
    if args.gate:
        if wl["kind"] != "mag":
            raise SystemExit("--gate applies to the single-lens position workloads")
        cfg["gate"] = True
        wl["gate"] = True
    if args.impl == "reference":
        run_reference(args, wl, cfg, metric, unit)
        return

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_2501_03322_gb300 as P

    prec = P.PREC_FP64 if args.mode == "fp64" else P.PREC_MIXED
    if args.graph:  # graph capture needs a stream other than the legacy default one
        torch.cuda.set_stream(torch.cuda.Stream(dev))
    stream = torch.cuda.current_stream(dev)
    kw = dict(precision=prec, autotune=args.autotune, use_graph=args.graph)

    def D(a, dt=torch.float64):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)

    if wl["kind"] == "mag" and wl.get("gate"):
        y1d, y2d = D(wl["y1"]), D(wl["y2"])
        sd, qd_, rd = (torch.full_like(y1d, wl[k]) for k in ("s", "q", "rho"))
        outd = torch.empty_like(y1d)
        wl["ncontour"] = []

        def step():
            _, nc = P.mag_gated(sd, qd_, rd, y1d, y2d, rel_tol=wl["rel_tol"], precision=prec, out=outd)
            wl["ncontour"].append(nc)
    elif wl["kind"] == "mag" and args.split:
        # one workload split across the ranks (strong scaling): contiguous
        # ranges balanced by the limb samples of the previous step, results
        # all-gathered (paper_2501_03322_gb300.shard)
        from paper_2501_03322_gb300 import shard

        y1d, y2d = D(wl["y1"]), D(wl["y2"])
        wl["costs"] = None

        def step():
            def compute(lo, hi):
                mu, _, ns, _ = P.mag(wl["s"], wl["q"], wl["rho"], y1d[lo:hi], y2d[lo:hi], rel_tol=wl["rel_tol"],
                                     details=True, **kw)
                wl["ns"] = ns.to(torch.float64)
                return mu

            if dist is None:
                out, bounds = compute(0, wl["n"]), np.array([0, wl["n"]])
                wl["costs"] = wl["ns"].cpu().numpy()
            else:
                out, bounds = shard.run_sharded(wl["n"], compute, dist, costs=wl["costs"], device=dev)
                wl["costs"] = shard.gather(wl["ns"], bounds, dist, dev).cpu().numpy()
            wl["out"] = out
            wl["bounds"] = bounds
    elif wl["kind"] == "mag":
        y1d, y2d = D(wl["y1"]), D(wl["y2"])
        outd = torch.empty_like(y1d)

        def step():
            P.mag(wl["s"], wl["q"], wl["rho"], y1d, y2d, rel_tol=wl["rel_tol"], out=outd, **kw)
    elif wl["kind"] == "multi":
        md = [D(a) for a in wl["arrays"]]
        outd = torch.empty_like(md[0])

        def step():
            P.mag_multi(*md, rel_tol=wl["rel_tol"], out=outd, **kw)
    elif wl["kind"] == "lc":
        td = D(wl["times"])
        outd = torch.empty_like(td)

        def step():
            P.lightcurve(wl["s"], wl["q"], wl["rho"], wl["u0"], wl["alpha"], wl["t0"], wl["tE"], td,
                         rel_tol=wl["rel_tol"], out=outd, **kw)
    elif wl["kind"] == "batch":
        pd, od, td = D(wl["params"]), D(wl["offsets"], torch.int64), D(wl["times"])
        outd = torch.empty_like(td)

        def step():
            P.lightcurve_batch(pd, od, td, rel_tol=wl["rel_tol"], out=outd, **kw)
    else:
        wpath = os.path.join(ROOT, "paper_2501_03322_gb300", "_build",
                             "surrogate_v2_s%d_n%d_e%d.bin" % (wl["seed_train"], wl["ntrain"], wl["epochs"]))
        t0 = time.perf_counter()
        if rank == 0 and not os.path.exists(wpath):  # one training run; the other ranks read its weights
            wl["train_stats"] = P.surrogate_train(wpath, wl["ntrain"], wl["seed_train"], wl["epochs"])
        if dist:
            dist.barrier()
        wl["train_s"] = time.perf_counter() - t0
        qd = P.surrogate_sample(rank_seed(wl["seed_query"], rank), wl["n"], device=dev)
        outd = torch.empty(wl["n"], dtype=torch.float64, device=dev)
        wl["nfb"] = []

        wl["sur_stats"] = []

        def step():
            _, cnt = P.surrogate_mag(wpath, *qd, rel_tol=wl["rel_tol"], kappa=wl["kappa"], precision=prec, out=outd,
                                     details=True)
            wl["nfb"].append(cnt)
            wl["sur_stats"].append(P.last_surrogate_stats())

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    f64 = f32 = 0.0
    kern_ms = []
    work = dict(samples=0, sweeps64=0, sweeps32=0, edges=0, newton64=0)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
        evs[i][1].synchronize()
        kern_ms.append(P.last_launch_ms() if launched_contour(wl) else 0.0)
        w = P.last_launch_work()
        for k in work:
            work[k] += w[k]
        a, b = flops_of(w, args.mode)
        f64 += a
        f32 += b
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    ms = [s.elapsed_time(e) for s, e in evs]
    t_step = sum(ms) / len(ms) / 1e3
    t_step = max_over_ranks(t_step, dist, dev)
    if dist:
        dist.barrier()
    value = (1 if args.split else world) * wl["n"] / t_step
    extra = {}
    if wl.get("gate"):
        extra = {"gate": {"contour_fraction": sum(wl["ncontour"][-args.steps:]) / (args.steps * wl["n"])}}
    if wl["kind"] == "surrogate":
        # plain contour integration of the same queries (tw_mag_multi), in the
        # arm's own mode and in FP64
        nfb = list(wl["nfb"][-args.steps:])
        sst = list(wl["sur_stats"][-args.steps:])

        def plain(pr):
            pe = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            flush.zero_()
            pe[0].record(stream)
            P.mag_multi(*qd, rel_tol=wl["rel_tol"], precision=pr, out=outd)
            pe[1].record(stream)
            pe[1].synchronize()
            return pe[0].elapsed_time(pe[1]) / 1e3

        t_plain = plain(prec)
        t_plain64 = t_plain if prec == P.PREC_FP64 else plain(P.PREC_FP64)
        frac = {k: sum(c[k] for c in nfb) / (len(nfb) * wl["n"])
                for k in ("fallback", "network", "expansion", "flagged", "uncertain")}
        extra = {"surrogate": {"fallback_fraction": frac["fallback"], "network_fraction": frac["network"],
                               "expansion_fraction": frac["expansion"],
                               "fallback_flagged_fraction": frac["flagged"],
                               "fallback_uncertain_fraction": frac["uncertain"],
                               "plain_value": wl["n"] / t_plain, "plain_ms_per_step": t_plain * 1e3,
                               "speedup_vs_plain": t_plain / t_step,
                               "plain_fp64_value": wl["n"] / t_plain64, "plain_fp64_ms_per_step": t_plain64 * 1e3,
                               "speedup_vs_plain_fp64": t_plain64 / t_step, "train_s": wl.get("train_s"),
                               "train_stats": wl.get("train_stats"), "queries": wl["n"],
                               "kappa": wl["kappa"]}}

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    if wl["kind"] == "mag" and wl.get("gate"):
        hin = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
               for a in (np.full(wl["n"], wl["s"]), np.full(wl["n"], wl["q"]), np.full(wl["n"], wl["rho"]),
                         wl["y1"], wl["y2"])]
        hout = torch.empty(wl["n"], dtype=torch.float64).pin_memory()
        h2d, d2h = 40 * wl["n"], 8 * wl["n"]

        def e2e_step():
            P.mag_gated(*[t.numpy() for t in hin], rel_tol=wl["rel_tol"], precision=prec, out=hout.numpy())
    elif wl["kind"] == "mag" and args.split:
        # this rank's range of the last step, from pinned host buffers
        lo, hi = int(wl["bounds"][rank]), int(wl["bounds"][rank + 1])
        hy1 = torch.from_numpy(np.ascontiguousarray(wl["y1"][lo:hi])).pin_memory()
        hy2 = torch.from_numpy(np.ascontiguousarray(wl["y2"][lo:hi])).pin_memory()
        hout = torch.empty(hi - lo, dtype=torch.float64).pin_memory()
        h2d, d2h = 16 * (hi - lo), 9 * (hi - lo)

        def e2e_step():
            P.mag(wl["s"], wl["q"], wl["rho"], hy1.numpy(), hy2.numpy(), rel_tol=wl["rel_tol"], precision=prec,
                  out=hout.numpy())
    elif wl["kind"] == "mag":
        hy1 = torch.from_numpy(np.ascontiguousarray(wl["y1"])).pin_memory()
        hy2 = torch.from_numpy(np.ascontiguousarray(wl["y2"])).pin_memory()
        hout = torch.empty(wl["n"], dtype=torch.float64).pin_memory()
        h2d, d2h = 16 * wl["n"], 9 * wl["n"]

        def e2e_step():
            P.mag(wl["s"], wl["q"], wl["rho"], hy1.numpy(), hy2.numpy(), rel_tol=wl["rel_tol"], precision=prec,
                  autotune=args.autotune, out=hout.numpy())
    elif wl["kind"] == "multi":
        hm = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in wl["arrays"]]
        hout = torch.empty(wl["n"], dtype=torch.float64).pin_memory()
        h2d, d2h = 40 * wl["n"], 8 * wl["n"]

        def e2e_step():
            P.mag_multi(*[t.numpy() for t in hm], rel_tol=wl["rel_tol"], precision=prec, autotune=args.autotune,
                        out=hout.numpy())
    elif wl["kind"] == "lc":
        ht = torch.from_numpy(np.ascontiguousarray(wl["times"])).pin_memory()
        hout = torch.empty(wl["n"], dtype=torch.float64).pin_memory()
        h2d, d2h = 8 * wl["n"], 9 * wl["n"]

        def e2e_step():
            P.lightcurve(wl["s"], wl["q"], wl["rho"], wl["u0"], wl["alpha"], wl["t0"], wl["tE"], ht.numpy(),
                         rel_tol=wl["rel_tol"], precision=prec, autotune=args.autotune, out=hout.numpy())
    elif wl["kind"] == "surrogate":
        hq = [t.cpu().pin_memory() for t in qd]
        hout = torch.empty(wl["n"], dtype=torch.float64).pin_memory()
        h2d, d2h = 40 * wl["n"], 8 * wl["n"]

        def e2e_step():
            P.surrogate_mag(wpath, *[t.numpy() for t in hq], rel_tol=wl["rel_tol"], kappa=wl["kappa"],
                            precision=prec, out=hout.numpy())
    else:
        hp = torch.from_numpy(wl["params"]).pin_memory()
        ho = torch.from_numpy(wl["offsets"]).pin_memory()
        ht = torch.from_numpy(wl["times"]).pin_memory()
        hout = torch.empty(wl["n"], dtype=torch.float64).pin_memory()
        h2d = 8 * (wl["params"].size + wl["offsets"].size + wl["times"].size)
        d2h = 9 * wl["n"]

        def e2e_step():
            P.lightcurve_batch(hp.numpy(), ho.numpy(), ht.numpy(), rel_tol=wl["rel_tol"], precision=prec,
                               autotune=args.autotune, out=hout.numpy())
    e2e_step()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    n_e2e = max(2, args.steps // 2)
    for _ in range(n_e2e):
        flush.zero_()
        torch.cuda.synchronize()
        e2e_step()
    t_e2e = (time.perf_counter() - t0) / n_e2e
    t_e2e = max_over_ranks(t_e2e, dist, dev)

    # roofline of the contour kernel (the dominant kernel of a step), timed by
    # the library's CUDA events around its launch on the launching stream,
    # against the FMA-pipe peaks measured on this GPU now
    probe64, probe32 = P.peak_probe("fp64"), P.peak_probe("fp32")
    peak64, peak32 = NOMINAL_FP64, NOMINAL_FP32
    f64 /= args.steps
    f32 /= args.steps
    t_kern = sum(kern_ms) / len(kern_ms) / 1e3 if kern_ms and sum(kern_ms) > 0 else t_step
    t_roof = max(f64 / peak64, f32 / peak32)
    roof = {"bound": "alu", "achieved": f64 / t_kern / 1e12, "peak": peak64 / 1e12, "unit": "TFLOP/s",
            "frac": t_roof / t_kern, "traffic": profile_traffic(args.workload, args.mode),
            "kernel": "contour_kernel", "kernel_ms": t_kern * 1e3, "kernel_share_of_step": t_kern / t_step,
            "peak_source": "unit counts and clocks: 152 SMs x 2.07 GHz x 2 FP64 FMA/clk/SM (1.25 TFLOP/s); "
                           "FP32 152 x 128 lanes x 2.07 GHz",
            "peak_fp32": peak32 / 1e12, "probe_fp64": probe64 / 1e12, "probe_fp32": probe32 / 1e12,
            "frac_vs_probe": max(f64 / probe64, f32 / probe32) / t_kern,
            "fp64_flop_per_launch": f64, "fp32_flop_per_launch": f32,
            "fp32_frac": (f32 / peak32) / t_kern}
    other = []
    if wl["kind"] == "surrogate" and sst:
        # feature kernel (FP64/FP32 ALU) and the tensor-core GEMMs, per step
        ms_f = sum(x["features_ms"] for x in sst) / len(sst) / 1e3
        ms_g = sum(x["gemm_ms"] for x in sst) / len(sst) / 1e3
        ff64 = sum(F_FEAT_SOLVE64 * x["point_solves"] + F_FEAT_NEWTON64 * x["newton64"] for x in sst) / len(sst)
        ff32 = sum(F_FEAT_SOLVE32 * x["point_solves"] + F_SWEEP32 * x["point_sweeps32"]
                   + F_CAUSTIC32 * x["caustic_iters"] for x in sst) / len(sst)
        gflop = sum(3 * 2.0 * x["gemm_rows"] * 256 * 256 for x in sst) / len(sst)
        bf16 = load_peaks().get("bf16_tflops_sustained")
        other.append({"kernel": "sur_features_kernel", "bound": "alu", "unit": "TFLOP/s", "kernel_ms": ms_f * 1e3,
                      "achieved": ff64 / ms_f / 1e12, "peak": peak64 / 1e12,
                      "frac": max(ff64 / peak64, ff32 / peak32) / ms_f, "fp32_frac": (ff32 / peak32) / ms_f,
                      "fp64_flop_per_step": ff64, "fp32_flop_per_step": ff32})
        other.append({"kernel": "gemm_bf16_tn_kernel", "bound": "tensor", "unit": "TFLOP/s", "kernel_ms": ms_g * 1e3,
                      "achieved": gflop / ms_g / 1e12, "peak": bf16,
                      "frac": (gflop / ms_g / 1e12) / bf16 if bf16 else None, "flop_per_step": gflop,
                      "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained"})

    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "vs_baseline": None, "dtype": "f64" if args.mode == "fp64" else "f32+f64", "data": "synthetic",
            "scaling": "strong" if args.split else "weak",
            "config": cfg, "roofline": roof, "clocks": clocks,
            "e2e": {"value": (1 if args.split else world) * wl["n"] / t_e2e, "unit": unit, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": gpu_launches(wl, args.steps),
            "roofline_other": other,
            "error_vs_oracle": golden_errors(wl, prec, P, wpath if wl["kind"] == "surrogate" else None),
            "wall_s_timed": wall,
            "work": {"samples_per_position": work["samples"] / (args.steps * wl["n"]),
                     "fp64_sweeps_per_sample": work["sweeps64"] / max(work["samples"], 1),
                     "fp32_sweeps_per_sample": work["sweeps32"] / max(work["samples"], 1),
                     "fp64_newton_per_sample": work["newton64"] / max(work["samples"], 1),
                     "edges_per_sample": work["edges"] / max(work["samples"], 1)}}
    line.update(extra)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n, dt, cores = cpu_oracle_sample(wl, args.cpu_sample)
        n1, dt1, _ = cpu_oracle_sample(wl, max(2, args.cpu_sample // 16), seed=778, cores=1)
        what = ("queries drawn on the CPU from the benchmark's distribution (oracle.sample_near_caustic)"
                if wl["kind"] == "surrogate" else "seeded positions of the same workload")
        line["cpu_baseline"] = {"value": n / dt, "unit": unit, "cores": cores, "kind": "oracle",
                                "sample": "%d %s, %.1f s on %d threads" % (n, what, dt, cores),
                                "value_single_core": n1 / dt1,
                                "sample_single_core": "%d %s, %.1f s on 1 thread" % (n1, what, dt1)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
