"""Writes the stored expected values of the GPU parity tests.

Every value here is computed by the CPU oracle (``oracle/``) from inputs drawn
by ``paper_2501_03322_gb300.workloads`` (seeded grids and random draws, no lens
arithmetic).  Run from the repository root:

    python tests/golden/make_golden.py [name ...]

Files (text, one position per line: inputs, mu, oracle status):
  lightcurve_central.txt  all 1000 points of the central-caustic light curve
  map_planetary.txt       256 sampled cells of the 512 x 512 planetary-caustic map, plus 96
                          cells whose limb passes within rho of the caustic (most cross it)
  stress_resonant.txt     200 sampled positions of the resonant large-source set
  stress_resonant_1e4.txt the first 10^4 positions of the resonant large-source set
  batch_lightcurves.txt   192 sampled (curve, time) points of the 4096-curve batch, plus 80
                          points (one per curve) whose limb passes within rho of the caustic
  paper_worked.txt        the paper's worked configurations (Fig. 1, 2, 5)
  surrogate_queries.txt   1024 positions near the caustics of 64 lenses of the surrogate's range
  surrogate_band.txt      2048 positions 4-12 rho off the caustics of 64 lenses of the surrogate's range
  narrow_crossings.txt    limbs that dip into a caustic fold over less than the initial sample spacing
  narrow_exits.txt        limbs that leave a caustic over less than the initial sample spacing
  central_wide.txt        4096 centres on the central caustic of a wide planetary lens
  lightcurve_orbital.txt  200 points of a central-caustic light curve of an orbiting lens (separation
                          and axis angle linear in time)
  limb_darkened.txt       32 positions of linearly limb-darkened sources (u = 0.6): 16 whose limb crosses a
                          caustic (central-caustic light curve, planetary-caustic map) and 16 that do not
  fig4_maps.txt           the paper's three Fig. 4 grids (480 x 340, q = 1e-4): per map 128
                          random cells and 64 cells within rho of the caustic
  fig6_sweep.txt          the (s, q) sweep (64 pairs x 30 x 30, rho = 1e-4): 4 random positions
                          of every pair

Positions "near the caustic" are chosen with the oracle's caustic (nearest of
its sampled points within rho of the limb's centre).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2501_03322_gb300 import workloads as W  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def _write(name, header, cols, rows):
    rows = list(rows)
    path = os.path.join(HERE, name)
    with open(path, "w") as f:
        for line in header.strip().splitlines():
            f.write("# " + line + "\n")
        f.write("# columns: " + " ".join(cols) + "\n")
        for r in rows:
            f.write(" ".join(repr(float(v)) if isinstance(v, (float, np.floating)) else str(int(v)) for v in r) + "\n")
    print("wrote", path, len(rows), "rows")


def lightcurve_central():
    c = W.LIGHTCURVE_CENTRAL
    t = W.lightcurve_central_times(c["n"])
    mu, st, nx = O.lightcurve(c["s"], c["q"], c["rho"], c["u0"], c["alpha"], c["t0"], c["tE"], t, scan_K=256)
    hdr = ("Central-caustic light curve: s=1, q=1e-3, rho=1e-3, u0=0.01, alpha=1 rad, t0=0, tE=20 d,\n"
           "1000 times linspace(-1, 1); oracle magnifications (binary128 linking-free contour integral).")
    _write("lightcurve_central.txt", hdr, ["t", "mu", "status", "ncross"], zip(t, mu, st, nx))


def _near_caustic(points, s, q, rho, M=8192):
    """Mask of points within rho of the oracle's caustic (sampled at M angles)."""
    from scipy.spatial import cKDTree

    _, cc = O.caustic(s, q, M)
    c = cc.ravel()
    d, _ = cKDTree(np.c_[c.real, c.imag]).query(points)
    return d < rho


def map_planetary():
    c = W.MAP_PLANETARY
    y1, y2 = W.map_grid()
    idx = W.sample_indices(y1.size, 256, seed=101)
    near = np.nonzero(_near_caustic(np.c_[y1, y2], c["s"], c["q"], c["rho"]))[0]
    near = np.setdiff1d(near, idx)
    extra = np.sort(np.random.default_rng(102).choice(near, size=min(96, near.size), replace=False))
    idx = np.r_[idx, extra]
    mu, st, nx = O.mag(c["s"], c["q"], c["rho"], y1[idx], y2[idx], scan_K=256)
    hdr = ("Planetary-caustic map: s=0.8, q=1e-4, rho=5e-4, 512x512 cell centres of the 0.1x0.1 box centred\n"
           "on (-0.44985, 0.016993); 256 cells sampled with seed 101, then 96 cells (seed 102) among those within\n"
           "rho of the oracle's caustic; oracle magnifications.")
    _write("map_planetary.txt", hdr, ["index", "y1", "y2", "mu", "status", "ncross"], zip(idx, y1[idx], y2[idx], mu, st, nx))


def stress_resonant():
    c = W.STRESS_RESONANT
    y1, y2 = W.stress_positions()
    idx = W.sample_indices(y1.size, 200, seed=202)
    mu, st, nx = O.mag(c["s"], c["q"], c["rho"], y1[idx], y2[idx], scan_K=256)
    hdr = ("Resonant large source: s=1, q=0.5, rho=0.05, 1e6 positions uniform in |y|<0.6 (seed 2);\n"
           "200 sampled with seed 202; oracle magnifications.")
    _write("stress_resonant.txt", hdr, ["index", "y1", "y2", "mu", "status", "ncross"], zip(idx, y1[idx], y2[idx], mu, st, nx))


def stress_resonant_1e4():
    c = W.STRESS_RESONANT
    y1, y2 = W.stress_positions()
    idx = np.arange(10000)
    mu, st, nx = O.mag(c["s"], c["q"], c["rho"], y1[idx], y2[idx], scan_K=256, nthreads=os.cpu_count())
    hdr = ("Resonant large source: s=1, q=0.5, rho=0.05, 1e6 positions uniform in |y|<0.6 (seed 2);\n"
           "the first 10^4 positions; oracle magnifications.")
    _write("stress_resonant_1e4.txt", hdr, ["index", "y1", "y2", "mu", "status", "ncross"],
           zip(idx, y1[idx], y2[idx], mu, st, nx))


def batch_lightcurves():
    params, offsets, times = W.batch_lightcurves()
    rng = np.random.default_rng(303)
    curves = np.sort(rng.choice(params.shape[0], 64, replace=False))
    jobs = []
    for k in curves:
        n_k = offsets[k + 1] - offsets[k]
        pick = np.sort(rng.choice(n_k, 3, replace=False)) + offsets[k]
        jobs.append((k, pick))

    def run(job):
        k, pick = job
        s, q, rho, u0, alpha, t0, tE = params[k]
        mu, st, nx = O.lightcurve(s, q, rho, u0, alpha, t0, tE, times[pick], scan_K=256, nthreads=1)
        return [(k, i, times[i], m, a, b) for i, m, a, b in zip(pick, mu, st, nx)]

    def near(k):
        """One time of curve k whose limb centre lies within rho of the caustic, or None."""
        s, q, rho, u0, alpha, t0, tE = params[k]
        t = times[offsets[k]:offsets[k + 1]]
        y1, y2 = O.trajectory(u0, alpha, t0, tE, t)
        m = np.nonzero(_near_caustic(np.c_[y1, y2], s, q, rho, M=2048))[0]
        if m.size == 0:
            return None
        return (k, np.array([offsets[k] + m[np.random.default_rng(int(k)).integers(m.size)]]))

    order = np.random.default_rng(304).permutation(params.shape[0])
    crossing = []
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count()) as ex:
        for start in range(0, order.size, 64):
            crossing += [j for j in ex.map(near, order[start:start + 64]) if j is not None]
            if len(crossing) >= 80:
                break
    jobs += sorted(crossing[:80], key=lambda j: j[0])

    rows = []
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count()) as ex:
        for r in ex.map(run, jobs):
            rows.extend(r)
    hdr = ("Batch of 4096 light curves (workloads.batch_lightcurves, seed 0); 64 curves x 3 times sampled\n"
           "with seed 303, then one time on each of 80 curves (curve order seed 304) whose limb centre lies\n"
           "within rho of the oracle's caustic; oracle magnifications.")
    _write("batch_lightcurves.txt", hdr, ["curve", "index", "t", "mu", "status", "ncross"], rows)


def paper_worked():
    rows = []
    # Fig. 1 (Sec. 2.2): s=0.5, q=1e-6, rho=1e-4, source centre -1.49981640625 + 0.0035i (limb near a cusp
    # of the planetary caustic)
    cases = [("fig1", 0.5, 1e-6, 1e-4, -1.49981640625, 0.0035)]
    # Fig. 2 (Sec. 2.3): s=1, q=0.1, rho=0.1, centre 0.2+0.2i (two caustic crossings)
    cases.append(("fig2", 1.0, 0.1, 0.1, 0.2, 0.2))
    # Fig. 5 (Sec. 4.2): s=0.5, q=1e-6, rho=1e-4, horizontal line y2 = -0.0035 near the planetary caustic;
    # the two positions where the paper reports spikes of another code, and a line across the caustic
    cases.append(("fig5_spike_a", 0.5, 1e-6, 1e-4, -1.49998960, -0.0035))
    cases.append(("fig5_spike_b", 0.5, 1e-6, 1e-4, -1.49993410, -0.0035))
    for x in np.linspace(-1.50012, -1.49988, 25):
        cases.append(("fig5_line", 0.5, 1e-6, 1e-4, float(x), -0.0035))

    def run(c):
        tag, s, q, rho, y1, y2 = c
        mu, st, nx = O.mag(s, q, rho, [y1], [y2], scan_K=512, nthreads=1)
        return (tag, s, q, rho, y1, y2, mu[0], st[0], nx[0])

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count()) as ex:
        out = list(ex.map(run, cases))
    path = os.path.join(HERE, "paper_worked.txt")
    with open(path, "w") as f:
        f.write("# The paper's worked configurations (it prints no magnification values for them):\n")
        f.write("#   fig1: Sec. 2.2, Fig. 1 (coefficient accuracy, limb next to a planetary-caustic cusp)\n")
        f.write("#   fig2: Sec. 2.3, Fig. 2 (two caustic crossings, three full images and two broken tracks)\n")
        f.write("#   fig5_*: Sec. 4.2, Fig. 5 (low-q light curve at y2=-0.0035; spike positions of another code)\n")
        f.write("# Values: CPU oracle magnifications.\n")
        f.write("# columns: tag s q rho y1 y2 mu status ncross\n")
        for r in out:
            f.write("%s %r %r %r %r %r %r %d %d\n" % (r[0], r[1], r[2], r[3], r[4], r[5], float(r[6]), int(r[7]), int(r[8])))
    print("wrote", path, len(out), "rows")


def surrogate_queries():
    """Query positions near caustics for the surrogate path: 64 lenses with
    log10 s ~ U[-0.5, 0.5], log10 q ~ U[-5, -1], log10 rho ~ U[-4, -2]; for
    each, 16 positions = a random point of a random branch of the oracle's
    caustic + a displacement uniform in a disc of 3x that branch's size."""
    rng = np.random.default_rng(404)
    rows = []
    jobs = []
    for k in range(64):
        s = 10 ** rng.uniform(-0.5, 0.5)
        q = 10 ** rng.uniform(-5, -1)
        rho = 10 ** rng.uniform(-4, -2)
        _, cc = O.caustic(s, q, 256)
        pts = []
        for _ in range(16):
            b = rng.integers(4)
            c = cc[rng.integers(256), b]
            w = max(np.ptp(cc[:, b].real), np.ptp(cc[:, b].imag))
            r = 3 * w * np.sqrt(rng.uniform())
            a = rng.uniform(0, 2 * np.pi)
            pts.append((c.real + r * np.cos(a), c.imag + r * np.sin(a)))
        jobs.append((s, q, rho, np.array(pts)))

    def run(job):
        s, q, rho, pts = job
        mu, st, nx = O.mag(s, q, rho, pts[:, 0], pts[:, 1], scan_K=256, nthreads=1)
        return [(s, q, rho, p[0], p[1], m, a, b) for p, m, a, b in zip(pts, mu, st, nx)]

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count()) as ex:
        for r in ex.map(run, jobs):
            rows.extend(r)
    hdr = ("Surrogate queries: 64 lenses (seed 404) x 16 positions near the oracle's caustic (random branch point +\n"
           "displacement within 3x the branch size); oracle magnifications.")
    _write("surrogate_queries.txt", hdr, ["s", "q", "rho", "y1", "y2", "mu", "status", "ncross"], rows)


def surrogate_band():
    """Query positions a few source radii off the caustic, where the source
    does not touch the caustic but its point-source expansion is uncertain
    (the network's band): 64 lenses of the surrogate's range (seed 405); for
    each, 32 positions = a random point of a random branch of the oracle's
    caustic + a displacement of 4-12 rho in a random direction."""
    rng = np.random.default_rng(405)
    rows = []
    jobs = []
    for k in range(64):
        s = 10 ** rng.uniform(-0.5, 0.5)
        q = 10 ** rng.uniform(-5, -1)
        rho = 10 ** rng.uniform(-4, -2)
        _, cc = O.caustic(s, q, 256)
        pts = []
        for _ in range(32):
            c = cc[rng.integers(256), rng.integers(4)]
            r = rho * rng.uniform(4.0, 12.0)
            a = rng.uniform(0, 2 * np.pi)
            pts.append((c.real + r * np.cos(a), c.imag + r * np.sin(a)))
        jobs.append((s, q, rho, np.array(pts)))

    def run(job):
        s, q, rho, pts = job
        mu, st, nx = O.mag(s, q, rho, pts[:, 0], pts[:, 1], scan_K=256, nthreads=1)
        return [(s, q, rho, p[0], p[1], m, a, b) for p, m, a, b in zip(pts, mu, st, nx)]

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count()) as ex:
        for r in ex.map(run, jobs):
            rows.extend(r)
    # positions the oracle itself reports as not converged are left out (a cusp
    # tip reaching just inside the limb between the oracle's caustic samples)
    nbad = sum(int(r[6]) != 0 for r in rows)
    rows = [r for r in rows if int(r[6]) == 0]
    hdr = ("Surrogate band queries: 64 lenses (seed 405) x 32 positions 4-12 rho from a random point of the oracle's\n"
           "caustic (random branch and angle, random direction); oracle magnifications; positions with a\n"
           "non-zero oracle status left out: %d." % nbad)
    _write("surrogate_band.txt", hdr, ["s", "q", "rho", "y1", "y2", "mu", "status", "ncross"], rows)


def _narrow(seed, side, name, title):
    """48 lenses of the surrogate's range; for each, a random fold point c of
    the oracle's caustic with normal n pointing to the three-image side
    (side = +1) or the five-image side (side = -1), the source centre at
    c + rho cos(w/2) n with w ~ U[0.02, 0.09] rad, so that the limb crosses
    the fold twice about w apart (2 pi/64 = 0.098).  Kept when the oracle
    finds exactly two crossings less than 0.098 apart and converges."""
    rng = np.random.default_rng(seed)
    rows = []
    jobs = []
    for k in range(48):
        s = 10 ** rng.uniform(-0.5, 0.5)
        q = 10 ** rng.uniform(-5, -1)
        rho = 10 ** rng.uniform(-4, -2)
        _, cc = O.caustic(s, q, 1024)
        for _ in range(64):  # a fold point: neighbouring chords nearly parallel, the caustic locally straight
            b = rng.integers(4)
            i = int(rng.integers(1024))
            c, t1, t2 = cc[i, b], cc[(i + 1) % 1024, b] - cc[i, b], cc[i, b] - cc[i - 1, b]
            if abs(t1) == 0 or abs(t2) == 0 or abs(np.angle(t1 / t2)) > 0.02:
                continue
            n = 1j * t1 / abs(t1)
            eps = 1e-3 * rho
            c_out = O.images(s, q, c + eps * n)["count"], O.images(s, q, c - eps * n)["count"]
            if c_out == (5, 3):
                n = -n
            elif c_out != (3, 5):
                continue
            w = rng.uniform(0.02, 0.09)
            z0 = c + side * rho * np.cos(0.5 * w) * n
            jobs.append((s, q, rho, z0.real, z0.imag))
            break

    def run(job):
        s, q, rho, y1, y2 = job
        mu, st, nx = O.mag(s, q, rho, [y1], [y2], scan_K=1024, nthreads=1)
        xs = O.crossings(s, q, rho, y1, y2, "caustic", 4096)
        gap = (xs[1] - xs[0]) if len(xs) == 2 else 9.0
        gap = min(gap, 2 * np.pi - gap)
        return (s, q, rho, y1, y2, mu[0], st[0], nx[0], gap)

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count()) as ex:
        for r in ex.map(run, jobs):
            if r[6] == 0 and r[7] == 2 and r[8] < 0.098:
                rows.append(r[:8])
    hdr = (title + ": 48 lenses (seed %d), the source centre rho cos(w/2) %s a fold point of the\n"
           "oracle's caustic, w ~ U[0.02, 0.09] rad; kept when the oracle finds two crossings < 0.098 rad apart\n"
           "(the initial sample spacing 2 pi/64) and converges; oracle magnifications."
           % (seed, "outside" if side > 0 else "inside"))
    _write(name, hdr, ["s", "q", "rho", "y1", "y2", "mu", "status", "ncross"], rows)


def narrow_crossings():
    """Limbs that dip into the caustic over less than the initial sample
    spacing (seed 406, centres on the three-image side)."""
    _narrow(406, 1.0, "narrow_crossings.txt", "Narrow crossings")


def narrow_exits():
    """Limbs that leave the caustic over less than the initial sample spacing
    (seed 407, centres on the five-image side)."""
    _narrow(407, -1.0, "narrow_exits.txt", "Narrow exits")


def central_wide():
    """All 4096 positions of the central-caustic set (wide planetary lens,
    source radius comparable to the caustic)."""
    c = W.CENTRAL_WIDE
    y1, y2 = W.central_wide_positions()
    mu, st, nx = O.mag(c["s"], c["q"], c["rho"], y1, y2, scan_K=256, nthreads=os.cpu_count())
    hdr = ("Central caustic of a wide planetary lens: s=3, q=1e-4, rho=1.1e-4; 4096 centres uniform in a disc of\n"
           "radius 2e-4 about the primary (seed 5); oracle magnifications.")
    _write("central_wide.txt", hdr, ["i", "y1", "y2", "mu", "status", "ncross"],
           zip(range(y1.size), y1, y2, mu, st, nx))


ORBITAL = dict(s=1.0, q=1e-3, rho=1e-3, u0=0.01, alpha=1.0, t0=0.0, tE=20.0, ds_dt=0.03, dalpha_dt=0.2)


def lightcurve_orbital():
    c = ORBITAL
    t = np.linspace(-1.0, 1.0, 200)
    mu, st, nx = O.lightcurve_orbital(c["s"], c["q"], c["rho"], c["u0"], c["alpha"], c["t0"], c["tE"], c["ds_dt"],
                                      c["dalpha_dt"], t, scan_K=256)
    hdr = ("Central-caustic light curve of an orbiting lens: s=1 + 0.03 (t - t0), q=1e-3, rho=1e-3, u0=0.01,\n"
           "alpha=1 + 0.2 (t - t0) rad, t0=0, tE=20 d, 200 times linspace(-1, 1); oracle magnifications.")
    _write("lightcurve_orbital.txt", hdr, ["t", "mu", "status", "ncross"], zip(t, mu, st, nx))


LD_U = 0.6


def limb_darkened():
    """Limb-darkened sources (linear law, u = 0.6) on two lenses: positions of
    the central-caustic light curve and of the planetary-caustic map, half of
    them crossing a caustic (oracle ncross >= 2)."""
    jobs = []
    lc = [ln.split() for ln in open(os.path.join(HERE, "lightcurve_central.txt")) if not ln.startswith("#")]
    c = W.LIGHTCURVE_CENTRAL
    t = np.array([float(r[0]) for r in lc])
    nx = np.array([int(r[3]) for r in lc])
    rng = np.random.default_rng(700)
    pick = np.r_[rng.choice(np.nonzero(nx >= 2)[0], 8, replace=False), rng.choice(np.nonzero(nx < 2)[0], 8, replace=False)]
    y1, y2 = O.trajectory(c["u0"], c["alpha"], c["t0"], c["tE"], t[pick])
    jobs += [("lightcurve_central", c["s"], c["q"], c["rho"], a, b) for a, b in zip(y1, y2)]
    mp = [ln.split() for ln in open(os.path.join(HERE, "map_planetary.txt")) if not ln.startswith("#")]
    m = W.MAP_PLANETARY
    xr = [r for r in mp if int(r[5]) >= 2]
    sr = [r for r in mp if int(r[5]) < 2]
    for r in [xr[i] for i in rng.choice(len(xr), 8, replace=False)] + [sr[i] for i in rng.choice(len(sr), 8, replace=False)]:
        jobs.append(("map_planetary", m["s"], m["q"], m["rho"], float(r[1]), float(r[2])))

    def run(j):
        tag, s, q, rho, a, b = j
        mu, st = O.mag_ld(s, q, rho, LD_U, a, b, epsrel=1e-8, nthreads=0)
        nxr = len(O.crossings(s, q, rho, a, b))
        return (tag, s, q, rho, LD_U, a, b, mu, st, nxr)

    rows = [run(j) for j in jobs]  # each position uses every core over its radii
    path = os.path.join(HERE, "limb_darkened.txt")
    with open(path, "w") as f:
        f.write("# Linearly limb-darkened sources, I(r) = 1 - u (1 - sqrt(1 - r^2/rho^2)), u = 0.6: 16 positions of\n")
        f.write("# the central-caustic light curve and 16 cells of the planetary-caustic map (seed 700), half of each\n")
        f.write("# crossing a caustic; oracle magnifications (oracle.mag_ld, adaptive in the annulus radius).\n")
        f.write("# columns: set s q rho u y1 y2 mu status ncross\n")
        for r in rows:
            f.write("%s %r %r %r %r %r %r %r %d %d\n" % (r[0], r[1], r[2], r[3], r[4], float(r[5]), float(r[6]), float(r[7]), int(r[8]), int(r[9])))
    print("wrote", path, len(rows), "rows")


def fig4_maps():
    rows = []
    for k, name in enumerate(sorted(W.FIG4)):
        c = W.FIG4[name]
        y1, y2 = W.fig4_grid(name)
        idx = W.sample_indices(y1.size, 128, seed=600 + k)
        near = np.nonzero(_near_caustic(np.c_[y1, y2], c["s"], c["q"], c["rho"]))[0]
        near = np.setdiff1d(near, idx)
        extra = np.sort(np.random.default_rng(610 + k).choice(near, size=min(64, near.size), replace=False))
        idx = np.r_[idx, extra]
        mu, st, nx = O.mag(c["s"], c["q"], c["rho"], y1[idx], y2[idx], scan_K=256)
        rows += [(name, i, a, b, m, t, x) for i, a, b, m, t, x in zip(idx, y1[idx], y2[idx], mu, st, nx)]
    path = os.path.join(HERE, "fig4_maps.txt")
    with open(path, "w") as f:
        f.write("# The paper's Fig. 4 speed maps (Sec. 4.1): q = 1e-4, s = 0.5 (rho 5e-5), 1 (rho 1e-3), 3 (rho 1e-4),\n")
        f.write("# 480 x 340 cells (workloads.fig4_grid); per map 128 random cells (seeds 600..602) and 64 cells\n")
        f.write("# within rho of the oracle's caustic (seeds 610..612); oracle magnifications.\n")
        f.write("# columns: map index y1 y2 mu status ncross\n")
        for r in rows:
            f.write("%s %d %r %r %r %d %d\n" % (r[0], int(r[1]), float(r[2]), float(r[3]), float(r[4]), int(r[5]), int(r[6])))
    print("wrote", path, len(rows), "rows")


def fig6_sweep():
    S, Q, R, Y1, Y2 = W.fig6_sweep()
    g2 = W.FIG6_GRID ** 2
    rng = np.random.default_rng(620)
    idx = np.concatenate([k * g2 + np.sort(rng.choice(g2, 4, replace=False)) for k in range(len(W.FIG6_BOXES))])

    def run(k):
        sel = idx[4 * k:4 * k + 4]
        mu, st, nx = O.mag(S[sel[0]], Q[sel[0]], R[sel[0]], Y1[sel], Y2[sel], scan_K=256, nthreads=1)
        return [(i, S[i], Q[i], R[i], Y1[i], Y2[i], m, a, b) for i, m, a, b in zip(sel, mu, st, nx)]

    rows = []
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count()) as ex:
        for r in ex.map(run, range(len(W.FIG6_BOXES))):
            rows.extend(r)
    hdr = ("The (s, q) sweep of Sec. 4.3 (Fig. 6): 64 pairs x 30 x 30 positions over the caustic on the planet's\n"
           "side (workloads.fig6_sweep), rho = 1e-4; 4 random positions per pair (seed 620); oracle magnifications.")
    _write("fig6_sweep.txt", hdr, ["index", "s", "q", "rho", "y1", "y2", "mu", "status", "ncross"], rows)


ALL = {"lightcurve_central": lightcurve_central, "central_wide": central_wide, "surrogate_queries": surrogate_queries,
       "surrogate_band": surrogate_band, "narrow_crossings": narrow_crossings, "narrow_exits": narrow_exits,
       "map_planetary": map_planetary, "stress_resonant": stress_resonant, "batch_lightcurves": batch_lightcurves,
       "paper_worked": paper_worked, "stress_resonant_1e4": stress_resonant_1e4, "fig4_maps": fig4_maps, "lightcurve_orbital": lightcurve_orbital,
       "limb_darkened": limb_darkened,
       "fig6_sweep": fig6_sweep}

if __name__ == "__main__":
    names = sys.argv[1:] or list(ALL)
    for nm in names:
        t = time.time()
        ALL[nm]()
        print(nm, "%.1fs" % (time.time() - t))
