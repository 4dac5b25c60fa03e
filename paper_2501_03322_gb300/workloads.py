"""Seeded synthetic workloads (source positions and light curves).

Pure random draws and grids: no lens arithmetic lives here, so the GPU path and
the CPU oracle can both be fed from it.  The paper's own workloads are
synthetic grids and light curves (Sec. 4.1-4.3); nothing here reads a dataset.

Workloads (sizes are those the benchmark and the parity tests use):

* ``lightcurve_central``: one resonant lens s=1, q=1e-3, rho=1e-3 and a straight
  trajectory u0=0.01, alpha=1 rad, t0=0, tE=20 d sampled at 1000 evenly spaced
  times in [-1, 1] d, which crosses the central caustic.
* ``map_planetary``: a 512 x 512 grid of cell centres in a 0.1 x 0.1 box centred
  on the upper planetary caustic of s=0.8, q=1e-4 (centre (-0.44985, 0.016993),
  the caustic's bounding-box centre), rho=5e-4.  Same convention as the paper's
  Fig. 4 maps, which are centred on a planetary caustic.
* ``batch_lightcurves``: 4096 light curves with log10 s ~ U[-0.5, 0.5],
  log10 q ~ U[-5, -1], log10 rho ~ U[-4, -2], u0 ~ U[-0.5, 0.5],
  alpha ~ U[0, 2 pi), tE ~ U[5, 100] d, t0 = 0, lengths ~ U{200..5000}, times
  ~ U[t0 - 1.5 tE, t0 + 1.5 tE] sorted.
* ``stress_resonant``: s=1, q=0.5, rho=0.05, positions uniform in the disc |y| < 0.6.
* ``fig4_*``: the three 480 x 340 source grids of the paper's speed maps
  (Sec. 4.1, Fig. 4), q = 1e-4: s = 0.5 (rho = 5e-5, centred on (-1.5,
  0.035), the upper planetary caustic), s = 1 (rho = 1e-3, centred on the
  origin, the resonant caustic) and s = 3 (rho = 1e-4, centred on (2.666, 0),
  the planetary caustic).  The paper prints the centres and the radii but not
  the box sizes; the boxes here cover each caustic with a margin.
* ``fig6_sweep``: the (s, q) exploration of Sec. 4.3 (Fig. 6): for each of
  8 x 8 (s, q) pairs a 30 x 30 grid over the caustic on the planet's side (or
  the resonant caustic), rho = 1e-4.  The paper's (s, q) axes are not in its
  text; the pairs span 0.45 <= s <= 2.2 and 1e-6 <= q <= 1e-2.
"""
from __future__ import annotations

import numpy as np

LIGHTCURVE_CENTRAL = dict(s=1.0, q=1e-3, rho=1e-3, u0=0.01, alpha=1.0, t0=0.0, tE=20.0, n=1000, rel_tol=1e-4)
MAP_PLANETARY = dict(s=0.8, q=1e-4, rho=5e-4, centre=(-0.44985, 0.016993), half=0.05, n=512, rel_tol=1e-4)
STRESS_RESONANT = dict(s=1.0, q=0.5, rho=0.05, radius=0.6, n=1_000_000, rel_tol=1e-5, seed=2)
BATCH_LIGHTCURVES = dict(ncurve=4096, nmin=200, nmax=5000, rel_tol=1e-4, seed=0)
# Source centres on the tiny central caustic of a wide planetary lens: a disc
# of radius 2e-4 around the primary lens (x = -q s/(1+q) for s=3, q=1e-4), a
# source radius comparable to the caustic, magnifications up to ~1e4.  The
# limb crosses the caustic next to its cusps, where ghost pairs come close.
CENTRAL_WIDE = dict(s=3.0, q=1e-4, rho=1.1e-4, centre=(-2.9997000299970003e-4, 0.0), radius=2e-4, n=4096,
                    rel_tol=1e-4, seed=5)


# Fig. 4 grids: (s, q, rho, centre, half-widths of the box); 480 x 340 cells.
# Box half-widths cover the caustic nearest the centre (its extent, from the
# CPU oracle's caustic at 4096 angles, is 1.9e-3 x 1.3e-3 for s = 0.5,
# 0.107 x 0.028 for s = 1 and 4.7e-3 x 4.2e-3 for s = 3) with the grid's
# aspect ratio 480:340.
FIG4 = {
    "fig4_s05": dict(s=0.5, q=1e-4, rho=5e-5, centre=(-1.5, 0.035), half=(1.6e-3, 1.6e-3 * 340 / 480)),
    "fig4_s1": dict(s=1.0, q=1e-4, rho=1e-3, centre=(0.0, 0.0), half=(0.09, 0.09 * 340 / 480)),
    "fig4_s3": dict(s=3.0, q=1e-4, rho=1e-4, centre=(2.666, 0.0), half=(4e-3, 4e-3 * 340 / 480)),
}
FIG4_SHAPE = (480, 340)

# Fig. 6 sweep: (s, q, box centre x, box centre y, half-width x, half-width y)
# per pair.  Each box is the bounding box of the caustic component on the
# planet's side (the upper one of a close binary's two planetary caustics;
# the resonant caustic near s = 1), from the CPU oracle's caustic at 2048
# angles, widened to 1.2 times its size plus 2e-4 on each side.  Written once
# from the oracle; rho = 1e-4 throughout.
FIG6_RHO = 1e-4
FIG6_GRID = 30
FIG6_BOXES = [
    (0.45, 1.000000e-06, -1.772218711, 0.004005821, 2.797384e-04, 2.565908e-04),
    (0.45, 3.162278e-06, -1.772211118, 0.007123386, 3.417963e-04, 3.007151e-04),
    (0.45, 1.000000e-05, -1.772187108, 0.012667070, 4.521501e-04, 3.793552e-04),
    (0.45, 3.162278e-05, -1.772111182, 0.022524422, 6.483727e-04, 5.197470e-04),
    (0.45, 1.000000e-04, -1.771871107, 0.040049823, 9.972161e-04, 7.711131e-04),
    (0.45, 3.162278e-04, -1.771112137, 0.071197544, 1.617021e-03, 1.223392e-03),
    (0.45, 1.000000e-03, -1.768714223, 0.126500912, 2.716197e-03, 2.043632e-03),
    (0.45, 1.000000e-02, -1.737454503, 0.396124582, 8.006754e-03, 6.344186e-03),
    (0.55, 1.000000e-06, -1.268179323, 0.003102659, 3.561792e-04, 3.002934e-04),
    (0.55, 3.162278e-06, -1.268173927, 0.005517242, 4.777285e-04, 3.785170e-04),
    (0.55, 1.000000e-05, -1.268156863, 0.009810687, 6.938723e-04, 5.179819e-04),
    (0.55, 3.162278e-05, -1.268102905, 0.017444360, 1.078201e-03, 7.671253e-04),
    (0.55, 1.000000e-04, -1.267932291, 0.031014371, 1.761453e-03, 1.213730e-03),
    (0.55, 3.162278e-04, -1.267392917, 0.055126151, 2.975383e-03, 2.018983e-03),
    (0.55, 1.000000e-03, -1.265688827, 0.097917712, 5.128036e-03, 3.484829e-03),
    (0.55, 1.000000e-02, -1.243477508, 0.306171410, 1.548095e-02, 1.128193e-02),
    (0.65, 1.000000e-06, -0.888459766, 0.002445334, 4.849594e-04, 3.613876e-04),
    (0.65, 3.162278e-06, -0.888455932, 0.004348204, 7.067348e-04, 4.873205e-04),
    (0.65, 1.000000e-05, -0.888443812, 0.007731399, 1.101104e-03, 7.119727e-04),
    (0.65, 3.162278e-05, -0.888405489, 0.013745538, 1.802340e-03, 1.113701e-03),
    (0.65, 1.000000e-04, -0.888284302, 0.024432995, 3.048999e-03, 1.835123e-03),
    (0.65, 3.162278e-04, -0.887901189, 0.043411469, 5.264018e-03, 3.140074e-03),
    (0.65, 1.000000e-03, -0.886690908, 0.077055982, 9.192314e-03, 5.529254e-03),
    (0.65, 1.000000e-02, -0.870929975, 0.240066953, 2.810424e-02, 1.853075e-02),
    (0.8, 1.000000e-06, -0.449998500, 0.001704603, 8.841907e-04, 4.970800e-04),
    (0.8, 3.162278e-06, -0.449995259, 0.003030474, 1.416680e-03, 7.292255e-04),
    (0.8, 1.000000e-05, -0.449985000, 0.005386515, 2.363612e-03, 1.144076e-03),
    (0.8, 3.162278e-05, -0.449952557, 0.009570636, 4.047550e-03, 1.888239e-03),
    (0.8, 1.000000e-04, -0.449849968, 0.016992877, 7.042282e-03, 3.232127e-03),
    (0.8, 3.162278e-04, -0.449525496, 0.030130129, 1.236898e-02, 5.687965e-03),
    (0.8, 1.000000e-03, -0.448498479, 0.053275908, 2.184864e-02, 1.027013e-02),
    (0.8, 1.000000e-02, -0.434814150, 0.162103539, 6.914794e-02, 3.747696e-02),
    (1, 1.000000e-06, 0.003937251, 0.000000000, 1.437320e-02, 1.897054e-03),
    (1, 3.162278e-06, 0.005757879, 0.000000000, 2.092552e-02, 3.217830e-03),
    (1, 1.000000e-05, 0.008399002, 0.000000000, 3.046149e-02, 5.566504e-03),
    (1, 3.162278e-05, 0.012220023, 0.000000000, 4.426949e-02, 9.742914e-03),
    (1, 1.000000e-04, 0.017697398, 0.000000000, 6.414480e-02, 1.716869e-02),
    (1, 3.162278e-04, 0.025443057, 0.000000000, 9.248823e-02, 3.036787e-02),
    (1, 1.000000e-03, 0.036145973, 0.000000000, 1.323345e-01, 5.380643e-02),
    (1, 1.000000e-02, 0.067823976, 0.032922046, 2.589792e-01, 1.285447e-01),
    (1.25, 1.000000e-06, 0.449990226, 0.000000000, 2.760075e-03, 1.399413e-03),
    (1.25, 3.162278e-06, 0.449969088, 0.000000000, 4.752819e-03, 2.332886e-03),
    (1.25, 1.000000e-05, 0.449902206, 0.000000000, 8.297816e-03, 3.992837e-03),
    (1.25, 3.162278e-05, 0.449690344, 0.000000000, 1.460938e-02, 6.944556e-03),
    (1.25, 1.000000e-04, 0.449016679, 0.000000000, 2.587612e-02, 1.219275e-02),
    (1.25, 3.162278e-04, 0.446847959, 0.000000000, 4.616170e-02, 2.152110e-02),
    (1.25, 1.000000e-03, 0.439551930, 0.000000000, 8.381402e-02, 3.808480e-02),
    (1.25, 1.000000e-02, 0.286805399, 0.000000000, 3.750070e-01, 1.187627e-01),
    (1.6, 1.000000e-06, 0.974997309, 0.000000000, 1.400964e-03, 9.949971e-04),
    (1.6, 3.162278e-06, 0.974991492, 0.000000000, 2.335658e-03, 1.613724e-03),
    (1.6, 1.000000e-05, 0.974973094, 0.000000000, 3.997847e-03, 2.713974e-03),
    (1.6, 3.162278e-05, 0.974914913, 0.000000000, 6.953922e-03, 4.670429e-03),
    (1.6, 1.000000e-04, 0.974730904, 0.000000000, 1.221198e-02, 8.149001e-03),
    (1.6, 3.162278e-04, 0.974148774, 0.000000000, 2.156978e-02, 1.433178e-02),
    (1.6, 1.000000e-03, 0.972305452, 0.000000000, 3.825313e-02, 2.530905e-02),
    (1.6, 1.000000e-02, 0.947645520, 0.000000000, 1.228747e-01, 7.872910e-02),
    (2.2, 1.000000e-06, 1.745452383, 0.000000000, 7.567018e-04, 6.514207e-04),
    (2.2, 3.162278e-06, 1.745447708, 0.000000000, 1.189970e-03, 1.002750e-03),
    (2.2, 1.000000e-05, 1.745432923, 0.000000000, 1.960434e-03, 1.627501e-03),
    (2.2, 3.162278e-05, 1.745386172, 0.000000000, 3.330491e-03, 2.738423e-03),
    (2.2, 1.000000e-04, 1.745238347, 0.000000000, 5.766599e-03, 4.713615e-03),
    (2.2, 3.162278e-04, 1.744771024, 0.000000000, 1.009734e-02, 8.224171e-03),
    (2.2, 1.000000e-03, 1.743294650, 0.000000000, 1.779110e-02, 1.445632e-02),
    (2.2, 1.000000e-02, 1.724062732, 0.000000000, 5.544903e-02, 4.475121e-02),
]


def fig4_grid(name: str):
    """Cell centres of one Fig. 4 map: 480 columns in y1 by 340 rows in y2, row-major."""
    c = FIG4[name]
    nx, ny = FIG4_SHAPE
    (cx, cy), (hx, hy) = c["centre"], c["half"]
    x = cx - hx + 2.0 * hx * (np.arange(nx) + 0.5) / nx
    y = cy - hy + 2.0 * hy * (np.arange(ny) + 0.5) / ny
    Y1, Y2 = np.meshgrid(x, y)
    return Y1.ravel().copy(), Y2.ravel().copy()


def fig6_sweep():
    """(s, q, rho, y1, y2) arrays of the (s, q) sweep: 64 pairs x 30 x 30 positions, pair-major."""
    g = FIG6_GRID
    u = (np.arange(g) + 0.5) / g * 2.0 - 1.0
    U1, U2 = np.meshgrid(u, u)
    out = [[], [], [], [], []]
    for s, q, cx, cy, hx, hy in FIG6_BOXES:
        out[0].append(np.full(g * g, s))
        out[1].append(np.full(g * g, q))
        out[2].append(np.full(g * g, FIG6_RHO))
        out[3].append(cx + hx * U1.ravel())
        out[4].append(cy + hy * U2.ravel())
    return tuple(np.concatenate(a) for a in out)


def lightcurve_central_times(n: int = 1000) -> np.ndarray:
    return np.linspace(-1.0, 1.0, n)


def map_grid(centre=MAP_PLANETARY["centre"], half=MAP_PLANETARY["half"], n=MAP_PLANETARY["n"]):
    """Cell centres of an n x n grid over [c1-half, c1+half] x [c2-half, c2+half], row-major in y2."""
    step = 2.0 * half / n
    x = centre[0] - half + step * (np.arange(n) + 0.5)
    y = centre[1] - half + step * (np.arange(n) + 0.5)
    Y1, Y2 = np.meshgrid(x, y)
    return Y1.ravel().copy(), Y2.ravel().copy()


def batch_lightcurves(ncurve=BATCH_LIGHTCURVES["ncurve"], nmin=BATCH_LIGHTCURVES["nmin"],
                      nmax=BATCH_LIGHTCURVES["nmax"], seed=BATCH_LIGHTCURVES["seed"]):
    """(params [ncurve, 7], offsets [ncurve+1], times [total]) of the batch workload."""
    rng = np.random.default_rng(seed)
    s = 10.0 ** rng.uniform(-0.5, 0.5, ncurve)
    q = 10.0 ** rng.uniform(-5.0, -1.0, ncurve)
    rho = 10.0 ** rng.uniform(-4.0, -2.0, ncurve)
    u0 = rng.uniform(-0.5, 0.5, ncurve)
    alpha = rng.uniform(0.0, 2.0 * np.pi, ncurve)
    tE = rng.uniform(5.0, 100.0, ncurve)
    t0 = np.zeros(ncurve)
    lens = rng.integers(nmin, nmax + 1, ncurve)
    offsets = np.zeros(ncurve + 1, np.int64)
    offsets[1:] = np.cumsum(lens)
    times = np.empty(int(offsets[-1]))
    for k in range(ncurve):
        t = rng.uniform(t0[k] - 1.5 * tE[k], t0[k] + 1.5 * tE[k], lens[k])
        times[offsets[k]:offsets[k + 1]] = np.sort(t)
    params = np.stack([s, q, rho, u0, alpha, t0, tE], axis=1)
    return np.ascontiguousarray(params), offsets, times


def stress_positions(n=STRESS_RESONANT["n"], radius=STRESS_RESONANT["radius"], seed=STRESS_RESONANT["seed"]):
    """n positions uniform in the disc |y| < radius."""
    rng = np.random.default_rng(seed)
    r = radius * np.sqrt(rng.uniform(0.0, 1.0, n))
    phi = rng.uniform(0.0, 2.0 * np.pi, n)
    return r * np.cos(phi), r * np.sin(phi)


def sample_indices(n_total: int, k: int, seed: int = 12345) -> np.ndarray:
    """k distinct indices of range(n_total), sorted (seeded)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_total, size=min(k, n_total), replace=False))


def central_wide_positions(n=CENTRAL_WIDE["n"], centre=CENTRAL_WIDE["centre"], radius=CENTRAL_WIDE["radius"],
                           seed=CENTRAL_WIDE["seed"]):
    """Seeded positions uniform in a disc (the central-caustic set)."""
    rng = np.random.default_rng(seed)
    r = radius * np.sqrt(rng.uniform(size=n))
    a = rng.uniform(0.0, 2.0 * np.pi, size=n)
    return centre[0] + r * np.cos(a), centre[1] + r * np.sin(a)
