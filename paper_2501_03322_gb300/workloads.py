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
