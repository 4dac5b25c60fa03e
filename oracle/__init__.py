"""CPU oracle for finite-source binary-lens magnification (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never calls it, and it
shares no code with the CUDA sources.

The computation lives in ``twinkle_oracle.c`` (long double C99, OpenMP over
source positions); this module compiles it in-tree on first use and wraps it
with ctypes.  Every function states the part of the paper it follows in the C
source; in short:

* ``quintic``      -- polynomial of Eq. 1 by generic expansion (not Eq. 6)
* ``images``       -- its roots, residuals (Eq. 12), Jacobians (Eq. 7), ghost pair test
* ``mag``          -- magnification = image area / source area (Sec. 1), image
                      area by a linking-free contour integral (Eq. 8)
* ``crossings``    -- limb/caustic crossing angles, by the caustic or an image-count scan
* ``close_approaches`` -- limb angles where the caustic nearly touches the limb
* ``caustic``      -- critical curve J = 0 and its caustic image
* ``trajectory``   -- straight-line source trajectory of a light curve
* ``lightcurve_orbital`` -- light curve of a lens with linear orbital motion
* ``mag_ld``       -- magnification of a linearly limb-darkened source
* ``rayshoot``     -- brute-force inverse ray shooting (Sec. 1), for pinning ``mag``

Per-position status codes from ``mag``: 0 ok, 1 crossing detectors disagree or
image counts are inconsistent, 2 quadrature did not converge, 3 root finder
failure, 4 invalid input.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "twinkle_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS_OK, STATUS_XING, STATUS_QUAD, STATUS_ROOT, STATUS_INPUT = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle shared library in-tree (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC]
        if platform.machine() in ("x86_64", "AMD64", "i686"):
            cmd.append("-lquadmath")  # binary128 working type on x86 (see the C source)
        cmd.append("-lm")
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_SO)
        d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
        P = ctypes.c_void_p
        lib.orc_quintic.argtypes = [d, d, d, d, P]
        lib.orc_quintic.restype = None
        lib.orc_images.argtypes = [d, d, d, d, P, P, P, P, P]
        lib.orc_images.restype = ctypes.c_int
        lib.orc_caustic.argtypes = [d, d, ctypes.c_int, P, P]
        lib.orc_caustic.restype = ctypes.c_int
        lib.orc_crossings.argtypes = [d, d, d, d, d, ctypes.c_int, ctypes.c_int, P, ctypes.c_int]
        lib.orc_crossings.restype = ctypes.c_int
        lib.orc_close_approaches.argtypes = [d, d, d, d, d, P, ctypes.c_int]
        lib.orc_close_approaches.restype = ctypes.c_int
        lib.orc_mag.argtypes = [d, d, d, P, P, i64, ctypes.c_int, ctypes.c_int, P, P, P]
        lib.orc_mag.restype = ctypes.c_int
        lib.orc_singular_radii.argtypes = [d, d, d, d, d, P, ctypes.c_int]
        lib.orc_singular_radii.restype = ctypes.c_int
        lib.orc_mag_radii.argtypes = [d, d, d, d, P, i64, ctypes.c_int, ctypes.c_int, P, P]
        lib.orc_mag_radii.restype = ctypes.c_int
        lib.orc_trajectory.argtypes = [d, d, d, d, P, i64, P, P]
        lib.orc_trajectory.restype = None
        lib.orc_rayshoot.argtypes = [d, d, d, d, d, d, d, d, d, i64, i64, ctypes.c_int]
        lib.orc_rayshoot.restype = d
        lib.orc_real_bits.argtypes = []
        lib.orc_real_bits.restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def real_bits() -> int:
    """Mantissa bits of the oracle's working type (113: IEEE binary128)."""
    return _load().orc_real_bits()


def quintic(s: float, q: float, zeta: complex) -> np.ndarray:
    """Ascending coefficients c0..c5 of the image polynomial (centre-of-mass frame)."""
    out = np.zeros(12)
    _load().orc_quintic(s, q, zeta.real, zeta.imag, _ptr(out))
    return out[0::2] + 1j * out[1::2]


def images(s: float, q: float, zeta: complex) -> dict:
    """Roots, residuals, Jacobians, real mask and image count of one point source."""
    roots, res, jac = np.zeros(10), np.zeros(10), np.zeros(5)
    isreal = np.zeros(5, np.int32)
    count = np.zeros(1, np.int32)
    st = _load().orc_images(s, q, zeta.real, zeta.imag, _ptr(roots), _ptr(res), _ptr(jac), _ptr(isreal), _ptr(count))
    if st:
        raise RuntimeError("oracle root finder failed (status %d)" % st)
    return dict(
        roots=roots[0::2] + 1j * roots[1::2],
        residuals=res[0::2] + 1j * res[1::2],
        jac=jac,
        real=isreal.astype(bool),
        count=int(count[0]),
    )


def caustic(s: float, q: float, M: int = 1024):
    """Critical curve and caustic at M angles: two complex arrays of shape (M, 4)."""
    zc, cc = np.zeros(8 * M), np.zeros(8 * M)
    st = _load().orc_caustic(s, q, M, _ptr(zc), _ptr(cc))
    if st:
        raise RuntimeError("oracle caustic failed")
    return (zc[0::2] + 1j * zc[1::2]).reshape(M, 4), (cc[0::2] + 1j * cc[1::2]).reshape(M, 4)


def crossings(s: float, q: float, rho: float, y1: float, y2: float, method: str = "caustic", K: int = 4096) -> np.ndarray:
    """Limb angles where the source limb crosses the caustic.

    method="caustic": limb/caustic intersections (caustic sampled at K angles);
    method="scan": changes of the image count on K limb points.
    """
    out = np.zeros(64)
    m = 1 if method == "caustic" else 2
    n = _load().orc_crossings(s, q, rho, y1, y2, m, K, _ptr(out), 64)
    if n < 0:
        raise RuntimeError("oracle crossings failed")
    return np.sort(out[: min(n, 64)])


def close_approaches(s: float, q: float, rho: float, y1: float, y2: float) -> np.ndarray:
    """Limb angles where the caustic comes within 5% of rho of the limb without
    crossing it (the extra split points of the quadrature in ``mag``)."""
    out = np.zeros(64)
    n = _load().orc_close_approaches(s, q, rho, y1, y2, _ptr(out), 64)
    if n < 0:
        raise RuntimeError("oracle caustic failed")
    return np.sort(out[: min(n, 64)])


def mag(s: float, q: float, rho: float, y1, y2, scan_K: int = 256, nthreads: int = 0):
    """Finite-source magnifications of positions (y1[i], y2[i]).

    Returns (mu, status, nxing) arrays.  ``scan_K`` > 0 cross-checks the caustic
    crossings by an image-count scan on that many limb points.
    """
    y1 = np.ascontiguousarray(np.atleast_1d(y1), dtype=np.float64)
    y2 = np.ascontiguousarray(np.atleast_1d(y2), dtype=np.float64)
    n = y1.size
    out = np.zeros(n)
    st = np.zeros(n, np.int32)
    nx = np.zeros(n, np.int32)
    rc = _load().orc_mag(s, q, rho, _ptr(y1), _ptr(y2), n, scan_K, nthreads, _ptr(out), _ptr(st), _ptr(nx))
    if rc:
        raise ValueError("oracle: invalid lens or source parameters")
    return out, st, nx


def sample_near_caustic(n: int, seed: int):
    """n positions of the surrogate workload's distribution, drawn on the CPU:
    a lens with log10 s ~ U[-0.5, 0.5], log10 q ~ U[-5, -1], log10 rho ~
    U[-4, -2] per position, a random point of a random branch of its caustic
    (this oracle's, 256 angles), displaced uniformly within a disc of three
    times that branch's bounding-box size.  Returns (s, q, rho, y1, y2)."""
    rng = np.random.default_rng(seed)
    out = np.zeros((5, n))
    for i in range(n):
        s = 10 ** rng.uniform(-0.5, 0.5)
        q = 10 ** rng.uniform(-5, -1)
        rho = 10 ** rng.uniform(-4, -2)
        _, cc = caustic(s, q, 256)
        b = rng.integers(4)
        c = cc[rng.integers(256), b]
        w = max(np.ptp(cc[:, b].real), np.ptp(cc[:, b].imag))
        r = 3 * w * np.sqrt(rng.uniform())
        a = rng.uniform(0, 2 * np.pi)
        out[:, i] = (s, q, rho, c.real + r * np.cos(a), c.imag + r * np.sin(a))
    return tuple(out)


def trajectory(u0: float, alpha: float, t0: float, tE: float, times):
    """Source positions along a straight-line trajectory."""
    t = np.ascontiguousarray(times, dtype=np.float64)
    y1, y2 = np.zeros(t.size), np.zeros(t.size)
    _load().orc_trajectory(u0, alpha, t0, tE, _ptr(t), t.size, _ptr(y1), _ptr(y2))
    return y1, y2


def lightcurve(s, q, rho, u0, alpha, t0, tE, times, scan_K: int = 256, nthreads: int = 0):
    """Magnification along a straight-line trajectory."""
    y1, y2 = trajectory(u0, alpha, t0, tE, times)
    return mag(s, q, rho, y1, y2, scan_K=scan_K, nthreads=nthreads)


def lightcurve_orbital(s, q, rho, u0, alpha, t0, tE, ds_dt, dalpha_dt, times, scan_K: int = 256, nthreads: int = 0):
    """Magnification along a straight-line trajectory behind an orbiting lens
    whose separation and axis angle change linearly in time: at time t the lens
    has separation s + ds_dt (t - t0) and the trajectory angle is alpha +
    dalpha_dt (t - t0) (the first-order reading of lens orbital motion).  Each
    time is its own lens: one ``mag`` per time, spread over threads."""
    import concurrent.futures as cf

    t = np.ascontiguousarray(np.atleast_1d(times), dtype=np.float64)
    st = s + ds_dt * (t - t0)
    at = alpha + dalpha_dt * (t - t0)

    def one(i):
        y1, y2 = trajectory(u0, at[i], t0, tE, t[i:i + 1])
        if not st[i] > 0:
            return np.nan, ORC_INPUT_STATUS, 0
        m, s_, n_ = mag(st[i], q, rho, y1, y2, scan_K=scan_K, nthreads=1)
        return m[0], s_[0], n_[0]

    workers = nthreads if nthreads > 0 else (os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        res = list(ex.map(one, range(t.size)))
    return (np.array([r[0] for r in res]), np.array([r[1] for r in res], np.int32),
            np.array([r[2] for r in res], np.int32))


ORC_INPUT_STATUS = STATUS_INPUT


def mag_radii(s: float, q: float, y1: float, y2: float, radii, scan_K: int = 0, nthreads: int = 0):
    """Uniform-disc magnifications of one position for many radii (one caustic build)."""
    r = np.ascontiguousarray(np.atleast_1d(radii), dtype=np.float64)
    out = np.zeros(r.size)
    st = np.zeros(r.size, np.int32)
    if _load().orc_mag_radii(s, q, y1, y2, _ptr(r), r.size, scan_K, nthreads, _ptr(out), _ptr(st)):
        raise ValueError("oracle: invalid lens")
    return out, st


def singular_radii(s: float, q: float, y1: float, y2: float, rmax: float) -> np.ndarray:
    """Radii below rmax where a circle about (y1, y2) touches a fold of the
    caustic or passes through a cusp (mu(r) is not smooth there)."""
    out = np.zeros(256)
    n = _load().orc_singular_radii(s, q, y1, y2, rmax, _ptr(out), 256)
    if n < 0:
        raise RuntimeError("oracle caustic failed")
    return np.sort(out[: min(n, 256)])


def mag_ld(s: float, q: float, rho: float, u: float, y1: float, y2: float, epsrel: float = 1e-9,
           nthreads: int = 0):
    """Magnification of a linearly limb-darkened disc, brightness
    I(r) = 1 - u (1 - sqrt(1 - r^2/rho^2)), centred at (y1, y2).

    The flux F = Int I dA_images is Int_0^rho I(r) dG(r) with G(r) = pi r^2
    mu(r) the image area of a uniform disc of radius r; by parts and with
    r = rho sin(phi),
        mu_LD = [(1 - u) mu(rho) + u Int_0^{pi/2} sin^3(phi) mu(rho sin phi) dphi] / (1 - u/3),
    evaluated with this oracle's uniform-disc magnification.  mu(r) is not
    smooth where the circle of radius r touches the caustic (G - G_t ~
    (r - r_t)^{3/2}), so the phi integral is cut at those radii
    (singular_radii) and each piece is halved; on each half, phi = end +- D t^2
    makes that behaviour smooth in t, and 16- and 24-point Gauss-Legendre
    rules in t are compared; a piece whose two values differ by more than its
    share of epsrel is halved again.
    Returns (mu_LD, worst oracle status of the radii used)."""
    xa, wa = np.polynomial.legendre.leggauss(16)
    xb, wb = np.polynomial.legendre.leggauss(24)
    xa, wa, xb, wb = 0.5 * (xa + 1), 0.5 * wa, 0.5 * (xb + 1), 0.5 * wb
    cuts = [np.arcsin(min(r / rho, 1.0)) for r in singular_radii(s, q, y1, y2, rho)]
    edges = [0.0]
    for c in sorted(c for c in cuts if 1e-6 < c < 0.5 * np.pi - 1e-6):
        if c - edges[-1] > 1e-6:  # cuts closer than that are one
            edges.append(c)
    edges = np.array(edges + [0.5 * np.pi])
    pieces = list(zip(edges[:-1], edges[1:]))
    mu_rho, st0 = mag_radii(s, q, y1, y2, [rho], nthreads=nthreads)
    worst = int(st0[0])
    done = 0.0

    def halves(a, b):
        m = 0.5 * (a + b)
        return [(a, m - a, xa, wa, xb, wb), (b, m - b, xa, wa, xb, wb)]

    for _ in range(30):
        nodes, plan = [], []
        for a, b in pieces:
            for end, D, x1, w1, x2, w2 in halves(a, b):
                i0 = len(nodes)
                nodes += list(end + D * x1 * x1) + list(end + D * x2 * x2)
                plan.append((abs(D), x1, w1, x2, w2, i0))
        ph = np.array(nodes)
        mu, st = mag_radii(s, q, y1, y2, rho * np.sin(ph), nthreads=nthreads)
        worst = max(worst, int(st.max()))
        f = np.sin(ph) ** 3 * mu
        va, vb = [], []
        for D, x1, w1, x2, w2, i0 in plan:
            n1 = x1.size
            va.append(D * np.sum(w1 * 2 * x1 * f[i0:i0 + n1]))
            vb.append(D * np.sum(w2 * 2 * x2 * f[i0 + n1:i0 + n1 + x2.size]))
        va = np.array(va).reshape(-1, 2).sum(1)
        vb = np.array(vb).reshape(-1, 2).sum(1)
        total = done + vb.sum()
        width = np.array([b - a for a, b in pieces])
        bad = np.abs(vb - va) > epsrel * abs(total) * (width / (0.5 * np.pi) + 1e-6)
        done += vb[~bad].sum()
        if not bad.any():
            break
        if 2 * bad.sum() + len(pieces) > 4096:
            worst = max(worst, STATUS_QUAD)
            done += vb[bad].sum()
            break
        pieces = [h for (pa, pb), keep in zip(pieces, bad) if keep for h in ((pa, 0.5 * (pa + pb)), (0.5 * (pa + pb), pb))]
    else:
        worst = max(worst, STATUS_QUAD)
    return ((1.0 - u) * float(mu_rho[0]) + u * done) / (1.0 - u / 3.0), worst


def rayshoot(s, q, rho, y1, y2, box, npix: int, nthreads: int = 0) -> float:
    """Brute-force inverse ray shooting over box=(x0, x1, y0, y1) with npix x npix rays."""
    x0, x1, yb0, yb1 = box
    return _load().orc_rayshoot(s, q, rho, y1, y2, x0, x1, yb0, yb1, npix, npix, nthreads)
