"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: an
independent formula printed in the paper (Eq. 6), closed forms of the
single-lens limit, algebraic invariants of the binary-lens polynomial
(Sec. 2.3-2.4), symmetries of the lens, brute-force inverse ray shooting
(Sec. 1), and the agreement of two independent caustic-crossing detectors.
"""
import math

import numpy as np
import pytest

import oracle as O


def eq6_planet_frame(s, q, y):
    """Coefficients c0..c5 of Eq. 6 (paper Sec. 2.2), origin at the secondary.

    Readings: the factor printed as "Im(y) i" is i*Im(y); m1 = 1 - m2."""
    m2 = q / (1 + q)
    yb = np.conj(y)
    vc = yb + s
    vp = 1 + s * yb
    iim = 1j * y.imag
    c5 = -yb * vc
    c4 = (yb * y - 1 - 2 * s * yb) * vc + m2 * s
    c3 = (2 * y - s) * (vp * vc + 2 * iim - m2 * s) + 4 * (m2 * s - y) * iim
    c2 = (vp.real ** 2 * vc.real + 1j * y.imag * vp.real * (1 - s * y).real + s * y.imag ** 2 * (2 + s * vc)
          + m2 * s * (2 * yb * (y - s) - (1 - s * y)))
    c1 = m2 * s * ((s + 2 * y) * vp + s * (2 * s * iim - m2))
    c0 = s * s * m2 * m2 * y
    return np.array([c0, c1, c2, c3, c4, c5])


def taylor_shift(c, a):
    """Coefficients of P(x + a) from those of P(x) (ascending)."""
    n = len(c)
    out = np.zeros(n, complex)
    for k in range(n):
        for j in range(k + 1):
            out[j] += c[k] * math.comb(k, j) * a ** (k - j)
    return out


@pytest.mark.parametrize("seed", range(6))
def test_generic_quintic_equals_eq6(seed):
    """The oracle's generically expanded polynomial is the paper's Eq. 6 (after
    moving the origin from the centre of mass to the secondary)."""
    rng = np.random.default_rng(seed)
    for _ in range(20):
        s = 10 ** rng.uniform(-0.5, 0.5)
        q = 10 ** rng.uniform(-3, 0)
        zeta = complex(rng.uniform(-1.5, 1.5), rng.uniform(-1.5, 1.5))
        z2 = s / (1 + q)
        c_cm = O.quintic(s, q, zeta)
        c_pl = taylor_shift(c_cm, z2)  # P(eta + z2)
        e6 = eq6_planet_frame(s, q, zeta - z2)
        r = c_pl / c_pl[5] * e6[5]
        assert np.max(np.abs(r - e6)) <= 1e-11 * np.max(np.abs(e6))


def test_roots_vieta_and_residual_sum():
    """Roots satisfy Vieta's sum rule, and the lens-equation residuals of the
    five roots sum to zero (Eq. 13-14); real images number 3 or 5 with parity
    sum -1 (Sec. 2.3); ghosts come as a pair of opposite residuals (Sec. 2.4.1)."""
    rng = np.random.default_rng(7)
    n3 = n5 = 0
    for k in range(300):
        if k % 2:  # wide lenses, sources anywhere
            s = 10 ** rng.uniform(-0.5, 0.5)
            q = 10 ** rng.uniform(-6, 0)
            zeta = complex(rng.uniform(-1, 1), rng.uniform(-0.6, 0.6))
        else:  # resonant lenses, sources near the large central caustic
            s = 10 ** rng.uniform(-0.1, 0.1)
            q = 10 ** rng.uniform(-1, 0)
            zeta = complex(rng.uniform(-0.15, 0.15), rng.uniform(-0.15, 0.15))
        c = O.quintic(s, q, zeta)
        im = O.images(s, q, zeta)
        r, R = im["roots"], im["residuals"]
        assert abs(r.sum() + c[4] / c[5]) <= 1e-9 * (1 + np.abs(r).max())
        assert abs(R.sum()) <= 1e-9
        assert im["count"] in (3, 5)
        real = im["real"]
        assert real.sum() == im["count"]
        par = np.sign(im["jac"][real])
        assert par.sum() == -1
        if im["count"] == 3:
            g = R[~real]
            assert abs(g[0] + g[1]) < 1e-6 * abs(g[0])
            assert np.abs(R[real]).max() < 1e-12
            n3 += 1
        else:
            n5 += 1
    assert n3 > 50 and n5 > 10


def test_image_count_matches_caustic_inside_outside():
    """Five images inside the caustic, three outside (Sec. 2.3): for X2's lens
    the centre of the central caustic has 5 images, a far point 3."""
    assert O.images(1.0, 0.1, complex(0.0, 0.0))["count"] == 5
    assert O.images(1.0, 0.1, complex(1.5, 1.0))["count"] == 3


@pytest.mark.parametrize("rho", [1.0, 0.1, 0.01])
def test_centred_disc_point_lens(rho):
    """Uniform disc centred on a point lens: image is an annulus, mu = sqrt(1 + 4/rho^2).

    The binary is made a point lens by a negligible companion far away
    (q = 1e-9 at s = 10); its effect on mu is ~1e-9."""
    s, q = 10.0, 1e-9
    x1 = -q * s / (1 + q)
    mu, st, _ = O.mag(s, q, rho, [x1], [0.0], scan_K=64)
    assert st[0] == 0
    assert abs(mu[0] / math.sqrt(1 + 4 / rho ** 2) - 1) < 3e-9


@pytest.mark.parametrize("u", [0.1, 0.5, 1.0])
def test_paczynski_limit(u):
    """rho -> 0 and q -> 0: mu -> (u^2 + 2)/(u sqrt(u^2 + 4)); the leading
    finite-source correction is O(rho^2/u^2)."""
    s, q, rho = 10.0, 1e-9, 1e-5
    x1 = -q * s / (1 + q)
    mu, st, _ = O.mag(s, q, rho, [x1 + u], [0.0], scan_K=64)
    A = (u * u + 2) / (u * math.sqrt(u * u + 4))
    assert st[0] == 0
    assert abs(mu[0] / A - 1) < 2e-9 + rho ** 2 / u ** 2


def single_lens_polygon(u, rho, n):
    """Area of the images of a disc under a unit point lens, by the polygon of
    the analytic images z = zeta/2 (1 +- sqrt(1 + 4/|zeta|^2)) of n limb
    points, each image weighted by its parity (+1 outer, -1 inner)."""
    th = 2 * np.pi * np.arange(n) / n
    zeta = u + rho * np.exp(1j * th)
    root = np.sqrt(1 + 4 / np.abs(zeta) ** 2)
    area = 0.0
    for sgn in (+1, -1):
        z = zeta / 2 * (1 + sgn * root)
        zn = np.roll(z, -1)
        area += sgn * 0.5 * np.sum(z.real * zn.imag - z.imag * zn.real)
    return area / (np.pi * rho * rho)


@pytest.mark.parametrize("u,rho", [(0.05, 0.1), (0.3, 0.1), (1.5, 0.4), (0.02, 0.01)])
def test_single_lens_finite_source(u, rho):
    """Finite-source single-lens magnification at any u: a periodic 1-D integral
    over the analytic images (Richardson-extrapolated polygon)."""
    n = 1 << 16
    ref = (4 * single_lens_polygon(u, rho, 2 * n) - single_lens_polygon(u, rho, n)) / 3
    s, q = 10.0, 1e-9
    x1 = -q * s / (1 + q)
    mu, st, _ = O.mag(s, q, rho, [x1 + u], [0.0], scan_K=64)
    assert st[0] == 0
    assert abs(mu[0] / ref - 1) < 5e-8


def test_symmetries():
    """Mirror about the lens axis, mu(y1, y2) = mu(y1, -y2); and mass swap,
    mu(s, q, y1, y2) = mu(s, 1/q, -y1, y2) (swapping the masses of Eq. 2
    reflects the lens through the centre of mass)."""
    s, q, rho = 1.0, 0.1, 0.05
    y1 = np.array([0.05, -0.1, 0.3])
    y2 = np.array([0.02, 0.1, -0.05])
    a, sa, _ = O.mag(s, q, rho, y1, y2, scan_K=64)
    b, sb, _ = O.mag(s, q, rho, y1, -y2, scan_K=64)
    c, sc, _ = O.mag(s, 1 / q, rho, -y1, y2, scan_K=64)
    assert (sa == 0).all() and (sb == 0).all() and (sc == 0).all()
    np.testing.assert_allclose(a, b, rtol=1e-10)
    np.testing.assert_allclose(a, c, rtol=1e-10)


def test_magnification_at_least_one_and_large_source_limit():
    """mu >= 1 for a lens of non-negative point masses; mu -> 1 as rho grows
    (a source much larger than the Einstein ring)."""
    rng = np.random.default_rng(3)
    y1 = rng.uniform(-1, 1, 12)
    y2 = rng.uniform(-1, 1, 12)
    mu, st, _ = O.mag(0.8, 0.3, 0.02, y1, y2, scan_K=32)
    assert (st == 0).all()
    assert (mu >= 1).all()
    big = O.mag(0.8, 0.3, 50.0, [0.0, 3.0], [0.0, -2.0], scan_K=32)[0]
    assert (big > 1).all() and (big < 1.002).all()


@pytest.mark.parametrize(
    "s,q,rho,y1,y2",
    [
        (1.0, 0.1, 0.1, 0.2, 0.2),  # Fig. 2 configuration: two caustic crossings
        (1.0, 0.5, 0.05, 0.0, 0.0),  # source inside the central caustic: 5 images
        (1.0, 0.5, 0.05, 0.12, 0.1),  # limb across a fold
        (0.8, 1e-2, 0.02, -0.3, 0.05),
    ],
)
def test_brute_force_ray_shooting(s, q, rho, y1, y2):
    """Inverse ray shooting on a fine image-plane grid (Sec. 1) agrees with the
    contour integral to its own resolution."""
    mu, st, _ = O.mag(s, q, rho, [y1], [y2], scan_K=128)
    ray = O.rayshoot(s, q, rho, y1, y2, (-2.2, 2.2, -2.2, 2.2), 8000)
    assert st[0] == 0
    assert abs(mu[0] / ray - 1) < 1.5e-3


def test_crossing_detectors_agree():
    """Limb/caustic intersections and the image-count scan find the same angles."""
    cases = [(1.0, 0.1, 0.1, 0.2, 0.2), (1.0, 1e-3, 1e-3, 0.0, 0.0), (0.8, 1e-4, 5e-4, -0.45, 0.0175)]
    for s, q, rho, y1, y2 in cases:
        a = O.crossings(s, q, rho, y1, y2, "caustic", 2048)
        b = O.crossings(s, q, rho, y1, y2, "scan", 1024)
        assert len(a) == len(b) and len(a) % 2 == 0
        assert np.max(np.abs(a - b), initial=0) < 1e-9


def test_trajectory_geometry():
    """Straight-line trajectory: closest approach |u0| at t0, direction alpha."""
    u0, alpha, t0, tE = 0.01, 1.0, 3.0, 20.0
    t = np.array([t0 - tE, t0, t0 + tE])
    y1, y2 = O.trajectory(u0, alpha, t0, tE, t)
    assert abs(math.hypot(y1[1], y2[1]) - abs(u0)) < 1e-15
    d = np.array([y1[2] - y1[1], y2[2] - y2[1]])
    assert abs(math.atan2(d[1], d[0]) - alpha) < 1e-14
    assert abs(np.hypot(*d) - 1) < 1e-14


def _merging_pairs(s, q, zeta0, rho, theta, dth):
    """Differences of the pair that is real on the five-image side of a
    crossing at limb angle theta (positive minus negative parity, the closest
    such pair) and of the ghost pair on its three-image side."""
    side = [O.images(s, q, zeta0 + rho * np.exp(1j * (theta + d))) for d in (-dth, dth)]
    five = side[0] if side[0]["count"] == 5 else side[1]
    three = side[1] if five is side[0] else side[0]
    assert five["count"] == 5 and three["count"] == 3
    R, J = five["roots"][five["real"]], five["jac"][five["real"]]
    pairs = [(abs(R[a] - R[b]), R[a] - R[b]) for a in range(5) for b in range(5) if J[a] > 0 > J[b]]
    d5 = min(pairs, key=lambda t: t[0])[1]
    g = three["roots"][~three["real"]]
    return d5, g[0] - g[1]


@pytest.mark.parametrize("cfg", [(1.0, 0.1, 0.1, 0.2, 0.2), (0.5, 1e-6, 1e-4, -1.49981640625, 0.0035)])
def test_slope_premise(cfg):
    """Sec. 2.4.2: across a caustic crossing the merging real pair and the ghost
    pair are perpendicular, with equal separations to leading order (the
    separation is the square root of a quantity that changes sign), and the
    real pair keeps its direction from one sample to the next."""
    s, q, rho, y1, y2 = cfg
    z0 = complex(y1, y2)
    xs = O.crossings(s, q, rho, y1, y2)
    gap = min(np.diff(np.r_[xs, xs[0] + 2 * np.pi]))
    h = min(1e-4, 1e-3 * gap)  # well inside the local (fold) regime of each crossing
    for th in xs:
        for dth in (h / 100, h):
            d5, d3 = _merging_pairs(s, q, z0, rho, th, dth)
            cos = abs((d5 * np.conj(d3)).real) / (abs(d5) * abs(d3))
            assert cos < 1e-2 and abs(abs(d5) / abs(d3) - 1) < 1e-2, (th, dth, cos)
            e5, _ = _merging_pairs(s, q, z0, rho, th, 2 * dth)
            assert abs((d5 * np.conj(e5)).real) / (abs(d5) * abs(e5)) > 0.99


def _point_mag_sum(s, q, zeta, count):
    """Point-source magnification sum_j 1/|J_j| (Eq. 7) over the `count`
    roots of smallest lens-equation residual (Eq. 12) at source point zeta."""
    im = O.images(s, q, zeta)
    real = np.argsort(np.abs(im["residuals"]))[:count]
    return float(np.sum(1.0 / np.abs(im["jac"][real])))


def _limb_mean_point_mag(s, q, rho, y1, y2):
    """(1/2 pi) Int_0^{2 pi} mu_ps(zeta0 + rho e^{i theta}) d theta by adaptive
    Gauss-Kronrod quadrature (QUADPACK) on each arc between caustic crossings.
    At a crossing the two merging images have 1/|J| ~ 1/sqrt(theta - a), an
    end-point singularity the extrapolation of QUADPACK absorbs; where the
    caustic nearly touches the limb the integrand peaks sharply, so those
    angles are given as break points."""
    from scipy.integrate import quad

    z0 = complex(y1, y2)
    xs = O.crossings(s, q, rho, y1, y2, "caustic", 2048)
    if len(xs) % 2 or not len(xs):  # crossings between the caustic samples: take the image-count changes
        xs = O.crossings(s, q, rho, y1, y2, "scan", 4096)
    near = O.close_approaches(s, q, rho, y1, y2)
    arcs = [(xs[i], xs[i + 1] if i + 1 < len(xs) else xs[0] + 2 * np.pi) for i in range(len(xs))]
    if not arcs:
        arcs = [(near[0], near[0] + 2 * np.pi)] if len(near) else [(0.0, 2 * np.pi)]
    tot = 0.0
    for a, b in arcs:
        c = O.images(s, q, z0 + rho * np.exp(1j * 0.5 * (a + b)))["count"]
        pts = sorted(t + 2 * np.pi * k for t in near for k in (0, 1) if a < t + 2 * np.pi * k < b)

        def f(x):
            return _point_mag_sum(s, q, z0 + rho * np.exp(1j * x), c)

        val, _ = quad(f, a, b, points=pts or None, epsabs=0.0, epsrel=1e-10, limit=4000)
        tot += val
    return tot / (2 * np.pi)


@pytest.mark.parametrize(
    "s,q,rho,y1,y2,h",
    [
        (1.0, 0.1, 0.1, 0.2, 0.2, 1e-3),  # Fig. 2 configuration: two fold crossings
        (1.0, 0.5, 0.05, 0.09635215498703824, 0.5675190958091779, 1e-3),  # resonant large source, four crossings
        (3.0, 1e-4, 1.1e-4, -0.00017032196187594936, -5.5429363083667814e-05, 1e-3),  # central caustic next to a cusp, mu ~ 1e4
        (0.5, 1e-6, 1e-4, -1.49998960, -0.0035, 1e-3),  # Fig. 5 spike position (Sec. 4.2): limb grazing a cusp
        # a cusp tip reaching 0.3% of rho into the limb between the caustic samples (crossings from the scan);
        # the tip enters the circle at 0.9967 rho, so the stencil in rho is kept well inside that
        (0.8609170617125291, 0.011058271392725569, 0.00022100735515155945, -0.18418949339547389, -0.09120884119378822, 2.5e-4),
        (0.8, 0.3, 0.02, 0.5, 0.3, 1e-3),  # no crossing
    ],
)
def test_area_derivative_identity(s, q, rho, y1, y2, h):
    """pi rho^2 mu(rho) is the integral of the point-source magnification over
    the disc of radius rho (Sec. 1), so d(rho^2 mu)/d rho = 2 rho <mu_ps>, the
    mean over the limb circle.  The left side differentiates the oracle's
    contour integral (its crossing pieces, the integration about critical
    points and their boundary terms, Eq. 8-11) in rho; the right side sums
    point-source magnifications 1/|J| directly, with no contour, linking or
    area formula.  A wrong sign, factor or piece in the assembly changes mu
    differently at each rho and breaks the equality."""
    import concurrent.futures as cf

    radii = rho * np.array([1 - 2 * h, 1 - h, 1 + h, 1 + 2 * h])
    with cf.ThreadPoolExecutor(max_workers=4) as ex:
        res = list(ex.map(lambda r: O.mag(s, q, r, [y1], [y2], scan_K=0, nthreads=1), radii))
    assert all(int(r[1][0]) == 0 for r in res)
    g = [r * r * m[0][0] for r, m in zip(radii, res)]
    dg = (-g[3] + 8 * g[2] - 8 * g[1] + g[0]) / (12 * h * rho)
    mean = _limb_mean_point_mag(s, q, rho, y1, y2)
    assert abs(dg / (2 * rho * mean) - 1) < 1e-7


def test_orbital_motion_point_lens_limit():
    """Lens orbital motion (separation and axis angle linear in time): turning
    the binary's axis only rotates the trajectory about the centre of mass, and
    for a negligible companion (q = 1e-9) the primary sits there whatever the
    separation, so the light curve is the single-lens finite-source curve at
    u = sqrt(tau^2 + u0^2) -- here against the independent polygon integral
    of the analytic point-lens images."""
    s, q, rho, u0, alpha, t0, tE = 1.3, 1e-9, 0.05, 0.2, 0.7, 0.0, 10.0
    t = np.array([-3.0, -1.0, 0.5, 2.5])
    mu, st, _ = O.lightcurve_orbital(s, q, rho, u0, alpha, t0, tE, 0.05, 0.3, t, scan_K=64)
    assert (st == 0).all()
    tau = (t - t0) / tE
    ref = np.array([(4 * single_lens_polygon(u, rho, 1 << 16) - single_lens_polygon(u, rho, 1 << 15)) / 3
                    for u in np.hypot(tau, u0)])
    assert np.max(np.abs(mu / ref - 1)) < 1e-7


def test_orbital_motion_mirror_symmetry():
    """Reflecting the trajectory in the lens axis, (u0, alpha, dalpha/dt) ->
    (-u0, -alpha, -dalpha/dt), maps y2 to -y2 at every time; the binary lens
    is symmetric about its axis, so the light curve is unchanged."""
    s, q, rho, u0, alpha, t0, tE, ds, da = 1.0, 0.1, 0.02, 0.05, 1.1, 0.0, 15.0, 0.02, 0.08
    t = np.linspace(-2.0, 2.0, 7)
    a, sa, _ = O.lightcurve_orbital(s, q, rho, u0, alpha, t0, tE, ds, da, t, scan_K=64)
    b, sb, _ = O.lightcurve_orbital(s, q, rho, -u0, -alpha, t0, tE, ds, -da, t, scan_K=64)
    assert (sa == 0).all() and (sb == 0).all()
    np.testing.assert_allclose(a, b, rtol=1e-10)


def _ld_profile(r, rho, u):
    return 1.0 - u * (1.0 - np.sqrt(np.clip(1.0 - (r / rho) ** 2, 0.0, None)))


def _point_mag(d):
    return (d * d + 2.0) / (d * np.sqrt(d * d + 4.0))


@pytest.mark.parametrize("rho,u", [(0.1, 0.6), (0.01, 0.3), (0.5, 1.0)])
def test_limb_darkening_centred_point_lens(rho, u):
    """A limb-darkened disc centred on a point lens (negligible companion):
    the definition mu = Int I mu_ps dA / Int I dA with the analytic point-lens
    magnification (r^2 + 2)/(r sqrt(r^2 + 4)) at distance r, as a 1-D radial
    integral -- no contour, no annuli."""
    from scipy.integrate import quad

    s, q = 10.0, 1e-9
    x1 = -q * s / (1 + q)
    num = quad(lambda r: _ld_profile(r, rho, u) * _point_mag(r) * 2 * np.pi * r, 0.0, rho, epsrel=1e-12,
               limit=200)[0]
    den = np.pi * rho * rho * (1.0 - u / 3.0)
    mu, st = O.mag_ld(s, q, rho, u, x1, 0.0)
    assert st == 0
    assert abs(mu / (num / den) - 1) < 1e-8


def test_limb_darkening_off_centre_point_lens():
    """Off-centre limb-darkened disc on a point lens: the definition as a 2-D
    integral over the disc in polar coordinates about its centre, with the
    analytic point-lens magnification; and u = 0 gives the uniform disc."""
    from scipy.integrate import dblquad

    s, q, rho, u, d = 10.0, 1e-9, 0.2, 0.7, 0.3
    x1 = -q * s / (1 + q)
    f = lambda th, r: _ld_profile(r, rho, u) * _point_mag(np.hypot(d + r * np.cos(th), r * np.sin(th))) * r
    num = dblquad(f, 0.0, rho, 0.0, 2 * np.pi, epsabs=0.0, epsrel=1e-10)[0]
    den = np.pi * rho * rho * (1.0 - u / 3.0)
    mu, st = O.mag_ld(s, q, rho, u, x1 + d, 0.0)
    assert st == 0 and abs(mu / (num / den) - 1) < 1e-7
    m0, _ = O.mag_ld(1.0, 0.1, 0.05, 0.0, 0.1, 0.05)
    assert abs(m0 / O.mag(1.0, 0.1, 0.05, [0.1], [0.05])[0][0] - 1) < 1e-12
