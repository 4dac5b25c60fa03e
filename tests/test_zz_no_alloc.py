"""tw_mag_noalloc: the magnification entry point for callers that cannot
allocate device memory (graph capture, caller-owned memory pools, real-time
loops).  Its scratch is a static device array inside the library; these tests
check that its output matches tw_mag_ex (which allocates its own working
memory) on two consecutive calls -- the second call reuses the static array as
the first one left it -- and that oversized requests are refused.

The file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2501_03322_gb300 as P  # noqa: E402
from paper_2501_03322_gb300 import workloads as W  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TOL = 1e-4


def positions():
    y1, y2 = W.map_grid()
    idx = W.sample_indices(y1.size, 3000, seed=55)
    s1, s2 = W.stress_positions(n=1000, seed=56)
    return np.concatenate([y1[idx], s1]), np.concatenate([y2[idx], s2])


def call_noalloc(s, q, rho, y1d, y2d, outd, prec, max_samples=512):
    stream = torch.cuda.current_stream().cuda_stream
    return P.lib().tw_mag_noalloc(s, q, rho, ctypes.c_void_p(y1d.data_ptr()), ctypes.c_void_p(y2d.data_ptr()),
                                  y1d.numel(), TOL, ctypes.c_void_p(outd.data_ptr()), prec, max_samples,
                                  ctypes.c_void_p(stream))


@pytest.mark.parametrize("prec", [P.PREC_FP64, P.PREC_MIXED])
def test_noalloc_matches_tw_mag_on_two_calls(prec):
    y1, y2 = positions()
    y1d = torch.as_tensor(y1, device="cuda")
    y2d = torch.as_tensor(y2, device="cuda")
    for lens in [(0.8, 1e-4, 5e-4), (1.0, 0.5, 0.05)]:
        s, q, rho = lens
        ref = P.mag(s, q, rho, y1d, y2d, rel_tol=TOL, precision=prec, max_samples=512).cpu().numpy()
        for _ in range(2):
            outd = torch.full_like(y1d, float("nan"))
            assert call_noalloc(s, q, rho, y1d, y2d, outd, prec) == P.TW_OK
            torch.cuda.synchronize()
            got = outd.cpu().numpy()
            assert np.isfinite(got).all()
            assert np.max(np.abs(got / ref - 1.0)) <= TOL


@pytest.mark.parametrize("prec", [P.PREC_FP64, P.PREC_MIXED])
def test_noalloc_caustic_crossings_against_oracle(prec):
    """Limbs that cross caustics, within the 512-sample cap of this entry
    point: the central-caustic light curve (its 1000 positions, from the
    oracle's trajectory) and the map cells within rho of the planetary caustic.
    tw_mag_noalloc matches tw_mag_ex at the same cap everywhere, and the
    oracle's stored values wherever that cap was not reached."""
    import os

    import oracle as O

    gold = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

    def rows(name):
        return [ln.split() for ln in open(os.path.join(gold, name)) if not ln.startswith("#") and ln.strip()]

    c = W.LIGHTCURVE_CENTRAL
    lc = rows("lightcurve_central.txt")
    y1, y2 = O.trajectory(c["u0"], c["alpha"], c["t0"], c["tE"], np.array([float(r[0]) for r in lc]))
    cases = [((c["s"], c["q"], c["rho"]), y1, y2, np.array([float(r[1]) for r in lc]))]
    m = W.MAP_PLANETARY
    mp = [r for r in rows("map_planetary.txt") if int(r[5]) >= 2]
    cases.append(((m["s"], m["q"], m["rho"]), np.array([float(r[1]) for r in mp]), np.array([float(r[2]) for r in mp]),
                  np.array([float(r[3]) for r in mp])))
    for lens, a, b, ref in cases:
        y1d = torch.as_tensor(a, device="cuda")
        y2d = torch.as_tensor(b, device="cuda")
        mu, err, ns, st = P.mag(*lens, y1d, y2d, rel_tol=TOL, precision=prec, max_samples=512, details=True)
        mu, st = mu.cpu().numpy(), st.cpu().numpy()
        outd = torch.full_like(y1d, float("nan"))
        assert call_noalloc(*lens, y1d, y2d, outd, prec) == P.TW_OK
        torch.cuda.synchronize()
        got = outd.cpu().numpy()
        assert np.max(np.abs(got / mu - 1.0)) <= TOL
        clean = (st & P.POS_CAP) == 0
        assert clean.sum() >= 0.95 * len(ref)
        assert np.max(np.abs(got[clean] / ref[clean] - 1.0)) <= TOL


def test_noalloc_rejects_oversized_and_host_requests():
    y1d = torch.zeros(8, dtype=torch.float64, device="cuda")
    outd = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert call_noalloc(1.0, 1e-3, 1e-3, y1d, y1d, outd, P.PREC_FP64, max_samples=1024) == P.TW_ETOOBIG
    assert "static scratch" in P.status_str(P.TW_ETOOBIG)
    h = np.zeros(8)
    rc = P.lib().tw_mag_noalloc(1.0, 1e-3, 1e-3, h.ctypes.data_as(ctypes.c_void_p), h.ctypes.data_as(ctypes.c_void_p),
                                8, TOL, h.ctypes.data_as(ctypes.c_void_p), 0, 512, None)
    assert rc == P.TW_EINVAL
