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
def test_noalloc_central_caustic_against_oracle(prec):
    """The central-caustic set (limbs crossing a tiny caustic next to its cusps,
    magnifications up to 1e4): tw_mag_noalloc matches tw_mag_ex at the same
    sample cap everywhere, and the oracle wherever that cap was not reached."""
    import os

    gold = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "central_wide.txt")
    rows = [ln.split() for ln in open(gold) if not ln.startswith("#") and ln.strip()]
    y1 = np.array([float(r[1]) for r in rows])
    y2 = np.array([float(r[2]) for r in rows])
    ref = np.array([float(r[3]) for r in rows])
    ok = np.array([int(r[4]) == 0 for r in rows])
    c = W.CENTRAL_WIDE
    y1d = torch.as_tensor(y1, device="cuda")
    y2d = torch.as_tensor(y2, device="cuda")
    mu, err, ns, st = P.mag(c["s"], c["q"], c["rho"], y1d, y2d, rel_tol=c["rel_tol"], precision=prec,
                            max_samples=512, details=True)
    st = st.cpu().numpy()
    mu = mu.cpu().numpy()
    outd = torch.full_like(y1d, float("nan"))
    assert P.lib().tw_mag_noalloc(c["s"], c["q"], c["rho"], ctypes.c_void_p(y1d.data_ptr()),
                                  ctypes.c_void_p(y2d.data_ptr()), y1d.numel(), c["rel_tol"],
                                  ctypes.c_void_p(outd.data_ptr()), prec, 512,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == P.TW_OK
    torch.cuda.synchronize()
    got = outd.cpu().numpy()
    assert np.max(np.abs(got / mu - 1.0)) <= TOL
    clean = ok & ((st & P.POS_CAP) == 0)
    assert clean.sum() >= 0.99 * len(rows)
    assert np.max(np.abs(got[clean] / ref[clean] - 1.0)) <= TOL


@pytest.mark.parametrize("prec", [P.PREC_FP64, P.PREC_MIXED])
def test_noalloc_runs_the_slope_repair_pass(prec):
    """Positions whose caustic crossing fails the slope test (Sec. 2.4.2) within
    512 limb samples, found among 2^20 seeded queries near caustics: tw_mag_ex
    repairs them in its second pass, and tw_mag_noalloc, which has that pass
    too, gives the same results (without it they differ by up to ~1e-3)."""
    s, q, rho, y1, y2 = P.surrogate_sample(3, 1 << 20)
    mu, err, ns, st = P.mag_multi(s, q, rho, y1, y2, rel_tol=TOL, precision=prec, max_samples=512, details=True)
    torch.cuda.synchronize()
    hit = np.nonzero((st.cpu().numpy() & P.POS_SLOPE) != 0)[0][:8]
    assert hit.size >= 1
    repaired = 0
    for i in hit:
        lens = [float(t[i]) for t in (s, q, rho)]
        ref, _, _, st1 = P.mag(*lens, y1[i:i + 1], y2[i:i + 1], rel_tol=TOL, precision=prec, max_samples=512,
                               details=True)
        repaired += int(int(st1[0]) & P.POS_SLOPE != 0)
        outd = torch.full_like(y1[i:i + 1], float("nan"))
        for _ in range(2):
            assert call_noalloc(*lens, y1[i:i + 1].contiguous(), y2[i:i + 1].contiguous(), outd, prec) == P.TW_OK
            torch.cuda.synchronize()
            assert abs(float(outd[0]) / float(ref[0]) - 1.0) <= 1e-12
    assert repaired >= 1  # the repair pass ran on at least one of them


def test_noalloc_rejects_oversized_and_host_requests():
    y1d = torch.zeros(8, dtype=torch.float64, device="cuda")
    outd = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert call_noalloc(1.0, 1e-3, 1e-3, y1d, y1d, outd, P.PREC_FP64, max_samples=1024) == P.TW_ETOOBIG
    assert "static scratch" in P.status_str(P.TW_ETOOBIG)
    h = np.zeros(8)
    rc = P.lib().tw_mag_noalloc(1.0, 1e-3, 1e-3, h.ctypes.data_as(ctypes.c_void_p), h.ctypes.data_as(ctypes.c_void_p),
                                8, TOL, h.ctypes.data_as(ctypes.c_void_p), 0, 512, None)
    assert rc == P.TW_EINVAL
