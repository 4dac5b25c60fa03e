"""Failure detection on the GPU without faulting it: a bounded device-side
wait that runs out reports TW_ETIMEOUT through the host, and an allocation
that the library's memory cap refuses reports TW_ENOMEM with nothing written;
in both cases the context stays usable for the next call."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2501_03322_gb300 as P  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _still_works():
    s, q = 10.0, 1e-9
    mu = P.mag(s, q, 0.1, np.array([-q * s / (1 + q)]), np.array([0.0]))
    assert abs(mu[0] / np.sqrt(1 + 4 / 0.01) - 1) < 1e-4


def test_bounded_wait_runs_out_and_reports():
    """An mbarrier that nothing arrives on: the kernel gives up after its poll
    limit, sets the error flag and returns; the host maps it to TW_ETIMEOUT."""
    for limit in (1 << 10, 1 << 16):
        assert P.lib().tw_selftest_timeout(limit) == P.TW_ETIMEOUT
    assert P.lib().tw_selftest_timeout(0) == P.TW_EINVAL
    _still_works()


def test_allocation_cap_refuses_the_arena(monkeypatch):
    """A cap above the smallest arena but below what the launch needs: the
    arena allocation is refused (TW_ENOMEM), the output is untouched, and
    without the cap the same call succeeds."""
    y1 = np.linspace(-0.1, 0.1, 1000)
    y2 = np.zeros(1000)
    out = np.full(1000, np.nan)
    monkeypatch.setenv("TW_DEVICE_MEMORY_LIMIT", str(20 << 20))
    with pytest.raises(P.TwError) as e:
        P.mag(1.0, 1e-3, 1e-3, y1, y2, max_samples=16384, out=out)
    assert e.value.code == P.TW_ENOMEM
    assert np.isnan(out).all()
    monkeypatch.delenv("TW_DEVICE_MEMORY_LIMIT")
    P.mag(1.0, 1e-3, 1e-3, y1, y2, max_samples=16384, out=out)
    assert np.isfinite(out).all() and (out >= 1.0 - 1e-4).all()
    _still_works()
