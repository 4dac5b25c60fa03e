"""Host-side checks of the C ABI: the library builds and loads, exports every
entry point declared in include/twinkle.h, and rejects invalid arguments
before any device work (so these run without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2501_03322_gb300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w \*]*?\b(tw_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    lib = P.lib()
    names = declared_functions()
    assert "tw_mag" in names and "tw_lightcurve_batch" in names
    for nm in names:
        assert hasattr(lib, nm), nm
    assert lib.tw_version() >= 100


def test_status_strings_and_defaults():
    for code in (0, -1, -2, -3, -4, 1):
        assert P.status_str(code) and P.status_str(code) != "unknown status"
    o = P.TwOpts()
    P.lib().tw_opts_default(ctypes.byref(o))
    assert (o.precision, o.samples_per_iter, o.max_samples, o.autotune) == (0, 64, 4096, 0)
    assert o.stream is None and o.err_out is None


def _mag(s=1.0, q=1e-3, rho=1e-3, n=4, tol=1e-4, opts=None, y=None):
    y1 = np.zeros(max(n, 1)) if y is None else y
    out = np.zeros(max(n, 1))
    return P.lib().tw_mag_ex(s, q, rho, y1.ctypes.data_as(ctypes.c_void_p), y1.ctypes.data_as(ctypes.c_void_p), n,
                             tol, out.ctypes.data_as(ctypes.c_void_p), None if opts is None else ctypes.byref(opts))


@pytest.mark.parametrize("kw", [dict(n=-1), dict(s=0.0), dict(q=-1.0), dict(rho=0.0), dict(rho=float("nan")),
                                dict(s=float("inf")), dict(tol=0.0), dict(tol=float("nan"))])
def test_invalid_arguments_rejected(kw):
    assert _mag(**kw) == P.TW_EINVAL


def test_invalid_options_rejected():
    for field, val in [("precision", 7), ("samples_per_iter", 48), ("samples_per_iter", 256), ("max_samples", 16),
                       ("max_samples", 1 << 20), ("warps_per_position", 3), ("warps_per_position", 8)]:
        o = P.TwOpts()
        P.lib().tw_opts_default(ctypes.byref(o))
        setattr(o, field, val)
        assert _mag(opts=o) == P.TW_EINVAL, field


def test_null_pointers_and_empty_calls():
    lib = P.lib()
    assert lib.tw_mag(1.0, 1e-3, 1e-3, None, None, 3, 1e-4, None) == P.TW_EINVAL
    assert lib.tw_mag(1.0, 1e-3, 1e-3, None, None, 0, 1e-4, None) == P.TW_OK  # nothing to do
    assert lib.tw_lightcurve(1.0, 1e-3, 1e-3, 0.1, 1.0, 0.0, 0.0, None, 0, 1e-4, None) == P.TW_EINVAL  # tE = 0
    assert lib.tw_lightcurve(1.0, 1e-3, 1e-3, 0.1, 1.0, 0.0, 20.0, None, 0, 1e-4, None) == P.TW_OK
    assert lib.tw_last_launch_work(None) == P.TW_EINVAL
    assert lib.tw_last_launch_ms(None) == P.TW_EINVAL
    assert lib.tw_mag_gated(None, None, None, None, None, 3, 1e-4, None, None, None) == P.TW_EINVAL
    assert lib.tw_mag_gated(None, None, None, None, None, 0, 1e-4, None, None, None) == P.TW_OK


def test_batch_offsets_validated_on_host():
    lib = P.lib()
    params = np.array([[1.0, 1e-3, 1e-3, 0.1, 1.0, 0.0, 20.0]] * 2)
    times = np.zeros(5)
    out = np.zeros(5)
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    for bad in ([1, 2, 5], [0, 3, 2]):
        off = np.array(bad, np.int64)
        assert lib.tw_lightcurve_batch(vp(params), vp(off), vp(times), 2, 1e-4, vp(out), None) == P.TW_EINVAL
    assert lib.tw_lightcurve_batch(vp(params), vp(np.array([0, 0, 0], np.int64)), vp(times), 2, 1e-4, vp(out),
                                   None) == P.TW_OK
    assert lib.tw_lightcurve_batch(None, None, None, 0, 1e-4, None, None) == P.TW_OK


def test_no_gpu_reports_cuda_error_not_a_fallback():
    """Without a GPU a valid call fails with TW_ECUDA: there is no CPU path."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    assert _mag(n=4) == P.TW_ECUDA
    with pytest.raises(P.TwError):
        P.mag(1.0, 1e-3, 1e-3, np.zeros(3), np.zeros(3))


def test_device_memory_cap_refuses_before_device_work(monkeypatch):
    """With TW_DEVICE_MEMORY_LIMIT below the smallest sample arena a launch
    needs, the call returns TW_ENOMEM before any device work and writes
    nothing (allocation failure injected on the host, no GPU involved)."""
    monkeypatch.setenv("TW_DEVICE_MEMORY_LIMIT", "4096")
    y = np.array([0.1, 0.2, 0.3, 0.4])
    out = np.full(4, -7.0)
    rc = P.lib().tw_mag_ex(1.0, 1e-3, 1e-3, y.ctypes.data_as(ctypes.c_void_p), y.ctypes.data_as(ctypes.c_void_p), 4,
                           1e-4, out.ctypes.data_as(ctypes.c_void_p), None)
    assert rc == P.TW_ENOMEM
    assert (out == -7.0).all()
    assert "memory" in P.status_str(rc)
