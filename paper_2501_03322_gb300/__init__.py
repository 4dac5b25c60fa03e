"""GB300-native finite-source binary-lens magnification by contour integration.

Thin ctypes binding over the C ABI of ``libtwinkle_gb300.so`` (declared in
``include/twinkle.h``).  Every step of the computation runs in the library's
CUDA kernels; this module only marshals arguments.  Arrays may be NumPy arrays
(host memory: the call is synchronous) or CUDA ``torch`` tensors (device
memory: the call is asynchronous on the given or current torch stream).

Functions mirror the C entry points:

* ``mag(s, q, rho, y1, y2, rel_tol, ...)``            -- ``tw_mag_ex``
* ``lightcurve(s, q, rho, u0, alpha, t0, tE, times, rel_tol, ...)`` -- ``tw_lightcurve_ex``
* ``lightcurve_batch(params, offsets, times, rel_tol, ...)``         -- ``tw_lightcurve_batch``

If the shared library is missing it is built from ``csrc/`` with nvcc; if that
is impossible the import of the library fails loudly.  There is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

TW_OK, TW_EINVAL, TW_ECUDA, TW_ENOMEM, TW_ETIMEOUT, TW_ETOOBIG, TW_WCAP = 0, -1, -2, -3, -4, -5, 1
POS_CAP, POS_IMAGECOUNT, POS_NONFINITE, POS_SOLVER, POS_SLOPE = 1, 2, 4, 8, 16
POS_EXPANSION, POS_NETWORK = 32, 64  # tw_surrogate_mag: answered without contour integration
PREC_FP64, PREC_MIXED = 0, 1

_lock = threading.Lock()
_lib = None


class TwError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (code %d)" % (msg, code))
        self.code = code


class TwOpts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("samples_per_iter", ctypes.c_int),
        ("max_samples", ctypes.c_int),
        ("autotune", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("err_out", ctypes.c_void_p),
        ("nsamp_out", ctypes.c_void_p),
        ("pos_status", ctypes.c_void_p),
        ("warps_per_position", ctypes.c_int),
    ]


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded shared library (built on first use if absent)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                path = _build.build()
            L = ctypes.CDLL(path)
            d, i64, P, I = ctypes.c_double, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
            L.tw_opts_default.argtypes = [P]
            L.tw_opts_default.restype = None
            L.tw_mag.argtypes = [d, d, d, P, P, i64, d, P]
            L.tw_mag.restype = I
            L.tw_mag_ex.argtypes = [d, d, d, P, P, i64, d, P, P]
            L.tw_mag_ex.restype = I
            L.tw_lightcurve.argtypes = [d, d, d, d, d, d, d, P, i64, d, P]
            L.tw_lightcurve.restype = I
            L.tw_lightcurve_ex.argtypes = [d, d, d, d, d, d, d, P, i64, d, P, P]
            L.tw_lightcurve_ex.restype = I
            L.tw_mag_ld.argtypes = [d, d, d, d, P, P, i64, d, P, P]
            L.tw_mag_ld.restype = I
            L.tw_lightcurve_orbital.argtypes = [d, d, d, d, d, d, d, d, d, P, i64, d, P, P]
            L.tw_lightcurve_orbital.restype = I
            L.tw_mag_multi.argtypes = [P, P, P, P, P, i64, d, P, P]
            L.tw_mag_gated.argtypes = [P, P, P, P, P, i64, d, P, P, P]
            L.tw_mag_gated.restype = I
            L.tw_mag_multi.restype = I
            L.tw_lightcurve_batch.argtypes = [P, P, P, i64, d, P, P]
            L.tw_lightcurve_batch.restype = I
            L.tw_status_str.argtypes = [I]
            L.tw_status_str.restype = ctypes.c_char_p
            L.tw_version.argtypes = []
            L.tw_version.restype = I
            L.tw_last_launch_work.argtypes = [P]
            L.tw_last_launch_work.restype = I
            L.tw_last_launch_ms.argtypes = [P]
            L.tw_last_launch_ms.restype = I
            L.tw_selftest_slope.argtypes = [d, d, d, d, d, P, I, I, P]
            L.tw_selftest_slope.restype = I
            L.tw_selftest_timeout.argtypes = [ctypes.c_uint]
            L.tw_selftest_timeout.restype = I
            L.tw_peak_probe.argtypes = [I, P]
            L.tw_peak_probe.restype = I
            L.tw_selftest.argtypes = [P]
            L.tw_selftest.restype = I
            L.tw_mag_noalloc.argtypes = [d, d, d, P, P, i64, d, P, I, I, P]
            L.tw_mag_noalloc.restype = I
            L.tw_gemm_bf16.argtypes = [P, P, I, I, I, P, P]
            L.tw_gemm_bf16.restype = I
            L.tw_surrogate_train.argtypes = [ctypes.c_char_p, i64, ctypes.c_uint64, I, P, P]
            L.tw_surrogate_train.restype = I
            L.tw_surrogate_mag.argtypes = [ctypes.c_char_p, P, P, P, P, P, i64, d, d, P, P, P]
            L.tw_surrogate_mag.restype = I
            L.tw_last_surrogate_stats.argtypes = [P]
            L.tw_last_surrogate_stats.restype = I
            L.tw_surrogate_sample.argtypes = [ctypes.c_uint64, i64, P, P, P, P, P, P]
            L.tw_surrogate_sample.restype = I
            _lib = L
    return _lib


def status_str(code: int) -> str:
    return lib().tw_status_str(code).decode()


def _is_torch_cuda(a) -> bool:
    return hasattr(a, "is_cuda") and bool(a.is_cuda)


def _ptr(a):
    if a is None:
        return None
    if _is_torch_cuda(a):
        return ctypes.c_void_p(a.data_ptr())
    if hasattr(a, "data_ptr"):  # CPU torch tensor
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int):
    if rc < 0:
        raise TwError(rc, status_str(rc))
    return rc


def _host(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def _alloc_like(ref, n, dtype_np, dtype_torch_name):
    if _is_torch_cuda(ref):
        import torch

        return torch.empty(n, dtype=getattr(torch, dtype_torch_name), device=ref.device)
    return np.empty(n, dtype=dtype_np)


def make_opts(precision=PREC_FP64, samples_per_iter=64, max_samples=4096, stream=None, err=None, nsamp=None,
              status=None, autotune=False, use_graph=False, warps_per_position=1) -> TwOpts:
    o = TwOpts()
    lib().tw_opts_default(ctypes.byref(o))
    o.warps_per_position = int(warps_per_position)
    o.autotune = int(bool(autotune))
    o.use_graph = int(bool(use_graph))
    o.precision = int(precision)
    o.samples_per_iter = int(samples_per_iter)
    o.max_samples = int(max_samples)
    o.stream = stream
    o.err_out = _ptr(err).value if err is not None else None
    o.nsamp_out = _ptr(nsamp).value if nsamp is not None else None
    o.pos_status = _ptr(status).value if status is not None else None
    return o


def _stream_of(ref, stream):
    if stream is not None:
        return getattr(stream, "cuda_stream", stream)
    if _is_torch_cuda(ref):
        import torch

        return torch.cuda.current_stream(ref.device).cuda_stream
    return None


def _prep(arr):
    if _is_torch_cuda(arr):
        return arr.contiguous()
    return _host(arr, np.float64)


def last_launch_work() -> dict:
    """Samples, FP64/FP32 Aberth sweeps, edge evaluations and FP64 Newton passes of the last launch."""
    a = np.zeros(5, np.int64)
    _check(lib().tw_last_launch_work(a.ctypes.data_as(ctypes.c_void_p)))
    return dict(samples=int(a[0]), sweeps64=int(a[1]), sweeps32=int(a[2]), edges=int(a[3]), newton64=int(a[4]))


def selftest_slope(s, q, rho, y1, y2, theta, mode) -> dict:
    """Device self-test of the slope test and repair on a planted misjudgment (tw_selftest_slope)."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    out = np.zeros(4)
    _check(lib().tw_selftest_slope(s, q, rho, y1, y2, th.ctypes.data_as(ctypes.c_void_p), int(th.size), int(mode),
                                   out.ctypes.data_as(ctypes.c_void_p)))
    return dict(detected=bool(out[0]), restored=bool(out[1]), area_change=float(out[2]), crossing=int(out[3]))


def last_launch_ms() -> float:
    """Device time (ms) of the last contour-integration kernel launch, from CUDA events on its stream."""
    a = np.zeros(1, np.float32)
    _check(lib().tw_last_launch_ms(a.ctypes.data_as(ctypes.c_void_p)))
    return float(a[0])


def gemm_bf16(A, B, out=None, stream=None):
    """C = A @ B.T on the tensor cores (tw_gemm_bf16); A [M, K], B [N, K] bf16 CUDA tensors."""
    import torch

    M, K = A.shape
    N = B.shape[0]
    if out is None:
        out = torch.empty(M, N, dtype=torch.float32, device=A.device)
    st = _stream_of(A, stream)
    _check(lib().tw_gemm_bf16(_ptr(A.contiguous()), _ptr(B.contiguous()), M, N, K, _ptr(out), st))
    return out


def surrogate_train(path, nsamples=1_000_000, seed=0, epochs=4, stream=None):
    """Train the MLP surrogate (tw_surrogate_train); returns its statistics."""
    st = np.zeros(9)
    o = make_opts(stream=getattr(stream, "cuda_stream", stream))
    _check(lib().tw_surrogate_train(str(path).encode(), int(nsamples), int(seed), int(epochs),
                                    st.ctypes.data_as(ctypes.c_void_p), ctypes.byref(o)))
    return dict(drawn=int(st[0]), labelled=int(st[1]), rows=int(st[2]), loss=float(st[3]), target_std=float(st[4]),
                heldout=int(st[5]), kappa_cal=float(st[6]), heldout_accepted=float(st[7]),
                heldout_accepted_max_err=float(st[8]))


def surrogate_sample(seed, n, device="cuda"):
    """n seeded query positions near caustics (tw_surrogate_sample): five CUDA tensors."""
    import torch

    a = [torch.empty(int(n), dtype=torch.float64, device=device) for _ in range(5)]
    st = torch.cuda.current_stream(a[0].device).cuda_stream
    _check(lib().tw_surrogate_sample(int(seed), int(n), *[_ptr(t) for t in a], st))
    return a


def surrogate_mag(path, s, q, rho, y1, y2, rel_tol=1e-4, kappa=3.0, precision=PREC_FP64, max_samples=4096, out=None,
                  stream=None, details=False, status=None):
    """Surrogate magnification with contour fallback (tw_surrogate_mag).

    Returns (out, n_fallback) or, with details=True, (out, counts) where counts =
    dict(fallback=..., network=..., expansion=...).  `status` (optional int8
    array of the inputs' kind) receives POS_EXPANSION / POS_NETWORK for the
    queries answered without contour integration, contour status bits for the
    others."""
    arrs = [_prep(a) for a in (s, q, rho, y1, y2)]
    n = int(arrs[0].shape[0])
    if out is None:
        out = _alloc_like(arrs[0], n, np.float64, "float64")
    c = np.zeros(5, np.int64)
    o = make_opts(precision, 64, max_samples, _stream_of(arrs[0], stream), status=status)
    _check(lib().tw_surrogate_mag(str(path).encode(), *[_ptr(a) for a in arrs], n, rel_tol, kappa, _ptr(out),
                                  c.ctypes.data_as(ctypes.c_void_p), ctypes.byref(o)))
    if details:
        return out, dict(fallback=int(c[0]), network=int(c[1]), expansion=int(c[2]), flagged=int(c[3]),
                         uncertain=int(c[4]))
    return out, int(c[0])


def last_surrogate_stats() -> dict:
    """Device times (ms) and work of the latest surrogate call (tw_last_surrogate_stats)."""
    a = np.zeros(8)
    _check(lib().tw_last_surrogate_stats(a.ctypes.data_as(ctypes.c_void_p)))
    return dict(features_ms=float(a[0]), network_ms=float(a[1]), gemm_ms=float(a[2]), point_solves=int(a[3]),
                point_sweeps32=int(a[4]), newton64=int(a[5]), caustic_iters=int(a[6]), gemm_rows=int(a[7]))


def peak_probe(kind: str = "fp64") -> float:
    """Measured FMA-pipe throughput (FLOP/s) of the current device (tw_peak_probe)."""
    v = np.zeros(1)
    _check(lib().tw_peak_probe(0 if kind == "fp64" else 1, v.ctypes.data_as(ctypes.c_void_p)))
    return float(v[0])


def selftest_rcp() -> tuple:
    """Largest relative errors of the device FP64 reciprocals (full, one-step) against IEEE division."""
    v = np.zeros(2)
    _check(lib().tw_selftest(v.ctypes.data_as(ctypes.c_void_p)))
    return float(v[0]), float(v[1])


def mag(s, q, rho, y1, y2, rel_tol=1e-4, precision=PREC_FP64, samples_per_iter=64, max_samples=4096,
        out=None, details=False, stream=None, autotune=False, use_graph=False, warps_per_position=1):
    """Finite-source magnification of positions (y1[i], y2[i]) (tw_mag_ex).

    Returns ``out`` or, with details=True, (out, err, nsamp, status)."""
    y1, y2 = _prep(y1), _prep(y2)
    n = int(y1.shape[0])
    if out is None:
        out = _alloc_like(y1, n, np.float64, "float64")
    err = nsamp = status = None
    if details:
        err = _alloc_like(y1, n, np.float64, "float64")
        nsamp = _alloc_like(y1, n, np.int32, "int32")
        status = _alloc_like(y1, n, np.int8, "int8")
    o = make_opts(precision, samples_per_iter, max_samples, _stream_of(y1, stream), err, nsamp, status, autotune,
                  use_graph, warps_per_position)
    _check(lib().tw_mag_ex(s, q, rho, _ptr(y1), _ptr(y2), n, rel_tol, _ptr(out), ctypes.byref(o)))
    return (out, err, nsamp, status) if details else out


def mag_ld(s, q, rho, u, y1, y2, rel_tol=1e-4, precision=PREC_FP64, max_samples=4096, out=None, details=False,
           stream=None):
    """Magnification of linearly limb-darkened sources (tw_mag_ld), brightness 1 - u (1 - sqrt(1 - r^2/rho^2))."""
    y1, y2 = _prep(y1), _prep(y2)
    n = int(y1.shape[0])
    if out is None:
        out = _alloc_like(y1, n, np.float64, "float64")
    err = nsamp = status = None
    if details:
        err = _alloc_like(y1, n, np.float64, "float64")
        nsamp = _alloc_like(y1, n, np.int32, "int32")
        status = _alloc_like(y1, n, np.int8, "int8")
    o = make_opts(precision, 64, max_samples, _stream_of(y1, stream), err, nsamp, status)
    _check(lib().tw_mag_ld(s, q, rho, u, _ptr(y1), _ptr(y2), n, rel_tol, _ptr(out), ctypes.byref(o)))
    return (out, err, nsamp, status) if details else out


def mag_noalloc(s, q, rho, y1, y2, rel_tol=1e-4, precision=PREC_FP64, max_samples=512, out=None, stream=None):
    """tw_mag_noalloc: like mag() but the library allocates no device memory
    (its scratch is a static device array).  y1, y2 and out must be CUDA
    tensors; the call is asynchronous on the given or current stream."""
    if not (_is_torch_cuda(y1) and _is_torch_cuda(y2)):
        raise TypeError("mag_noalloc needs CUDA tensors")
    y1, y2 = y1.contiguous(), y2.contiguous()
    n = int(y1.shape[0])
    if out is None:
        out = _alloc_like(y1, n, np.float64, "float64")
    st = _stream_of(y1, stream)
    _check(lib().tw_mag_noalloc(s, q, rho, _ptr(y1), _ptr(y2), n, rel_tol, _ptr(out), int(precision),
                                int(max_samples), st))
    return out


def mag_multi(s, q, rho, y1, y2, rel_tol=1e-4, precision=PREC_FP64, samples_per_iter=64, max_samples=4096,
              out=None, details=False, stream=None, autotune=False, use_graph=False, warps_per_position=1):
    """Magnification of positions each with its own lens and source radius (tw_mag_multi)."""
    arrs = [_prep(a) for a in (s, q, rho, y1, y2)]
    n = int(arrs[0].shape[0])
    if out is None:
        out = _alloc_like(arrs[0], n, np.float64, "float64")
    err = nsamp = status = None
    if details:
        err = _alloc_like(arrs[0], n, np.float64, "float64")
        nsamp = _alloc_like(arrs[0], n, np.int32, "int32")
        status = _alloc_like(arrs[0], n, np.int8, "int8")
    o = make_opts(precision, samples_per_iter, max_samples, _stream_of(arrs[0], stream), err, nsamp, status,
                  autotune, use_graph, warps_per_position)
    _check(lib().tw_mag_multi(*[_ptr(a) for a in arrs], n, rel_tol, _ptr(out), ctypes.byref(o)))
    return (out, err, nsamp, status) if details else out


def mag_gated(s, q, rho, y1, y2, rel_tol=1e-4, precision=PREC_FP64, max_samples=4096, out=None, stream=None):
    """Magnification with the point-source adequacy gate (tw_mag_gated): positions
    whose expansion is certified take its value, the rest are contour-integrated.
    Returns (out, number of contour-integrated positions)."""
    arrs = [_prep(a) for a in (s, q, rho, y1, y2)]
    n = int(arrs[0].shape[0])
    if out is None:
        out = _alloc_like(arrs[0], n, np.float64, "float64")
    o = make_opts(precision, 64, max_samples, _stream_of(arrs[0], stream), None, None, None, False, False)
    nc = np.zeros(1, np.int64)
    _check(lib().tw_mag_gated(*[_ptr(a) for a in arrs], n, rel_tol, _ptr(out), nc.ctypes.data_as(ctypes.c_void_p),
                              ctypes.byref(o)))
    return out, int(nc[0])


def lightcurve(s, q, rho, u0, alpha, t0, tE, times, rel_tol=1e-4, precision=PREC_FP64, samples_per_iter=64,
               max_samples=4096, out=None, details=False, stream=None, autotune=False, use_graph=False, warps_per_position=1):
    """Magnification along a straight-line trajectory (tw_lightcurve_ex)."""
    times = _prep(times)
    n = int(times.shape[0])
    if out is None:
        out = _alloc_like(times, n, np.float64, "float64")
    err = nsamp = status = None
    if details:
        err = _alloc_like(times, n, np.float64, "float64")
        nsamp = _alloc_like(times, n, np.int32, "int32")
        status = _alloc_like(times, n, np.int8, "int8")
    o = make_opts(precision, samples_per_iter, max_samples, _stream_of(times, stream), err, nsamp, status, autotune,
                  use_graph, warps_per_position)
    _check(lib().tw_lightcurve_ex(s, q, rho, u0, alpha, t0, tE, _ptr(times), n, rel_tol, _ptr(out), ctypes.byref(o)))
    return (out, err, nsamp, status) if details else out


def lightcurve_orbital(s, q, rho, u0, alpha, t0, tE, ds_dt, dalpha_dt, times, rel_tol=1e-4, precision=PREC_FP64,
                       max_samples=4096, out=None, details=False, stream=None, warps_per_position=1):
    """Light curve of an orbiting lens, s and alpha linear in time (tw_lightcurve_orbital)."""
    times = _prep(times)
    n = int(times.shape[0])
    if out is None:
        out = _alloc_like(times, n, np.float64, "float64")
    err = nsamp = status = None
    if details:
        err = _alloc_like(times, n, np.float64, "float64")
        nsamp = _alloc_like(times, n, np.int32, "int32")
        status = _alloc_like(times, n, np.int8, "int8")
    o = make_opts(precision, 64, max_samples, _stream_of(times, stream), err, nsamp, status, False, False,
                  warps_per_position)
    _check(lib().tw_lightcurve_orbital(s, q, rho, u0, alpha, t0, tE, ds_dt, dalpha_dt, _ptr(times), n, rel_tol,
                                       _ptr(out), ctypes.byref(o)))
    return (out, err, nsamp, status) if details else out


def lightcurve_batch(params, offsets, times, rel_tol=1e-4, precision=PREC_FP64, samples_per_iter=64,
                     max_samples=4096, out=None, details=False, stream=None, autotune=False, use_graph=False, warps_per_position=1):
    """Many light curves in one launch (tw_lightcurve_batch).

    params: [ncurve, 7] (s, q, rho, u0, alpha, t0, tE); offsets: [ncurve + 1] int64."""
    if _is_torch_cuda(params):
        params, offsets, times = params.contiguous(), offsets.contiguous(), times.contiguous()
        total = int(offsets[-1].item())
    else:
        params = _host(params, np.float64)
        offsets = _host(offsets, np.int64)
        times = _host(times, np.float64)
        total = int(offsets[-1]) if offsets.size else 0
    ncurve = int(params.shape[0])
    if out is None:
        out = _alloc_like(times, total, np.float64, "float64")
    err = nsamp = status = None
    if details:
        err = _alloc_like(times, total, np.float64, "float64")
        nsamp = _alloc_like(times, total, np.int32, "int32")
        status = _alloc_like(times, total, np.int8, "int8")
    o = make_opts(precision, samples_per_iter, max_samples, _stream_of(times, stream), err, nsamp, status, autotune,
                  use_graph, warps_per_position)
    _check(lib().tw_lightcurve_batch(_ptr(params), _ptr(offsets), _ptr(times), ncurve, rel_tol, _ptr(out),
                                     ctypes.byref(o)))
    return (out, err, nsamp, status) if details else out
