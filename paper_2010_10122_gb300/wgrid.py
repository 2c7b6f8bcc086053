"""Thin Python binding of libwgrid.so (include/wgrid.h): argument marshalling only.

Every step of degrid / grid runs in the library's CUDA kernels (and cuFFT for the plane
transforms); this module checks shapes and dtypes, moves host inputs to the device when
given host arrays, passes raw pointers and the current torch CUDA stream, and turns error
codes into exceptions.  There is no CPU fallback: without the compiled library, or without
a CUDA device, the calls raise.

Names follow the paper (Arras et al., App. B): ``dirty2ms`` = degrid = R, ``ms2dirty`` =
grid = R^dagger; ``uvw`` (nrows, 3) metres, ``freq`` (nchan,) Hz, ``dirty`` (npix_x, npix_y),
``ms`` / ``vis`` (nrows, nchan) complex.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libwgrid.so")

WG_OK, WG_ERR_ARG, WG_ERR_OOM, WG_ERR_CUDA, WG_ERR_CUFFT, WG_ERR_TIMEOUT, WG_ERR_INTERNAL = range(7)
WG_F32, WG_F64 = 0, 1
NOALLOC_SCRATCH_BYTES = 64 << 20   # WG_NOALLOC_SCRATCH_BYTES of include/wgrid.h


class WgridError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"wgrid error {code}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("do_wstacking", ctypes.c_int), ("w_shift", ctypes.c_int),
                ("eps_safety", ctypes.c_double), ("max_workspace", ctypes.c_size_t),
                ("force_alpha", ctypes.c_int), ("force_sigma", ctypes.c_double),
                ("tile", ctypes.c_int), ("grid_variant", ctypes.c_int),
                ("fft_impl", ctypes.c_int), ("compact_index", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("ms_total", ctypes.c_double), ("ms_prep", ctypes.c_double),
                ("ms_screen", ctypes.c_double), ("ms_fft", ctypes.c_double),
                ("ms_grid", ctypes.c_double), ("ms_accum", ctypes.c_double),
                ("n_batches", ctypes.c_int64), ("n_planes", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_size_t), ("n_kernels", ctypes.c_int64),
                ("n_fft_calls", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class PlanInfo(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_int), ("sigma", ctypes.c_double), ("beta", ctypes.c_double),
                ("mu", ctypes.c_double), ("eps_kernel", ctypes.c_double),
                ("nu", ctypes.c_int64), ("nv", ctypes.c_int64), ("nw", ctypes.c_int64),
                ("dw", ctypes.c_double), ("w0", ctypes.c_double), ("nshift", ctypes.c_double),
                ("tile", ctypes.c_int), ("ntiles", ctypes.c_int64), ("nvis", ctypes.c_int64),
                ("batch", ctypes.c_int64), ("index_bytes", ctypes.c_size_t),
                ("workspace_bytes", ctypes.c_size_t), ("umax", ctypes.c_double),
                ("vmax", ctypes.c_double), ("wmin", ctypes.c_double), ("wmax", ctypes.c_double),
                ("fft_impl", ctypes.c_int), ("rounding_gain", ctypes.c_double),
                ("err_model", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# exported symbols and their ctypes signatures (checked by the ABI test)
_VP, _I64, _D, _I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
SIGNATURES = {
    "wg_default_options": (None, [ctypes.POINTER(Options)]),
    "wg_plan_create": (_I, [_VP, _VP, _I64, _I64, _I64, _I64, _D, _D, _D, _I, _VP,
                            ctypes.POINTER(Options), _VP, ctypes.POINTER(_VP)]),
    "wg_plan_destroy": (_I, [_VP]),
    "wg_plan_get_info": (_I, [_VP, ctypes.POINTER(PlanInfo)]),
    "wg_degrid": (_I, [_VP, _VP, _VP, _VP, _VP, ctypes.POINTER(Stats)]),
    "wg_grid": (_I, [_VP, _VP, _VP, _VP, _VP, ctypes.POINTER(Stats)]),
    "wg_degrid_noalloc": (_I, [_VP, _VP, _VP, _VP, _VP]),
    "wg_dirty2ms": (_I, [_VP, _VP, _I64, _I64, _VP, _VP, _I64, _I64, _D, _D, _D, _I, _I, _VP,
                         _VP, _VP]),
    "wg_ms2dirty": (_I, [_VP, _VP, _I64, _I64, _VP, _VP, _I64, _I64, _D, _D, _D, _I, _I, _VP,
                         _VP, _VP]),
    "wg_last_error": (ctypes.c_char_p, []),
    "wg_wait": (_I, [_VP, _D]),
    "wg_pool_trim": (_I, [ctypes.c_size_t]),
    "wg_kernel_table_size": (_I, []),
    "wg_kernel_table_row": (_I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_D), ctypes.POINTER(_D),
                                 ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "wg_kernel_phi": (_I, [_I, _D, _D, _VP, _VP, _I64]),
    "wg_kernel_poly": (_I, [_I, _D, _D, _VP, _VP, _I64]),
    "wg_kernel_psi": (_I, [_I, _D, _D, _VP, _VP, _I64]),
    "wg_kernel_design_size": (_I, []),
    "wg_kernel_design_row": (_I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_D), ctypes.POINTER(_D),
                                  ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "wg_kernel_eps": (_I, [_I, _D, _D, _D, ctypes.POINTER(_D)]),
    "wg_kernel_search": (_I, [_I, _D, _D, _D, ctypes.POINTER(_D), ctypes.POINTER(_D),
                              ctypes.POINTER(_D)]),
    "wg_plan_params": (_I, [_I64, _I64, _D, _D, _D, _I, ctypes.POINTER(Options), _D, _D, _D, _D,
                            _I64, ctypes.POINTER(PlanInfo)]),
    "wg_fft_time": (_I, [_I64, _I, _I64, _I, _I, ctypes.POINTER(_D)]),
    "wg_fft2d": (_I, [_VP, _I64, _I64, _I64, _I, _I, _I, _VP]),
    "wg_fma_peak": (_I, [_I, ctypes.POINTER(_D)]),
    "wg_fft_f32_tune": (_I, [_I, _I, _I]),
    "wg_version": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """Load libwgrid.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libwgrid.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != WG_OK:
        raise WgridError(rc, lib().wg_last_error().decode(errors="replace"))


def default_options(**kw) -> Options:
    o = Options()
    lib().wg_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if v is not None:
            setattr(o, k, v)
    return o


# ----------------------------------------------------------------------------------------
# tensor marshalling
# ----------------------------------------------------------------------------------------
def _device(dev=None) -> torch.device:
    if not torch.cuda.is_available():
        raise RuntimeError("wgrid needs a CUDA device; there is no CPU fallback")
    if dev is None:
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device(dev)


def _to_dev(x, dtype, dev, name, shape=None) -> torch.Tensor:
    if x is None:
        return None
    t = x if isinstance(x, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(x))
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")
    if t.device != dev:
        t = t.to(dev, non_blocking=True)
    return t.contiguous()


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream, dev):
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    return ctypes.c_void_p(s.cuda_stream)


def _order(stream, dev, *tensors):
    """A call on a caller-given stream reads tensors that were staged (or produced) on torch's
    current stream: the given stream first waits for the current one, and the device tensors
    are marked as used on it, so that the caching allocator does not hand their memory out
    again before the call's kernels are done with it."""
    if stream is None:
        return
    cur = torch.cuda.current_stream(dev)
    if stream.cuda_stream == cur.cuda_stream:
        return
    stream.wait_stream(cur)
    for t in tensors:
        if t is not None and t.is_cuda:
            t.record_stream(stream)


def _prec(precision) -> int:
    if precision in ("f32", "float32", torch.float32, np.float32, WG_F32):
        return WG_F32
    if precision in ("f64", "float64", torch.float64, np.float64, WG_F64):
        return WG_F64
    raise ValueError(f"unknown precision {precision!r}")


_REAL = {WG_F32: torch.float32, WG_F64: torch.float64}
_CPLX = {WG_F32: torch.complex64, WG_F64: torch.complex128}


class Plan:
    """A resident w-gridding plan for one observation (uvw, freq, mask), image geometry,
    accuracy and precision (wg_plan_create).  ``degrid`` applies R, ``grid`` R^dagger."""

    def __init__(self, uvw, freq, npix_x, npix_y, pixsize_x, pixsize_y, epsilon,
                 precision="f32", mask=None, do_wstacking=True, w_shift=True, eps_safety=None,
                 max_workspace=0, force_alpha=0, force_sigma=0.0, tile=0, grid_variant=0,
                 fft_impl=0, compact_index=False, stream=None, device=None):
        self._h = None
        dev = _device(device)
        self.device = dev
        self.prec = _prec(precision)
        uvw_t = _to_dev(uvw, torch.float64, dev, "uvw")
        if uvw_t.ndim != 2 or uvw_t.shape[1] != 3:
            raise ValueError("uvw must have shape (nrows, 3)")
        freq_t = _to_dev(freq, torch.float64, dev, "freq").reshape(-1)
        self.nrows, self.nchan = int(uvw_t.shape[0]), int(freq_t.numel())
        mask_t = _to_dev(mask, torch.uint8, dev, "mask", (self.nrows, self.nchan))
        self.npix_x, self.npix_y = int(npix_x), int(npix_y)
        opt = default_options(do_wstacking=int(bool(do_wstacking)), w_shift=int(bool(w_shift)),
                              eps_safety=None if eps_safety is None else float(eps_safety),
                              max_workspace=int(max_workspace),
                              force_alpha=int(force_alpha), force_sigma=float(force_sigma),
                              tile=int(tile), grid_variant=int(grid_variant),
                              fft_impl=int(fft_impl), compact_index=int(bool(compact_index)))
        h = ctypes.c_void_p()
        _order(stream, dev, uvw_t, freq_t, mask_t)
        with torch.cuda.device(dev):
            rc = lib().wg_plan_create(_ptr(uvw_t), _ptr(freq_t), self.nrows, self.nchan,
                                      self.npix_x, self.npix_y, float(pixsize_x),
                                      float(pixsize_y), float(epsilon), self.prec,
                                      _ptr(mask_t), ctypes.byref(opt),
                                      _stream_handle(stream, dev), ctypes.byref(h))
        _check(rc)
        self._h = h
        self.epsilon = float(epsilon)

    @property
    def info(self) -> dict:
        inf = PlanInfo()
        _check(lib().wg_plan_get_info(self._h, ctypes.byref(inf)))
        return inf.as_dict()

    def degrid(self, dirty, wgt=None, out=None, stream=None, stats=False):
        """vis = R(dirty): (nrows, nchan) complex on the plan's device."""
        dev = self.device
        d = _to_dev(dirty, _REAL[self.prec], dev, "dirty", (self.npix_x, self.npix_y))
        w = _to_dev(wgt, _REAL[self.prec], dev, "wgt", (self.nrows, self.nchan))
        if out is None:
            out = torch.empty((self.nrows, self.nchan), dtype=_CPLX[self.prec], device=dev)
        elif out.dtype != _CPLX[self.prec] or tuple(out.shape) != (self.nrows, self.nchan) \
                or not out.is_contiguous() or out.device != dev:
            raise ValueError("out: wrong dtype, shape, layout or device")
        st = Stats() if stats else None
        _order(stream, dev, d, w, out)
        with torch.cuda.device(dev):
            rc = lib().wg_degrid(self._h, _ptr(d), _ptr(w), _ptr(out), _stream_handle(stream, dev),
                                 ctypes.byref(st) if st is not None else None)
        _check(rc)
        return (out, st.as_dict()) if stats else out

    def degrid_noalloc(self, dirty, out, wgt=None, stream=None):
        """vis = R(dirty) through wg_degrid_noalloc: no allocation inside the call; ``out`` and
        the inputs must already be device tensors of the right dtype and shape, and the plan
        must have been made with max_workspace <= NOALLOC_SCRATCH_BYTES.  The call runs on
        ``stream`` (default: the current stream) as given: the caller orders it after the work
        that produced the inputs."""
        dev = self.device
        for t in (dirty, out) + (() if wgt is None else (wgt,)):
            if not isinstance(t, torch.Tensor) or t.device != dev or not t.is_contiguous():
                raise ValueError("degrid_noalloc needs contiguous tensors on the plan's device")
        if dirty.dtype != _REAL[self.prec] or out.dtype != _CPLX[self.prec] \
                or tuple(dirty.shape) != (self.npix_x, self.npix_y) \
                or tuple(out.shape) != (self.nrows, self.nchan):
            raise ValueError("degrid_noalloc: wrong dtype or shape")
        if wgt is not None and (wgt.dtype != _REAL[self.prec]
                                or tuple(wgt.shape) != (self.nrows, self.nchan)):
            raise ValueError("degrid_noalloc: wgt must be real of the plan's precision, "
                             "shape (nrows, nchan)")
        with torch.cuda.device(dev):
            rc = lib().wg_degrid_noalloc(self._h, _ptr(dirty), _ptr(wgt), _ptr(out),
                                         _stream_handle(stream, dev))
        _check(rc)
        return out

    def grid(self, vis, wgt=None, out=None, stream=None, stats=False):
        """dirty = R^dagger(vis): (npix_x, npix_y) real on the plan's device."""
        dev = self.device
        v = _to_dev(vis, _CPLX[self.prec], dev, "vis", (self.nrows, self.nchan))
        w = _to_dev(wgt, _REAL[self.prec], dev, "wgt", (self.nrows, self.nchan))
        if out is None:
            out = torch.empty((self.npix_x, self.npix_y), dtype=_REAL[self.prec], device=dev)
        elif out.dtype != _REAL[self.prec] or tuple(out.shape) != (self.npix_x, self.npix_y) \
                or not out.is_contiguous() or out.device != dev:
            raise ValueError("out: wrong dtype, shape, layout or device")
        st = Stats() if stats else None
        _order(stream, dev, v, w, out)
        with torch.cuda.device(dev):
            rc = lib().wg_grid(self._h, _ptr(v), _ptr(w), _ptr(out), _stream_handle(stream, dev),
                               ctypes.byref(st) if st is not None else None)
        _check(rc)
        return (out, st.as_dict()) if stats else out

    def close(self):
        if self._h is not None:
            lib().wg_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def dirty2ms(uvw, freq, dirty, wgt=None, pixsize_x=None, pixsize_y=None, epsilon=1e-5,
             do_wstacking=True, mask=None, stream=None, device=None):
    """One-shot degrid with the paper's argument order (App. B); the dtype of ``dirty``
    (float32 / float64) selects the precision."""
    dev = _device(device)
    d = dirty if isinstance(dirty, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(dirty))
    prec = _prec(d.dtype)
    d = _to_dev(d, _REAL[prec], dev, "dirty")
    uvw_t = _to_dev(uvw, torch.float64, dev, "uvw")
    freq_t = _to_dev(freq, torch.float64, dev, "freq").reshape(-1)
    nrows, nchan = int(uvw_t.shape[0]), int(freq_t.numel())
    w = _to_dev(wgt, _REAL[prec], dev, "wgt", (nrows, nchan))
    m = _to_dev(mask, torch.uint8, dev, "mask", (nrows, nchan))
    out = torch.empty((nrows, nchan), dtype=_CPLX[prec], device=dev)
    _order(stream, dev, d, uvw_t, freq_t, w, m, out)
    with torch.cuda.device(dev):
        rc = lib().wg_dirty2ms(_ptr(uvw_t), _ptr(freq_t), nrows, nchan, _ptr(d), _ptr(w),
                               int(d.shape[0]), int(d.shape[1]), float(pixsize_x),
                               float(pixsize_y), float(epsilon), prec, int(bool(do_wstacking)),
                               _ptr(m), _ptr(out), _stream_handle(stream, dev))
    _check(rc)
    return out


def ms2dirty(uvw, freq, ms, wgt=None, npix_x=None, npix_y=None, pixsize_x=None, pixsize_y=None,
             epsilon=1e-5, do_wstacking=True, mask=None, stream=None, device=None):
    """One-shot grid with the paper's argument order (App. B); the dtype of ``ms``
    (complex64 / complex128) selects the precision."""
    dev = _device(device)
    v = ms if isinstance(ms, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(ms))
    prec = WG_F64 if v.dtype == torch.complex128 else WG_F32
    v = _to_dev(v, _CPLX[prec], dev, "ms")
    uvw_t = _to_dev(uvw, torch.float64, dev, "uvw")
    freq_t = _to_dev(freq, torch.float64, dev, "freq").reshape(-1)
    nrows, nchan = int(uvw_t.shape[0]), int(freq_t.numel())
    w = _to_dev(wgt, _REAL[prec], dev, "wgt", (nrows, nchan))
    m = _to_dev(mask, torch.uint8, dev, "mask", (nrows, nchan))
    out = torch.empty((int(npix_x), int(npix_y)), dtype=_REAL[prec], device=dev)
    _order(stream, dev, v, uvw_t, freq_t, w, m, out)
    with torch.cuda.device(dev):
        rc = lib().wg_ms2dirty(_ptr(uvw_t), _ptr(freq_t), nrows, nchan, _ptr(v), _ptr(w),
                               int(npix_x), int(npix_y), float(pixsize_x), float(pixsize_y),
                               float(epsilon), prec, int(bool(do_wstacking)), _ptr(m),
                               _ptr(out), _stream_handle(stream, dev))
    _check(rc)
    return out


# ----------------------------------------------------------------------------------------
# host-only helpers (no GPU needed)
# ----------------------------------------------------------------------------------------
def kernel_design_table():
    """Searched kernels for the supports App. A does not print: [(alpha, sigma, eps, beta, mu)]."""
    rows = []
    for i in range(lib().wg_kernel_design_size()):
        a, sg, e, b, m = ctypes.c_int(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib().wg_kernel_design_row(i, ctypes.byref(a), ctypes.byref(sg), ctypes.byref(e),
                                          ctypes.byref(b), ctypes.byref(m)))
        rows.append((a.value, sg.value, e.value, b.value, m.value))
    return rows


def kernel_eps(alpha, beta, mu, sigma) -> float:
    """Supremum of the map error function of the exact modified ES kernel over |x| <= 1/(2 sigma)."""
    e = ctypes.c_double()
    _check(lib().wg_kernel_eps(int(alpha), float(beta), float(mu), float(sigma), ctypes.byref(e)))
    return e.value


def kernel_search(alpha, sigma, beta0, mu0):
    """(beta, mu, eps) minimising kernel_eps for (alpha, sigma), from (beta0, mu0)."""
    b, m, e = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().wg_kernel_search(int(alpha), float(sigma), float(beta0), float(mu0),
                                  ctypes.byref(b), ctypes.byref(m), ctypes.byref(e)))
    return b.value, m.value, e.value


def kernel_table():
    """Rows (alpha, sigma, eps, beta, mu) of the library's built-in table (App. A)."""
    L = lib()
    out = []
    a, s, e, b, m = ctypes.c_int(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    for i in range(L.wg_kernel_table_size()):
        _check(L.wg_kernel_table_row(i, ctypes.byref(a), ctypes.byref(s), ctypes.byref(e),
                                     ctypes.byref(b), ctypes.byref(m)))
        out.append((a.value, s.value, e.value, b.value, m.value))
    return out


def _vec_call(fn, alpha, beta, mu, x):
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    out = np.empty_like(x)
    _check(fn(int(alpha), float(beta), float(mu), x.ctypes.data_as(ctypes.c_void_p),
              out.ctypes.data_as(ctypes.c_void_p), x.size))
    return out


def kernel_phi(alpha, beta, mu, x):
    return _vec_call(lib().wg_kernel_phi, alpha, beta, mu, x)


def kernel_poly(alpha, beta, mu, x):
    return _vec_call(lib().wg_kernel_poly, alpha, beta, mu, x)


def kernel_psi(alpha, beta, mu, k):
    return _vec_call(lib().wg_kernel_psi, alpha, beta, mu, k)


def plan_params(npix_x, npix_y, pixsize_x, pixsize_y, epsilon, precision="f32", umax=0.0,
                vmax=0.0, wmin=0.0, wmax=0.0, nvis=0, **opts) -> dict:
    o = default_options(**opts)
    inf = PlanInfo()
    _check(lib().wg_plan_params(int(npix_x), int(npix_y), float(pixsize_x), float(pixsize_y),
                                float(epsilon), _prec(precision), ctypes.byref(o), float(umax),
                                float(vmax), float(wmin), float(wmax), int(nvis), ctypes.byref(inf)))
    return inf.as_dict()


def fft_time(n, precision="f32", batch=1, reps=3, impl=1) -> float:
    """Milliseconds per plane of the batched n x n plane FFT (planner calibration);
    impl 1 = cuFFT, 2 = the library's double-float FFT (f64)."""
    ms = ctypes.c_double()
    _check(lib().wg_fft_time(int(n), _prec(precision), int(batch), int(reps), int(impl),
                             ctypes.byref(ms)))
    return ms.value


def fft2d(planes, sign=-1, impl=1, stream=None):
    """In-place unnormalised 2-D FFT of a contiguous (batch, nu, nv) complex CUDA tensor with the
    library's transforms (impl 1 = cuFFT, 2 = double-float, complex128 only)."""
    if not isinstance(planes, torch.Tensor) or not planes.is_cuda or not planes.is_contiguous():
        raise ValueError("planes must be a contiguous CUDA tensor")
    prec = WG_F64 if planes.dtype == torch.complex128 else WG_F32
    b, nu, nv = planes.shape if planes.ndim == 3 else (1,) + tuple(planes.shape)
    _check(lib().wg_fft2d(_ptr(planes), int(nu), int(nv), int(b), prec, int(impl), int(sign),
                          _stream_handle(stream, planes.device)))
    return planes


def pool_trim(keep_bytes=0, device=None) -> None:
    """Release the library's cached per-call workspace memory on the device beyond keep_bytes."""
    dev = _device(device)
    with torch.cuda.device(dev):
        _check(lib().wg_pool_trim(int(keep_bytes)))


def wait(stream=None, timeout_ms=-1.0) -> bool:
    """Bounded host wait on a CUDA stream (wg_wait): True when its work has finished, False
    if it is still running after ``timeout_ms`` (negative: wait without bound)."""
    dev = _device(None) if stream is None else stream.device
    rc = lib().wg_wait(_stream_handle(stream, dev), float(timeout_ms))
    if rc == WG_ERR_TIMEOUT:
        return False
    _check(rc)
    return True


def fma_peak(precision="f32") -> float:
    """Measured FMA throughput (flop/s, an FMA = 2) of the current device in FP32 or FP64."""
    f = ctypes.c_double()
    _check(lib().wg_fma_peak(_prec(precision), ctypes.byref(f)))
    return f.value


def fft_f32_tune(cols=0, max_points=0, per_thread=0):
    """Shape of the library's FP32 plane FFT for transforms and plans created afterwards
    (wg_fft_f32_tune; 0 keeps a default)."""
    _check(lib().wg_fft_f32_tune(int(cols), int(max_points), int(per_thread)))


def version() -> str:
    return lib().wg_version().decode()
