"""Direct-sum FP64 oracle for degrid (Eq. rime) and grid (its direct adjoint, Sec. 5.2).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s ``cpu_baseline`` / ``--impl reference`` legs may import this module.
The product path (``paper_2010_10122_gb300``) never imports, links or runs it, and it
shares no code with the CUDA path.

The arithmetic lives in ``oracle/direct.c`` (plain C, POSIX threads); this module
only compiles it with gcc and marshals numpy arrays to it.

Conventions (paper Sec. 2 and App. B):
  * uvw: (nrows, 3) float64 in metres; freq: (nchan,) float64 in Hz;
  * visibility k = (row, chan), data array (nrows, nchan) complex;
  * dirty image (nx, ny), pixel (jx, jy) at l = (jx - nx/2) dl, m = (jy - ny/2) dm;
  * degrid:  d_k = sum_lm exp(-2 pi i [u_k l + v_k m - w_k (n_lm - 1)]) I_lm / n_lm
  * grid:    I_lm = Re sum_k exp(+2 pi i [...]) d_k / n_lm
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "direct.c")
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lib = None

SPEED_OF_LIGHT = 299792458.0


def build(force: bool = False) -> str:
    """Compile oracle/direct.c into oracle/_build/liboracle.so with gcc."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-shared",
                               "-fPIC", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, dp, u8p, i64p = ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p
        sig = [dp, dp, i64, i64, dp, i64, i64, ctypes.c_double, ctypes.c_double,
               dp, u8p, ctypes.c_int, i64p, i64, dp, ctypes.c_int]
        lib.oracle_degrid.argtypes = sig
        lib.oracle_degrid.restype = ctypes.c_int
        lib.oracle_grid.argtypes = sig
        lib.oracle_grid.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _prep(uvw, freq, wgt, mask, nvis):
    uvw = np.ascontiguousarray(uvw, dtype=np.float64)
    freq = np.ascontiguousarray(freq, dtype=np.float64)
    assert uvw.ndim == 2 and uvw.shape[1] == 3
    if wgt is not None:
        wgt = np.ascontiguousarray(wgt, dtype=np.float64).reshape(-1)
        assert wgt.size == nvis
    if mask is not None:
        mask = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        assert mask.size == nvis
    return uvw, freq, wgt, mask


def degrid(uvw, freq, dirty, pixsize_x, pixsize_y, wgt=None, mask=None,
           do_wstacking=True, vis_index=None, nthreads=0):
    """(R0 I)_k for all visibilities, or for the flat indices ``vis_index`` only.

    Returns complex128 of shape (nrows, nchan), or (len(vis_index),).
    """
    uvw = np.asarray(uvw)
    nrows, nchan = uvw.shape[0], np.asarray(freq).size
    uvw, freq, wgt, mask = _prep(uvw, freq, wgt, mask, nrows * nchan)
    dirty = np.ascontiguousarray(dirty, dtype=np.float64)
    nx, ny = dirty.shape
    if vis_index is None:
        sel, nsel = None, nrows * nchan
    else:
        sel = np.ascontiguousarray(vis_index, dtype=np.int64)
        nsel = sel.size
    out = np.zeros(2 * nsel, dtype=np.float64)
    used = _load().oracle_degrid(_ptr(uvw), _ptr(freq), nrows, nchan, _ptr(dirty), nx, ny,
                                 float(pixsize_x), float(pixsize_y), _ptr(wgt), _ptr(mask),
                                 int(bool(do_wstacking)), _ptr(sel), nsel, _ptr(out), int(nthreads))
    if used < 0:
        raise ValueError("a pixel lies outside the unit disc (l^2 + m^2 > 1)")
    res = out.view(np.complex128)
    return res.reshape(nrows, nchan) if vis_index is None else res


def grid(uvw, freq, vis, nx, ny, pixsize_x, pixsize_y, wgt=None, mask=None,
         do_wstacking=True, pixel_index=None, nthreads=0):
    """(R0^dagger d)_lm for all pixels (shape (nx, ny)), or for flat ``pixel_index`` only."""
    uvw = np.asarray(uvw)
    nrows, nchan = uvw.shape[0], np.asarray(freq).size
    uvw, freq, wgt, mask = _prep(uvw, freq, wgt, mask, nrows * nchan)
    vis = np.ascontiguousarray(vis, dtype=np.complex128).reshape(-1)
    assert vis.size == nrows * nchan
    visf = vis.view(np.float64)
    if pixel_index is None:
        sel, nsel = None, nx * ny
    else:
        sel = np.ascontiguousarray(pixel_index, dtype=np.int64)
        nsel = sel.size
    out = np.zeros(nsel, dtype=np.float64)
    used = _load().oracle_grid(_ptr(uvw), _ptr(freq), nrows, nchan, _ptr(visf), nx, ny,
                               float(pixsize_x), float(pixsize_y), _ptr(wgt), _ptr(mask),
                               int(bool(do_wstacking)), _ptr(sel), nsel, _ptr(out), int(nthreads))
    if used < 0:
        raise ValueError("a pixel lies outside the unit disc (l^2 + m^2 > 1)")
    return out.reshape(nx, ny) if pixel_index is None else out


def threads_used(nthreads=0):
    """Thread count the oracle uses for a given request (0 = all online cores)."""
    return nthreads if nthreads > 0 else (os.cpu_count() or 1)


def rel_l2(x, ref):
    """Relative L2 error ||x - ref|| / ||ref|| (Sec. 5.2, eps_rms)."""
    x = np.asarray(x); ref = np.asarray(ref)
    return float(np.linalg.norm((x - ref).ravel()) / np.linalg.norm(ref.ravel()))


def adjointness_error(I, RI, d, Rd):
    """eps_adj of Sec. 5.1: |Re<R I, d> - <I, R^dagger d>| / min(|d||R I|, |I||R^dagger d|)."""
    I = np.asarray(I, dtype=np.float64).ravel(); Rd = np.asarray(Rd, dtype=np.float64).ravel()
    RI = np.asarray(RI, dtype=np.complex128).ravel(); d = np.asarray(d, dtype=np.complex128).ravel()
    lhs = np.real(np.vdot(RI, d))
    rhs = float(np.dot(I, Rd))
    den = min(np.linalg.norm(d) * np.linalg.norm(RI), np.linalg.norm(I) * np.linalg.norm(Rd))
    return abs(lhs - rhs) / den
