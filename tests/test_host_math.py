"""Host-side checks of libwgrid.so that need no GPU: the C ABI exports, the built-in kernel
table (App. A), the piecewise-polynomial kernel (Sec. 4.2), its Fourier transform psi, and
the planner's definitions (Sec. 2: N = ceil(sigma n), Delta w, w_0, N_w; Sec. 4.1: smallest
sigma per alpha that meets epsilon, cost-model choice across alpha)."""
import math
import os
import re

import numpy as np
import pytest

from oracle import kernel_math as km

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def wg():
    from paper_2010_10122_gb300 import _build
    _build.build()
    import paper_2010_10122_gb300 as wg
    return wg


def test_library_exports_every_declared_symbol(wg):
    import ctypes
    hdr = open(os.path.join(ROOT, "include", "wgrid.h")).read()
    declared = set(re.findall(r"\b(wg_[a-z0-9_]+)\s*\(", hdr))
    assert len(declared) >= 15
    L = ctypes.CDLL(wg.wgrid.LIB_PATH)
    missing = [s for s in sorted(declared) if not hasattr(L, s)]
    assert not missing, missing
    assert set(wg.wgrid.SIGNATURES) == declared


def test_builtin_table_equals_paper_table(wg):
    from tests.test_kernel_table_pin import table_rows
    assert wg.kernel_table() == table_rows()


def test_phi_direct_matches_oracle(wg):
    x = np.linspace(-4.2, 4.2, 301)
    np.testing.assert_allclose(wg.kernel_phi(8, 1.7876782642, 0.5176319503, x),
                               km.phi(x, 8, 1.7876782642, 0.5176319503), rtol=1e-14, atol=0)


@pytest.mark.parametrize("row", [0, 20, 40, 60, 80])
def test_polynomial_kernel_close_to_phi(wg, row):
    """Sec. 4.2: alpha pieces of degree alpha + 3 through Chebyshev nodes.  The pointwise error
    is largest next to the support edge, where phi has its (1 - s^2)^mu branch point; it
    stays below the edge value exp(-alpha beta) of the kernel (plus FP64 rounding)."""
    a, s, e, b, m = wg.kernel_table()[row]
    x = np.linspace(-a / 2, a / 2, 4001)
    err = np.abs(wg.kernel_poly(a, b, m, x) - km.phi(x, a, b, m)).max()
    assert err < 2.0 * math.exp(-a * b) + 1e-14  # edge term + FP64 Horner rounding
    assert wg.kernel_poly(a, b, m, np.array([a / 2 + 1e-9, -a / 2 - 1e-9, 7.0 * a])).max() == 0


def test_psi_of_polynomial_matches_oracle_psi(wg):
    a, s, e, b, m = 12, 1.55, 8.0989276e-10, 2.0129847811, 0.5085327805
    k = np.linspace(-0.5, 0.5, 41)
    np.testing.assert_allclose(wg.kernel_psi(a, b, m, k), km.psi(k, a, b, m), rtol=0, atol=1e-10)


@pytest.mark.parametrize("row", [0, 5, 17, 18, 26, 35, 40, 47, 55, 60, 66, 73, 78])
def test_polynomial_kernel_meets_table_epsilon(wg, row):
    """The kernel the GPU actually evaluates (piecewise polynomial, with the psi computed from
    it) has sup-norm map error (Eq. maperror) within 5% of the table epsilon."""
    a, s, e, b, m = wg.kernel_table()[row]
    k = np.linspace(0.0, 0.5 / s, 48)
    l = km.map_error_of(k, a, lambda x: wg.kernel_poly(a, b, m, x),
                        lambda kk: wg.kernel_psi(a, b, m, kk))
    assert l.max() <= 1.05 * e


def _planner_case(wg, **kw):
    ps = math.radians(20 / 3600)
    base = dict(npix_x=2048, npix_y=1536, pixsize_x=ps, pixsize_y=0.8 * ps, epsilon=1e-5,
                precision="f32", umax=4000.0, vmax=3000.0, wmin=12.0, wmax=3600.0, nvis=10**6)
    base.update(kw)
    return base, wg.plan_params(**base)


@pytest.mark.parametrize("w_shift", [0, 1])
@pytest.mark.parametrize("prec,eps", [("f32", 1e-5), ("f64", 1e-12), ("f64", 1e-9), ("f32", 1e-3)])
def test_planner_follows_sec2_definitions(wg, w_shift, prec, eps):
    a, info = _planner_case(wg, precision=prec, epsilon=eps, w_shift=w_shift)
    alpha, sigma = info["alpha"], info["sigma"]
    # chosen kernel meets epsilon and is the smallest such sigma for its alpha (Sec. 4.1)
    safety = 0.8   # default: table epsilon <= 0.8 x requested
    rows = [r for r in wg.kernel_table() if r[0] == alpha and r[2] <= safety * eps]
    assert info["eps_kernel"] <= safety * eps and sigma == min(r[1] for r in rows)
    # N >= ceil(sigma n), an FFT-friendly (11-smooth) multiple of the tile, and not much above
    for n, N in ((a["npix_x"], info["nu"]), (a["npix_y"], info["nv"])):
        assert N >= math.ceil(sigma * n) and N % info["tile"] == 0
        assert N <= 1.25 * math.ceil(sigma * n) + 64
        q = N // info["tile"]
        for pr in (2, 3, 5, 7, 11):
            while q % pr == 0:
                q //= pr
        assert q == 1
    # Delta w = 1 / (2 sigma max|n - 1 - shift|) (Sec. 2), corner pixel extreme
    l, m = a["npix_x"] / 2 * a["pixsize_x"], a["npix_y"] / 2 * a["pixsize_y"]
    nm1 = -(l * l + m * m) / (1 + math.sqrt(1 - l * l - m * m))
    span = abs(nm1) / 2 if w_shift else abs(nm1)
    assert info["nshift"] == pytest.approx(nm1 / 2 if w_shift else 0.0, rel=1e-15, abs=0)
    assert info["dw"] == pytest.approx(1 / (2 * sigma * span), rel=1e-14)
    # Eq. (wcirc) and N_w = (max w - min w) / Delta w + alpha (rounded up, + 1 slack plane)
    assert info["w0"] == pytest.approx(a["wmin"] - info["dw"] * (alpha - 1) / 2, rel=1e-14)
    assert info["nw"] == math.ceil((a["wmax"] - a["wmin"]) / info["dw"]) + alpha + 1


def test_planner_without_wstacking_has_one_plane(wg):
    _, info = _planner_case(wg, do_wstacking=0)
    assert info["nw"] == 1 and info["nshift"] == 0.0


def test_planner_cost_prefers_cheap_fp32_kernels(wg):
    """Sec. 4.1: across alpha the predicted cheapest kernel wins; FP64 at 1e-12 needs alpha 16."""
    _, f64 = _planner_case(wg, precision="f64", epsilon=1e-12)
    assert f64["alpha"] == 16 and f64["sigma"] == 1.55
    _, f32 = _planner_case(wg)
    assert f32["alpha"] in (7, 8, 12)


@pytest.mark.parametrize("bad", [dict(npix_x=31), dict(npix_x=30), dict(npix_y=33),
                                 dict(epsilon=1e-13), dict(precision="f32", epsilon=9e-6),
                                 dict(pixsize_x=0.1, npix_x=64),   # corner beyond the unit disc
                                 dict(tile=24)])
def test_planner_rejects_invalid_arguments(wg, bad):
    with pytest.raises(wg.WgridError) as ei:
        _planner_case(wg, **bad)
    assert ei.value.code == 1


def test_gpu_calls_fail_loudly_without_a_device(wg):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(RuntimeError):
        wg.Plan(np.zeros((1, 3)), np.array([1e9]), 64, 64, 1e-4, 1e-4, 1e-5)
