"""Host-side checks of libwgrid.so that need no GPU: the C ABI exports, the built-in kernel
table (App. A), the piecewise-polynomial kernel (Sec. 4.2), its Fourier transform psi, and
the planner's definitions (Sec. 2: N = ceil(sigma n), Delta w, w_0, N_w; Sec. 4.1: smallest
sigma per alpha that meets epsilon, cost-model choice across alpha), and the planner's model of
plane rounding (the gain by which it reaches the result through the 1 / psi correction)."""
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
    # chosen kernel meets epsilon and is the smallest such sigma for its alpha (Sec. 4.1), the
    # error counting the kernel term and the plane rounding of the chosen FFT kind
    safety = 0.8   # default: table epsilon <= 0.8 x requested
    rows = [r for r in list(wg.kernel_table()) + wg.kernel_design_table()
            if r[0] == alpha and r[2] <= safety * eps]
    assert info["eps_kernel"] <= safety * eps and info["err_model"] <= eps
    for r in rows:
        if r[1] < sigma:
            alt = wg.plan_params(**a, force_alpha=alpha, force_sigma=r[1],
                                 fft_impl=info["fft_impl"])
            assert alt["err_model"] > eps
    assert info["fft_impl"] == 1 if prec == "f32" else info["fft_impl"] in (2, 3)
    assert info["err_model"] >= info["eps_kernel"] / safety
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
    """Sec. 4.1: across alpha the predicted cheapest kernel wins; FP64 at 1e-12 needs alpha 16
    (sigma 1.55 with FP64 planes; the double-float FFT's larger rounding needs more)."""
    _, f64 = _planner_case(wg, precision="f64", epsilon=1e-12, fft_impl=3)
    assert f64["alpha"] >= 15 and f64["fft_impl"] == 3
    _, df = _planner_case(wg, precision="f64", epsilon=1e-12, fft_impl=2)
    assert df["alpha"] >= 15 and df["sigma"] > 1.55 and df["fft_impl"] == 2
    _, auto = _planner_case(wg, precision="f64", epsilon=1e-12)
    assert auto["alpha"] >= 15 and auto["fft_impl"] in (2, 3) and auto["err_model"] <= 1e-12
    # with only the printed supports (forced), FP64 planes at 1e-12 need alpha 16, sigma 1.55
    _, f16 = _planner_case(wg, precision="f64", epsilon=1e-12, fft_impl=3, force_alpha=16)
    assert f16["sigma"] == 1.55
    _, f32 = _planner_case(wg)
    assert 6 <= f32["alpha"] <= 12 and f32["fft_impl"] == 1


def _gain_reference(nx, ny, psx, psy, nu, nv, alpha, beta, mu, nshift, dw):
    """rms of 1 / (n psi_u psi_v psi_w) over a 64 x 64 midpoint lattice of pixels, times
    (int phi^2)^(3/2): the factor by which a relative rounding of the plane values reaches
    degridded visibilities of an image with uniformly spread flux (unnormalised FFT: the rms
    per cell of FFT(I corr) is ||I corr||; the footprint sums phi-weighted cells per axis).
    Written with the oracle's phi and psi (the exponential of a semicircle itself)."""
    x = np.linspace(-alpha / 2, alpha / 2, 40001)
    phi2 = np.trapezoid(km.phi(x, alpha, beta, mu) ** 2, x)
    jx = -nx / 2 + (np.arange(64) + 0.5) * nx / 64
    jy = -ny / 2 + (np.arange(64) + 0.5) * ny / 64
    L, M = np.meshgrid(jx * psx, jy * psy, indexing="ij")
    r2 = L * L + M * M
    n = np.sqrt(1 - r2)
    nm1 = -r2 / (1 + n)
    pu = km.psi(jx / nu, alpha, beta, mu)
    pv = km.psi(jy / nv, alpha, beta, mu)
    pw = km.psi(((nm1 - nshift) * dw).ravel(), alpha, beta, mu).reshape(nm1.shape)
    corr = 1 / (n * pu[:, None] * pv[None, :] * pw)
    return math.sqrt(np.mean(corr ** 2)) * phi2 ** 1.5


@pytest.mark.parametrize("prec,eps,impl", [("f64", 1e-12, 2), ("f64", 1e-10, 3), ("f32", 1e-5, 0),
                                           ("f32", 1e-3, 0)])
def test_rounding_gain_matches_its_definition(wg, prec, eps, impl):
    a, info = _planner_case(wg, precision=prec, epsilon=eps, fft_impl=impl)
    ref = _gain_reference(a["npix_x"], a["npix_y"], a["pixsize_x"], a["pixsize_y"], info["nu"],
                          info["nv"], info["alpha"], info["beta"], info["mu"], info["nshift"],
                          info["dw"])
    assert info["rounding_gain"] == pytest.approx(ref, rel=2e-3)
    # the planner's rounding term: c(G) u log2(nu nv) G, u the unit roundoff of the plane
    # arithmetic, c(G) = 0.065 (1 + G / 2000)
    u = {1: 2.0 ** -24 if prec == "f32" else 2.0 ** -53, 2: 2.0 ** -47, 3: 2.0 ** -53}[info["fft_impl"]]
    g = info["rounding_gain"]
    r = 0.065 * (1 + g / 2000) * u * math.log2(info["nu"] * info["nv"]) * g
    k = info["eps_kernel"] / 0.8
    assert info["err_model"] == pytest.approx(math.hypot(k, r), rel=1e-12)


def test_rounding_gain_grows_as_sigma_shrinks(wg):
    """1 / psi at the image edge grows as the oversampling drops (Sec. 2: the kernel's Fourier
    transform decays towards |k| = 1 / (2 sigma))."""
    gains = [wg.plan_params(**_planner_case(wg)[0] | dict(precision="f64", epsilon=1e-6,
                                                          force_alpha=16, force_sigma=s))["rounding_gain"]
             for s in (1.3, 1.5, 1.7, 2.0)]
    assert all(g1 > g2 for g1, g2 in zip(gains, gains[1:]))


def test_planner_fft_kind_arguments(wg):
    with pytest.raises(wg.WgridError):
        _planner_case(wg, precision="f32", fft_impl=2)
    with pytest.raises(wg.WgridError):
        _planner_case(wg, precision="f32", fft_impl=3)
    with pytest.raises(wg.WgridError):
        _planner_case(wg, precision="f64", epsilon=1e-9, fft_impl=4)
    # grid sides beyond the double-float FFT's 25600
    with pytest.raises(wg.WgridError) as ei:
        _planner_case(wg, precision="f64", epsilon=1e-9, fft_impl=2, npix_x=24576, npix_y=24576,
                      pixsize_x=math.radians(1 / 3600), pixsize_y=math.radians(1 / 3600))
    assert "25600" in str(ei.value)


def test_planner_double_float_fft_split_sides(wg):
    """Sides above 6400 run each line on 2 or 4 CTAs: an 8192^2 image at eps = 1e-12 gets a
    double-float plan whose grid side is 2 or 4 times a side the line kernel supports."""
    _, p = _planner_case(wg, precision="f64", epsilon=1e-12, fft_impl=2, npix_x=8192, npix_y=8192,
                         pixsize_x=math.radians(4 / 3600), pixsize_y=math.radians(4 / 3600))
    assert p["fft_impl"] == 2 and 6400 < p["nu"] <= 25600 and p["err_model"] <= 1e-12
    ok = False
    for s in (2, 4):
        m = p["nu"] // s
        if p["nu"] % s or m > 6400:
            continue
        for f in (2, 3, 5, 7, 11):
            while m % f == 0:
                m //= f
        ok = ok or m == 1
    assert ok, p


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


@pytest.mark.parametrize("bad", [(3, 0, 0), (16, 0, 0), (0, 32, 0), (0, 12801, 0), (0, 0, 1),
                                 (0, 0, 65), (-1, 0, 0)])
def test_fft_f32_tune_rejects_out_of_range(wg, bad):
    """The FP32 FFT's shape knob (host-side only) takes cols 1, 2, 4, 8, max_points 64 .. 12800
    and per_thread 2 .. 64, and rejects anything else with WG_ERR_ARG."""
    with pytest.raises(wg.WgridError) as ei:
        wg.wgrid.fft_f32_tune(*bad)
    assert ei.value.code == 1
    wg.wgrid.fft_f32_tune(8, 64, 2)        # extremes are accepted
    wg.wgrid.fft_f32_tune(1, 12800, 64)
    wg.wgrid.fft_f32_tune(0, 0, 0)         # back to the defaults


def test_planner_f32_library_fft_sides(wg):
    """fft_impl 4 plans grid sides the FP32 line kernels support: 1, 2, 4 or 8 times a part of at
    most 12800 points with prime factors 2, 3, 5, 7, 11 (and at most 46340, 32-bit offsets)."""
    for npix, pix in ((2048, 20), (8192, 4)):
        _, p = _planner_case(wg, precision="f32", epsilon=1e-5, fft_impl=4, npix_x=npix,
                             npix_y=npix, pixsize_x=math.radians(pix / 3600),
                             pixsize_y=math.radians(pix / 3600))
        assert p["fft_impl"] == 4 and p["nu"] <= 46340
        ok = False
        for s in (1, 2, 4, 8):
            m = p["nu"] // s
            if p["nu"] % s or m > 12800:
                continue
            for f in (2, 3, 5, 7, 11):
                while m % f == 0:
                    m //= f
            ok = ok or m == 1
        assert ok, p


def test_calibration_table_merge(tmp_path):
    """calibrate_fft re-measures only the selected columns in [min_n, max_n] and keeps every
    other entry of the existing table, including sizes beyond max_n (a range-limited run once
    dropped them)."""
    from paper_2010_10122_gb300 import calibrate_fft as cf
    src = open(os.path.join(os.path.dirname(__file__), "..", "paper_2010_10122_gb300", "csrc",
                            "fft_table.inc")).read()
    path = tmp_path / "t.inc"
    path.write_text(src)
    old = cf.read_table(str(path))
    assert len(old) > 100 and all(len(v) == 4 for v in old.values())
    plan = dict(cf.table_plan(old, ["df64"], 2049, 6400))
    assert set(plan) == set(old)                          # no size lost or added
    for n, measure in plan.items():
        assert measure == [False, False, 2049 <= n <= 6400, False]
    # a fresh table: every column of every size measured
    fresh = cf.table_plan({}, list(cf.COLUMNS), 0, 1024)
    assert [n for n, _ in fresh] == [32 * m for m in range(4, 33) if cf.smooth(m)]
    assert all(all(m) for _, m in fresh)
    # the written form reads back
    rows = [[n] + old[n] for n in sorted(old)]
    path.write_text(cf.format_table(rows, "GPU"))
    assert cf.read_table(str(path)) == {n: [float(f"{x:.6g}") for x in v] for n, v in old.items()}
