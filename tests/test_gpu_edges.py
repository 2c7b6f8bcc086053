"""Parity edge cases of the method's geometry, element by element against the FP64 oracle.

  * uv coordinates beyond +-1 / (2 dl): Eq. (rime) evaluated on the pixel lattice l = j dl is
    periodic in u with period 1 / dl, and the gridding realises that period by wrapping the
    kernel footprint around the uv grid (Sec. 2, the index sets U, V are periodic);
  * grid coordinates that are exact integers, on uv-tile edges, at the grid's wrap point and
    at the band edge u = +-1 / (2 dl) (the first footprint cell is ceil(x - alpha / 2), with
    ties at the kernel's support edge where phi is ~exp(-alpha beta));
  * a w range that spans a single plane position (N_w = alpha + 1, Eq. wcirc);
  * the bounded host wait on a stream (wg_wait) running out while device work is pending.
"""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2010_10122_gb300 import synthetic as S  # noqa: E402

C = S.SPEED_OF_LIGHT


@pytest.fixture(scope="module")
def wg():
    from paper_2010_10122_gb300 import _build
    _build.build()
    import paper_2010_10122_gb300 as wg
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return wg


def _dt(prec):
    return (np.float32, np.complex64) if prec == "f32" else (np.float64, np.complex128)


def _pair(wg, oracle_lib, obs, eps, prec, seed, **opts):
    rdt, cdt = _dt(prec)
    I = S.gaussian_image(obs.npix_x, obs.npix_y, seed=seed)
    d = S.complex_normal((obs.nrows, obs.nchan), seed=seed + 1)
    plan = wg.Plan(obs.uvw, obs.freq, obs.npix_x, obs.npix_y, obs.pixsize_x, obs.pixsize_y, eps, prec,
                   **opts)
    vis = plan.degrid(torch.from_numpy(I.astype(rdt)).cuda()).cpu().numpy()
    img = plan.grid(torch.from_numpy(d.astype(cdt)).cuda()).cpu().numpy()
    rv = oracle_lib.degrid(obs.uvw, obs.freq, I, obs.pixsize_x, obs.pixsize_y)
    ri = oracle_lib.grid(obs.uvw, obs.freq, d, obs.npix_x, obs.npix_y, obs.pixsize_x, obs.pixsize_y)
    return plan, oracle_lib.rel_l2(vis, rv), oracle_lib.rel_l2(img, ri)


@pytest.mark.parametrize("prec,eps", [("f64", 1e-12), ("f64", 1e-9), ("f32", 1e-5)])
def test_uv_beyond_the_band_wraps(wg, oracle_lib, prec, eps):
    """|u| dl and |v| dm up to 1.4 (the band is +-0.5): the gridded operator equals the direct
    sum, which is periodic in u with period 1 / dl on the pixel lattice."""
    rng = np.random.default_rng(41)
    nx, ny, f = 96, 64, 1.2e9
    psx, psy = math.radians(6.0) / nx, math.radians(4.0) / ny
    n = 1200
    u = rng.uniform(-1.4, 1.4, n) / psx
    v = rng.uniform(-1.4, 1.4, n) / psy
    w = rng.uniform(-0.3, 0.3, n) / psx
    uvw = np.stack([u, v, w], axis=1) * (C / f)
    obs = S.Observation(uvw, np.array([f]), nx, ny, psx, psy)
    assert np.abs(u).max() * psx > 1.3 and np.abs(v).max() * psy > 1.3
    _, ev, ei = _pair(wg, oracle_lib, obs, eps, prec, seed=5)
    assert ev <= eps and ei <= eps, (ev, ei)


def _coordinates_at(k, scale):
    """float64 u~ whose grid coordinate u~ * scale (formed in FP64 by the library) is exactly k
    when some u~ lands there, else the nearest coordinates just below and just above k."""
    u = np.nextafter(k / scale, -np.inf)
    for _ in range(8):
        u = np.nextafter(u, -np.inf)
    below = above = None
    for _ in range(24):
        x = u * scale
        if x == k:
            return [u]
        if x < k:
            below = u
        elif above is None:
            above = u
        u = np.nextafter(u, np.inf)
    return [c for c in (below, above) if c is not None]


@pytest.mark.parametrize("prec,eps", [("f64", 1e-12), ("f64", 1e-10), ("f32", 1e-5)])
def test_integer_coordinates_and_tile_edges(wg, oracle_lib, prec, eps):
    """Grid coordinates x = u dl N that are exact integers (fractional offset 0) on uv-tile
    edges, one cell either side, at the wrap point N and at the band edges +-N / 2, plus half
    cells; w on exact plane positions as well."""
    nx, ny, f = 128, 96, 1.0e9
    psx, psy = math.radians(5.0) / nx, math.radians(5.0) / ny
    rng = np.random.default_rng(42)
    w_lam = np.concatenate([rng.uniform(-800.0, 800.0, 256), [0.0, 800.0, -800.0]])
    base = np.stack([np.zeros_like(w_lam), np.zeros_like(w_lam), w_lam * C / f], axis=1)
    probe = wg.Plan(base, np.array([f]), nx, ny, psx, psy, eps, prec)
    info = probe.info
    probe.close()
    N, M, T, a = info["nu"], info["nv"], info["tile"], info["alpha"]
    s = f / C
    scale_u, scale_v = s * psx * N, s * psy * M   # left to right, as the library forms it
    ks_u = sorted({0, 1, T - 1, T, T + 1, 2 * T, N // 2, -N // 2, N - 1, N - a // 2,
                   a // 2, -(a // 2), T - a // 2, 2 * T - a // 2 - 1, N // 2 - a // 2})
    ks_v = sorted({0, 1, T - 1, T, M // 2, -M // 2, M - 1, M - a // 2, a // 2, T - a // 2})
    rows = []
    for ku in ks_u:
        for kv in ks_v:
            for half in (0.0, 0.5):
                for uu in _coordinates_at(ku + half, scale_u):
                    for vv in _coordinates_at(kv + half, scale_v):
                        rows.append((uu, vv))
    rows = np.array(rows)
    nr = rows.shape[0]
    w = w_lam[rng.integers(len(w_lam), size=nr)] * C / f
    w[: len(w_lam)] = (w_lam * C / f)[: min(nr, len(w_lam))]
    uvw = np.stack([rows[:, 0], rows[:, 1], w], axis=1)
    obs = S.Observation(uvw, np.array([f]), nx, ny, psx, psy)
    # the planner's cost model depends on the visibility count: keep the probe's choice
    plan, ev, ei = _pair(wg, oracle_lib, obs, eps, prec, seed=7, force_alpha=a,
                         force_sigma=info["sigma"], fft_impl=info["fft_impl"] if prec == "f64" else 0)
    assert (plan.info["nu"], plan.info["nv"]) == (N, M)
    assert ev <= eps and ei <= eps, (ev, ei, plan.info)


@pytest.mark.parametrize("prec,eps", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("wval", [0.0, 350.0])
def test_single_plane_position(wg, oracle_lib, prec, eps, wval):
    """Every visibility at the same |w| (wmax = wmin): N_w = alpha + 1 planes (Eq. wcirc with
    an empty w range, plus the slack plane), with w = 0 and with w on both sides of zero (the
    Hermitian fold maps them onto one plane position)."""
    rng = np.random.default_rng(43)
    nx, ny, f = 64, 64, 1.1e9
    ps = math.radians(8.0) / nx
    n = 700
    u = rng.uniform(-0.45, 0.45, n) / ps
    v = rng.uniform(-0.45, 0.45, n) / ps
    w = np.full(n, wval) * rng.choice([-1.0, 1.0], n)
    obs = S.Observation(np.stack([u, v, w], axis=1) * (C / f), np.array([f]), nx, ny, ps, ps)
    plan, ev, ei = _pair(wg, oracle_lib, obs, eps, prec, seed=9)
    assert plan.info["nw"] == plan.info["alpha"] + 1, plan.info
    assert ev <= eps and ei <= eps, (ev, ei)


def test_bounded_wait_runs_out_and_recovers(wg):
    """wg_wait returns WG_ERR_TIMEOUT while a bounded sleep kernel (about 0.5 s) is pending on
    the stream, and WG_OK once it has finished; the context stays usable."""
    L = wg.lib()
    s = torch.cuda.Stream()
    h = ctypes.c_void_p(s.cuda_stream)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        torch.cuda._sleep(int(1e9))        # ~0.5 s at the GB300's clock; ends by itself
    assert L.wg_wait(h, 5.0) == wg.wgrid.WG_ERR_TIMEOUT
    assert b"not finished" in L.wg_last_error()
    assert not wg.wait(s, timeout_ms=1.0)
    assert L.wg_wait(h, 30000.0) == wg.wgrid.WG_OK
    assert wg.wait(s, timeout_ms=0.0)
    x = torch.ones(4, device="cuda").sum().item()
    assert x == 4.0


def test_calls_on_another_stream_wait_for_their_inputs():
    """Inputs staged by the binding on torch's current stream (here: pinned host arrays copied
    behind a busy kernel) are ready before a plan built, or an operator run, on another stream
    reads them."""
    import paper_2010_10122_gb300 as wg
    obs = S.random_uvw_observation(3000, 4, 96, 80, 12.0, seed=71)
    img = S.gaussian_image(obs.npix_x, obs.npix_y, seed=72, dtype=np.float32)
    ref = wg.Plan(obs.uvw, obs.freq, obs.npix_x, obs.npix_y, obs.pixsize_x, obs.pixsize_y,
                  1e-5, "f32")
    want = ref.degrid(torch.from_numpy(img).cuda())
    side = torch.cuda.Stream()
    uvw = torch.from_numpy(obs.uvw).pin_memory()
    freq = torch.from_numpy(obs.freq).pin_memory()
    x = torch.from_numpy(img).pin_memory()
    torch.cuda._sleep(50_000_000)            # ~25 ms of clock cycles on the current stream
    p = wg.Plan(uvw, freq, obs.npix_x, obs.npix_y, obs.pixsize_x, obs.pixsize_y, 1e-5, "f32",
                stream=side)
    torch.cuda._sleep(50_000_000)
    got = p.degrid(x, stream=side)
    torch.cuda.synchronize()
    assert torch.equal(got, want)
