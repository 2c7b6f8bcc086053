"""Compact index (wg_options.compact_index): the plan keeps 4 bytes per visibility plus a copy of
uvw, and every call recomputes the visibilities' records into its workspace with the same FP64
arithmetic as the full index.  The records are therefore identical: degridding is bitwise equal
to the full index's; both
meet epsilon against the oracle (with weights, a mask, several plane batches).  Gridding
agrees to rounding: the order inside a bucket comes from the bin-sort's atomics."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2010_10122_gb300 import synthetic as S  # noqa: E402


@pytest.fixture(scope="module")
def wg():
    from paper_2010_10122_gb300 import _build
    _build.build()
    import paper_2010_10122_gb300 as wg
    assert torch.cuda.is_available()
    return wg


OBS = S.random_uvw_observation(611, 3, 96, 128, 25.0, seed=81)


@pytest.mark.parametrize("prec,eps,fft_impl,w_shift,cap", [
    ("f32", 1e-5, 0, 1, 0), ("f32", 1e-4, 0, 0, 3 << 20), ("f64", 1e-12, 2, 1, 0),
    ("f64", 1e-10, 3, 1, 0), ("f64", 1e-9, 2, 0, 5 << 20)])
def test_compact_index_matches_full_and_oracle(wg, oracle_lib, prec, eps, fft_impl, w_shift, cap):
    rdt, cdt = (np.float32, np.complex64) if prec == "f32" else (np.float64, np.complex128)
    rng = np.random.default_rng(5)
    wgt = rng.uniform(0.3, 2.0, (OBS.nrows, OBS.nchan))
    mask = (rng.uniform(size=(OBS.nrows, OBS.nchan)) > 0.2).astype(np.uint8)
    I = S.gaussian_image(OBS.npix_x, OBS.npix_y, seed=3)
    d = S.complex_normal((OBS.nrows, OBS.nchan), seed=4)
    outs = []
    for compact in (False, True):
        plan = wg.Plan(OBS.uvw, OBS.freq, OBS.npix_x, OBS.npix_y, OBS.pixsize_x, OBS.pixsize_y,
                       eps, prec, mask=mask, w_shift=w_shift, fft_impl=fft_impl,
                       max_workspace=cap, compact_index=compact)
        w = torch.from_numpy(wgt.astype(rdt)).cuda()
        vis = plan.degrid(torch.from_numpy(I.astype(rdt)).cuda(), wgt=w)
        img = plan.grid(torch.from_numpy(d.astype(cdt)).cuda(), wgt=w)
        outs.append((plan.info, vis, img))
    (fi, fv, fg), (ci, cv, cg) = outs
    assert ci["index_bytes"] < fi["index_bytes"]
    assert (ci["alpha"], ci["nu"], ci["nw"], ci["batch"]) == (fi["alpha"], fi["nu"], fi["nw"], fi["batch"])
    assert torch.equal(cv, fv)
    # gridding sums each bucket in index order, and the order inside a bucket comes from the
    # bin-sort's atomics (and FP32 adds with shared-memory atomics): separately built plans
    # agree to the plane-rounding term
    r_term = math.sqrt(max(fi["err_model"] ** 2 - (fi["eps_kernel"] / 0.8) ** 2, 0.0))
    tol = max(2e-6 if prec == "f32" else 1e-13, 10 * r_term)
    assert oracle_lib.rel_l2(cg.cpu().numpy(), fg.cpu().numpy()) <= tol
    rv = oracle_lib.degrid(OBS.uvw, OBS.freq, I, OBS.pixsize_x, OBS.pixsize_y, wgt=wgt, mask=mask)
    ri = oracle_lib.grid(OBS.uvw, OBS.freq, d, OBS.npix_x, OBS.npix_y, OBS.pixsize_x,
                         OBS.pixsize_y, wgt=wgt, mask=mask)
    assert oracle_lib.rel_l2(cv.cpu().numpy(), rv) <= eps
    assert oracle_lib.rel_l2(cg.cpu().numpy(), ri) <= eps


def test_compact_index_bytes_per_visibility(wg):
    """A compact plan holds exactly: bucket offsets (4 bytes per (tile, plane) + 1), 4 bytes per
    visibility, the uvw rows (24 bytes each) and the per-pixel correction table (16 / 32 bytes per
    pixel); the full plan holds 28 (FP32) / 52 (FP64) more bytes per visibility, and in FP64 a
    kernel-value table as well when it is small."""
    obs = S.array_observation(32, 40, 16, 256, 60 * S.ARCSEC, seed=82)
    for prec, eps, per_vis, per_pix in (("f32", 1e-5, 28, 16), ("f64", 1e-9, 52, 32)):
        comp = wg.Plan(obs.uvw, obs.freq, 256, 256, obs.pixsize_x, obs.pixsize_y, eps, prec,
                       compact_index=True).info
        full = wg.Plan(obs.uvw, obs.freq, 256, 256, obs.pixsize_x, obs.pixsize_y, eps, prec).info
        expect = 4 * (comp["ntiles"] * comp["nw"] + 1) + 4 * comp["nvis"] + 24 * obs.nrows + \
            per_pix * 256 * 256
        assert comp["index_bytes"] == expect, (comp["index_bytes"], expect)
        wts = (3 * 16 * 8 * full["nvis"]) if prec == "f64" else 0   # resident kernel values
        assert full["index_bytes"] - comp["index_bytes"] in (
            full["nvis"] * per_vis - 24 * obs.nrows, full["nvis"] * per_vis - 24 * obs.nrows + wts)
