"""wg_degrid_noalloc: degridding for callers that cannot allocate device memory while they run
(memory owned by another allocator or a fixed arena, real-time loops).  Its workspace is a fixed
device array inside the library (WG_NOALLOC_SCRATCH_BYTES), so the plan must be made with a
workspace cap at or below that size.  Checked through the C ABI against wg_degrid on the same
plan, on two calls in a row (the second reuses the scratch the first left behind), with one
plane batch and with several; the device's free memory must not change across a warmed-up
call.  This file is collected last so a failure here stops a -x run only after every other test
has run."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wg():
    from paper_2010_10122_gb300 import _build
    _build.build()
    import paper_2010_10122_gb300 as wg
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return wg


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("prec,eps,cap", [("f32", 1e-5, None), ("f64", 1e-10, None),
                                          ("f32", 1e-5, 1 << 20), ("f64", 1e-12, 3 << 20)])
def test_noalloc_matches_degrid_twice(wg, prec, eps, cap):
    from paper_2010_10122_gb300 import synthetic as S
    obs = S.random_uvw_observation(1500, 3, 128, 96, 20.0, seed=31)
    rdt, cdt = (torch.float32, torch.complex64) if prec == "f32" else (torch.float64, torch.complex128)
    plan = wg.Plan(obs.uvw, obs.freq, 128, 96, obs.pixsize_x, obs.pixsize_y, eps, prec,
                   max_workspace=cap or wg.wgrid.NOALLOC_SCRATCH_BYTES)
    info = plan.info
    assert info["workspace_bytes"] <= wg.wgrid.NOALLOC_SCRATCH_BYTES
    if cap is not None:   # several plane batches share the scratch in turn
        assert info["batch"] < info["nw"], info
    L = wg.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    wgt = torch.from_numpy(np.random.default_rng(3).uniform(0.5, 2.0, (obs.nrows, obs.nchan))).to("cuda", rdt)
    for call in range(2):
        img = torch.from_numpy(S.gaussian_image(128, 96, seed=call)).to("cuda", rdt)
        w = wgt if call == 1 else None
        ref = torch.empty((obs.nrows, obs.nchan), dtype=cdt, device="cuda")
        got = torch.full((obs.nrows, obs.nchan), float("nan"), dtype=cdt, device="cuda")
        assert L.wg_degrid(plan._h, _p(img), _p(w), _p(ref), stream, None) == 0
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0] if call == 1 else None
        rc = L.wg_degrid_noalloc(plan._h, _p(img), _p(w), _p(got), stream)
        assert rc == 0, L.wg_last_error().decode()
        torch.cuda.synchronize()
        if free0 is not None:   # the first call loaded any lazily loaded kernels
            assert torch.cuda.mem_get_info()[0] == free0
        # the same plan, plane batches and summation order: identical results
        assert torch.equal(got, ref), (call, (got - ref).abs().max().item())
    plan.close()


def test_noalloc_rejects_plans_beyond_the_scratch(wg):
    from paper_2010_10122_gb300 import synthetic as S
    obs = S.random_uvw_observation(200, 2, 1024, 1024, 20.0, seed=32)
    plan = wg.Plan(obs.uvw, obs.freq, 1024, 1024, obs.pixsize_x, obs.pixsize_y, 1e-10, "f64")
    assert plan.info["workspace_bytes"] > wg.wgrid.NOALLOC_SCRATCH_BYTES
    img = torch.zeros((1024, 1024), dtype=torch.float64, device="cuda")
    out = torch.empty((200, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(wg.WgridError) as ei:
        plan.degrid_noalloc(img, out)
    assert ei.value.code == wg.wgrid.WG_ERR_ARG


def test_noalloc_binding_checks_weights(wg):
    from paper_2010_10122_gb300 import synthetic as S
    obs = S.random_uvw_observation(100, 2, 64, 64, 20.0, seed=33)
    plan = wg.Plan(obs.uvw, obs.freq, 64, 64, obs.pixsize_x, obs.pixsize_y, 1e-5, "f32",
                   max_workspace=wg.wgrid.NOALLOC_SCRATCH_BYTES)
    img = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    out = torch.empty((100, 2), dtype=torch.complex64, device="cuda")
    for bad in (torch.ones((100, 2), dtype=torch.float64, device="cuda"),
                torch.ones((100, 1), dtype=torch.float32, device="cuda")):
        with pytest.raises(ValueError):
            plan.degrid_noalloc(img, out, wgt=bad)
    plan.degrid_noalloc(img, out, wgt=torch.ones((100, 2), dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    assert not out.abs().any()
