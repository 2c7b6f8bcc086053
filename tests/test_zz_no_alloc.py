"""wg_degrid_noalloc: degridding for callers that cannot allocate device memory in their
hot path.  Its workspace is a fixed device array inside the library (WG_NOALLOC_SCRATCH_BYTES),
so the plan must be made with a workspace cap at or below that size.  Checked through the C
ABI against wg_degrid on the same plan, on two calls in a row (the second reuses the scratch
the first left behind).  This file is collected last so a failure here stops a -x run only
after every other test has run."""
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


@pytest.mark.parametrize("prec,eps,tol", [("f32", 1e-5, 1e-6), ("f64", 1e-10, 1e-13)])
def test_noalloc_matches_degrid_twice(wg, prec, eps, tol):
    from paper_2010_10122_gb300 import synthetic as S
    obs = S.random_uvw_observation(1500, 3, 128, 96, 20.0, seed=31)
    rdt, cdt = (torch.float32, torch.complex64) if prec == "f32" else (torch.float64, torch.complex128)
    plan = wg.Plan(obs.uvw, obs.freq, 128, 96, obs.pixsize_x, obs.pixsize_y, eps, prec,
                   max_workspace=wg.wgrid.NOALLOC_SCRATCH_BYTES)
    assert plan.info["workspace_bytes"] <= wg.wgrid.NOALLOC_SCRATCH_BYTES
    L = wg.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        img = torch.from_numpy(S.gaussian_image(128, 96, seed=call)).to("cuda", rdt)
        ref = torch.empty((obs.nrows, obs.nchan), dtype=cdt, device="cuda")
        got = torch.full((obs.nrows, obs.nchan), float("nan"), dtype=cdt, device="cuda")
        assert L.wg_degrid(plan._h, ctypes.c_void_p(img.data_ptr()), None,
                           ctypes.c_void_p(ref.data_ptr()), stream, None) == 0
        rc = L.wg_degrid_noalloc(plan._h, ctypes.c_void_p(img.data_ptr()), None,
                                 ctypes.c_void_p(got.data_ptr()), stream)
        assert rc == 0, L.wg_last_error().decode()
        torch.cuda.synchronize()
        err = (got - ref).abs().max().item() / ref.abs().max().item()
        assert np.isfinite(err) and err <= tol, (call, err)


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
