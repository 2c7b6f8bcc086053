"""torch.autograd over the operator: WDegrid (forward degrid, backward grid) and WGrid.

The loss of the differentiable-operator workload, L = 0.5 ||degrid(x) - d||^2 with
d = degrid(x_true) + complex noise, has dL/dx = R^dagger(R x - d).  The autograd gradient
(backward = the hand-written grid kernel) is checked against central finite differences of L
at sampled pixels and against the oracle's direct adjoint applied to the same residual.
"""
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


def _loss(ag, x, plan, d):
    r = ag.degrid(x, plan) - d
    return 0.5 * (r.real.double() ** 2 + r.imag.double() ** 2).sum()


@pytest.mark.parametrize("prec,eps,fd_tol", [("f64", 1e-10, 1e-7), ("f32", 1e-5, 2e-3)])
def test_gradient_fd_and_oracle_small(wg, oracle_lib, prec, eps, fd_tol):
    from paper_2010_10122_gb300 import autograd as ag
    obs = S.random_uvw_observation(600, 2, 64, 64, 20.0, seed=41)
    rdt, cdt = (torch.float32, torch.complex64) if prec == "f32" else (torch.float64, torch.complex128)
    plan = wg.Plan(obs.uvw, obs.freq, 64, 64, obs.pixsize_x, obs.pixsize_y, eps, prec)
    x_true = torch.from_numpy(S.gaussian_image(64, 64, seed=1)).to("cuda", rdt)
    noise = torch.from_numpy(0.01 * S.complex_normal((600, 2), seed=2)).to("cuda", cdt)
    with torch.no_grad():
        d = plan.degrid(x_true) + noise
    x = (x_true + 0.3 * torch.from_numpy(S.gaussian_image(64, 64, seed=3)).to("cuda", rdt)).requires_grad_(True)
    L = _loss(ag, x, plan, d)
    L.backward()
    g = x.grad.detach().double().cpu().numpy()
    # central finite differences at sampled pixels
    rng = np.random.default_rng(0)
    pix = rng.choice(64 * 64, 16, replace=False)
    # the loss is quadratic, so central differences are exact up to rounding for any step; a
    # large step keeps single-precision rounding of the forward passes small against it
    h = (1e-3 if prec == "f64" else 0.5) * float(x.detach().double().pow(2).mean().sqrt())
    fd = []
    with torch.no_grad():
        for p in pix:
            e = torch.zeros(64 * 64, dtype=rdt, device="cuda"); e[p] = h
            e = e.reshape(64, 64)
            fd.append(float(_loss(ag, x + e, plan, d) - _loss(ag, x - e, plan, d)) / (2 * h))
    fd = np.array(fd)
    scale = np.abs(g).max()
    assert np.abs(fd - g.reshape(-1)[pix]).max() <= fd_tol * scale
    # oracle adjoint of the same residual: dL/dx = R0^dagger (R x - d)
    with torch.no_grad():
        r = (plan.degrid(x.detach()) - d).cpu().numpy().astype(np.complex128)
    go = oracle_lib.grid(obs.uvw, obs.freq, r, 64, 64, obs.pixsize_x, obs.pixsize_y)
    assert oracle_lib.rel_l2(g, go) <= eps


def test_wgrid_backward_is_degrid(wg):
    from paper_2010_10122_gb300 import autograd as ag
    obs = S.random_uvw_observation(400, 2, 64, 64, 20.0, seed=42)
    plan = wg.Plan(obs.uvw, obs.freq, 64, 64, obs.pixsize_x, obs.pixsize_y, 1e-10, "f64")
    v = torch.from_numpy(S.complex_normal((400, 2), seed=4)).cuda().requires_grad_(True)
    b = torch.from_numpy(S.gaussian_image(64, 64, seed=5)).cuda()
    img = ag.grid(v, plan)
    L = 0.5 * ((img - b) ** 2).sum()
    L.backward()
    with torch.no_grad():
        ref = plan.degrid(plan.grid(v.detach()) - b)
    assert torch.allclose(v.grad, ref, rtol=0, atol=1e-12 * ref.abs().max().item())


def test_no_activations_saved(wg):
    from paper_2010_10122_gb300 import autograd as ag
    obs = S.random_uvw_observation(300, 2, 64, 64, 20.0, seed=43)
    plan = wg.Plan(obs.uvw, obs.freq, 64, 64, obs.pixsize_x, obs.pixsize_y, 1e-5, "f32")
    x = torch.from_numpy(S.gaussian_image(64, 64, seed=6)).to("cuda", torch.float32).requires_grad_(True)
    y = ag.degrid(x, plan)
    assert y.grad_fn.saved_tensors == ()


def test_differentiable_workload_4k(wg, oracle_lib):
    """4096^2 float32 image, 9,999,360 visibilities (64 antennas x 310 x 16 channels), eps 1e-5:
    the autograd gradient at 64 random pixels against central finite differences and against
    the oracle adjoint applied to the residual; activation memory of the graph reported."""
    from paper_2010_10122_gb300 import autograd as ag
    obs = S.diff_4k()
    n = obs.npix_x
    plan = wg.Plan(obs.uvw, obs.freq, n, n, obs.pixsize_x, obs.pixsize_y, 1e-5, "f32")
    x_true = torch.from_numpy(S.point_source_image(n, n, seed=7)).to("cuda", torch.float32)
    noise = torch.from_numpy(0.01 * S.complex_normal((obs.nrows, obs.nchan), seed=8)).to("cuda", torch.complex64)
    with torch.no_grad():
        d = plan.degrid(x_true) + noise
    del noise
    x = (0.5 * x_true).requires_grad_(True)
    torch.cuda.synchronize()
    m0 = torch.cuda.memory_allocated()
    L = _loss(ag, x, plan, d)
    m_graph = torch.cuda.memory_allocated() - m0
    L.backward()
    g = x.grad.detach().double().cpu().numpy().reshape(-1)
    print(f"activation memory held by the graph: {m_graph} bytes (output + loss scalars)")
    rng = np.random.default_rng(1)
    pix = rng.choice(np.flatnonzero(S.point_source_image(n, n, seed=7).reshape(-1)), 64, replace=False)
    h = 0.05
    fd = []
    with torch.no_grad():
        xd = x.detach()
        for p in pix:
            e = torch.zeros(n * n, dtype=torch.float32, device="cuda"); e[p] = h
            e = e.reshape(n, n)
            fd.append(float(_loss(ag, xd + e, plan, d) - _loss(ag, xd - e, plan, d)) / (2 * h))
        r = (plan.degrid(xd) - d).cpu().numpy().astype(np.complex128)
    fd = np.array(fd)
    scale = np.abs(g[pix]).max()
    assert np.abs(fd - g[pix]).max() <= 1e-2 * scale
    go = oracle_lib.grid(obs.uvw, obs.freq, r, n, n, obs.pixsize_x, obs.pixsize_y, pixel_index=pix)
    assert oracle_lib.rel_l2(g[pix], go) <= 1e-5
