"""Continuous batching on the GPU: mixed degrid / grid requests of several sizes, epsilons and
precisions over resident observations run concurrently on stream slots; every result equals
the same request run alone, within the parity tolerances; the memory budget bounds admission."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2010_10122_gb300 import synthetic as S  # noqa: E402


@pytest.fixture(scope="module")
def env():
    from paper_2010_10122_gb300 import _build
    _build.build()
    import paper_2010_10122_gb300 as wg  # noqa: F401
    from paper_2010_10122_gb300.server import CudaExecutor, Request, Server, run_serial
    assert torch.cuda.is_available()
    obs = {
        "o128": S.random_uvw_observation(2000, 4, 128, 128, 15.0, seed=51),
        "o256": S.random_uvw_observation(6000, 8, 256, 256, 10.0, seed=52),
        "o192": S.random_uvw_observation(500, 16, 192, 160, 20.0, seed=53),
        "a512": S.array_observation(16, 40, 8, 512, 60 * S.ARCSEC, seed=54),
    }
    return obs, CudaExecutor, Request, Server, run_serial


def make_requests(obs, Request, n=24, seed=0):
    rng = np.random.default_rng(seed)
    keys = sorted(obs)
    reqs = []
    t = 0.0
    for i in range(n):
        k = keys[rng.integers(len(keys))]
        o = obs[k]
        eps, prec = [(1e-4, "f32"), (1e-5, "f32"), (1e-12, "f64")][rng.integers(3)]
        rdt = torch.float32 if prec == "f32" else torch.float64
        cdt = torch.complex64 if prec == "f32" else torch.complex128
        if rng.uniform() < 0.5:
            data = torch.from_numpy(S.gaussian_image(o.npix_x, o.npix_y, seed=i)).to("cuda", rdt)
            direction = "degrid"
        else:
            data = torch.from_numpy(S.complex_normal((o.nrows, o.nchan), seed=i)).to("cuda", cdt)
            direction = "grid"
        t += rng.exponential(0.002)
        reqs.append(Request(k, direction, data, eps, prec, arrival=t))
    return reqs


def test_results_same_alone_and_in_the_mix(env):
    obs, CudaExecutor, Request, Server, run_serial = env
    mixed = make_requests(obs, Request)
    ex = CudaExecutor(obs, slots=4)
    srv = Server(ex, slots=4, memory_budget=40 << 30)
    srv.run(mixed)
    torch.cuda.synchronize()
    assert all(r.error is None for r in mixed)
    assert srv.max_inflight >= 2, "requests never overlapped"
    alone = make_requests(obs, Request)          # same seeds -> same data
    ex1 = CudaExecutor(obs, slots=1)
    run_serial(ex1, alone)
    torch.cuda.synchronize()
    for a, b in zip(mixed, alone):
        x, y = a.result, b.result
        # relative L2 difference (the parity metric).  Degrid is order-independent, so bitwise
        # equal.  Grid sums footprints in an order that depends on the plan's bin-sort (the
        # order inside a bucket comes from atomics) and, in FP32, on shared-memory atomics; the
        # two runs build separate plans, so they differ by rounding: well below epsilon, and at
        # most a few times the plan's plane-rounding term where that dominates (double-float
        # planes: the rounding of two slightly different inputs is uncorrelated)
        err = ((x - y).abs().pow(2).sum() / y.abs().pow(2).sum()).sqrt().item()
        info = ex1.plans[(b.obs, b.epsilon, b.precision)].info
        k_term = info["eps_kernel"] / 0.8
        r_term = math.sqrt(max(info["err_model"] ** 2 - k_term ** 2, 0.0))
        tol = max(0.1 * a.epsilon, 3 * r_term) if a.direction == "grid" else 0.0
        assert err <= tol, (a.obs, a.direction, a.precision, a.epsilon, err, tol)
    rep = srv.report()
    assert rep["completed"] == len(mixed) and rep["p99_s"] >= rep["p50_s"]


def test_memory_budget_bounds_concurrency(env):
    obs, CudaExecutor, Request, Server, run_serial = env
    reqs = [r for r in make_requests(obs, Request, n=12, seed=3)]
    ex = CudaExecutor(obs, slots=8)
    for r in reqs:
        ex.plan_bytes(r.obs, r.epsilon, r.precision)
    resident = sum(p.info["index_bytes"] for p in ex.plans.values())
    biggest = max(p.info["workspace_bytes"] for p in ex.plans.values())
    budget = resident + int(1.5 * biggest)
    srv = Server(ex, slots=8, memory_budget=budget)
    srv.run(reqs)
    torch.cuda.synchronize()
    assert all(r.error is None for r in reqs)
    assert srv.peak_memory <= budget


def test_workspace_cap_is_a_target(env):
    """An observation whose single w-plane needs more than the executor's workspace cap gets a
    plan with a larger workspace (the cap doubled until it fits) instead of failing."""
    obs, CudaExecutor, Request, Server, run_serial = env
    ex = CudaExecutor(obs, slots=1, workspace_cap=1 << 20)
    _, ws, _ = ex.plan_bytes("a512", 1e-5, "f32")
    assert ws > 1 << 20
    o = obs["a512"]
    r = Request("a512", "degrid",
                torch.from_numpy(S.gaussian_image(o.npix_x, o.npix_y, seed=4, dtype=np.float32)).cuda(),
                1e-5, "f32")
    run_serial(ex, [r])
    torch.cuda.synchronize()
    assert r.error is None and torch.isfinite(r.result.abs()).all()
    ex.close()
