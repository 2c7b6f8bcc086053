"""Host logic of the continuous-batching server, with a fake executor (no GPU): admission by
slots and memory, skip-ahead, plan residency with LRU eviction, failures and timeouts."""
import concurrent.futures as cf

import pytest

from paper_2010_10122_gb300.server import Executor, Request, Server, ServerTimeout


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-3          # every query advances time a little
        return self.t


class FakeExecutor(Executor):
    """Plans of given sizes; a request takes `duration[obs]` clock seconds; result = 2 * data."""

    def __init__(self, clock, sizes, duration, fail_launch=(), never_finish=()):
        self.clock, self.sizes, self.duration = clock, sizes, duration
        self.created, self.dropped = [], []
        self.fail_launch, self.never_finish = set(fail_launch), set(never_finish)
        self.running = {}

    def plan_bytes(self, obs, epsilon, precision):
        if (obs, epsilon, precision) not in self.created:
            self.created.append((obs, epsilon, precision))
        resident, ws = self.sizes[obs]
        return resident, ws, 100

    def drop_plan(self, obs, epsilon, precision):
        self.dropped.append((obs, epsilon, precision))
        self.created.remove((obs, epsilon, precision))

    def launch(self, req, slot):
        if req.obs in self.fail_launch:
            raise RuntimeError("launch failed")
        assert slot not in self.running, "slot reused while busy"
        self.running[slot] = req
        return (slot, self.clock.t + self.duration[req.obs])

    def poll(self, h):
        slot, t_end = h
        req = self.running[slot]
        if req.obs in self.never_finish:
            return False
        if self.clock.t >= t_end:
            del self.running[slot]
            return True
        return False

    def finish(self, req, h):
        req.result = 2 * req.data


def make(n, obs="a", t=0.0, dt=0.0):
    return [Request(obs, "degrid", i, 1e-5, "f32", arrival=t + i * dt) for i in range(n)]


def test_all_complete_with_correct_results_and_bounded_concurrency():
    clk = FakeClock()
    ex = FakeExecutor(clk, {"a": (10, 5)}, {"a": 0.05})
    srv = Server(ex, slots=3, memory_budget=1000, clock=clk)
    out = srv.run(make(20, dt=0.002))
    assert len(out) == 20 and all(r.error is None and r.result == 2 * r.data for r in out)
    assert srv.max_inflight == 3
    rep = srv.report()
    assert rep["completed"] == 20 and rep["p99_s"] >= rep["p50_s"] > 0


def test_memory_budget_limits_admission_and_small_requests_skip_ahead():
    clk = FakeClock()
    ex = FakeExecutor(clk, {"big": (0, 60), "small": (0, 10)}, {"big": 0.05, "small": 0.01})
    srv = Server(ex, slots=8, memory_budget=100, clock=clk)
    reqs = make(3, "big") + make(4, "small", t=0.0)
    out = srv.run(reqs)
    assert len(out) == 7 and all(r.error is None for r in out)
    assert srv.peak_memory <= 100
    first_small = min(r.start for r in out if r.obs == "small")
    second_big = sorted(r.start for r in out if r.obs == "big")[1]
    assert first_small < second_big        # smaller requests used the space the big one left


def test_request_larger_than_budget_fails_alone_others_complete():
    clk = FakeClock()
    ex = FakeExecutor(clk, {"huge": (0, 500), "a": (0, 5)}, {"huge": 0.01, "a": 0.01})
    srv = Server(ex, slots=2, memory_budget=100, clock=clk)
    out = srv.run(make(1, "huge") + make(3, "a"))
    errs = [r for r in out if r.error is not None]
    assert len(errs) == 1 and errs[0].obs == "huge" and isinstance(errs[0].error, MemoryError)
    assert sum(r.error is None for r in out) == 3


def test_idle_plans_are_evicted_lru_to_make_room():
    clk = FakeClock()
    ex = FakeExecutor(clk, {"a": (50, 5), "b": (50, 5), "c": (50, 5)}, {"a": .01, "b": .01, "c": .01})
    srv = Server(ex, slots=1, memory_budget=120, clock=clk)
    out = srv.run(make(1, "a") + make(1, "b", t=0.1) + make(1, "c", t=0.2))
    assert all(r.error is None for r in out)
    assert ("a", 1e-5, "f32") in ex.dropped
    assert srv.peak_memory <= 120


def test_launch_failure_releases_slot():
    clk = FakeClock()
    ex = FakeExecutor(clk, {"bad": (0, 5), "a": (0, 5)}, {"bad": .01, "a": .01}, fail_launch={"bad"})
    srv = Server(ex, slots=1, memory_budget=100, clock=clk)
    out = srv.run(make(2, "bad") + make(2, "a"))
    assert sum(r.error is not None for r in out) == 2 and sum(r.error is None for r in out) == 2
    assert srv.workspace_in_use == 0 and len(srv.free_slots) == 1


class ClockFuture(cf.Future):
    """A future that completes (with fn()) once the fake clock reaches t_ready."""

    def __init__(self, clock, t_ready, fn):
        super().__init__()
        self.clock, self.t_ready, self.fn = clock, t_ready, fn

    def done(self):
        if not super().done() and self.clock.t >= self.t_ready:
            self.set_result(self.fn())
        return super().done()


class SlowPlanExecutor(FakeExecutor):
    """Plans of `slow` observations take `build` clock seconds to build (a future that
    completes later, as a worker thread would); outputs take `out` bytes."""

    def __init__(self, clock, sizes, duration, slow=(), build=0.2, out=0):
        super().__init__(clock, sizes, duration)
        self.slow, self.build, self.out = set(slow), build, out
        self.futures = {}

    def plan_async(self, obs, epsilon, precision):
        key = (obs, epsilon, precision)
        if obs not in self.slow or key in self.created:
            return super().plan_async(obs, epsilon, precision)
        if key not in self.futures:
            self.futures[key] = ClockFuture(self.clock, self.clock.t + self.build,
                                            lambda: self.plan_bytes(obs, epsilon, precision))
        return self.futures[key]

    def output_bytes(self, req):
        return self.out


def test_requests_go_ahead_of_a_plan_being_built():
    """A request whose plan is still being built does not hold up later requests whose plans
    are resident; it is admitted once the build finishes."""
    clk = FakeClock()
    ex = SlowPlanExecutor(clk, {"cold": (10, 5), "hot": (10, 5)}, {"cold": 0.01, "hot": 0.01},
                          slow={"cold"}, build=0.3)
    srv = Server(ex, slots=2, memory_budget=1000, clock=clk)
    out = srv.run(make(1, "cold") + make(6, "hot", t=0.001, dt=0.01))
    assert all(r.error is None for r in out)
    cold = [r for r in out if r.obs == "cold"][0]
    hot_starts = sorted(r.start for r in out if r.obs == "hot")
    assert cold.start >= 0.3 and hot_starts[0] < 0.1 and srv.plan_waits > 0
    assert cold.latency < 0.5          # admitted soon after its plan exists


def test_outputs_are_charged_to_the_memory_budget():
    clk = FakeClock()
    ex = SlowPlanExecutor(clk, {"a": (0, 10)}, {"a": 0.05}, out=40)
    srv = Server(ex, slots=8, memory_budget=100, clock=clk)
    out = srv.run(make(6, "a"))
    assert all(r.error is None for r in out)
    assert srv.max_inflight == 2 and srv.peak_memory <= 100    # 2 x (10 + 40) fit, 3 do not


def test_stuck_request_times_out_on_the_host():
    clk = FakeClock()
    ex = FakeExecutor(clk, {"stuck": (0, 5)}, {"stuck": 0.01}, never_finish={"stuck"})
    srv = Server(ex, slots=2, memory_budget=100, timeout_s=0.5, clock=clk)
    with pytest.raises(ServerTimeout):
        srv.run(make(1, "stuck"))


def test_workspace_cap_is_a_target_host():
    """plan_with_cap_target doubles the cap while the plan reports that one w-plane needs more,
    up to the limit; other errors and the cap error at the limit are raised unchanged."""
    from paper_2010_10122_gb300.server import plan_with_cap_target

    class Err(RuntimeError):
        def __init__(self, code, msg):
            super().__init__(msg)
            self.code = code

    OOM, ARG = 2, 1
    calls = []

    def make_needing(need):
        def make(cap):
            calls.append(cap)
            if cap != 0 and cap < need:
                raise Err(OOM, f"one w-plane needs {need} bytes of workspace, above the cap {cap}")
            return ("plan", cap)
        return make

    assert plan_with_cap_target(make_needing(5), 1, 64, Err, OOM) == ("plan", 8)
    assert calls == [1, 2, 4, 8]
    calls.clear()
    assert plan_with_cap_target(make_needing(18), 8, 20, Err, OOM) == ("plan", 20)   # capped at the limit
    assert calls == [8, 16, 20]
    calls.clear()
    with pytest.raises(Err):                       # beyond the limit: the last cap error
        plan_with_cap_target(make_needing(100), 8, 20, Err, OOM)
    assert calls == [8, 16, 20]

    def other(cap):
        raise Err(ARG, "frequencies must be positive")
    with pytest.raises(Err):
        plan_with_cap_target(other, 8, 64, Err, OOM)

    def real_oom(cap):                             # a device allocation failure is not the cap
        raise Err(OOM, "device allocation of 123 bytes failed")
    with pytest.raises(Err):
        plan_with_cap_target(real_oom, 8, 64, Err, OOM)
