"""Continuous-batching server for degrid / grid requests over resident observations.

The paper has no serving layer; this is the system pattern the build adds on top of the
operator: many observations' plans (visibility index + per-pixel tables) stay resident on the
device, requests (degrid of an image, or grid of visibilities, at a requested epsilon and
precision) arrive over time, and each is admitted as soon as a stream slot is free and the
device-memory budget has room for its workspace and its output.  Plans are built off the
scheduler's thread (the executor builds them on a worker thread with its own CUDA stream):
while a request's plan is being built the request waits and later arrivals whose plans are
resident go ahead of it.  Admitted requests run concurrently on their own CUDA streams, so
their kernels overlap on the GPU; completions are detected by polling CUDA events (bounded host
waits, no device-side spin), which frees the slot and the memory for the next request.  Latency
is measured from arrival to completion.

The scheduler itself (admission, FIFO with skip-ahead, memory accounting, plan residency with
LRU eviction, timeouts) is host logic over an executor interface, so it can be exercised on the
CPU with a fake executor; ``CudaExecutor`` runs requests through libwgrid.so.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import itertools
import threading
import time
from typing import Any, Callable, Dict, List, Optional, Tuple


class ServerTimeout(RuntimeError):
    """A request did not complete within the server's deadline (host-side detection)."""


@dataclasses.dataclass(eq=False)   # identity: requests carry tensors, and a pending queue is
class Request:                       # searched for the one being admitted
    obs: str                      # observation key
    direction: str                # "degrid" (image -> vis) or "grid" (vis -> image)
    data: Any                     # image (degrid) or visibilities (grid)
    epsilon: float
    precision: str                # "f32" / "f64"
    arrival: float = 0.0          # seconds on the server clock
    rid: int = -1
    # filled by the server
    start: Optional[float] = None
    done: Optional[float] = None
    result: Any = None
    error: Optional[BaseException] = None
    nvis: int = 0
    workspace: int = 0

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival


class Executor:
    """Interface the scheduler drives."""

    def plan_bytes(self, obs: str, epsilon: float, precision: str) -> Tuple[int, int, int]:
        """(resident bytes of the plan, per-call workspace bytes, visibilities); creates the
        plan if needed (blocking)."""
        raise NotImplementedError

    def plan_async(self, obs: str, epsilon: float, precision: str) -> "cf.Future":
        """A future of plan_bytes(...).  The default builds the plan right away on the calling
        thread; executors whose plans take long to build override it with a worker thread."""
        f: cf.Future = cf.Future()
        try:
            f.set_result(self.plan_bytes(obs, epsilon, precision))
        except Exception as e:  # noqa: BLE001 - handed to the scheduler through the future
            f.set_exception(e)
        return f

    def output_bytes(self, req: "Request") -> int:
        """Device bytes of the request's output (charged to the memory budget while it runs)."""
        return 0

    def drop_plan(self, obs: str, epsilon: float, precision: str) -> None:
        raise NotImplementedError

    def launch(self, req: Request, slot: int) -> Any:
        """Enqueue the request on slot `slot`; return a handle."""
        raise NotImplementedError

    def poll(self, handle: Any) -> bool:
        """True once the request's device work has finished (non-blocking)."""
        raise NotImplementedError

    def finish(self, req: Request, handle: Any) -> None:
        """Collect the result into req.result (called after poll() returned True)."""
        raise NotImplementedError


class Server:
    def __init__(self, executor: Executor, slots: int = 8, memory_budget: int = 150 << 30,
                 timeout_s: float = 600.0, clock: Callable[[], float] = time.perf_counter):
        self.ex = executor
        self.slots = slots
        self.budget = memory_budget
        self.timeout_s = timeout_s
        self.clock = clock
        self.t0 = clock()
        self.pending: collections.deque = collections.deque()
        self.inflight: Dict[int, Tuple[Request, Any]] = {}   # slot -> (request, handle)
        self.free_slots = list(range(slots))[::-1]
        self.resident: "collections.OrderedDict[tuple, int]" = collections.OrderedDict()
        self.busy_plans: Dict[tuple, int] = collections.Counter()
        self.workspace_in_use = 0
        self.completed: List[Request] = []
        self.max_inflight = 0
        self.peak_memory = 0
        self.plan_waits = 0          # admission passes that skipped a request whose plan was building
        self._building: Dict[tuple, "cf.Future"] = {}
        self._ids = itertools.count()

    # ------------------------------------------------------------------ accounting
    def now(self) -> float:
        return self.clock() - self.t0

    def memory_in_use(self) -> int:
        return sum(self.resident.values()) + self.workspace_in_use

    def _plan_state(self, key):
        """(resident, workspace, nvis) of a plan that is ready, None while it is being built
        (the build is started on first use); raises the build's exception if it failed."""
        f = self._building.get(key)
        if f is None:
            if key in self.resident:
                f = self.ex.plan_async(*key)   # resident: returns at once
            else:
                f = self._building[key] = self.ex.plan_async(*key)
        if not f.done():
            return None
        self._building.pop(key, None)
        resident, ws, nvis = f.result()
        if key in self.resident:
            self.resident.move_to_end(key)
        else:
            self.resident[key] = resident
        return resident, ws, nvis

    def _evict_for(self, need: int, keep) -> None:
        """Drop least-recently used idle plans until `need` more bytes fit."""
        for key in list(self.resident):
            if self.memory_in_use() + need <= self.budget:
                return
            if key == keep or self.busy_plans.get(key, 0) > 0:
                continue
            self.ex.drop_plan(*key)
            del self.resident[key]

    # ------------------------------------------------------------------ API
    def adopt(self, plans: Dict[tuple, int]) -> None:
        """Account for plans the executor already holds ({(obs, epsilon, precision): bytes}), so
        that they count against the budget and can be evicted."""
        for key, nbytes in plans.items():
            self.resident[key] = nbytes

    def submit(self, req: Request) -> Request:
        req.rid = next(self._ids)
        if req.arrival is None or req.arrival == 0.0:
            req.arrival = self.now()
        self.pending.append(req)
        return req

    def _admit(self) -> int:
        """Admit pending requests in arrival order; a request that does not fit the memory
        left is skipped over (it keeps its place) so smaller ones can use the space."""
        admitted = 0
        for req in list(self.pending):
            if not self.free_slots:
                break
            key = (req.obs, req.epsilon, req.precision)
            try:
                st = self._plan_state(key)
            except Exception as e:  # plan creation failed: the request fails, others go on
                req.error = e
                req.done = self.now()
                self.pending.remove(req)
                self.completed.append(req)
                continue
            if st is None:          # plan still being built: later requests may go first
                self.plan_waits += 1
                continue
            resident, ws, nvis = st
            ws += self.ex.output_bytes(req)     # the output lives on the device too
            if self.memory_in_use() + ws > self.budget:
                self._evict_for(ws, key)
            if self.memory_in_use() + ws > self.budget:
                if resident + ws > self.budget:   # can never fit, even alone
                    req.error = MemoryError("request does not fit the memory budget")
                    req.done = self.now()
                    self.pending.remove(req)
                    self.completed.append(req)
                continue
            slot = self.free_slots.pop()
            self.pending.remove(req)
            req.workspace, req.nvis = ws, nvis
            req.start = self.now()
            self.workspace_in_use += ws
            self.busy_plans[key] += 1
            try:
                handle = self.ex.launch(req, slot)
            except Exception as e:
                self._release(req, slot, key)
                req.error = e
                req.done = self.now()
                self.completed.append(req)
                continue
            self.inflight[slot] = (req, handle)
            admitted += 1
            self.max_inflight = max(self.max_inflight, len(self.inflight))
            self.peak_memory = max(self.peak_memory, self.memory_in_use())
        return admitted

    def _release(self, req, slot, key):
        self.workspace_in_use -= req.workspace
        self.busy_plans[key] -= 1
        self.free_slots.append(slot)

    def _reap(self) -> int:
        done = 0
        for slot, (req, handle) in list(self.inflight.items()):
            if self.ex.poll(handle):
                try:
                    self.ex.finish(req, handle)
                except Exception as e:
                    req.error = e
                req.done = self.now()
                del self.inflight[slot]
                self._release(req, slot, (req.obs, req.epsilon, req.precision))
                self.completed.append(req)
                done += 1
            elif self.now() - req.start > self.timeout_s:
                raise ServerTimeout(f"request {req.rid} ({req.obs}, {req.direction}) exceeded "
                                    f"{self.timeout_s} s")
        return done

    def step(self) -> bool:
        """One scheduler iteration; returns True if anything happened."""
        r = self._reap()
        a = self._admit()
        return (r + a) > 0

    def run(self, requests: List[Request], idle_sleep: float = 2e-5) -> List[Request]:
        """Serve `requests`, each released into the queue at its `arrival` time (seconds from
        now).  Returns them completed, in completion order."""
        stream = sorted(requests, key=lambda r: r.arrival)
        self.t0 = self.clock()
        i = 0
        while i < len(stream) or self.pending or self.inflight:
            t = self.now()
            while i < len(stream) and stream[i].arrival <= t:
                self.submit(stream[i])
                i += 1
            if not self.step():
                if not self.inflight and not self.pending and i < len(stream):
                    wait = stream[i].arrival - self.now()
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
                else:
                    time.sleep(idle_sleep)
        return self.completed

    # ------------------------------------------------------------------ metrics
    def report(self) -> dict:
        lat = sorted(r.latency for r in self.completed if r.error is None)
        if not lat:
            return {"completed": 0}
        q = lambda p: lat[min(len(lat) - 1, int(round(p * (len(lat) - 1))))]
        span = max(r.done for r in self.completed) - min(r.arrival for r in self.completed)
        nvis = sum(r.nvis for r in self.completed if r.error is None)
        errors = collections.Counter(f"{type(r.error).__name__}: {str(r.error)[:80]}"
                                     for r in self.completed if r.error is not None)
        return {"completed": len(lat), "failed": sum(r.error is not None for r in self.completed),
                "errors": dict(errors.most_common(5)),
                "p50_s": q(0.5), "p99_s": q(0.99), "mean_s": sum(lat) / len(lat),
                "span_s": span, "vis_per_s": nvis / span if span > 0 else None,
                "max_inflight": self.max_inflight, "peak_memory": self.peak_memory,
                "plan_waits": self.plan_waits}


class CudaExecutor(Executor):
    """Runs requests through libwgrid.so, one CUDA stream per slot; plans are built by a worker
    thread on a stream of its own (wg_plan_create synchronises only that stream, and ctypes
    releases the interpreter lock during the call, so the scheduler keeps running)."""

    def __init__(self, observations: Dict[str, Any], slots: int, workspace_cap: int = 8 << 30,
                 device=None, keep_results: bool = True, compact: bool = True):
        import torch
        from . import wgrid
        self.torch = torch
        self.wg = wgrid
        self.obs = observations        # key -> synthetic.Observation-like (uvw, freq, npix, pixsize)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        self.plan_stream = torch.cuda.Stream(device=self.device)
        self.plans: Dict[tuple, Any] = {}
        self.cap = workspace_cap
        self._lock = threading.Lock()
        self._builder = cf.ThreadPoolExecutor(max_workers=1, thread_name_prefix="wg-plan")
        self._futures: Dict[tuple, "cf.Future"] = {}
        self.keep_results = keep_results   # False: outputs are dropped once complete (benchmarks)
        self.compact = compact             # compact plans: index 4 B / visibility, no resident tables

    def _build(self, key):
        obs, epsilon, precision = key
        o = self.obs[obs]
        # cached workspace beyond what the slots can use at once goes back to the driver first,
        # so that it does not crowd out the plan
        self.wg.pool_trim(len(self.streams) * self.cap, device=self.device)
        limit = max(self.cap, self.torch.cuda.get_device_properties(self.device).total_memory // 4)

        def make(cap):
            with self.torch.cuda.device(self.device):
                return self.wg.Plan(o.uvw, o.freq, o.npix_x, o.npix_y, o.pixsize_x, o.pixsize_y,
                                    epsilon, precision, max_workspace=cap, device=self.device,
                                    stream=self.plan_stream, compact_index=self.compact)
        p = plan_with_cap_target(make, self.cap, limit, self.wg.WgridError, self.wg.WG_ERR_OOM)
        with self._lock:
            self.plans[key] = p
        info = p.info
        return info["index_bytes"], info["workspace_bytes"], info["nvis"]

    def plan_async(self, obs, epsilon, precision):
        key = (obs, epsilon, precision)
        with self._lock:
            p = self.plans.get(key)
            if p is not None:
                f = cf.Future()
                info = p.info
                f.set_result((info["index_bytes"], info["workspace_bytes"], info["nvis"]))
                return f
            f = self._futures.get(key)
            if f is None or (f.done() and f.exception() is not None):
                f = self._futures[key] = self._builder.submit(self._build, key)
            return f

    def plan_bytes(self, obs, epsilon, precision):
        return self.plan_async(obs, epsilon, precision).result()

    def resident_plans(self) -> Dict[tuple, int]:
        with self._lock:
            return {k: p.info["index_bytes"] for k, p in self.plans.items()}

    def output_bytes(self, req):
        o = self.obs[req.obs]
        if req.direction == "degrid":
            return o.nrows * o.nchan * (8 if req.precision == "f32" else 16)
        return o.npix_x * o.npix_y * (4 if req.precision == "f32" else 8)

    def drop_plan(self, obs, epsilon, precision):
        """Forget the plan now; free it on the builder thread (wg_plan_destroy waits for the
        device, which the scheduler thread must not do)."""
        key = (obs, epsilon, precision)
        with self._lock:
            p = self.plans.pop(key, None)
            self._futures.pop(key, None)
        if p is not None:
            self._builder.submit(p.close)

    def close(self):
        """Wait for pending plan builds and frees, then free every plan."""
        self._builder.shutdown(wait=True)
        with self._lock:
            plans, self.plans = list(self.plans.values()), {}
        for p in plans:
            p.close()

    def launch(self, req, slot):
        torch = self.torch
        s = self.streams[slot]
        p = self.plans[(req.obs, req.epsilon, req.precision)]
        s.wait_stream(torch.cuda.current_stream(self.device))   # inputs produced before submit
        with torch.cuda.stream(s):
            data = req.data
            if data.device != self.device:
                data = data.to(self.device, non_blocking=True)
            data.record_stream(s)
            out = p.degrid(data, stream=s) if req.direction == "degrid" else p.grid(data, stream=s)
            ev = torch.cuda.Event()
            ev.record(s)
        return (ev, out, s)

    def poll(self, handle):
        return handle[0].query()

    def finish(self, req, handle):
        req.result = handle[1] if self.keep_results else None


def plan_with_cap_target(make: Callable[[int], Any], cap: int, limit: int, error_type,
                         oom_code: int) -> Any:
    """make(cap) with the workspace cap as a per-request target: an observation whose single
    w-plane (with its per-visibility partial sums and records) needs more than the cap gets
    twice the cap, and so on up to `limit`; the server then admits the plan by the workspace it
    reports.  Other errors, and the cap error at the limit (or with no cap), are raised."""
    while True:
        try:
            return make(cap)
        except error_type as e:
            if getattr(e, "code", None) != oom_code or "above the cap" not in str(e) \
                    or cap == 0 or cap >= limit:
                raise
            cap = min(2 * cap, limit)


def run_serial(executor: Executor, requests: List[Request]) -> float:
    """One-at-a-time execution of the same requests (the baseline a continuous-batching server is
    compared with): the plans are built first (not timed), then each request is launched on slot
    0 and waited for.  Returns seconds."""
    for req in requests:
        executor.plan_bytes(req.obs, req.epsilon, req.precision)
    t0 = time.perf_counter()
    for req in requests:
        h = executor.launch(req, 0)
        while not executor.poll(h):
            time.sleep(1e-5)
        executor.finish(req, h)
    return time.perf_counter() - t0
