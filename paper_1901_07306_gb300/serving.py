"""Continuous-batching server for many watch points on one GPU.

Routers (watch points, Sec. 4.1) send batches of <hip, oip> pairs; the
server keeps every router's sketch resident in one library context, plus one
extra router that plays the global server of Sec. 4.2.  All arithmetic runs
in the library's kernels; this module only schedules.

Engine (``SketchServer.run``):
  * admission -- requests are admitted in arrival order while their bytes fit
    a fixed budget of pinned host memory in flight (``budget_bytes``: bytes
    admitted and not yet scanned); a request that does not fit waits until
    earlier ones have been scanned and freed their room.
  * continuous batching -- every engine step scans all newly admitted
    requests with ONE ``sp_update_batched`` call on the compute stream.  The
    kernels read each request's pinned host pairs in place, across the host
    link (NVLink-C2C to the Grace CPU on a GB300; pinned memory is mapped into
    the device's address space), so a step has no staging copy, no copy
    stream and no device arena, and its scan streams its input once.  While
    the GPU works on step s the host admits and issues step s + 1.
  * windows -- every ``detect_every`` admitted pairs close a window (a time
    slice): the routers are OR-merged into the global router, it is detected
    asynchronously, and the routers start the next window (reset, or slide
    when ``window_slices`` > 1, Sec. 5).  A request belongs to the window in
    which it was admitted, so window contents depend only on arrival order.
  * failure detection -- every device wait of the engine (a step's scan, a
    window's detection) is bounded: when the oldest outstanding one has not
    completed ``timeout_s`` after it was issued, ``run`` raises
    ``ServingTimeout`` (the paper has no such step; a watch point whose GPU
    stopped making progress is reported instead of waited on forever).

The device side sits behind ``GpuOps`` (context, stream, result buffers),
so the scheduling, admission and deadline logic of ``SketchServer`` can also
be driven by a stand-in with the same methods.

Latencies are host wall-clock times: ``ack`` = arrival to the moment its scan
is seen complete; ``result`` = arrival to the moment the detection of its
window is available on the host.
"""
from __future__ import annotations

import gc
import time
from collections import deque
from dataclasses import dataclass

import numpy as np
import torch


@dataclass
class Request:
    router: int
    pairs: torch.Tensor          # int32 tensor of 2 n values: pinned host memory or CUDA
    arrival: float               # seconds after the start of the run
    window: int = -1
    t_ack: float = float("nan")
    t_result: float = float("nan")

    @property
    def n_pairs(self) -> int:
        return self.pairs.numel() // 2

    @property
    def nbytes(self) -> int:
        return self.pairs.numel() * 4


@dataclass
class WindowResult:
    index: int
    n_pairs: int
    records: np.ndarray = None
    n_found: int = 0
    t_ready: float = float("nan")


class ServingTimeout(TimeoutError):
    """A device wait of the server passed its bound; the work is still in
    flight and the server cannot be reused (``close`` waits for the device)."""


class _Budget:
    """Admission by a fixed budget: bytes of admitted requests whose scan has
    not completed yet (their pinned host memory is still read by the GPU)."""

    def __init__(self, budget_bytes: int):
        self.budget = int(budget_bytes)
        self.in_use = 0

    def fits(self, nbytes: int) -> bool:
        if nbytes > self.budget:
            raise ValueError(f"a {nbytes}-byte request exceeds the {self.budget}-byte budget")
        return self.in_use + nbytes <= self.budget

    def take(self, nbytes: int):
        self.in_use += nbytes

    def give(self, nbytes: int):
        self.in_use -= nbytes


class GpuOps:
    """The server's device side: one library context holding routers
    0 .. n_routers - 1 plus the global router n_routers, on one compute
    stream.  The batched engine scans a step's requests where they lie
    (pinned host or device memory); the plain path copies each request
    through the library's staging buffers (sp_update_host)."""

    def __init__(self, n_routers: int, params: dict | None, window_slices: int, batched: bool, report_cap: int):
        from . import sp
        self.sp = sp
        self.n_routers = n_routers
        self.gs = n_routers                                  # the global server's router slot
        kw = dict(params or {})
        kw.update(n_routers=n_routers + 1, window_slices=window_slices)
        self.compute = torch.cuda.Stream()
        self.ctx = sp.SuperPoint(sp.make_params(**kw), stream=self.compute)
        self.window_slices = window_slices
        self.batched = batched
        self.report_cap = report_cap
        # nothing in the serving loop allocates: the library's lazy buffers
        # (staging, batch tables, bin lists, planes) and a few pinned result
        # buffers are made here (a pinned or device allocation can stall the
        # host for milliseconds)
        sp.sp_reserve(self.ctx.ctx, 0, n_routers)
        self.result_bufs = [self._result_buf() for _ in range(4)]

    def close(self):
        self.ctx.close()

    def _result_buf(self):
        out_t = torch.empty(self.report_cap * self.sp.CANDIDATE.itemsize, dtype=torch.uint8).pin_memory()
        return out_t, torch.zeros(2, dtype=torch.int32).pin_memory()

    def synchronize(self):
        torch.cuda.synchronize()

    def issue_step(self, step: list):
        """Scans the step's requests: one batched call that reads every
        request in place (batched engine), or one copy + one launch per
        request (plain path).  Returns the event that completes with the
        step's scan; the requests' memory must stay valid until then."""
        sp, c = self.sp, self.ctx.ctx
        with torch.cuda.stream(self.compute):
            if self.batched:
                for r in step:
                    if not (r.pairs.is_cuda or r.pairs.is_pinned()):
                        raise ValueError("the batched engine reads requests in place: give pinned host tensors "
                                         "(Tensor.pin_memory) or CUDA tensors")
                sp.sp_update_batched(c, [r.router for r in step], [r.pairs for r in step])
            else:
                for r in step:
                    sp.sp_update_host(c, r.router, r.pairs)
        ev = torch.cuda.Event()
        ev.record(self.compute)
        return ev

    def close_window(self):
        """Window end: OR-merge the routers into the global router, detect it
        asynchronously (results copied to pinned host memory), start the next
        window.  Returns (event, handle for read_window)."""
        sp, c = self.sp, self.ctx.ctx
        with torch.cuda.stream(self.compute):
            sp.sp_merge(c, list(range(self.n_routers)), self.gs)
            sp.sp_detect_async(c, self.gs, 0)
            out_t, status = self.result_bufs.pop() if self.result_bufs else self._result_buf()
            sp.sp_results_async(c, out_t, self.report_cap, status)
            if self.window_slices > 1:
                for r in range(self.n_routers + 1):
                    sp.sp_slide(c, r)
            else:
                sp.sp_reset_range(c, 0, self.n_routers + 1)           # every router and the global one, one launch
            ev = torch.cuda.Event()
            ev.record(self.compute)
        return ev, (out_t, status)

    def read_window(self, handle):
        """(super points found, their records) of a completed detection."""
        out_t, status = handle
        cnt, _flags = (int(x) for x in status.numpy().view(np.uint32))
        recs = out_t.numpy().view(self.sp.CANDIDATE)[:min(cnt, self.report_cap)].copy()
        self.result_bufs.append(handle)                       # free for a later window
        return cnt, recs


class SketchServer:
    """Routers 0 .. n_routers-1 plus the global router n_routers, one context.

    batched=True is the continuous-batching engine described above;
    batched=False is the plain path: every request is copied and scanned on
    its own (one sp_update_host per request) as soon as it arrives, with the
    same windows, so both paths produce the same detection results.
    ``ops`` replaces the device side (default: a ``GpuOps`` on the current
    GPU); ``timeout_s`` bounds every device wait.
    """

    def __init__(self, n_routers: int, params: dict | None = None, budget_bytes: int = 1 << 30,
                 detect_every: int = 1 << 24, window_slices: int = 1, max_step_requests: int = 1024,
                 report_cap: int = 4096, batched: bool = True, timeout_s: float = 60.0, ops=None):
        self.n_routers = n_routers
        self.budget = _Budget(budget_bytes)
        self.detect_every = int(detect_every)
        self.max_step = max_step_requests
        self.batched = batched
        self.timeout_s = float(timeout_s)
        self.ops = ops if ops is not None else GpuOps(n_routers, params, window_slices, batched, report_cap)
        self.windows: list[WindowResult] = []
        self.elapsed = float("nan")

    def close(self):
        self.ops.close()

    def run(self, requests: list[Request]):
        """Serves the requests (sorted by arrival); returns self.windows, the
        windows of this call (a server may run several request lists in turn:
        every call ends with its last window closed and the routers reset).
        Raises ServingTimeout when a step's scan or a window's detection has
        not completed timeout_s after it was issued.  Python's cyclic garbage
        collector is paused while the loop runs (a collection can stall the
        host for tens of milliseconds, a latency spike for every request in
        flight)."""
        self.windows = []
        was_enabled = gc.isenabled()
        gc.disable()
        try:
            return self._run(requests)
        finally:
            if was_enabled:
                gc.enable()

    def _run(self, requests: list[Request]):
        ops = self.ops
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        steps = deque()           # (event, issued at, requests, bytes, step index)
        detects = deque()         # (event, issued at, WindowResult, handle, requests)
        window, window_pairs, window_reqs = 0, 0, []
        n_steps = 0
        ops.synchronize()
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        while pending or steps or detects:
            progressed = False
            while steps and steps[0][0].query():                     # scans done: ack, free
                _, _, reqs, nbytes, _ = steps.popleft()
                t = now()
                for r in reqs:
                    r.t_ack = t
                self.budget.give(nbytes)
                progressed = True
            while detects and detects[0][0].query():                 # detections on the host
                _, _, res, handle, reqs = detects.popleft()
                t = now()
                res.n_found, res.records = ops.read_window(handle)
                res.t_ready = t
                for r in reqs:
                    r.t_result = t
                self.windows.append(res)
                progressed = True
            # the stream runs in order: the oldest outstanding wait is the first to pass its bound
            t = now()
            if steps and t - steps[0][1] > self.timeout_s:
                raise ServingTimeout(f"the scan of step {steps[0][4]} ({len(steps[0][2])} requests) has not "
                                     f"completed {self.timeout_s:g} s after it was issued")
            if detects and t - detects[0][1] > self.timeout_s:
                raise ServingTimeout(f"the detection of window {detects[0][2].index} has not completed "
                                     f"{self.timeout_s:g} s after it was issued")
            # admit what has arrived, in order, within the budget and the window
            step = []
            boundary = False
            while pending and pending[0].arrival <= now() and len(step) < self.max_step \
                    and self.budget.fits(pending[0].nbytes):
                r = pending[0]
                pending.popleft()
                self.budget.take(r.nbytes)                            # charged as it is admitted
                r.window = window
                window_pairs += r.n_pairs
                window_reqs.append(r)
                step.append(r)
                if window_pairs >= self.detect_every:
                    boundary = True
                    break
            if not pending and window_reqs and not step and not boundary:
                boundary = True                                       # the last, partial window
            if step:
                ev = ops.issue_step(step)
                steps.append((ev, now(), step, sum(r.nbytes for r in step), n_steps))
                n_steps += 1
                progressed = True
            if boundary:
                ev, handle = ops.close_window()
                detects.append((ev, now(), WindowResult(index=window, n_pairs=window_pairs), handle, window_reqs))
                window, window_pairs, window_reqs = window + 1, 0, []
                progressed = True
            if not progressed:
                if steps or detects:
                    time.sleep(0)                                     # device work in flight: yield, poll again
                elif pending:
                    time.sleep(min(1e-3, max(0.0, pending[0].arrival - now())))   # until the next arrival

        ops.synchronize()
        self.elapsed = now()
        return self.windows


def poisson_requests(seed: int, n_routers: int, n_requests: int, rate_pairs_per_s: float,
                     lo_log2: int = 12, hi_log2: int = 22, streams=None) -> list[Request]:
    """Requests with log-uniform sizes in [2^lo, 2^hi] pairs, routers uniform,
    Poisson arrivals whose mean pair rate is rate_pairs_per_s.  ``streams`` is
    a callable (router, n, seed) -> uint32 pairs array, default uniform."""
    from . import workloads as W
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(2.0 ** lo_log2), np.log(2.0 ** hi_log2), n_requests)).astype(np.int64)
    routers = rng.integers(0, n_routers, n_requests)
    gaps = rng.exponential(sizes.mean() / rate_pairs_per_s, n_requests)
    arrivals = np.cumsum(gaps) - gaps[0]
    out = []
    for i in range(n_requests):
        n = int(sizes[i])
        pairs = (streams(int(routers[i]), n, seed * 100003 + i) if streams is not None
                 else W.uniform_pairs(n, seed=seed * 100003 + i, n_hosts=max(1, n // 4)))
        t = torch.from_numpy(np.ascontiguousarray(pairs, np.uint32).reshape(-1).view(np.int32))
        out.append(Request(router=int(routers[i]), pairs=t.pin_memory() if torch.cuda.is_available() else t,
                           arrival=float(arrivals[i])))
    return out


def latency_summary(requests: list[Request]) -> dict:
    ack = np.array([r.t_ack - r.arrival for r in requests])
    res = np.array([r.t_result - r.arrival for r in requests])
    return {"ack_ms": {"p50": float(np.percentile(ack, 50) * 1e3), "p99": float(np.percentile(ack, 99) * 1e3)},
            "result_ms": {"p50": float(np.percentile(res, 50) * 1e3), "p99": float(np.percentile(res, 99) * 1e3)}}
