"""Continuous-batching P-NDF serving over several resident hierarchies.

Requests (a batch of P-NDF queries, or of projected-area requests, on one
map) arrive over time.  The batcher admits arrived requests while their
working buffers (evaluation order and results, 8 bytes per query) fit a
device-memory budget and the admitted work not yet in a step stays under
what the in-flight steps can take (so a burst does not hold the GPU idle
while it is admitted), optionally sorts each once on a copy stream (queries
that arrive in a coherent order, such as a camera's pixels, run faster as
they come; the autotuner decides), and runs steps: each step takes up to
`step_queries` P-NDF queries and `max_area_requests` projected-area requests
from the admitted requests in arrival order (a large request spans several
steps; small ones share a step) and evaluates them in one graph-replayed step
(pndf_server_step).  Steps alternate over two streams and up to slots - 1 are
in flight, so requests that arrive while the GPU works join the next step.

A request's latency runs from its arrival to the device completion of the step
that holds its last queries, on one clock: the device timeline anchored by an
event recorded when the run starts.

The plain baseline launches each batch alone with pndf_eval_batch (or
pndf_diffuse_projected_area) in arrival order: no graphs, no sharing of
launches, with the library's default query sort or none.
"""

from __future__ import annotations

import gc
import math
import statistics
import time
from collections import deque
from dataclasses import dataclass, field

import torch

from . import pndf

BYTES_PER_QUERY = 8  # order (4) + result (4) held while a request is admitted


@dataclass
class Request:
    rid: int
    map: int
    queries: torch.Tensor            # (n, 8) float32 on the serving device, owned by the client
    arrival: float                   # seconds from the run's time origin
    kind: int = 0                    # pndf.PNDF_SEGMENT_PNDF, or _PROJECTED_AREA (then D receives P)
    omega: torch.Tensor | None = None  # projected area: (n, 3) float32 unit directions
    D: torch.Tensor | None = None    # results, filled by the run
    order: torch.Tensor | None = None
    ready: torch.cuda.Event | None = None
    next: int = 0
    waited: list = field(default_factory=list)   # step streams that waited for its sort
    slices: list = field(default_factory=list)   # completion events of the steps holding its slices
    done: torch.cuda.Event | None = None
    latency: float = math.nan

    @property
    def n(self) -> int:
        return int(self.queries.shape[0])


def percentile(xs, p):
    xs = sorted(xs)
    if not xs:
        return math.nan
    k = (len(xs) - 1) * p
    lo, hi = math.floor(k), math.ceil(k)
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


def summarize(reqs, t_first, t_last):
    lat = [r.latency for r in reqs]
    nq = sum(r.n for r in reqs)
    span = max(t_last - t_first, 1e-9)
    return {"requests": len(reqs), "queries": nq, "p50_ms": 1e3 * percentile(lat, 0.5),
            "p99_ms": 1e3 * percentile(lat, 0.99), "mean_ms": 1e3 * statistics.fmean(lat),
            "queries_per_s": nq / span, "span_s": span}


class ContinuousBatcher:
    """Continuous batching over `maps` (same texel and bounds formats)."""

    _queued = 0  # queries admitted and not yet in a step (reset per run)

    def __init__(self, maps, step_queries: int = 1 << 20, memory_budget: int = 2 << 30, max_segments: int = 1024,
                 warps_per_cta: int = 0, ctas_per_sm: int = 0, slots: int = 4, sort: bool = True,
                 kernel: int = pndf.PNDF_KERNEL_GAUSS, tau: float = 0.0, jac_eps: float = 0.0, streams: int = 2,
                 max_area_requests: int = 0):
        """kernel / tau / jac_eps: what every query evaluates (the footprint
        kernel, the cluster cut, the Eq. 6 clamp), as in pndf_eval_batch_ex.
        streams: steps alternate over this many streams, so that a step's
        persistent kernel can start on the SMs the previous step's last
        queries leave idle (its tail).  max_area_requests: projected-area
        requests a step can hold beside its P-NDF queries (0: none)."""
        self.maps = list(maps)
        self.sort = bool(sort)
        self.device = self.maps[0].device
        self.step_queries = int(step_queries)
        self.budget = int(memory_budget)
        self.area_cap = int(max_area_requests)
        self.server = pndf.pndf_server_create(self.maps, max_segments=max_segments, warps_per_cta=warps_per_cta,
                                              ctas_per_sm=ctas_per_sm, slots=slots, kernel=kernel, tau=tau,
                                              jac_eps=jac_eps, max_area_requests=self.area_cap)
        self.max_inflight = max(1, slots - 1)
        self.max_segments = max_segments
        self.copy_stream = torch.cuda.Stream(self.device)
        self.step_streams = [torch.cuda.Stream(self.device) for _ in range(max(1, int(streams)))]
        self.step_stream = self.step_streams[0]
        self.steps = 0

    def close(self):
        self.server.destroy()

    def _admit(self, r: Request):
        with torch.cuda.stream(self.copy_stream):
            sort = self.sort and r.kind == pndf.PNDF_SEGMENT_PNDF
            r.order = pndf.pndf_sort_queries(self.maps[r.map], r.queries, stream=self.copy_stream) if sort else None
            r.D = torch.empty(r.n, dtype=torch.float32, device=self.device)
            r.ready = torch.cuda.Event()
            r.ready.record(self.copy_stream)
        r.queries.record_stream(self.copy_stream)
        for st in self.step_streams:
            if r.order is not None:
                r.order.record_stream(st)
            if r.omega is not None:
                r.omega.record_stream(st)
            r.D.record_stream(st)
            r.queries.record_stream(st)

    def _form_step(self, active: deque, stream, ev):
        """Up to step_queries queries from the admitted requests in arrival
        order, for a step on `stream` completing with event `ev`; returns the
        segments and the requests whose last slice is in it."""
        segs, finishing = [], []
        total = area = 0
        while active and len(segs) < self.max_segments:
            r = active[0]
            is_area = r.kind == pndf.PNDF_SEGMENT_PROJECTED_AREA
            room = self.area_cap - area if is_area else self.step_queries - total
            if room <= 0:  # FIFO: the step ends at the first request it has no room for
                break
            if stream not in r.waited:
                stream.wait_event(r.ready)
                r.waited.append(stream)
            take = min(r.n - r.next, room)
            self._queued -= take
            seg = (r.map, r.queries, r.order, r.D, None, r.next, take)
            segs.append(seg + (r.kind, r.omega) if is_area else seg)
            r.slices.append(ev)
            r.next += take
            if is_area:
                area += take
            else:
                total += take
            if r.next == r.n:
                finishing.append(active.popleft())
        return segs, finishing

    def run(self, requests, realtime: bool = True):
        """Serve `requests` (arrival times relative to the start of the run;
        with realtime=False every request is present at time 0).  Returns the
        summary dict; each request gets `latency`, `D` and `done`."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        for r in reqs:
            r.next, r.waited, r.done, r.latency, r.slices = 0, [], None, math.nan, []
        self._queued = 0
        torch.cuda.synchronize(self.device)
        t0_ev = torch.cuda.Event(enable_timing=True)
        t0_ev.record(self.step_stream)
        t0_ev.synchronize()
        gc_was = gc.isenabled()
        gc.disable()  # no collector pauses inside the host's step loop
        t0 = time.perf_counter()
        pending = deque(reqs)
        active: deque = deque()
        inflight: deque = deque()
        waiting: list = []
        used = 0
        submit_s = wait_s = 0.0  # host time forming and launching steps / blocked on the device
        # admit only what the steps that can be in flight will take, so the
        # first steps start while later requests are still being admitted
        ahead = (self.max_inflight + 1) * self.step_queries
        while pending or active or inflight or waiting:
            now = time.perf_counter() - t0
            progressed = False
            while pending and (not realtime or pending[0].arrival <= now) and self._queued < ahead and \
                    (used + pending[0].n * BYTES_PER_QUERY <= self.budget or (not active and not inflight)):
                r = pending.popleft()
                self._admit(r)
                active.append(r)
                used += r.n * BYTES_PER_QUERY
                self._queued += r.n
                progressed = True
            if active and len(inflight) < self.max_inflight:
                ts = time.perf_counter()
                stream = self.step_streams[self.steps % len(self.step_streams)]
                ev = torch.cuda.Event(enable_timing=True)
                segs, fin = self._form_step(active, stream, ev)
                pndf.pndf_server_step(self.server, segs, stream=stream, ev_done=ev)
                self.steps += 1
                inflight.append((ev, fin, segs))
                submit_s += time.perf_counter() - ts
                continue
            while inflight and inflight[0][0].query():
                _, fin, _ = inflight.popleft()
                waiting.extend(fin)
                progressed = True
            # a request is finished when every step holding one of its slices
            # is (its slices may have run on different streams)
            if waiting:
                still = []
                for r in waiting:
                    if all(e.query() for e in r.slices):
                        r.done = r.slices[-1]
                        used -= r.n * BYTES_PER_QUERY
                        progressed = True
                    else:
                        still.append(r)
                waiting = still
            if progressed:
                continue
            if inflight and (not pending or not realtime or pending[0].arrival > now + 2e-4 or
                             used + pending[0].n * BYTES_PER_QUERY > self.budget):
                tw = time.perf_counter()
                inflight[0][0].synchronize()
                wait_s += time.perf_counter() - tw
            elif waiting and not inflight:
                tw = time.perf_counter()
                waiting[0].slices[0].synchronize()
                wait_s += time.perf_counter() - tw
            elif pending and realtime:
                time.sleep(max(0.0, min(pending[0].arrival - (time.perf_counter() - t0), 5e-4)))
        torch.cuda.synchronize(self.device)
        if gc_was:
            gc.enable()
        for r in reqs:
            # a request is done when the last of its slices' steps completes
            r.latency = max(t0_ev.elapsed_time(e) for e in r.slices) / 1e3 - r.arrival
        t_last = max(r.latency + r.arrival for r in reqs)
        out = summarize(reqs, min(r.arrival for r in reqs), t_last)
        wall = time.perf_counter() - t0
        out["host"] = {"submit_s": submit_s, "blocked_on_device_s": wait_s, "wall_s": wall}
        return out


def run_plain(maps, requests, realtime: bool = True, sort: int = pndf.PNDF_SORT_DEFAULT):
    """Baseline: each batch launched alone (pndf_eval_batch, or
    pndf_diffuse_projected_area for projected-area requests) in arrival
    order; sort = the query order within a P-NDF batch (the library default
    unless given)."""
    reqs = sorted(requests, key=lambda r: r.arrival)
    dev = maps[0].device
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize(dev)
    t0_ev = torch.cuda.Event(enable_timing=True)
    t0_ev.record(stream)
    t0_ev.synchronize()
    t0 = time.perf_counter()
    for r in reqs:
        if realtime:
            wait = r.arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        with torch.cuda.stream(stream):
            r.D = torch.empty(r.n, dtype=torch.float32, device=dev)
            if r.kind == pndf.PNDF_SEGMENT_PROJECTED_AREA:
                pndf.pndf_diffuse_projected_area(maps[r.map], r.queries, r.omega, out=r.D, stream=stream)
            else:
                pndf.pndf_eval_batch_ex(maps[r.map], r.queries, out=r.D, sort=sort, stream=stream)
            r.done = torch.cuda.Event(enable_timing=True)
            r.done.record(stream)
    torch.cuda.synchronize(dev)
    for r in reqs:
        r.latency = t0_ev.elapsed_time(r.done) / 1e3 - r.arrival
    t_last = max(t0_ev.elapsed_time(r.done) / 1e3 for r in reqs)
    return summarize(reqs, min(r.arrival for r in reqs), t_last)


def poisson_arrivals(n: int, rate: float, seed: int):
    g = torch.Generator().manual_seed(seed)
    gaps = -torch.log(1.0 - torch.rand(n, generator=g, dtype=torch.float64)) / rate
    return torch.cumsum(gaps, 0).tolist()


@dataclass
class TuneResult:
    step_queries: int
    ctas_per_sm: int
    warps_per_cta: int
    p99_ms: float
    queries_per_s: float
    sort: bool = True
    table: list = field(default_factory=list)


def autotune(maps, sample, arrivals=None, step_candidates=(1 << 16, 1 << 18, 1 << 20, 1 << 22),
             cta_candidates=(0,), warp_candidates=(8, 4), sort_candidates=(True, False), streams: int = 2,
             capacity_margin: float = 0.97, p99_margin: float = 1.05, capacity_sample=None):
    """Pick step size, launch shape and whether to sort each request for the
    served path on a sample of requests.  Every candidate's saturated
    throughput is measured; with `arrivals` (a Poisson stream at the target
    load) the candidates within `capacity_margin` of the best saturated
    throughput qualify (a latency gain is not bought with capacity), and among
    those whose p99 is within `p99_margin` of the lowest (differences below
    that are run-to-run noise) the highest saturated throughput wins;
    without, the highest saturated throughput wins.  The saturated throughput
    is measured on `capacity_sample` when given (a longer run ranks step
    sizes more reliably than the latency sample)."""
    runs = []
    table = []
    for sort in sort_candidates:
        for ctas in cta_candidates:
            for warps in warp_candidates:
                for step in step_candidates:
                    b = ContinuousBatcher(maps, step_queries=step, warps_per_cta=warps, ctas_per_sm=ctas, sort=sort,
                                          streams=streams)
                    for r in sample:
                        r.arrival = 0.0
                    b.run(sample, realtime=False)  # warm
                    cap = b.run(capacity_sample or sample, realtime=False)["queries_per_s"]
                    s = None
                    if arrivals is not None:
                        for r, a in zip(sample, arrivals):
                            r.arrival = a
                        s = b.run(sample, realtime=True)
                    b.close()
                    p99 = s["p99_ms"] if s else math.nan
                    qps = s["queries_per_s"] if s else cap
                    table.append((step, ctas, warps, int(sort), p99, qps, cap))
                    runs.append((TuneResult(step, ctas, warps, p99, qps, sort), cap))
    for r in sample:
        r.arrival = 0.0
    best_cap = max(c for _, c in runs)
    if arrivals is not None:
        ok = [(t, c) for t, c in runs if c >= capacity_margin * best_cap]
        p99 = min(t.p99_ms for t, _ in ok)
        out = max((tc for tc in ok if tc[0].p99_ms <= p99_margin * p99), key=lambda tc: tc[1])[0]
    else:
        out = max(runs, key=lambda tc: tc[1])[0]
    out.table = table
    return out
