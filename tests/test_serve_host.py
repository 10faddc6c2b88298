"""Host logic of the continuous batcher (CPU only): latency percentiles and
summaries, Poisson arrivals, and how a step is formed from the admitted
requests (large requests span steps, small ones share one, FIFO, at most
`step_queries` queries and `max_segments` slices per step)."""

import math
from collections import deque

import numpy as np
import pytest
import torch

serve = pytest.importorskip("paper_2505_08985_gb300.serve")


def test_percentile_matches_linear_interpolation():
    rng = np.random.default_rng(1)
    for n in (1, 2, 7, 100):
        xs = rng.exponential(size=n).tolist()
        for p in (0.0, 0.5, 0.9, 0.99, 1.0):
            assert serve.percentile(xs, p) == pytest.approx(float(np.percentile(xs, 100 * p)), rel=1e-12)
    assert math.isnan(serve.percentile([], 0.5))


def test_summarize():
    reqs = []
    for k, (n, lat) in enumerate(((10, 0.001), (30, 0.003), (60, 0.002))):
        r = serve.Request(rid=k, map=0, queries=torch.zeros(n, 8), arrival=0.0)
        r.latency = lat
        reqs.append(r)
    s = serve.summarize(reqs, 1.0, 3.0)
    assert s["requests"] == 3 and s["queries"] == 100
    assert s["p50_ms"] == pytest.approx(2.0) and s["mean_ms"] == pytest.approx(2.0)
    assert s["queries_per_s"] == pytest.approx(50.0) and s["span_s"] == pytest.approx(2.0)


def test_poisson_arrivals():
    a = serve.poisson_arrivals(20000, rate=500.0, seed=3)
    assert a == serve.poisson_arrivals(20000, rate=500.0, seed=3)
    gaps = np.diff([0.0] + a)
    assert (gaps > 0).all()
    assert gaps.mean() == pytest.approx(1 / 500.0, rel=0.03)
    assert gaps.std() == pytest.approx(1 / 500.0, rel=0.05)  # exponential: std = mean


class _Stream:
    def __init__(self):
        self.waits = 0

    def wait_event(self, ev):
        self.waits += 1


def _batcher(step_queries, max_segments):
    b = serve.ContinuousBatcher.__new__(serve.ContinuousBatcher)  # host logic only: no server
    b.step_queries, b.max_segments, b.step_stream = step_queries, max_segments, _Stream()
    return b


def test_step_formation_slices_fifo():
    sizes = [50, 1000, 30, 30, 400]
    reqs = deque()
    for k, n in enumerate(sizes):
        r = serve.Request(rid=k, map=k % 2, queries=torch.zeros(n, 8), arrival=0.0)
        r.next, r.waited, r.slices = 0, [], []
        reqs.append(r)
    all_reqs = list(reqs)
    b = _batcher(step_queries=256, max_segments=3)
    covered = {k: [] for k in range(len(sizes))}
    shape = []
    streams = [b.step_stream, _Stream()]
    nstep = 0
    while reqs:
        segs, fin = b._form_step(reqs, streams[nstep % 2], object())
        nstep += 1
        shape.append((sum(s[6] for s in segs), len(segs)))
        assert 0 < shape[-1][0] <= 256 and shape[-1][1] <= 3
        for m, q, order, D, flags, first, count in segs:
            rid = next(r.rid for r in [*fin, *reqs] if r.queries is q)
            covered[rid].append((first, count))
    for k, n in enumerate(sizes):  # every query of every request exactly once, in order
        pos = 0
        for first, count in covered[k]:
            assert first == pos and count > 0
            pos += count
        assert pos == n
    # each request's readiness awaited once per step stream that runs a slice of it
    waits = sum(len(r.waited) for r in all_reqs)
    assert streams[0].waits + streams[1].waits == waits and len(sizes) <= waits <= 2 * len(sizes)
    assert all(len(r.slices) == len(covered[r.rid]) for r in all_reqs)  # one completion event per slice
    # a step stops only when full or out of slices (or out of requests)
    assert all(total == 256 or nsegs == 3 for total, nsegs in shape[:-1])
    assert shape == [(256, 2), (256, 1), (256, 1), (256, 1), (86, 3), (256, 1), (144, 1)]


def test_step_formation_keeps_area_and_pndf_budgets():
    """Projected-area requests join steps under their own budget
    (max_area_requests per step) beside the P-NDF queries (step_queries);
    the step ends, FIFO, at the first request it has no room for."""
    AREA = serve.pndf.PNDF_SEGMENT_PROJECTED_AREA
    spec = [(0, 100), (AREA, 3), (0, 300), (AREA, 9), (0, 20)]
    reqs = deque()
    for k, (kind, n) in enumerate(spec):
        r = serve.Request(rid=k, map=0, queries=torch.zeros(n, 8), arrival=0.0, kind=kind,
                          omega=torch.zeros(n, 3) if kind == AREA else None)
        r.next, r.waited, r.slices = 0, [], []
        reqs.append(r)
    all_reqs = list(reqs)
    b = _batcher(step_queries=256, max_segments=8)
    b.area_cap = 4
    steps = []
    while reqs:
        segs, fin = b._form_step(reqs, b.step_stream, object())
        steps.append(segs)
        area = sum(s[6] for s in segs if len(s) > 7)
        pn = sum(s[6] for s in segs if len(s) == 7)
        assert area <= 4 and pn <= 256 and segs
        for s in segs:
            if len(s) > 7:
                assert s[7] == AREA and s[8] is not None and s[2] is None
    covered = {r.rid: sum(s[6] for st in steps for s in st if s[1] is r.queries) for r in all_reqs}
    assert covered == {k: n for k, (_, n) in enumerate(spec)}
    shape = [[(len(s) > 7, s[5], s[6]) for s in st] for st in steps]
    assert shape[0] == [(False, 0, 100), (True, 0, 3), (False, 0, 156)]
    assert shape[1] == [(False, 156, 144), (True, 0, 4)]
    assert shape[2] == [(True, 4, 4)]
    assert shape[3] == [(True, 8, 1), (False, 0, 20)]
