"""Serving: continuous batching over several resident hierarchies.

Each request's densities must be the same alone (pndf_eval_batch on its map)
and in the mix (sliced across steps, sharing steps with other requests and
maps): a query's sum is exact whichever warps evaluate it, so equality is
bitwise.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2505_08985_gb300 import synth
from parity import check_pndf

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_08985_gb300 import pndf
    return pndf


@pytest.fixture(scope="module")
def maps_and_requests(P):
    from paper_2505_08985_gb300 import serve
    sts = [synth.bumps_map(n=256, n_bumps=40, seed=21, device=DEV),
           synth.scratch_map(n=512, n_grooves=120, seed=22, device=DEV),
           synth.flake_normals(1024, 3000, seed=23, device=DEV)]
    rng = np.random.default_rng(5)
    reqs = []
    for k in range(40):
        m = int(rng.integers(0, 3))
        n = int(np.exp(rng.uniform(np.log(50), np.log(30000))))
        q = synth.camera_queries(sts[m].shape[0], n, seed=1000 + k, device=DEV)
        reqs.append(serve.Request(rid=k, map=m, queries=q, arrival=0.0))
    return sts, reqs


def test_served_equals_alone(P, maps_and_requests):
    from paper_2505_08985_gb300 import serve
    sts, reqs = maps_and_requests
    hs = [P.pndf_build_hierarchy(st, bounds_fmt=P.PNDF_BOUNDS_F16_OUTWARD) for st in sts]
    alone = [P.pndf_eval_batch(hs[r.map], r.queries).cpu() for r in reqs]
    b = serve.ContinuousBatcher(hs, step_queries=20000, max_segments=64)
    s = b.run(reqs, realtime=False)
    assert b.steps >= 5  # requests really were sliced across and shared steps
    for r, a in zip(reqs, alone):
        assert torch.equal(r.D.cpu(), a), r.rid
    assert s["requests"] == len(reqs) and s["queries"] == sum(r.n for r in reqs)
    # Poisson arrivals in real time give the same results
    times = serve.poisson_arrivals(len(reqs), rate=2000.0, seed=3)
    for r, t in zip(reqs, times):
        r.arrival = t
    s2 = b.run(reqs, realtime=True)
    for r, a in zip(reqs, alone):
        assert torch.equal(r.D.cpu(), a), r.rid
    assert np.isfinite(s2["p99_ms"]) and s2["p99_ms"] >= s2["p50_ms"] >= 0
    b.close()
    # requests kept in arrival order (no per-request sort) give the same results
    b = serve.ContinuousBatcher(hs, step_queries=20000, max_segments=64, sort=False)
    for r in reqs:
        r.arrival = 0.0
    b.run(reqs, realtime=False)
    for r, a in zip(reqs, alone):
        assert torch.equal(r.D.cpu(), a), r.rid
    b.close()
    # the plain per-batch path agrees too
    sp = serve.run_plain(hs, reqs, realtime=False)
    for r, a in zip(reqs, alone):
        assert torch.equal(r.D.cpu(), a), r.rid
    assert sp["requests"] == len(reqs)
    serve.run_plain(hs, reqs, realtime=False, sort=P.PNDF_SORT_NONE)
    for r, a in zip(reqs, alone):
        assert torch.equal(r.D.cpu(), a), r.rid
    for h in hs:
        h.free()


def test_served_matches_oracle(P, maps_and_requests):
    from paper_2505_08985_gb300 import serve
    sts, reqs = maps_and_requests
    hs = [P.pndf_build_hierarchy(st, bounds_fmt=P.PNDF_BOUNDS_F16_OUTWARD) for st in sts]
    sub = [r for r in reqs if r.n < 3000][:6]
    b = serve.ContinuousBatcher(hs, step_queries=4096)
    b.run(sub, realtime=False)
    b.close()
    for r in sub:
        ref = oracle.pndf(sts[r.map].cpu(), r.queries.cpu())
        check_pndf(r.D.cpu().double().numpy(), ref, label=f"served request {r.rid}")
    for h in hs:
        h.free()


@pytest.mark.parametrize("variant", ["tau", "disk", "box", "clamp"])
def test_served_variant_equals_alone(P, maps_and_requests, variant):
    """A server fixed to the cluster cut, the disk or box kernel or the Eq. 6
    clamp gives, for every request, exactly what pndf_eval_batch_ex gives on
    its map with the same setting."""
    from paper_2505_08985_gb300 import serve
    sts, _ = maps_and_requests
    kw = {"tau": {"tau": 1e-3}, "disk": {"kernel": P.PNDF_KERNEL_DISK}, "box": {"kernel": P.PNDF_KERNEL_BOX},
          "clamp": {"jac_eps": 1e-6}}[variant]
    hs = [P.pndf_build_hierarchy(st, bounds_fmt=P.PNDF_BOUNDS_F16_OUTWARD, clusters=variant == "tau") for st in sts]
    # footprints of 1-24 texels, so that the cut applies (camera footprints are mostly sub-texel)
    rng = np.random.default_rng(11)
    mix = synth.QueryMix(sigma=(1.0, 24.0), aspect=(1.0, 3.0), frac_near=0.8)
    sub = []
    for k in range(16):
        m = int(rng.integers(0, 3))
        n = int(np.exp(rng.uniform(np.log(100), np.log(6000))))
        sub.append(serve.Request(rid=k, map=m, queries=synth.make_queries(sts[m], n, mix, 500 + k), arrival=0.0))
    alone = [P.pndf_eval_batch_ex(hs[r.map], r.queries, **kw).cpu() for r in sub]
    b = serve.ContinuousBatcher(hs, step_queries=20000, max_segments=64, **kw)
    b.run(sub, realtime=False)
    b.close()
    for r, a in zip(sub, alone):
        assert torch.equal(r.D.cpu(), a), (variant, r.rid)
    if variant != "clamp":  # (the clamp only moves hits in triangles of |cross| < 1e-6, rare here)
        exact = [P.pndf_eval_batch(hs[r.map], r.queries).cpu() for r in sub]
        assert any(not torch.equal(a, e) for a, e in zip(alone, exact))  # the variant changes the densities
    for h in hs:
        h.free()


def test_server_variant_validation(P):
    st = synth.bumps_map(n=64, n_bumps=4, seed=1).to(DEV)
    plain = P.pndf_build_hierarchy(st, bounds_fmt=1)
    clustered = P.pndf_build_hierarchy(st, bounds_fmt=1, clusters=True)
    for kw, code in (({"tau": 1e-3}, 6), ({"tau": 1e-3, "kernel": P.PNDF_KERNEL_DISK}, 6), ({"kernel": 7}, 1),
                     ({"tau": -1.0}, 1), ({"jac_eps": 1e-12}, 1), ({"jac_eps": 1e-6, "kernel": P.PNDF_KERNEL_BOX}, 6)):
        maps = [clustered] if "kernel" in kw and "tau" in kw else [plain]
        with pytest.raises(P.PndfError) as ei:
            P.pndf_server_create(maps, **kw)
        assert ei.value.code == code, kw
    with pytest.raises(P.PndfError) as ei:  # the clamp and the cut together
        P.pndf_server_create([clustered], tau=1e-3, jac_eps=1e-6)
    assert ei.value.code == 6
    P.pndf_server_create([clustered], tau=1e-3).destroy()
    plain.free()
    clustered.free()


def test_server_rejects_mixed_formats(P):
    a = P.pndf_build_hierarchy(synth.bumps_map(n=64, n_bumps=4, seed=1).to(DEV), bounds_fmt=0)
    b = P.pndf_build_hierarchy(synth.bumps_map(n=64, n_bumps=4, seed=2).to(DEV), bounds_fmt=1)
    with pytest.raises(P.PndfError):
        P.pndf_server_create([a, b])
    srv = P.pndf_server_create([a], max_segments=4)
    q = synth.camera_queries(64, 10, seed=1, device=DEV)
    D = torch.empty(10, device=DEV)
    with pytest.raises(P.PndfError):  # map index out of range
        P.pndf_server_step(srv, [(1, q, None, D, None, 0, 10)])
    P.pndf_server_step(srv, [(0, q, None, D, None, 0, 10)])
    P.pndf_server_sync(srv)
    assert torch.equal(D, P.pndf_eval_batch(a, q))
    srv.destroy()
    a.free()
    b.free()


def test_autotune_picks_from_its_table(P, maps_and_requests):
    """The autotuner tries every candidate (step size, warps, sort or arrival
    order); among those within 0.97 of the best saturated throughput and
    within 1.05 of their lowest p99 at the offered load it returns the one
    with the highest saturated throughput."""
    from paper_2505_08985_gb300 import serve
    sts, reqs = maps_and_requests
    hs = [P.pndf_build_hierarchy(st, bounds_fmt=P.PNDF_BOUNDS_F16_OUTWARD) for st in sts]
    sample = [serve.Request(rid=r.rid, map=r.map, queries=r.queries, arrival=0.0) for r in reqs[:20]]
    arr = serve.poisson_arrivals(len(sample), rate=4000.0, seed=2)
    t = serve.autotune(hs, sample, arrivals=arr, step_candidates=(1 << 14, 1 << 16), warp_candidates=(8,))
    assert len(t.table) == 4 and {row[3] for row in t.table} == {0, 1}
    cap = max(row[6] for row in t.table)
    ok = [row for row in t.table if row[6] >= 0.97 * cap]
    p99 = min(row[4] for row in ok)
    best = max((row for row in ok if row[4] <= 1.05 * p99), key=lambda row: row[6])
    assert (t.step_queries, t.warps_per_cta, int(t.sort)) == (best[0], best[2], best[3])
    for h in hs:
        h.free()


def test_mixed_steps_with_projected_area_equal_alone(P):
    """Projected-area requests served in the same steps as P-NDF queries (a
    binary16 scratches + flakes map, the glint + diffuse mix): every P equals
    pndf_diffuse_projected_area on the same request alone, and every D equals
    pndf_eval_batch_ex, bit for bit, through the C ABI steps and through the
    continuous batcher."""
    from paper_2505_08985_gb300 import serve
    st = synth.mixed_map(n=512, n_cells=1200, n_grooves=40, seed=5, device=DEV).half()
    h = P.pndf_build_hierarchy(st, bounds_fmt=P.PNDF_BOUNDS_F16_OUTWARD)
    mix = synth.QueryMix(sigma=(1.0, 40.0), frac_near=0.7)
    qp = synth.make_queries(st.float(), 3000, mix, 5)
    qa = synth.make_queries(st.float(), 200, mix, 6)
    w = synth.hemisphere_dirs(200, seed=7, device=DEV)
    ref_D = P.pndf_eval_batch_ex(h, qp)
    ref_P = P.pndf_diffuse_projected_area(h, qa, w)
    A = P.PNDF_SEGMENT_PROJECTED_AREA
    srv = P.pndf_server_create([h], max_area_requests=128)
    D = torch.full((3000,), float("nan"), device=DEV)
    Pv = torch.full((200,), float("nan"), device=DEV)
    P.pndf_server_step(srv, [(0, qp, None, D, None, 0, 2000), (0, qa, None, Pv, None, 0, 128, A, w)])
    P.pndf_server_step(srv, [(0, qa, None, Pv, None, 128, 72, A, w), (0, qp, None, D, None, 2000, 1000)])
    P.pndf_server_sync(srv)
    assert torch.equal(D, ref_D) and torch.equal(Pv, ref_P)
    with pytest.raises(P.PndfError) as ei:  # more area requests than a step holds
        P.pndf_server_step(srv, [(0, qa, None, Pv, None, 0, 129, A, w)])
    assert ei.value.code == 5
    srv.destroy()
    plain = P.pndf_server_create([h])
    with pytest.raises(P.PndfError) as ei:  # a server created without area capacity
        P.pndf_server_step(plain, [(0, qa, None, Pv, None, 0, 10, A, w)])
    assert ei.value.code == 6
    plain.destroy()
    # through the batcher: a stream alternating P-NDF batches and area batches
    reqs = []
    for k in range(12):
        if k % 2:
            lo = 20 * (k // 2)
            reqs.append(serve.Request(rid=k, map=0, queries=qa[lo:lo + 20].contiguous(), arrival=0.0,
                                      kind=A, omega=w[lo:lo + 20].contiguous()))
        else:
            lo = 500 * (k // 2)
            reqs.append(serve.Request(rid=k, map=0, queries=qp[lo:lo + 500].contiguous(), arrival=0.0))
    b = serve.ContinuousBatcher([h], step_queries=700, max_area_requests=16)
    b.run(reqs, realtime=False)
    for r in reqs:
        lo = (20 if r.kind == A else 500) * (r.rid // 2)
        want = ref_P[lo:lo + 20] if r.kind == A else ref_D[lo:lo + 500]
        assert torch.equal(r.D, want), r.rid
    b.close()
    h.free()


def test_served_large_footprints_divided_same_bits(P):
    """Steps holding a few footprints much larger than the step's average
    share per warp divide them into tiles evaluated by several warps (as
    pndf_eval_batch does); each result equals one warp per query to the bit."""
    from paper_2505_08985_gb300 import serve
    st = synth.flake_normals(2048, 12000, seed=31, device=DEV)
    h = P.pndf_build_hierarchy(st, bounds_fmt=P.PNDF_BOUNDS_F16_OUTWARD)
    reqs = []
    for k in range(12):
        sig = (60.0, 250.0) if k % 3 == 0 else (1.0, 8.0)
        q = synth.make_queries(st, 40 if k % 3 == 0 else 400, synth.QueryMix(sigma=sig, frac_near=0.9), 300 + k)
        reqs.append(serve.Request(rid=k, map=0, queries=q.to(DEV), arrival=0.0))
    whole = [P.pndf_eval_batch_ex(h, r.queries, split=False).cpu() for r in reqs]
    b = serve.ContinuousBatcher([h], step_queries=1000, max_segments=16)
    b.run(reqs, realtime=False)
    assert b.steps >= 3
    for r, a in zip(reqs, whole):
        assert torch.equal(r.D.cpu(), a), r.rid
    b.close()
    assert P.pndf_last_device_status(h) == 0
    h.free()
