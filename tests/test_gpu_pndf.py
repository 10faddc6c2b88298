"""GPU parity of the P-NDF path (pndf_build_hierarchy + pndf_eval_batch)
against the FP64 oracle, through the C ABI.

Bar: per-query relative error <= 1e-4 on every query the oracle does not flag
(normal-space edge ties within 1e-6, hits within 1e-4 of the q = 16 cut,
zero-area ties, invalid covariance), exact zeros where the oracle has no
hit, and identical hit counts and hit-set fingerprints.
"""

import math

import numpy as np
import pytest
import torch

import oracle
from paper_2505_08985_gb300 import synth
from parity import RTOL, check_pndf, rel_err

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_08985_gb300 import pndf
    return pndf


def run(P, st, q, bounds=0, mode=0, sort=1, warps=0, stats=True):
    h = P.pndf_build_hierarchy(st.to(DEV), bounds_fmt=bounds)
    qd = q.to(DEV)
    flags = torch.zeros(q.shape[0], dtype=torch.int32, device=DEV)
    stt = torch.zeros(q.shape[0], P.STATS_FIELDS, dtype=torch.int32, device=DEV) if stats else None
    D = P.pndf_eval_batch_ex(h, qd, flags=flags, stats=stt, mode=mode, sort=sort, warps_per_cta=warps)
    torch.cuda.synchronize()
    out = (D.cpu().double().numpy(), flags.cpu().numpy().astype(np.uint32),
           None if stt is None else stt.cpu().numpy().astype(np.int64))
    h.free()
    return out


def test_bumps256_4096_queries(P):
    """The small plain-method workload: 256^2 bumps map, 4096 isotropic sigma=4 queries."""
    cfg = synth.BUMPS_256
    st = synth.bumps_map(n=cfg["n"], seed=cfg["seed"])
    q = synth.make_queries(st, cfg["queries"], cfg["mix"], cfg["seed"])
    ref = oracle.pndf(st, q)
    D, fl, stt = run(P, st, q)
    s = check_pndf(D, ref, hits_gpu=stt[:, 3], hash_gpu=stt[:, 4], label="bumps256")
    assert s["nonzero"] > 0.8 * s["compared"]
    assert s["excluded"] < 0.05 * q.shape[0]
    assert P.pndf_device_status() == 0


def test_stats_match_host_count(P):
    """Stats mode counts what it claims (the work figures behind the roofline):
    in flat mode each query's leaf blocks and triangle tests equal a host count
    of the 4 x 4-quad blocks whose closed extent meets the support's bounding
    box and of the triangles inside the map in them; queries whose box edge
    lies within 1e-3 texel of a block boundary are skipped (FP32 vs FP64
    rounding), and there must be few."""
    cfg = synth.BUMPS_256
    st = synth.bumps_map(n=cfg["n"], seed=cfg["seed"])
    mix = synth.QueryMix(sigma=(0.5, 20.0), aspect=(1.0, 3.0), frac_near=0.8, centre_margin=-10.0)
    q = synth.make_queries(st, 4096, mix, cfg["seed"])
    _, _, s = run(P, st, q, mode=1)
    n = st.shape[0]
    S = 1 << (P.top_level(n) - 2)
    qd = q.double().numpy()
    det = qd[:, 2] * qd[:, 4] - qd[:, 3] ** 2
    assert (det > 0).all()
    rx = 4.0 * np.sqrt(qd[:, 2]) * (1 + 1e-5) + 1e-6
    ry = 4.0 * np.sqrt(qd[:, 4]) * (1 + 1e-5) + 1e-6
    blocks = np.zeros(len(qd), np.int64)
    tris = np.zeros(len(qd), np.int64)
    ambiguous = np.zeros(len(qd), bool)
    quads_in = np.clip(n - 1 - 4 * np.arange(S), 0, 4)  # quads of block column (row) a inside the map
    for k in range(len(qd)):
        lo_hi = []
        for c, r in ((qd[k, 0], rx[k]), (qd[k, 1], ry[k])):
            e0, e1 = (c - r) / 4.0, (c + r) / 4.0
            ambiguous[k] |= min(abs(e0 - round(e0)), abs(e1 - round(e1))) < 2.5e-4
            lo_hi.append((max(math.ceil(e0) - 1, 0), min(math.floor(e1), S - 1)))
        (a0, a1), (c0, c1) = lo_hi
        if a0 <= a1 and c0 <= c1:
            blocks[k] = (a1 - a0 + 1) * (c1 - c0 + 1)
            tris[k] = 2 * quads_in[a0:a1 + 1].sum() * quads_in[c0:c1 + 1].sum()
    ok = ~ambiguous
    assert ambiguous.sum() < 0.01 * len(qd)
    assert np.array_equal(s[ok, 1], blocks[ok])
    assert np.array_equal(s[ok, 2], tris[ok])
    assert (tris[ok] > 0).mean() > 0.9


def test_hierarchy_prunes_only(P):
    """Pyramid traversal and flat evaluation test exactly the same contributing
    triangles (every query, ties included: both use the same leaf predicate)."""
    st = synth.bumps_map(n=200, n_bumps=40, seed=7)
    q = synth.make_queries(st, 3000, synth.QueryMix(sigma=(0.7, 12.0), aspect=(1.0, 4.0), frac_near=0.8), 7)
    Dh, _, sh = run(P, st, q, mode=0)
    Df, _, sf = run(P, st, q, mode=1)
    assert np.array_equal(sh[:, 3], sf[:, 3]) and np.array_equal(sh[:, 4], sf[:, 4])
    assert rel_err(Dh, Df).max() <= 1e-5  # same hits, different summation order
    # and pruning is real: far fewer triangle tests than the flat scan
    assert sh[:, 2].sum() < 0.5 * sf[:, 2].sum()


@pytest.mark.parametrize("bounds", [0, 1])
def test_quad_capsules_prune_only(P, bounds):
    """The per-quad capsule (segment between the quad's farthest normals plus
    a radius) only prunes: with query normals placed exactly on texel normals,
    on midpoints of quad edges and diagonals, and on the farthest points of
    the triangles (the cases where a capsule rounded too tightly would drop a
    hit), the pyramid traversal hits exactly the triangles the flat scan hits.
    Flake cells (long slivers across cell borders), bumps and scratches."""
    rng = np.random.default_rng(31)
    maps = [synth.flake_normals(256, 700, seed=31), synth.bumps_map(n=192, n_bumps=30, seed=32),
            synth.scratch_map(n=192, n_grooves=60, seed=33)]
    for st in maps:
        n = st.shape[0]
        nq = 3000
        i = rng.integers(0, n - 1, nq)
        j = rng.integers(0, n - 1, nq)
        stn = st.double().numpy()
        v = [stn[j, i], stn[j, i + 1], stn[j + 1, i], stn[j + 1, i + 1]]
        kind = rng.integers(0, 4, nq)
        a, b = rng.integers(0, 4, nq), rng.integers(0, 4, nq)
        pa = np.stack(v, 0)[a, np.arange(nq)]
        pb = np.stack(v, 0)[b, np.arange(nq)]
        m = np.where((kind == 0)[:, None], pa, 0.5 * (pa + pb))  # a vertex or a midpoint of two
        m = np.where((kind == 3)[:, None], pa + 1e-7 * rng.normal(size=(nq, 2)), m)
        m = m.astype(np.float32).astype(np.float64)
        x = i + rng.uniform(-2, 3, nq)
        y = j + rng.uniform(-2, 3, nq)
        sg = rng.uniform(0.8, 6.0, nq)
        q = torch.from_numpy(np.stack([x, y, sg * sg, np.zeros(nq), sg * sg, m[:, 0], m[:, 1], np.zeros(nq)],
                                      1).astype(np.float32))
        Dh, _, sh = run(P, st, q, mode=0, bounds=bounds)
        Df, _, sf = run(P, st, q, mode=1, bounds=bounds)
        assert (sf[:, 3] > 0).mean() > 0.5
        assert np.array_equal(sh[:, 3], sf[:, 3]) and np.array_equal(sh[:, 4], sf[:, 4])
        assert rel_err(Dh, Df).max() <= 1e-5


def test_fp16_outward_bounds_keep_hit_sets(P):
    """FP16 bounds rounded outward only prune less: hit sets are identical to
    FP32 bounds and D agrees to summation-order rounding."""
    st = synth.scratch_map(n=512, n_grooves=120, seed=3)
    q = synth.make_queries(st, 4000, synth.QueryMix(sigma=(1.0, 32.0), aspect=(1.0, 4.0), frac_near=0.7), 3)
    D32, _, s32 = run(P, st, q, bounds=0)
    D16, _, s16 = run(P, st, q, bounds=1)
    assert np.array_equal(s32[:, 3], s16[:, 3]) and np.array_equal(s32[:, 4], s16[:, 4])
    assert rel_err(D16, D32).max() <= 1e-5
    assert s16[:, 0].sum() >= s32[:, 0].sum()  # looser boxes visit at least as many nodes
    ref = oracle.pndf(st, q)
    check_pndf(D16, ref, hits_gpu=s16[:, 3], hash_gpu=s16[:, 4], label="scratch512 fp16 bounds")


@pytest.mark.parametrize("n", [256, 203, 129])
def test_fp16_texels(P, n):
    """A binary16-stored map: the map is its FP16 values (decoded exactly by
    the oracle).  256: 16-byte vector loads; 203: rows not a multiple of four
    texels (scalar loads); 129: the map's last column is a tile's shared edge.
    The tile build also writes the hierarchy's own copy of the texels, which
    every leaf test reads."""
    st = synth.flake_normals(n, 300 * n * n // 65536 + 20, seed=4).half()
    mix = synth.QueryMix(sigma=(1.0, 20.0), frac_near=0.7, centre_margin=-4)
    q = synth.make_queries(st.float(), 2000, mix, 4)
    ref = oracle.pndf(st.float(), q)
    for bounds in (0, 1):
        D, _, stt = run(P, st, q, bounds=bounds)
        check_pndf(D, ref, hits_gpu=stt[:, 3], hash_gpu=stt[:, 4], label=f"fp16 texels n={n} bounds={bounds}")


@pytest.mark.parametrize("n", [2, 3, 5, 6, 37, 100, 129, 257])
def test_ragged_map_sizes(P, n):
    """Maps whose quad count is not a power of two (padded pyramid, partial
    tiles, odd rows that disable vector loads), footprints crossing or outside
    the border."""
    st = synth.bumps_map(n=n, n_bumps=max(1, n // 8), seed=n)
    mix = synth.QueryMix(sigma=(0.5, max(1.0, n / 4)), aspect=(1.0, 3.0), frac_near=0.8,
                         centre_margin=-0.2 * n - 2)
    q = synth.make_queries(st, 600, mix, n)
    ref = oracle.pndf(st, q)
    D, _, stt = run(P, st, q)
    check_pndf(D, ref, hits_gpu=stt[:, 3], hash_gpu=stt[:, 4], label=f"n={n}")


def test_affine_field_closed_form(P):
    """Affine normal field: D = k_r(M^-1 (m - n0) - x) / |det M| (Eq. 2),
    independent of the oracle."""
    n0 = (-0.2001953125, -0.150390625)
    M = np.array(((44 / 4096, 8 / 4096), (-12 / 4096, 40 / 4096)))
    N = 32
    st = synth.affine_normals(N, n0, M)
    rng = np.random.default_rng(11)
    nq = 2000
    us = rng.uniform(0.01, N - 1.01, (nq, 2))
    m = (np.asarray(n0)[None] + us @ M.T).astype(np.float32).astype(np.float64)
    x = rng.uniform(4, 27, nq)
    y = rng.uniform(4, 27, nq)
    s = rng.uniform(0.8, 3.0, nq)
    q = np.stack([x, y, s * s, np.zeros(nq), s * s, m[:, 0], m[:, 1], np.zeros(nq)], 1).astype(np.float32)
    qt = torch.from_numpy(q)
    D, _, stt = run(P, st, qt)
    q64 = q.astype(np.float64)
    ustar = np.linalg.solve(M[None], (q64[:, 5:7] - np.asarray(n0)[None])[:, :, None])[:, :, 0]
    d = ustar - q64[:, :2]
    qq = (d ** 2).sum(1) / q64[:, 2]
    expect = np.where(qq <= 16, np.exp(-0.5 * qq) / (2 * np.pi * q64[:, 2]) / abs(np.linalg.det(M)), 0.0)
    ref = oracle.pndf(st, qt)
    ok = (ref[1] & oracle.F_EXCLUDE) == 0
    assert ok.mean() > 0.95
    r = rel_err(D[ok], expect[ok])
    assert r.max() <= RTOL, r.max()


def test_near_singular_triangles_take_fp64(P):
    """Normal triangles of area below 1e-10 (the fold / caustic case of Eq. 4,
    where the Jacobian ratio is ill-conditioned) are hit-tested and weighted
    in FP64.  The affine field n(u) = n0 + 2^-17 u (dyadic, exact in binary32)
    makes every triangle a right triangle of legs 2^-17: |cross| = 2^-34, below
    the FP32 cut-off of 2e-10, yet with an inradius (2.2e-6) above the 1e-6
    edge-tie band, so D can be checked against the closed form
    k_r(M^-1 (m - n0) - x) / |det M| (Eq. 2) and against the oracle, and the
    FP64 flag and counter must show on every query that hits."""
    n0 = (-0.125, 0.0625)
    c = 2.0 ** -17
    M = np.array(((c, 0.0), (0.0, c)))
    N = 64
    st = synth.affine_normals(N, n0, M)
    assert np.array_equal(st.double().numpy()[..., 0], n0[0] + c * np.arange(N)[None, :].repeat(N, 0))
    rng = np.random.default_rng(23)
    nq = 1500
    us = rng.uniform(0.05, N - 1.05, (nq, 2))
    m = (np.asarray(n0)[None] + us @ M.T).astype(np.float32).astype(np.float64)
    x = us[:, 0] + rng.uniform(-3, 3, nq)
    y = us[:, 1] + rng.uniform(-3, 3, nq)
    s = rng.uniform(1.0, 4.0, nq)
    q = np.stack([x, y, s * s, np.zeros(nq), s * s, m[:, 0], m[:, 1], np.zeros(nq)], 1).astype(np.float32)
    qt = torch.from_numpy(q)
    for bounds in (P.PNDF_BOUNDS_F32, P.PNDF_BOUNDS_F16_OUTWARD):
        D, fl, stt = run(P, st, qt, bounds=bounds)
        ref = oracle.pndf(st, qt)
        summary = check_pndf(D, ref, hits_gpu=stt[:, 3], hash_gpu=stt[:, 4], label="near-singular affine")
        assert summary["compared"] > 300 and summary["nonzero"] > 200
        hit = stt[:, 3] > 0
        assert hit.sum() > 200
        assert (stt[hit, 5] > 0).all(), "hits on tiny triangles must come from the FP64 branch"
        assert ((fl[hit] & P.PNDF_QF_FP64) != 0).all()
        assert (ref[1][hit] & oracle.F_TINY).all()  # the oracle sees the same tiny-area hits
        # the closed form, away from edge ties
        q64 = q.astype(np.float64)
        ustar = (q64[:, 5:7] - np.asarray(n0)[None]) / c
        d = ustar - q64[:, :2]
        qq = (d ** 2).sum(1) / q64[:, 2]
        expect = np.where(qq <= 16, np.exp(-0.5 * qq) / (2 * np.pi * q64[:, 2]) / (c * c), 0.0)
        ok = (ref[1] & oracle.F_EXCLUDE) == 0
        assert rel_err(D[ok], expect[ok]).max() <= RTOL
    assert P.pndf_device_status() == 0


def test_fold_slivers_take_fp64(P):
    """A fold line: s falls linearly towards column 32 and rises again after
    it, with columns 32 and 33 equal up to a few binary32 ulps, so the
    triangles of quad column 32 have normal-space areas of order 1e-11 (not
    zero).  Queries whose normal lies on that sliver band must be tested in
    FP64 (flag and counter); everything away from edge ties matches the
    oracle."""
    N = 64
    rng = np.random.default_rng(5)
    i = np.arange(N)
    s_col = np.where(i <= 32, 0.25 - 0.002 * (32 - i), 0.25 - 0.002 * (i - 33)).astype(np.float32)
    ulp = np.spacing(np.float32(0.25))
    s_col[33] = np.float32(0.25) + np.float32(2) * ulp
    t_row = (0.001 * np.arange(N) - 0.03).astype(np.float32)
    st = np.zeros((N, N, 2), np.float32)
    st[..., 0] = s_col[None, :] + (rng.integers(-1, 2, (N, N)) * ulp).astype(np.float32) * (i[None, :] >= 32)
    st[..., 1] = t_row[:, None]
    st = torch.from_numpy(st)
    nq = 800
    # normals on the sliver band (s within the fold columns' values) and elsewhere
    ms = np.where(rng.uniform(size=nq) < 0.5, 0.25 + rng.uniform(-4, 6, nq) * ulp, rng.uniform(0.19, 0.25, nq))
    mt = rng.uniform(-0.028, 0.03, nq)
    x = rng.uniform(24, 40, nq)
    y = rng.uniform(4, 59, nq)
    sg = rng.uniform(1.0, 5.0, nq)
    q = torch.from_numpy(np.stack([x, y, sg * sg, np.zeros(nq), sg * sg, ms, mt, np.zeros(nq)], 1).astype(np.float32))
    D, fl, stt = run(P, st, q)
    ref = oracle.pndf(st, q)
    check_pndf(D, ref, hits_gpu=stt[:, 3], hash_gpu=stt[:, 4], label="fold slivers")
    fp64 = stt[:, 5] > 0
    assert fp64.sum() > 50, int(fp64.sum())
    assert ((fl[fp64] & P.PNDF_QF_FP64) != 0).all()
    assert ((fl[~fp64] & P.PNDF_QF_FP64) == 0).all()
    # the tiny-area hits the oracle reports all come from FP64-tested queries
    tiny = (ref[1] & oracle.F_TINY) != 0
    assert tiny.any() and fp64[tiny].all()


def test_large_footprints_deep_traversal(P):
    """Footprints up to sigma = 150 on a 1024^2 flake map (deep descent, many entry nodes)."""
    st = synth.flake_normals(1024, 3000, seed=9)
    q = synth.make_queries(st, 300, synth.QueryMix(sigma=(20.0, 150.0), frac_near=0.8), 9)
    ref = oracle.pndf(st, q)
    D, _, stt = run(P, st, q)
    s = check_pndf(D, ref, hits_gpu=stt[:, 3], hash_gpu=stt[:, 4], label="flake1024 large")
    assert s["nonzero"] > 100


def test_empty_and_single(P):
    st = synth.bumps_map(n=64, n_bumps=4, seed=2)
    h = P.pndf_build_hierarchy(st.to(DEV))
    D = P.pndf_eval_batch(h, torch.zeros(0, 8, dtype=torch.float32, device=DEV))
    assert D.shape == (0,)
    q = synth.make_queries(st, 1, synth.QueryMix(sigma=(3.0, 3.0)), 2)
    D1 = P.pndf_eval_batch(h, q.to(DEV)).cpu().double().numpy()
    check_pndf(D1, oracle.pndf(st, q), label="single")
    h.free()


def test_invalid_queries_flagged(P):
    st = synth.bumps_map(n=64, n_bumps=4, seed=2)
    q = synth.make_queries(st, 8, synth.QueryMix(sigma=(3.0, 3.0)), 2)
    q[1, 2] = -1.0                      # sxx < 0
    q[2, 3] = 100.0                     # not positive definite
    q[3, 0] = float("nan")
    h = P.pndf_build_hierarchy(st.to(DEV))
    flags = torch.zeros(8, dtype=torch.int32, device=DEV)
    D = P.pndf_eval_batch(h, q.to(DEV), flags=flags).cpu().numpy()
    fl = flags.cpu().numpy()
    assert np.all(np.isnan(D[1:4])) and np.all(fl[1:4] & P.PNDF_QF_INVALID)
    assert not np.isnan(D[0]) and not np.isnan(D[4:]).any()
    assert P.pndf_device_status() & P.PNDF_QF_INVALID
    assert P.pndf_device_status() == 0  # cleared by the read
    h.free()


def test_status_word_per_hierarchy(P):
    """Each hierarchy keeps its own status word: an invalid query evaluated on
    one map (P-NDF or projected area) sets that map's word and the device-wide
    one, not another map's; reading a word clears it."""
    st = synth.bumps_map(n=64, n_bumps=4, seed=2)
    a = P.pndf_build_hierarchy(st.to(DEV))
    b = P.pndf_build_hierarchy(st.to(DEV))
    P.pndf_device_status()  # start from a clean device word
    q = synth.make_queries(st, 8, synth.QueryMix(sigma=(3.0, 3.0)), 2).to(DEV)
    bad = q.clone()
    bad[5, 4] = -2.0  # syy < 0
    P.pndf_eval_batch(a, bad)
    P.pndf_eval_batch(b, q)
    assert P.pndf_last_device_status(b) == 0
    assert P.pndf_last_device_status(a) == P.PNDF_QF_INVALID
    assert P.pndf_last_device_status(a) == 0  # cleared by the read
    assert P.pndf_device_status() == P.PNDF_QF_INVALID
    w = torch.tensor([[0.3, 0.2, math.sqrt(1 - 0.13)]], device=DEV).repeat(8, 1)
    P.pndf_diffuse_projected_area(b, bad, w)
    assert P.pndf_last_device_status(a) == 0
    assert P.pndf_last_device_status(b) == P.PNDF_QF_INVALID
    assert P.pndf_device_status() == P.PNDF_QF_INVALID
    assert P.pndf_device_status() == 0
    a.free()
    b.free()


def test_result_independent_of_batch(P):
    """A query's D is bit-identical alone, in a batch, sorted or unsorted and
    with another launch shape: its sum is exact (fixed point), so neither the
    order of its hits nor the warps that find them change it."""
    st = synth.scratch_map(n=256, n_grooves=40, seed=12)
    q = synth.make_queries(st, 2048, synth.QueryMix(sigma=(1.0, 24.0), aspect=(1.0, 4.0), frac_near=0.8), 12)
    D_all, _, _ = run(P, st, q, stats=False)
    D_uns, _, _ = run(P, st, q, sort=0, stats=False)
    D_tile, _, _ = run(P, st, q, sort=2, stats=False)
    D_w4, _, _ = run(P, st, q, warps=4, stats=False)
    D_sub, _, _ = run(P, st, q[100:117], stats=False)
    assert np.array_equal(D_all, D_uns) and np.array_equal(D_all, D_w4) and np.array_equal(D_all, D_tile)
    assert np.array_equal(D_all[100:117], D_sub)


def test_split_large_footprints_same_bits(P):
    """In a small batch, footprints far larger than the batch's average share
    per warp are divided into tiles of pyramid nodes, each descended by its own
    warp.  The result is the same bits as one warp per query (split=False),
    with the same hits, and the oracle agrees; the node counts differ (a tile
    starts its descent below the entry level), which shows the division."""
    st = synth.flake_normals(2048, 12000, seed=21)
    q = synth.make_queries(st, 48, synth.QueryMix(sigma=(60.0, 250.0), frac_near=0.9), 21)
    h = P.pndf_build_hierarchy(st.to(DEV))
    qd = q.to(DEV)
    out = {}
    for split in (True, False):
        fl = torch.zeros(q.shape[0], dtype=torch.int32, device=DEV)
        stt = torch.zeros(q.shape[0], P.STATS_FIELDS, dtype=torch.int32, device=DEV)
        D = P.pndf_eval_batch_ex(h, qd, flags=fl, stats=stt, split=split)
        D2 = P.pndf_eval_batch_ex(h, qd, split=split, sort=0)
        out[split] = (D.cpu(), fl.cpu(), stt.cpu(), D2.cpu())
    Dn = P.pndf_eval_batch_noalloc(h, qd).cpu()  # whole queries only
    torch.cuda.synchronize()
    h.free()
    (Ds, fs, ss, Ds2), (Dw, fw, sw, Dw2) = out[True], out[False]
    assert torch.equal(Ds, Dw) and torch.equal(Ds, Ds2) and torch.equal(Ds, Dw2) and torch.equal(Ds, Dn)
    assert torch.equal(fs, fw)
    cols = [P.STATS_NAMES.index(c) for c in ("leaf_blocks", "tri_tests", "hits", "hit_hash", "quads")]
    assert torch.equal(ss[:, cols], sw[:, cols])
    nodes = P.STATS_NAMES.index("nodes")
    assert (ss[:, nodes] != sw[:, nodes]).sum() >= 10
    ref = oracle.pndf(st, q)
    s = check_pndf(Ds.double().numpy(), ref, hits_gpu=ss[:, 3].numpy(), hash_gpu=ss[:, 4].numpy(),
                   label="split flake2048")
    assert s["nonzero"] > 20


def test_flat_and_hierarchy_same_bits(P):
    """The exact per-query sum makes the flat scan (every leaf block of the
    support, no pruning) and the hierarchy agree to the bit wherever they find
    the same hits (hit count and fingerprint)."""
    st = synth.scratch_map(n=256, n_grooves=40, seed=12)
    q = synth.make_queries(st, 2048, synth.QueryMix(sigma=(1.0, 24.0), aspect=(1.0, 4.0), frac_near=0.8), 13)
    Dh, _, sh = run(P, st, q)
    Df, _, sf = run(P, st, q, mode=P.PNDF_MODE_FLAT)
    same = (sh[:, 3] == sf[:, 3]) & (sh[:, 4] == sf[:, 4])
    assert same.mean() > 0.99 and (Dh[same] > 0).sum() > 500
    assert np.array_equal(Dh[same], Df[same])


def test_host_buffer_entry_point(P):
    st = synth.bumps_map(n=128, n_bumps=16, seed=5)
    q = synth.make_queries(st, 3000, synth.QueryMix(sigma=(1.0, 8.0)), 5)
    h = P.pndf_build_hierarchy(st.to(DEV))
    Dh = P.pndf_eval_batch_host(h, q.pin_memory())
    Dd = P.pndf_eval_batch(h, q.to(DEV)).cpu()
    assert torch.equal(Dh, Dd)
    h.free()


def _sampled(nq_total, k, rng):
    return np.sort(rng.choice(nq_total, size=k, replace=False))


def test_scratch2048_1m_sampled(P):
    """The 2048^2 scratch workload at full size (1M anisotropic queries) in the
    default launch configuration; a sample is checked against the oracle."""
    cfg = synth.SCRATCH_2048
    st = synth.scratch_map(n=cfg["n"], seed=cfg["seed"], device=DEV)
    q = synth.make_queries(st, cfg["queries"], cfg["mix"], cfg["seed"])
    for bounds in (0, 1):
        h = P.pndf_build_hierarchy(st, bounds_fmt=bounds)
        stt = torch.zeros(q.shape[0], P.STATS_FIELDS, dtype=torch.int32, device=DEV)
        D = P.pndf_eval_batch(h, q, stats=stt).cpu().double().numpy()
        stt = stt.cpu().numpy().astype(np.int64)
        h.free()
        idx = _sampled(q.shape[0], 3000, np.random.default_rng(bounds))
        ref = oracle.pndf(st.cpu(), q.cpu()[idx])
        s = check_pndf(D[idx], ref, hits_gpu=stt[idx, 3], hash_gpu=stt[idx, 4], label=f"scratch2048 b={bounds}")
        assert s["nonzero"] > 500
        assert np.isfinite(D).all()


def test_flake8192_4m_sampled(P):
    """The 8192^2 flake workload at full size (4M queries, sigma 1..512), FP32
    and FP16-outward bounds; a sigma-stratified sample checked against the oracle."""
    cfg = synth.FLAKE_8192
    st = synth.flake_map(n=cfg["n"], seed=cfg["seed"], device=DEV)
    q = synth.make_queries(st, cfg["queries"], cfg["mix"], cfg["seed"])
    sig = torch.sqrt(q[:, 2]).cpu().numpy()
    rng = np.random.default_rng(5)
    # stratify: 8 log-sigma bins, 40 queries each (large ones are expensive for the oracle)
    edges = np.exp(np.linspace(0, math.log(512), 9))
    idx = []
    for a, b in zip(edges[:-1], edges[1:]):
        cand = np.flatnonzero((sig >= a) & (sig < b))
        idx.append(rng.choice(cand, size=min(40, cand.size), replace=False))
    idx = np.sort(np.concatenate(idx))
    ref = oracle.pndf(st.cpu(), q.cpu()[idx])
    Ds = {}
    for bounds in (0, 1):
        h = P.pndf_build_hierarchy(st, bounds_fmt=bounds)
        stt = torch.zeros(q.shape[0], P.STATS_FIELDS, dtype=torch.int32, device=DEV)
        D = P.pndf_eval_batch(h, q, stats=stt).cpu().double().numpy()
        stt = stt.cpu().numpy().astype(np.int64)
        h.free()
        check_pndf(D[idx], ref, hits_gpu=stt[idx, 3], hash_gpu=stt[idx, 4], label=f"flake8192 b={bounds}")
        Ds[bounds] = (D, stt)
    assert np.array_equal(Ds[0][1][:, 4], Ds[1][1][:, 4])
    assert rel_err(Ds[1][0], Ds[0][0]).max() <= 1e-5


def test_update_in_place_matches_fresh_build(P):
    st_a = synth.bumps_map(n=96, n_bumps=10, seed=31)
    st_b = synth.flake_normals(96, 40, seed=32)
    q = synth.make_queries(st_b, 1000, synth.QueryMix(sigma=(1.0, 10.0)), 33)
    h = P.pndf_build_hierarchy(st_a.to(DEV), bounds_fmt=1)
    P.pndf_update_hierarchy(h, st_b.to(DEV))
    D_upd = P.pndf_eval_batch(h, q.to(DEV)).cpu()
    h.free()
    h2 = P.pndf_build_hierarchy(st_b.to(DEV), bounds_fmt=1)
    D_new = P.pndf_eval_batch(h2, q.to(DEV)).cpu()
    h2.free()
    assert torch.equal(D_upd, D_new)


@pytest.mark.parametrize("n,half", [(96, False), (97, False), (128, True), (131, True)])
def test_pinned_host_texels(P, n, half):
    """Texels in page-locked host memory are read by the build kernel itself
    (no staging copy): build and update from them give exactly the hierarchy
    built from device texels (vector and scalar staging paths, FP32 and FP16)."""
    st = synth.flake_normals(n, 60, seed=n)
    st = st.half() if half else st
    q = synth.make_queries(st.float(), 1500, synth.QueryMix(sigma=(1.0, 12.0), frac_near=0.8), n)
    qd = q.to(DEV)
    h_dev = P.pndf_build_hierarchy(st.to(DEV), bounds_fmt=1)
    D_dev = P.pndf_eval_batch(h_dev, qd).cpu()
    h_dev.free()
    pinned = st.pin_memory()
    h = P.pndf_build_hierarchy(pinned, bounds_fmt=1)
    D_build = P.pndf_eval_batch(h, qd).cpu()
    other = synth.bumps_map(n=n, n_bumps=5, seed=n + 1)
    P.pndf_update_hierarchy(h, (other.half() if half else other).to(DEV))
    P.pndf_update_hierarchy(h, pinned)
    D_upd = P.pndf_eval_batch(h, qd).cpu()
    h.free()
    assert torch.equal(D_build, D_dev) and torch.equal(D_upd, D_dev)
    assert P.pndf_device_status() == 0


def test_unreadable_texels_rejected(P):
    """A pointer the device cannot read (pageable host memory) is refused on the
    host with INVALID_ARG before any work is queued, by the C ABI itself and
    by the binding."""
    import ctypes
    st = synth.bumps_map(n=64, n_bumps=4, seed=3)
    h = P.pndf_build_hierarchy(st.to(DEV), bounds_fmt=1)
    pageable = st.clone()
    assert not pageable.is_pinned()
    s = torch.cuda.current_stream().cuda_stream
    assert P.LIB.pndf_update_hierarchy(h.handle, ctypes.c_void_p(pageable.data_ptr()), ctypes.c_void_p(s)) == 1
    with pytest.raises(ValueError):
        P.pndf_update_hierarchy(h, pageable)
    with pytest.raises(ValueError):
        P.pndf_build_hierarchy(pageable)
    D = P.pndf_eval_batch(h, synth.make_queries(st, 100, synth.QueryMix(sigma=(1.0, 4.0)), 1).to(DEV))
    assert torch.isfinite(D).all()
    h.free()
