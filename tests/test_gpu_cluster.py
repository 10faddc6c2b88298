"""GPU parity of the cluster hierarchy and tau cut (Sec. 4.2, Eq. 7-8) with
the FP64 oracle, through the C ABI.

The fits (corner normals and residuals of every node) are compared node by
node; D with the cut is held to the same per-query bar as the exact path on
every query the oracle does not flag (edge and cut ties, and residuals or
entry radii within 1e-5 / 3e-5 of their thresholds on a node whose normal
hull holds m, where FP32 and FP64 may decide the cut differently).
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2505_08985_gb300 import synth
from parity import check_pndf, rel_err

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_08985_gb300 import pndf
    return pndf


def run(P, h, q, tau, sort=1):
    qd = q.to(DEV)
    flags = torch.zeros(q.shape[0], dtype=torch.int32, device=DEV)
    stt = torch.zeros(q.shape[0], P.STATS_FIELDS, dtype=torch.int32, device=DEV)
    D = P.pndf_eval_batch_ex(h, qd, flags=flags, stats=stt, tau=tau, sort=sort)
    torch.cuda.synchronize()
    return D.cpu().double().numpy(), flags.cpu().numpy(), stt.cpu().numpy().astype(np.int64)


def big_footprints(st, n, seed, sigma=(2.0, 48.0)):
    return synth.make_queries(st, n, synth.QueryMix(sigma=sigma, aspect=(1.0, 3.0), frac_near=0.8), seed)


def maps():
    return {"bumps256": synth.bumps_map(n=256, n_bumps=40, seed=21),
            "scratch257": synth.scratch_map(n=257, n_grooves=60, seed=22),
            "flakes256": synth.flake_normals(256, 600, seed=23)}


@pytest.mark.parametrize("name", ["bumps256", "scratch257", "flakes256"])
def test_cluster_fits_match_oracle(P, name):
    """Every node's corner normals and residual agree with the oracle's FP64
    fit (the GPU combines its children's quadratic forms up the tree; the
    oracle integrates each node directly)."""
    st = maps()[name]
    fits = oracle.cluster_fits(st)
    for bf in (0, 1):
        h = P.pndf_build_hierarchy(st.to(DEV), bounds_fmt=bf, clusters=True)
        for l in range(2, fits.L + 1):
            rec, e = P.pndf_cluster_level(h, l)
            rec, e = rec.cpu().double().numpy(), e.cpu().double().numpy()
            c_o, e_o = fits.level(l)
            inside = np.isfinite(e_o)
            assert np.array_equal(np.isfinite(e), inside), (name, l)
            if not inside.any():
                continue
            c00 = rec[..., 0:2]
            corners = np.stack([c00, c00 + rec[..., 2:4], c00 + rec[..., 4:6], c00 + rec[..., 6:8]], -2)
            np.testing.assert_allclose(corners[inside], c_o[inside], rtol=0, atol=2e-6, err_msg=f"{name} l={l}")
            # differences, which carry the cluster's Jacobian, to FP32 relative precision
            d_o = c_o[inside][:, 1:] - c_o[inside][:, :1]
            d_g = rec[inside][:, 2:].reshape(-1, 3, 2)
            scale = np.abs(d_o).max(axis=(1, 2), keepdims=True)
            assert (np.abs(d_g - d_o) <= 1e-6 * scale + 1e-12).all(), (name, l)
            # FP32 storage of e; an exactly linear (e.g. clamped constant) node has e = 0 and
            # both sides return rounding-level values there
            err = np.abs(e[inside] - e_o[inside])
            assert (err <= 1e-6 * e_o[inside] + 1e-7).all(), (name, l, err.max())
        h.free()


@pytest.mark.parametrize("name", ["bumps256", "scratch257", "flakes256"])
@pytest.mark.parametrize("tau", [1e-3, 1e-2, 0.1])
def test_cluster_cut_matches_oracle(P, name, tau):
    st = maps()[name]
    q = big_footprints(st, 1500, 5)
    fits = oracle.cluster_fits(st)
    ref = oracle.pndf_cluster(st, q, tau, fits)
    h = P.pndf_build_hierarchy(st.to(DEV), bounds_fmt=1, clusters=True)
    D, fl, stt = run(P, h, q, tau)
    h.free()
    s = check_pndf(D, ref, hits_gpu=stt[:, 3], hash_gpu=stt[:, 4], label=f"{name} tau={tau}")
    assert s["excluded"] < 0.1 * q.shape[0], s
    assert s["nonzero"] > 0.3 * s["compared"], s
    if tau >= 1e-2:
        assert stt[:, 9].sum() > 0, "no node was cut"  # clusters were really used
    assert P.pndf_device_status() == 0


def test_cluster_cut_reduces_work_and_keeps_mass_close(P):
    """A larger tau cuts higher in the tree: fewer triangle tests; D stays
    close to exact in aggregate (the surrogate approximates the map)."""
    st = synth.bumps_map(n=512, n_bumps=60, seed=3)
    q = big_footprints(st, 2000, 9, sigma=(8.0, 64.0))
    h = P.pndf_build_hierarchy(st.to(DEV), bounds_fmt=1, clusters=True)
    D0, _, s0 = run(P, h, q, 0.0)
    tests = [s0[:, 2].sum()]
    for tau in (1e-3, 1e-2, 1e-1):
        D, _, s = run(P, h, q, tau)
        tests.append(s[:, 2].sum() + 2 * s[:, 9].sum())
    h.free()
    assert tests[1] <= tests[0] and tests[3] < 0.5 * tests[0], tests
    assert tests[3] <= tests[2] <= tests[1], tests


def test_tau_zero_on_cluster_hierarchy_is_exact(P):
    """tau = 0 on a hierarchy built with clusters (widened boxes) gives the
    exact P-NDF: the same hit sets as the plain hierarchy and the oracle."""
    st = synth.scratch_map(n=512, n_grooves=120, seed=3)
    q = big_footprints(st, 2000, 4)
    ha = P.pndf_build_hierarchy(st.to(DEV), bounds_fmt=1)
    hb = P.pndf_build_hierarchy(st.to(DEV), bounds_fmt=1, clusters=True)
    Da, _, sa = run(P, ha, q, 0.0)
    Db, _, sb = run(P, hb, q, 0.0)
    assert hb.nbytes > ha.nbytes
    ha.free()
    hb.free()
    assert np.array_equal(sa[:, 3], sb[:, 3]) and np.array_equal(sa[:, 4], sb[:, 4])
    assert rel_err(Db, Da).max() <= 1e-5
    sub = np.arange(0, 2000, 10)
    check_pndf(Db[sub], oracle.pndf(st, q[sub]), hits_gpu=sb[sub, 3], hash_gpu=sb[sub, 4], label="tau=0")


def test_cut_does_not_depend_on_bounds_format(P):
    """The cut depends on the footprint only; FP16 outward and FP32 bounds
    prune differently but give the same hit sets."""
    st = synth.flake_normals(512, 1500, seed=5)
    q = big_footprints(st, 2000, 6)
    out = []
    for bf in (0, 1):
        h = P.pndf_build_hierarchy(st.to(DEV), bounds_fmt=bf, clusters=True)
        out.append(run(P, h, q, 3e-3))
        h.free()
    (D32, _, s32), (D16, _, s16) = out
    assert np.array_equal(s32[:, 3], s16[:, 3]) and np.array_equal(s32[:, 4], s16[:, 4])
    assert rel_err(D16, D32).max() <= 1e-5


def test_update_rebuilds_clusters(P):
    """pndf_update_hierarchy refits the clusters: the same results as a fresh build."""
    a = synth.bumps_map(n=256, n_bumps=30, seed=1)
    b = synth.bumps_map(n=256, n_bumps=30, seed=2)
    q = big_footprints(b, 1000, 2)
    h = P.pndf_build_hierarchy(a.to(DEV), bounds_fmt=1, clusters=True)
    P.pndf_update_hierarchy(h, b.to(DEV))
    Du, _, su = run(P, h, q, 1e-2)
    h.free()
    h = P.pndf_build_hierarchy(b.to(DEV), bounds_fmt=1, clusters=True)
    Df, _, sf = run(P, h, q, 1e-2)
    h.free()
    assert np.array_equal(Du, Df) and np.array_equal(su, sf)


def test_tau_errors(P):
    st = synth.bumps_map(n=64, n_bumps=4, seed=1).to(DEV)
    q = synth.camera_queries(64, 10, seed=1, device=DEV)
    h = P.pndf_build_hierarchy(st, bounds_fmt=1)
    with pytest.raises(P.PndfError) as ei:
        P.pndf_eval_batch_ex(h, q, tau=1e-3)
    assert ei.value.code == 6  # UNSUPPORTED: built without clusters
    with pytest.raises(P.PndfError):
        P.pndf_cluster_level(h, 2)
    h.free()
    h = P.pndf_build_hierarchy(st, bounds_fmt=1, clusters=True)
    for bad in (float("nan"), -1.0, float("inf")):
        with pytest.raises(P.PndfError) as ei:
            P.pndf_eval_batch_ex(h, q, tau=bad)
        assert ei.value.code == 1
    with pytest.raises(P.PndfError) as ei:
        P.pndf_eval_batch_ex(h, q, tau=1e-3, mode=1)
    assert ei.value.code == 6  # flat mode has no cut
    with pytest.raises(P.PndfError):
        P.pndf_cluster_level(h, 1)
    h.free()


@pytest.mark.slow
def test_flake8192_cluster_cut_sampled(P):
    """The 8192^2 flake workload with tau = 1e-3 in the benchmark's launch
    configuration (4,194,304 queries, FP16 bounds, sorted): a stratified
    sample of queries against the oracle's cut."""
    cfg = synth.FLAKE_8192
    st = synth.flake_map(n=8192, seed=cfg["seed"], device=DEV)
    q = synth.make_queries(st, cfg["queries"], cfg["mix"], cfg["seed"])
    h = P.pndf_build_hierarchy(st, bounds_fmt=1, clusters=True)
    D = P.pndf_eval_batch_ex(h, q, tau=1e-3)
    torch.cuda.synchronize()
    h.free()
    sig = q[:, 2].sqrt().cpu().numpy()
    order = np.argsort(sig, kind="stable")
    sub = np.sort(order[np.linspace(0, len(order) - 1, 600).astype(np.int64)])  # across the sigma range
    stc = st.cpu()
    fits = oracle.cluster_fits(stc)
    ref = oracle.pndf_cluster(stc, q[sub].cpu(), 1e-3, fits)
    s = check_pndf(D[sub].cpu().double().numpy(), ref, label="flake8192 tau=1e-3")
    assert s["excluded"] < 0.1 * len(sub), s
