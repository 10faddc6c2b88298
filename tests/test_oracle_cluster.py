"""Pins for the oracle's cluster hierarchy (Sec. 4.2 on mesh clustering,
Eq. 7-8, App. A) and its tau cut.

Expected values come by other routes than the oracle's: exact recovery of
piecewise-linear data, a weighted least-squares fit by numpy over a dense
sub-triangle sample (centroid rule, not the oracle's edge midpoints), the
mass invariant of Eq. 2 for the surrogate map the cut defines, the binning
reference (Fig. 3) of that surrogate with the cut taken by this file's own
top-down walk, and metamorphic relations.
"""

import math

import numpy as np
import pytest

from paper_2505_08985_gb300 import synth
from test_oracle_pins import gauss, interp_normal

JAC_EPS = 1e-6


# ---------------------------------------------------------------------------
# helpers (independent of the oracle's arithmetic)
# ---------------------------------------------------------------------------

def pl_map(N, corners):
    """Texels of the function that is linear on the two triangles of the
    whole map (split like a quad, Eq. 3) with corner normals
    (c00, c10, c01, c11) at the four map corners."""
    a = N - 1
    C = np.asarray(corners, np.float64).reshape(2, 2, 2)  # [t][s] -> normal
    j, i = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    return interp_normal(C, (i / a).ravel(), (j / a).ravel()).reshape(N, N, 2)


def cluster_eval(c, s, t):
    """n^l at normalised local coordinates: Eq. 3 interpolation of the 2 x 2
    corner grid."""
    C = np.asarray(c, np.float64).reshape(2, 2, 2)
    return interp_normal(C, np.asarray(s, np.float64), np.asarray(t, np.float64))


def subtri_points(K):
    """Centroids of the K^2 congruent sub-triangles of the unit lower
    triangle {u, v >= 0, u + v <= 1}; each has area 1 / (2 K^2)."""
    pts = []
    for a in range(K):
        for b in range(K - a):
            pts.append(((a + 1 / 3) / K, (b + 1 / 3) / K))
            if a + b <= K - 2:
                pts.append(((a + 2 / 3) / K, (b + 2 / 3) / K))
    return np.asarray(pts)


def fine_cross(st, i, j, tri):
    n0, n1, n2, n3 = st[j, i], st[j, i + 1], st[j + 1, i], st[j + 1, i + 1]
    a, b, c = (n0, n1, n2) if tri == 0 else (n3, n2, n1)
    return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])


def dense_fit(st, l, I, J, K):
    """Weighted least squares (Eq. 7) over sub-triangle centroids of every
    fine triangle of node (l, I, J), solved by numpy's lstsq."""
    a = 1 << l
    P = subtri_points(K)
    w_sub = 1.0 / (2 * K * K)
    rows_u, rows_v, rows_w = [], [], []
    for j in range(a * J, a * J + a):
        for i in range(a * I, a * I + a):
            for tri in range(2):
                w = w_sub / max(abs(fine_cross(st, i, j, tri)), JAC_EPS)
                u, v = (P[:, 0], P[:, 1]) if tri == 0 else (1 - P[:, 0], 1 - P[:, 1])
                rows_u.append(i + u)
                rows_v.append(j + v)
                rows_w.append(np.full(len(P), w))
    ux, uy, w = np.concatenate(rows_u), np.concatenate(rows_v), np.concatenate(rows_w)
    n = interp_normal(st, ux, uy)
    s, t = (ux - a * I) / a, (uy - a * J) / a
    basis = np.stack([cluster_eval(np.eye(4)[k].repeat(2).reshape(4, 2) * [1, 0], s, t)[:, 0] for k in range(4)], 1)
    sw = np.sqrt(w)[:, None]
    c, *_ = np.linalg.lstsq(basis * sw, n * sw, rcond=None)
    F = float(np.sum(w * np.sum((basis @ c - n) ** 2, axis=1)))
    return c, math.sqrt(F)


def walk_cut(fits, N, x, y, sxx, syy, tau):
    """The cut of Sec. 4.2 taken top down from the entry nodes: returns the
    cut nodes (l, I, J) and the level-2 nodes evaluated exactly."""
    L = fits.L
    rx, ry = 4 * math.sqrt(sxx), 4 * math.sqrt(syy)
    r = max(rx, ry)
    le = 2
    while le < L and 2 ** le < r:
        le += 1
    cut, exact = [], []

    def visit(l, I, J):
        a = 1 << l
        if a * I > N - 2 or a * J > N - 2:
            return
        if a * I > x + rx or a * (I + 1) < x - rx or a * J > y + ry or a * (J + 1) < y - ry:
            return
        _, e = fits.level(l)
        if tau > 0 and np.isfinite(e[J, I]) and e[J, I] <= rx * ry * tau:
            cut.append((l, I, J))
            return
        if l == 2:
            exact.append((I, J))
            return
        for dj in range(2):
            for di in range(2):
                visit(l - 1, 2 * I + di, 2 * J + dj)

    a = 1 << le
    S = 1 << (L - le)
    for J in range(max(math.ceil((y - ry) / a) - 1, 0), min(math.floor((y + ry) / a), S - 1) + 1):
        for I in range(max(math.ceil((x - rx) / a) - 1, 0), min(math.floor((x + rx) / a), S - 1) + 1):
            visit(le, I, J)
    return cut, exact


def surrogate_normal(st, fits, cut, ux, uy):
    """The surrogate map the cut defines: the cluster of a cut node where u
    falls in one, the normal map elsewhere (Eq. 3)."""
    n = interp_normal(st, ux, uy)
    for (l, I, J) in cut:
        a = 1 << l
        inside = (ux >= a * I) & (ux < a * I + a) & (uy >= a * J) & (uy < a * J + a)
        if np.any(inside):
            c, _ = fits.level(l)
            n[inside] = cluster_eval(c[J, I], (ux[inside] - a * I) / a, (uy[inside] - a * J) / a)
    return n


def smooth_map(N, seed):
    return synth.normals_from_height(synth.bumps_height(N, 6, seed=seed, noise=0.0, sig=(3.0, 8.0))).double().numpy()


# ---------------------------------------------------------------------------
# Eq. 7-8: the fit
# ---------------------------------------------------------------------------

PL_CORNERS = ((-0.25, 0.125), (0.1875, -0.0625), (-0.0625, 0.3125), (0.25, 0.1875))


def test_fit_recovers_piecewise_linear_data(oracle_mod):
    """Data that is linear on the two triangles of the whole map is linear on
    every node's two cluster triangles (the anti-diagonals line up), so every
    fit is exact: corner normals = the data at the node corners, e = 0."""
    N = 33
    st = pl_map(N, PL_CORNERS)
    fits = oracle_mod.cluster_fits(st)
    for l in range(2, fits.L + 1):
        c, e = fits.level(l)
        a = 1 << l
        for J in range(1 << (fits.L - l)):
            for I in range(1 << (fits.L - l)):
                expect = np.stack([st[a * J, a * I], st[a * J, a * I + a], st[a * J + a, a * I],
                                   st[a * J + a, a * I + a]])
                np.testing.assert_allclose(c[J, I], expect, rtol=0, atol=1e-12)
                assert 0 <= e[J, I] < 1e-9, (l, I, J, e[J, I])


def test_fit_only_inside_the_map(oracle_mod):
    """A node with a quad outside the map has no cluster."""
    st = smooth_map(32, 3)  # 31 quads per side, L = 5
    fits = oracle_mod.cluster_fits(st)
    c, e = fits.level(3)
    assert np.isfinite(e[:3, :3]).all() and np.isinf(e[3, :]).all() and np.isinf(e[:, 3]).all()
    assert oracle_mod.cluster_fit(st, 3, 3, 0) is None
    assert np.isinf(fits.level(fits.L)[1]).all()


@pytest.mark.parametrize("l,I,J", [(2, 1, 2), (2, 4, 3), (3, 1, 1)])
def test_fit_matches_dense_least_squares(oracle_mod, l, I, J):
    """The oracle's fit and residual (the 2-norm of the weighted error, Eq. 8)
    agree with a dense weighted least-squares solve (numpy lstsq over
    sub-triangle centroids); the gap shrinks as the sample is refined."""
    st = smooth_map(40, 8)
    c, e = oracle_mod.cluster_fit(st, l, I, J)
    errs = []
    for K in (4, 16):
        cd, Fd = dense_fit(st, l, I, J, K)
        errs.append((np.abs(cd - c).max() / np.abs(c).max(), abs(Fd - e) / e))
    assert errs[1][0] < 2e-4 and errs[1][1] < 2e-3, errs
    assert errs[1][0] < 0.2 * errs[0][0] and errs[1][1] < 0.2 * errs[0][1], errs


def test_fit_weights_follow_inverse_jacobian(oracle_mod):
    """Making one fine triangle nearly flat in normal space raises its weight
    (1 / |det J|, Eq. 7) and pulls the fit toward it: the misfit there drops."""
    st = smooth_map(40, 8)
    l, I, J = 2, 2, 2
    c0, _ = oracle_mod.cluster_fit(st, l, I, J)
    st2 = st.copy()
    i, j = 9, 9  # lower triangle of quad (9, 9): make n1 and n2 nearly equal to n0
    st2[j, i + 1] = st2[j, i] + [1e-4, 0]
    st2[j + 1, i] = st2[j, i] + [0, 1e-4]
    c1, _ = oracle_mod.cluster_fit(st2, l, I, J)
    cd1, _ = dense_fit(st2, l, I, J, 16)
    np.testing.assert_allclose(c1, cd1, rtol=0, atol=2e-4 * np.abs(c1).max())
    s, t = (i + 1 / 3 - 4 * I) / 4, (j + 1 / 3 - 4 * J) / 4
    target = interp_normal(st2, np.array([i + 1 / 3]), np.array([j + 1 / 3]))[0]
    miss0 = np.linalg.norm(cluster_eval(c0, [s], [t])[0] - target)
    miss1 = np.linalg.norm(cluster_eval(c1, [s], [t])[0] - target)
    assert miss1 < 0.5 * miss0, (miss0, miss1)


# ---------------------------------------------------------------------------
# the cut and the cluster P-NDF
# ---------------------------------------------------------------------------

def _queries(st, n, seed, sig=(1.0, 4.0), margin=6):
    import torch
    return synth.make_queries(torch.as_tensor(st, dtype=torch.float32), n,
                              synth.QueryMix(sigma=sig, aspect=(1.0, 3.0), frac_near=0.8, centre_margin=margin),
                              seed).double().numpy()


def test_tau_zero_is_exact(oracle_mod):
    """tau = 0 cuts nothing: D, hits and hit fingerprints equal the exact P-NDF."""
    st = smooth_map(48, 2)
    q = _queries(st, 300, 4)
    D, f, h, hh = oracle_mod.pndf(st, q)
    Dc, fc, hc, hhc = oracle_mod.pndf_cluster(st, q, 0.0)
    np.testing.assert_allclose(Dc, D, rtol=1e-13, atol=0)
    assert np.array_equal(h, hc) and np.array_equal(hh, hhc) and np.array_equal(f, fc)


def test_piecewise_linear_map_is_unchanged_by_any_cut(oracle_mod):
    """On data linear on the map's two triangles every cluster is exact, so
    the surrogate is the map itself and D does not depend on tau."""
    N = 65
    st = pl_map(N, PL_CORNERS)
    q = _queries(st, 400, 5, sig=(1.0, 6.0), margin=4)
    D, f, *_ = oracle_mod.pndf(st, q)
    hh = oracle_mod.pndf(st, q)[3]
    for tau in (1e-3, 1e9):
        Dc, fc, hc, hhc = oracle_mod.pndf_cluster(st, q, tau)
        ok = ((f | fc) & oracle_mod.F_EXCLUDE) == 0
        assert ok.sum() > 0.9 * len(q)
        np.testing.assert_allclose(Dc[ok], D[ok], rtol=1e-9, atol=1e-300)
        assert ((hhc != hh) & (hc > 0)).mean() > 0.2  # cluster hits replaced triangle hits


def _cluster_mass(oracle_mod, st, fits, x, y, sxx, syy, tau, res, seed):
    rng = np.random.default_rng(seed)
    rx, ry = 4 * math.sqrt(sxx), 4 * math.sqrt(syy)
    cut, exact = walk_cut(fits, st.shape[0], x, y, sxx, syy, tau)
    pts = [st[max(0, int(y - ry) - 1):int(y + ry) + 3, max(0, int(x - rx) - 1):int(x + rx) + 3].reshape(-1, 2)]
    for (l, I, J) in cut:
        pts.append(fits.level(l)[0][J, I])
    pts = np.concatenate(pts)
    lo, hi = pts.min(0) - 1e-3, pts.max(0) + 1e-3
    h = (hi - lo) / res
    off = rng.uniform(0, 1, 2)
    mx, my = np.meshgrid(lo[0] + (np.arange(res) + off[0]) * h[0], lo[1] + (np.arange(res) + off[1]) * h[1])
    q = np.zeros((mx.size, 7))
    q[:, 0], q[:, 1], q[:, 2], q[:, 4] = x, y, sxx, syy
    q[:, 5], q[:, 6] = mx.ravel(), my.ravel()
    D, *_ = oracle_mod.pndf_cluster(st, q, tau, fits)
    return D.sum() * h[0] * h[1], len(cut), len(exact)


@pytest.mark.parametrize("tau", [1e9, "mixed"])
def test_cluster_mass_invariant(oracle_mod, tau):
    """Each piece of the surrogate map (a cut node's two cluster triangles or
    an exact triangle) maps its uv area onto the normal plane with the
    Jacobian of Eq. 4 (|cross| / 2^(2l) for a cluster), so D still
    integrates to the kernel mass 1 - e^-8 over the footprint."""
    st = smooth_map(40, 11)
    fits = oracle_mod.cluster_fits(st)
    x, y, sxx, syy = 19.5, 19.25, 4.0, 2.25
    if tau == "mixed":  # about half of the entry nodes cut
        rx, ry = 4 * math.sqrt(sxx), 4 * math.sqrt(syy)
        e = fits.level(3)[1][1:4, 1:4].ravel()
        tau = float(np.median(e[np.isfinite(e)])) / (rx * ry)
    target = 1.0 - math.exp(-8.0)
    m1, ncut, nex = _cluster_mass(oracle_mod, st, fits, x, y, sxx, syy, tau, 300, 1)
    m2, _, _ = _cluster_mass(oracle_mod, st, fits, x, y, sxx, syy, tau, 700, 2)
    assert ncut > 0
    assert abs(m2 - target) / target < 0.01, (m1, m2, ncut, nex)
    assert abs(m2 - target) < abs(m1 - target) or abs(m2 - target) / target < 2e-3


def _surrogate_binning_l1(oracle_mod, st, fits, x, y, sxx, syy, tau, nbins, nsamp, seed, sub):
    rng = np.random.default_rng(seed)
    rx, ry = 4 * math.sqrt(sxx), 4 * math.sqrt(syy)
    cut, _ = walk_cut(fits, st.shape[0], x, y, sxx, syy, tau)
    k = int(math.sqrt(nsamp))
    gx = (np.arange(k)[None, :] + rng.uniform(0, 1, (k, k))) / k
    gy = (np.arange(k)[:, None] + rng.uniform(0, 1, (k, k))) / k
    ux = ((x - rx) + 2 * rx * gx).ravel()
    uy = ((y - ry) + 2 * ry * gy).ravel()
    w, _ = gauss(ux - x, uy - y, sxx, 0.0, syy)
    w *= 4 * rx * ry / ux.size
    n = surrogate_normal(st, fits, cut, ux, uy)
    lo, hi = n[w > 0].min(0), n[w > 0].max(0)
    ex, ey = np.linspace(lo[0], hi[0], nbins + 1), np.linspace(lo[1], hi[1], nbins + 1)
    hist, _, _ = np.histogram2d(n[:, 0], n[:, 1], bins=[ex, ey], weights=w)
    bx, by = ex[1] - ex[0], ey[1] - ey[0]
    fx = (np.arange(nbins * sub) + rng.uniform(0, 1, nbins * sub)) / sub
    fy = (np.arange(nbins * sub) + rng.uniform(0, 1, nbins * sub)) / sub
    mx, my = np.meshgrid(ex[0] + fx * bx, ey[0] + fy * by, indexing="ij")
    q = np.zeros((mx.size, 7))
    q[:, 0], q[:, 1], q[:, 2], q[:, 4] = x, y, sxx, syy
    q[:, 5], q[:, 6] = mx.ravel(), my.ravel()
    D, *_ = oracle_mod.pndf_cluster(st, q, tau, fits)
    Dm = D.reshape(nbins, sub, nbins, sub).mean(axis=(1, 3)) * bx * by
    return np.abs(Dm - hist).sum() / hist.sum(), len(cut)


def test_cluster_binning_with_anisotropic_cut(oracle_mod):
    """The binned normals of the surrogate map (cut by this file's own walk
    with threshold r_x r_y tau) match the cluster P-NDF.  tau is set so that
    some entry nodes lie between r_x r_y tau and max(r_x, r_y)^2 tau: a cut
    taken on the wrong footprint size changes the surrogate there."""
    st = smooth_map(40, 11)
    fits = oracle_mod.cluster_fits(st)
    x, y, sxx, syy = 19.5, 19.25, 4.0, 1.0
    rx, ry = 4 * math.sqrt(sxx), 4 * math.sqrt(syy)
    e = np.sort(fits.level(3)[1][1:3, 1:4].ravel())  # the six entry nodes
    tau = 0.75 * e[3] / (rx * ry)
    assert ((e > rx * ry * tau) & (e <= max(rx, ry) ** 2 * tau)).any()
    l1_small, ncut = _surrogate_binning_l1(oracle_mod, st, fits, x, y, sxx, syy, tau, 16, 250_000, 1, 8)
    l1_big, _ = _surrogate_binning_l1(oracle_mod, st, fits, x, y, sxx, syy, tau, 16, 4_000_000, 2, 48)
    assert ncut > 0
    assert l1_big < 0.01, (l1_small, l1_big)
    assert l1_big < 0.5 * l1_small


def test_cluster_transpose_symmetry(oracle_mod):
    """Transposing the map (i <-> j, s <-> t) with the query transposed
    leaves the cluster fits (transposed) and the cut D unchanged."""
    st = smooth_map(48, 4)
    stT = np.ascontiguousarray(st.transpose(1, 0, 2)[:, :, ::-1])
    f, fT = oracle_mod.cluster_fits(st), oracle_mod.cluster_fits(stT)
    for l in range(2, f.L + 1):
        c, e = f.level(l)
        cT, eT = fT.level(l)
        np.testing.assert_allclose(eT, e.T, rtol=1e-10, atol=1e-300)
        ok = np.isfinite(e)
        swap = c[:, :, [0, 2, 1, 3], ::-1].transpose(1, 0, 2, 3)  # c10 <-> c01, s <-> t
        np.testing.assert_allclose(cT[ok.T], swap[ok.T], rtol=0, atol=1e-12)
    q = _queries(st, 300, 6, sig=(1.0, 6.0))
    qT = q[:, [1, 0, 4, 3, 2, 6, 5]]
    tau = 3e-3
    D, fl, h, _ = oracle_mod.pndf_cluster(st, q, tau, f)
    DT, flT, hT, _ = oracle_mod.pndf_cluster(stT, qT, tau, fT)
    ok = ((fl | flT) & oracle_mod.F_EXCLUDE) == 0
    np.testing.assert_allclose(DT[ok], D[ok], rtol=1e-9, atol=1e-300)


def test_near_tau_flag_covers_every_close_call(oracle_mod):
    """A cut decision within rounding of its threshold is flagged: with tau
    set exactly at one visited node's residual, nudging tau by less than the
    flag's band flips that node, and every query whose D changes is flagged
    (and some do change)."""
    st = smooth_map(64, 5)
    fits = oracle_mod.cluster_fits(st)
    x, y, sxx, syy = 31.5, 30.75, 9.0, 6.25
    rx, ry = 4 * math.sqrt(sxx), 4 * math.sqrt(syy)
    # an entry node (level 4) that is cut at tau = e / (r_x r_y) and not just below
    e = fits.level(4)[1][1:3, 1:3].ravel()
    tau = float(np.sort(e[np.isfinite(e)])[1]) / (rx * ry)
    rng = np.random.default_rng(3)
    pts = st[12:52, 12:52].reshape(-1, 2)
    m = pts[rng.integers(0, len(pts), 3000)] + rng.normal(0, 0.01, (3000, 2))
    q = np.zeros((3000, 7))
    q[:, 0], q[:, 1], q[:, 2], q[:, 4], q[:, 5], q[:, 6] = x, y, sxx, syy, m[:, 0], m[:, 1]
    D0, f0, *_ = oracle_mod.pndf_cluster(st, q, tau, fits)
    changed = np.zeros(len(q), bool)
    for k in (1 - 5e-6, 1 + 5e-6):
        D1, *_ = oracle_mod.pndf_cluster(st, q, tau * k, fits)
        changed |= D1 != D0
    assert changed.sum() > 20, changed.sum()
    assert np.all(f0[changed] & oracle_mod.F_NEAR_TAU), np.flatnonzero(changed & ((f0 & oracle_mod.F_NEAR_TAU) == 0))
