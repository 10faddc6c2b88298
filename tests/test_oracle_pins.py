"""Pins for the FP64 oracle: facts the paper and the mathematics fix.

Every pin computes its expected value by a route other than the oracle's own
formula: a closed form (affine field, Eq. 2 by change of variables), an
integral invariant, the paper's binning reference (Fig. 3), metamorphic
symmetries, and for the projected area a shoelace sum, 2D quadrature of the
area integrand (App. B, Stokes check) and uv-space quadrature of Eq. 13.
"""

import math

import numpy as np
import pytest
import torch

from paper_2505_08985_gb300 import synth

QCUT = 16.0


def gauss(dx, dy, sxx, sxy, syy):
    det = sxx * syy - sxy * sxy
    q = (syy * dx * dx - 2 * sxy * dx * dy + sxx * dy * dy) / det
    g = np.exp(-0.5 * q) / (2 * np.pi * np.sqrt(det))
    return np.where(q <= QCUT, g, 0.0), q


def interp_normal(st, ux, uy):
    """Eq. 3: barycentric interpolation of the normal map at uv (ux, uy)."""
    N = st.shape[0]
    i = np.clip(np.floor(ux).astype(np.int64), 0, N - 2)
    j = np.clip(np.floor(uy).astype(np.int64), 0, N - 2)
    u = ux - i
    v = uy - j
    n0 = st[j, i]
    n1 = st[j, i + 1]
    n2 = st[j + 1, i]
    n3 = st[j + 1, i + 1]
    lower = (u + v < 1.0)[:, None]
    a = n0 * (1 - u - v)[:, None] + n1 * u[:, None] + n2 * v[:, None]
    b = n3 * (u + v - 1)[:, None] + n2 * (1 - u)[:, None] + n1 * (1 - v)[:, None]
    return np.where(lower, a, b)


# ---------------------------------------------------------------------------
# (a) affine normal field: closed form
# ---------------------------------------------------------------------------

AFF_N0 = (-0.2001953125, -0.150390625)
AFF_M = ((44 / 4096, 8 / 4096), (-12 / 4096, 40 / 4096))


def _affine_cases(seed, nq=400):
    N = 32
    st = synth.affine_normals(N, AFF_N0, AFF_M)
    assert np.all(st.double().numpy() == np.asarray(
        [[[AFF_N0[0] + AFF_M[0][0] * i + AFF_M[0][1] * j, AFF_N0[1] + AFF_M[1][0] * i + AFF_M[1][1] * j]
          for i in range(N)] for j in range(N)])), "affine texels must be exact in float32"
    rng = np.random.default_rng(seed)
    x = rng.uniform(4, 27, nq)
    y = rng.uniform(4, 27, nq)
    s1 = rng.uniform(0.7, 3.0, nq)
    s2 = rng.uniform(0.7, 3.0, nq)
    th = rng.uniform(0, np.pi, nq)
    c, s = np.cos(th), np.sin(th)
    sxx = (c * c * s1 * s1 + s * s * s2 * s2).astype(np.float32).astype(np.float64)
    syy = (s * s * s1 * s1 + c * c * s2 * s2).astype(np.float32).astype(np.float64)
    sxy = (c * s * (s1 * s1 - s2 * s2)).astype(np.float32).astype(np.float64)
    # preimages inside and outside the map
    us = rng.uniform(-3, N + 2, (nq, 2))
    M = np.asarray(AFF_M)
    m = (np.asarray(AFF_N0)[None, :] + us @ M.T).astype(np.float32).astype(np.float64)
    q = np.stack([x, y, sxx, sxy, syy, m[:, 0], m[:, 1]], 1).astype(np.float32).astype(np.float64)
    return st, q


def test_affine_closed_form(oracle_mod):
    """n(u) = n0 + M u: the unique preimage u* = M^-1 (m - n0) gives
    D = k_r(u* - x) / |det M| inside the map, 0 outside (Eq. 2)."""
    st, q = _affine_cases(7)
    D, flags, hits, _ = oracle_mod.pndf(st, q)
    M = np.asarray(AFF_M)
    ustar = np.linalg.solve(M[None, :, :], (q[:, 5:7] - np.asarray(AFF_N0)[None, :])[:, :, None])[:, :, 0]
    N = st.shape[0]
    inside = np.all((ustar > 0) & (ustar < N - 1), axis=1)
    g, qq = gauss(ustar[:, 0] - q[:, 0], ustar[:, 1] - q[:, 1], q[:, 2], q[:, 3], q[:, 4])
    expect = np.where(inside, g / abs(np.linalg.det(M)), 0.0)
    ok = (flags & oracle_mod.F_EXCLUDE) == 0
    assert ok.sum() > 0.95 * len(q)
    assert np.any(expect[ok] > 0) and np.any(expect[ok] == 0)
    np.testing.assert_allclose(D[ok], expect[ok], rtol=1e-12, atol=0)
    contributing = inside & (qq <= QCUT)
    assert np.array_equal(hits[ok], contributing[ok].astype(np.int64))


# ---------------------------------------------------------------------------
# (b) mass: the P-NDF integrates to the footprint's kernel mass
# ---------------------------------------------------------------------------

def _mass_estimate(oracle_mod, st, x, y, sig, res, seed):
    rng = np.random.default_rng(seed)
    N = st.shape[0]
    r = 4 * sig
    i0, i1 = int(max(0, math.floor(x - r) - 1)), int(min(N - 1, math.ceil(x + r) + 1))
    j0, j1 = int(max(0, math.floor(y - r) - 1)), int(min(N - 1, math.ceil(y + r) + 1))
    sub = st[j0:j1 + 1, i0:i1 + 1].reshape(-1, 2)
    lo = sub.min(0) - 1e-3
    hi = sub.max(0) + 1e-3
    h = (hi - lo) / res
    off = rng.uniform(0, 1, 2)
    gx = lo[0] + (np.arange(res) + off[0]) * h[0]
    gy = lo[1] + (np.arange(res) + off[1]) * h[1]
    mx, my = np.meshgrid(gx, gy)
    n = mx.size
    q = np.zeros((n, 7))
    q[:, 0] = x
    q[:, 1] = y
    q[:, 2] = sig * sig
    q[:, 4] = sig * sig
    q[:, 5] = mx.ravel()
    q[:, 6] = my.ravel()
    D, *_ = oracle_mod.pndf(st, q)
    return D.sum() * h[0] * h[1]


def test_mass_invariant(oracle_mod):
    """Integrating D over the normal plane gives the kernel mass over the
    footprint: 1 - e^-8 for the 4-sigma-cut Gaussian inside the map (Eq. 2,
    change of variables per triangle).  The jittered-grid estimate converges."""
    st = synth.normals_from_height(synth.bumps_height(40, 6, seed=11, noise=0.0, sig=(3.0, 6.0))).double().numpy()
    target = 1.0 - math.exp(-8.0)
    e_coarse = abs(_mass_estimate(oracle_mod, st, 19.5, 19.25, 2.0, 150, 1) - target) / target
    e_fine = abs(_mass_estimate(oracle_mod, st, 19.5, 19.25, 2.0, 600, 2) - target) / target
    assert e_fine < 0.01, (e_coarse, e_fine)
    assert e_fine < e_coarse or e_fine < 2e-3


# ---------------------------------------------------------------------------
# (c) binning: the paper's reference (Fig. 3)
# ---------------------------------------------------------------------------

def _binning_l1(oracle_mod, st, x, y, sig, nbins, nsamp, seed, sub=8):
    """L1 distance between the normalised binned histogram of n(u), u ~ k_r,
    and the oracle's bin averages of D, relative to the total mass."""
    rng = np.random.default_rng(seed)
    r = 4 * sig
    # stratified uv sampling over the footprint box, weights k_r
    k = int(math.sqrt(nsamp))
    g = (np.arange(k)[None, :] + rng.uniform(0, 1, (k, k))) / k
    ux = (x - r) + 2 * r * g
    uy = (y - r) + 2 * r * ((np.arange(k)[:, None] + rng.uniform(0, 1, (k, k))) / k)
    ux, uy = ux.ravel(), uy.ravel()
    w, _ = gauss(ux - x, uy - y, sig * sig, 0.0, sig * sig)
    w *= (2 * r) ** 2 / ux.size
    n = interp_normal(st, ux, uy)
    lo = n[w > 0].min(0)
    hi = n[w > 0].max(0)
    edges_x = np.linspace(lo[0], hi[0], nbins + 1)
    edges_y = np.linspace(lo[1], hi[1], nbins + 1)
    hist, _, _ = np.histogram2d(n[:, 0], n[:, 1], bins=[edges_x, edges_y], weights=w)
    # oracle: bin average of D on a sub x sub jittered sub-grid per bin
    bx = (edges_x[1] - edges_x[0])
    by = (edges_y[1] - edges_y[0])
    fx = (np.arange(nbins * sub) + rng.uniform(0, 1, nbins * sub)) / sub
    fy = (np.arange(nbins * sub) + rng.uniform(0, 1, nbins * sub)) / sub
    mx, my = np.meshgrid(edges_x[0] + fx * bx, edges_y[0] + fy * by, indexing="ij")
    qq = np.zeros((mx.size, 7))
    qq[:, 0], qq[:, 1], qq[:, 2], qq[:, 4] = x, y, sig * sig, sig * sig
    qq[:, 5], qq[:, 6] = mx.ravel(), my.ravel()
    D, *_ = oracle_mod.pndf(st, qq)
    Dm = D.reshape(nbins, sub, nbins, sub).mean(axis=(1, 3)) * bx * by
    return np.abs(Dm - hist).sum() / hist.sum()


def test_binning_converges(oracle_mod):
    """A dense uv sample of n(u) (Eq. 3 interpolation), binned in m with
    weights k_r, matches the bin-integrated P-NDF (the paper's binning
    reference, Fig. 3); the gap shrinks with more samples."""
    st = synth.normals_from_height(synth.bumps_height(32, 5, seed=5, noise=0.0, sig=(3.0, 8.0))).double().numpy()
    l1_small = _binning_l1(oracle_mod, st, 15.5, 15.5, 1.5, 16, 250_000, 1, sub=8)
    l1_big = _binning_l1(oracle_mod, st, 15.5, 15.5, 1.5, 16, 4_000_000, 2, sub=64)
    assert l1_big < 0.01, (l1_small, l1_big)
    assert l1_big < 0.5 * l1_small


# ---------------------------------------------------------------------------
# (e) metamorphic relations
# ---------------------------------------------------------------------------

def _rand_queries(st, n, seed, sig=(1.0, 3.0), margin=14):
    return synth.make_queries(torch.as_tensor(st, dtype=torch.float32), n,
                              synth.QueryMix(sigma=sig, aspect=(1.0, 3.0), frac_near=0.8, centre_margin=margin),
                              seed).double().numpy()


def test_translation_invariance(oracle_mod):
    """Shifting the map and the footprint centre by whole texels leaves D unchanged."""
    big = synth.bumps_map(n=64, n_bumps=12, seed=9).double().numpy()
    a = big[0:48, 0:48]
    b = big[5:53, 3:51]  # b[j, i] = a[j + 5, i + 3]
    q = _rand_queries(b, 300, 3, margin=15)
    qa = q.copy()
    qa[:, 0] += 3
    qa[:, 1] += 5
    Da, fa, ha, _ = oracle_mod.pndf(a, qa)
    Db, fb, hb, _ = oracle_mod.pndf(b, q)
    np.testing.assert_allclose(Db, Da, rtol=1e-12, atol=0)
    assert np.array_equal(ha, hb) and np.array_equal(fa, fb)


def test_transpose_symmetry(oracle_mod):
    """Transposing the map (i <-> j, s <-> t) with x, Sigma and m transposed
    leaves D unchanged: the u1-u2 diagonal maps onto itself."""
    st = synth.bumps_map(n=48, n_bumps=10, seed=4).double().numpy()
    stT = np.ascontiguousarray(st.transpose(1, 0, 2)[:, :, ::-1])
    q = _rand_queries(st, 300, 8)
    qT = q[:, [1, 0, 4, 3, 2, 6, 5]]
    D, f, h, _ = oracle_mod.pndf(st, q)
    DT, fT, hT, _ = oracle_mod.pndf(stT, qT)
    np.testing.assert_allclose(DT, D, rtol=1e-12, atol=1e-300)
    assert np.array_equal(h, hT)


def test_constant_map_is_zero(oracle_mod):
    """A constant map has only zero-area normal triangles: every one is a
    delta, skipped, so D = 0 and the queries on the constant are flagged."""
    st = np.full((24, 24, 2), 0.125)
    q = np.array([[11.0, 12.0, 4.0, 0.5, 3.0, 0.125, 0.125],
                  [11.0, 12.0, 4.0, 0.5, 3.0, 0.1, 0.125]])
    D, f, h, _ = oracle_mod.pndf(st, q)
    assert np.all(D == 0) and np.all(h == 0)
    assert f[0] & oracle_mod.F_DEGENERATE and not f[1] & oracle_mod.F_DEGENERATE


def test_invalid_covariance_flagged(oracle_mod):
    st = synth.bumps_map(n=16, n_bumps=3, seed=1)
    q = np.array([[7.0, 7.0, 1.0, 1.0, 1.0, 0.0, 0.0], [7.0, 7.0, -1.0, 0.0, 1.0, 0.0, 0.0]])
    D, f, h, _ = oracle_mod.pndf(st, q)
    assert np.all(np.isnan(D)) and np.all(f & oracle_mod.F_INVALID)


# ---------------------------------------------------------------------------
# (f) projected area
# ---------------------------------------------------------------------------

def _tri_quadrature(n0, n1, n2, w, K=700):
    """Midpoint rule on K^2 sub-triangles of the normal triangle of
    max(m~ . w, 0) / m~_z (Eq. 10, second line)."""
    n0, n1, n2 = map(np.asarray, (n0, n1, n2))
    a = np.arange(K)
    I, J = np.meshgrid(a, a, indexing="ij")
    keep = I + J < K
    I, J = I[keep], J[keep]
    # upright sub-triangles: centroid at (I + 1/3, J + 1/3)/K; inverted: (I + 2/3, J + 2/3)/K (I + J < K - 1)
    cu = np.stack([(I + 1 / 3) / K, (J + 1 / 3) / K], 1)
    inv = I + J < K - 1
    ci = np.stack([(I[inv] + 2 / 3) / K, (J[inv] + 2 / 3) / K], 1)
    c = np.concatenate([cu, ci])
    m = n0[None] + c[:, :1] * (n1 - n0)[None] + c[:, 1:] * (n2 - n0)[None]
    mz = np.sqrt(1 - (m ** 2).sum(1))
    f = np.maximum(m[:, 0] * w[0] + m[:, 1] * w[1] + mz * w[2], 0) / mz
    area = 0.5 * abs((n1[0] - n0[0]) * (n2[1] - n0[1]) - (n1[1] - n0[1]) * (n2[0] - n0[0]))
    return f.mean() * area


def test_stokes_matches_area_quadrature(oracle_mod):
    """Per triangle, the boundary-integral evaluation (Eq. 11 with Alg. 1)
    equals a 2D quadrature of the area integrand over the visible part of the
    normal triangle (App. B, correctness of the area-line conversion)."""
    rng = np.random.default_rng(3)
    checked_clipped = 0
    for k in range(90):
        th = rng.uniform(0.02, np.pi / 2) if k % 3 else rng.uniform(1.2, 1.55)
        ph = rng.uniform(0, 2 * np.pi)
        w = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        if k % 3 == 0:
            # straddle the visibility boundary, which crosses -w_z * w_xy/|w_xy| (App. B)
            c = -w[2] * w[:2] / np.linalg.norm(w[:2]) + rng.uniform(-0.05, 0.05, 2)
        else:
            c = rng.uniform(-0.45, 0.45, 2)
        size = rng.choice([0.02, 0.1, 0.3])
        pts = c[None] + size * rng.uniform(-1, 1, (3, 2))
        pts = np.clip(pts, -0.56, 0.56)
        got = oracle_mod.tri_integral(pts[0], pts[1], pts[2], w)
        ref = _tri_quadrature(pts[0], pts[1], pts[2], w)
        e1, e2 = pts[1] - pts[0], pts[2] - pts[0]
        area = 0.5 * abs(e1[0] * e2[1] - e1[1] * e2[0])
        # full visibility would give the quadrature of (w.m~)/m~_z; count the clipped cases
        m = pts
        vis = m[:, 0] * w[0] + m[:, 1] * w[1] + np.sqrt(1 - (m ** 2).sum(1)) * w[2]
        checked_clipped += int(np.any(vis < 0) and np.any(vis > 0))
        assert abs(got - ref) <= 2e-4 * area + 1e-4 * abs(ref), (k, got, ref, area)
    assert checked_clipped >= 15, checked_clipped


def test_projarea_normal_incidence_is_shoelace(oracle_mod):
    """w = (0, 0, 1): every triangle is fully visible and the integrand is 1,
    so P = sum over footprint triangles of k_r(T) * area / (2 area) = sum k_r(T) / 2."""
    st = synth.bumps_map(n=40, n_bumps=8, seed=3).double().numpy()
    rng = np.random.default_rng(0)
    nq = 20
    q = np.zeros((nq, 7))
    q[:, 0] = rng.uniform(10, 29, nq)
    q[:, 1] = rng.uniform(10, 29, nq)
    q[:, 2] = rng.uniform(1, 5, nq)
    q[:, 4] = rng.uniform(1, 5, nq)
    q[:, 3] = rng.uniform(-0.5, 0.5, nq)
    w = np.tile([0.0, 0.0, 1.0], (nq, 1))
    P = oracle_mod.projarea(st, q, w)
    N = st.shape[0]
    I, J = np.meshgrid(np.arange(N - 1), np.arange(N - 1))
    for k in range(nq):
        tot = 0.0
        for off in (1 / 3, 2 / 3):
            g, _ = gauss(I + off - q[k, 0], J + off - q[k, 1], q[k, 2], q[k, 3], q[k, 4])
            tot += 0.5 * g.sum()
        assert abs(P[k] - tot) <= 1e-12 * tot


def test_projarea_uv_form(oracle_mod):
    """Eq. 13: with k_r constant per triangle, P(w) equals the uv-space
    integral of k_r(T) max(n~(u) . w, 0) / n~_z(u), n(u) from Eq. 3."""
    st = synth.bumps_map(n=24, n_bumps=4, seed=8).double().numpy()
    N = st.shape[0]
    rng = np.random.default_rng(5)
    nq = 6
    q = np.zeros((nq, 7))
    q[:, 0] = rng.uniform(9, 14, nq)
    q[:, 1] = rng.uniform(9, 14, nq)
    q[:, 2] = 4.0
    q[:, 4] = 3.0
    q[:, 3] = 0.7
    th = np.array([0.1, 0.8, 1.3, 1.5, 1.55, 1.2])
    ph = rng.uniform(0, 2 * np.pi, nq)
    w = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    P = oracle_mod.projarea(st, q, w)
    K = 40  # sub-samples per uv axis per quad
    f = (np.arange(K) + 0.5) / K
    U, V = np.meshgrid(f, f, indexing="ij")
    U, V = U.ravel(), V.ravel()
    lower = U + V < 1
    for k in range(nq):
        tot = 0.0
        for j in range(N - 1):
            for i in range(N - 1):
                for tri, sel, off in ((0, lower, 1 / 3), (1, ~lower, 2 / 3)):
                    g, _ = gauss(i + off - q[k, 0], j + off - q[k, 1], q[k, 2], q[k, 3], q[k, 4])
                    if g == 0:
                        continue
                    n = interp_normal(st, i + U[sel], j + V[sel])
                    nz = np.sqrt(1 - (n ** 2).sum(1))
                    val = np.maximum(n[:, 0] * w[k, 0] + n[:, 1] * w[k, 1] + nz * w[k, 2], 0) / nz
                    tot += g * val.sum() / (K * K)
        assert abs(P[k] - tot) <= 2e-3 * tot, (k, P[k], tot)


def test_projarea_uv_form_collapsed_triangles(oracle_mod):
    """Steep bumps clamp |s|, |t| to 0.4, so many normal triangles collapse onto
    segments (exactly zero area); Eq. 13's uv-space integral still fixes their
    contribution, and the oracle must match dense uv quadrature there too."""
    h = synth.bumps_height(20, 3, seed=4, amp=(4.0, 5.0), sig=(2.5, 3.0), noise=0.0)
    st = synth.normals_from_height(h).double().numpy()
    N = st.shape[0]
    n0, n1, n2 = st[:-1, :-1], st[:-1, 1:], st[1:, :-1]
    cr = (n1[..., 0] - n0[..., 0]) * (n2[..., 1] - n0[..., 1]) - (n1[..., 1] - n0[..., 1]) * (n2[..., 0] - n0[..., 0])
    collinear = (np.abs(cr) < 1e-12) & (np.abs(n1 - n0).sum(-1) + np.abs(n2 - n0).sum(-1) > 0.05)
    assert collinear.sum() >= 10, int(collinear.sum())
    q = np.array([[9.5, 9.7, 6.0, 0.5, 5.0, 0, 0], [10.2, 9.1, 3.0, -0.3, 4.0, 0, 0]])
    w = np.array([[0.3, -0.5, math.sqrt(1 - 0.34)], [-0.9, 0.2, math.sqrt(1 - 0.85)]])
    _check_uv_form(oracle_mod, st, q, w, 1e-3)
    # long collapsed segments: s = 0.4 everywhere, t alternating +-0.4, so every
    # normal triangle is a segment of length 0.8
    N = 8
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    st2 = np.stack([np.full((N, N), 0.4), np.where((ii + jj) % 2 == 0, 0.4, -0.4)], -1)
    q2 = np.array([[3.5, 3.5, 1.5, 0.2, 1.2, 0, 0], [3.2, 3.9, 2.5, -0.4, 2.0, 0, 0]])
    w2 = np.array([[0.0, 0.95, math.sqrt(1 - 0.9025)], [-0.6, -0.6, math.sqrt(1 - 0.72)]])
    _check_uv_form(oracle_mod, st2, q2, w2, 1e-3)


def _check_uv_form(oracle_mod, st, q, w, rtol):
    N = st.shape[0]
    P = oracle_mod.projarea(st, q, w)
    K = 60
    f = (np.arange(K) + 0.5) / K
    U, V = np.meshgrid(f, f, indexing="ij")
    U, V = U.ravel(), V.ravel()
    lower = U + V < 1
    for k in range(len(q)):
        tot = 0.0
        for j in range(N - 1):
            for i in range(N - 1):
                for sel, off in ((lower, 1 / 3), (~lower, 2 / 3)):
                    g, _ = gauss(i + off - q[k, 0], j + off - q[k, 1], q[k, 2], q[k, 3], q[k, 4])
                    if g == 0:
                        continue
                    n = interp_normal(st, i + U[sel], j + V[sel])
                    nz = np.sqrt(1 - (n ** 2).sum(1))
                    val = np.maximum(n[:, 0] * w[k, 0] + n[:, 1] * w[k, 1] + nz * w[k, 2], 0) / nz
                    tot += g * val.sum() / (K * K)
        assert abs(P[k] - tot) <= rtol * tot, (k, P[k], tot)


# ---------------------------------------------------------------------------
# disk and box footprint kernels (kernel ablation: (3 sigma)^2 footprints)
# ---------------------------------------------------------------------------

def support_weight(kernel, dx, dy, sxx, sxy, syy):
    """Disk / box kernel from their definitions by library routines: the disk
    is q = d^T S^-1 d <= 1.5^2 (numpy solve), the box |L^-1 d|_inf <= 1.5 with
    L = numpy's Cholesky factor; each normalised by its support's area."""
    out = np.zeros(len(dx))
    for k in range(len(dx)):
        S = np.array([[sxx[k], sxy[k]], [sxy[k], syy[k]]])
        d = np.array([dx[k], dy[k]])
        if kernel == 1:
            inside = d @ np.linalg.solve(S, d) <= 2.25
            area = np.pi * 2.25 * math.sqrt(np.linalg.det(S))
        else:
            v = np.linalg.solve(np.linalg.cholesky(S), d)
            inside = np.abs(v).max() <= 1.5
            area = 9.0 * math.sqrt(np.linalg.det(S))
        out[k] = 1.0 / area if inside else 0.0
    return out


@pytest.mark.parametrize("kernel", [1, 2])
def test_affine_closed_form_disk_box(oracle_mod, kernel):
    """Affine field, disk and box kernels: D = k(u* - x) / |det M| (Eq. 2)."""
    st, q = _affine_cases(11)
    q[:, 2:5] *= 4.0  # larger footprints so preimages land inside and outside the support
    D, flags, hits, _ = oracle_mod.pndf(st, q, kernel=kernel)
    M = np.asarray(AFF_M)
    ustar = np.linalg.solve(M[None, :, :], (q[:, 5:7] - np.asarray(AFF_N0)[None, :])[:, :, None])[:, :, 0]
    N = st.shape[0]
    inside = np.all((ustar > 0) & (ustar < N - 1), axis=1)
    w = support_weight(kernel, ustar[:, 0] - q[:, 0], ustar[:, 1] - q[:, 1], q[:, 2], q[:, 3], q[:, 4])
    expect = np.where(inside, w / abs(np.linalg.det(M)), 0.0)
    ok = (flags & oracle_mod.F_EXCLUDE) == 0
    assert ok.sum() > 0.95 * len(q)
    assert np.any(expect[ok] > 0) and np.any(expect[ok] == 0)
    np.testing.assert_allclose(D[ok], expect[ok], rtol=1e-12, atol=0)


def _mass_estimate_kernel(oracle_mod, st, x, y, S, kernel, res, seed):
    rng = np.random.default_rng(seed)
    N = st.shape[0]
    r = 4 * math.sqrt(max(S[0], S[2]))
    i0, i1 = int(max(0, math.floor(x - r) - 1)), int(min(N - 1, math.ceil(x + r) + 1))
    j0, j1 = int(max(0, math.floor(y - r) - 1)), int(min(N - 1, math.ceil(y + r) + 1))
    sub = st[j0:j1 + 1, i0:i1 + 1].reshape(-1, 2)
    lo, hi = sub.min(0) - 1e-3, sub.max(0) + 1e-3
    h = (hi - lo) / res
    off = rng.uniform(0, 1, 2)
    mx, my = np.meshgrid(lo[0] + (np.arange(res) + off[0]) * h[0], lo[1] + (np.arange(res) + off[1]) * h[1])
    q = np.zeros((mx.size, 7))
    q[:, 0], q[:, 1], q[:, 2], q[:, 3], q[:, 4] = x, y, S[0], S[1], S[2]
    q[:, 5], q[:, 6] = mx.ravel(), my.ravel()
    D, *_ = oracle_mod.pndf(st, q, kernel=kernel)
    return D.sum() * h[0] * h[1]


@pytest.mark.parametrize("kernel", [1, 2])
def test_mass_invariant_disk_box(oracle_mod, kernel):
    """The disk and box kernels are normalised with no truncation: D
    integrates to exactly 1 over the normal plane (change of variables per
    triangle, Eq. 2), for an anisotropic, correlated S."""
    st = synth.normals_from_height(synth.bumps_height(40, 6, seed=11, noise=0.0, sig=(3.0, 6.0))).double().numpy()
    S = (9.0, 3.0, 5.0)
    e_coarse = abs(_mass_estimate_kernel(oracle_mod, st, 19.5, 19.25, S, kernel, 200, 1) - 1.0)
    e_fine = abs(_mass_estimate_kernel(oracle_mod, st, 19.5, 19.25, S, kernel, 700, 2) - 1.0)
    assert e_fine < 0.01, (e_coarse, e_fine)
    assert e_fine < e_coarse or e_fine < 2e-3


def test_binning_box_kernel(oracle_mod):
    """Binning with the box kernel and a correlated S: uv samples uniform in
    the sheared square L [-1.5, 1.5]^2 (numpy's Cholesky factor), binned in m,
    converge to the bin-integrated D."""
    st = synth.normals_from_height(synth.bumps_height(32, 5, seed=5, noise=0.0, sig=(3.0, 8.0))).double().numpy()
    x, y, S = 15.5, 15.5, np.array([[6.0, 2.5], [2.5, 3.0]])
    L = np.linalg.cholesky(S)

    def l1(nsamp, seed, sub):
        rng = np.random.default_rng(seed)
        k = int(math.sqrt(nsamp))
        v = np.stack([((np.arange(k)[None, :] + rng.uniform(0, 1, (k, k))) / k).ravel(),
                      ((np.arange(k)[:, None] + rng.uniform(0, 1, (k, k))) / k).ravel()], 1) * 3.0 - 1.5
        u = v @ L.T + np.array([x, y])
        w = np.full(len(u), 1.0 / len(u))  # uniform density over the support, total mass 1
        n = interp_normal(st, u[:, 0], u[:, 1])
        lo, hi = n.min(0), n.max(0)
        nb = 16
        ex, ey = np.linspace(lo[0], hi[0], nb + 1), np.linspace(lo[1], hi[1], nb + 1)
        hist, _, _ = np.histogram2d(n[:, 0], n[:, 1], bins=[ex, ey], weights=w)
        bx, by = ex[1] - ex[0], ey[1] - ey[0]
        fx = (np.arange(nb * sub) + rng.uniform(0, 1, nb * sub)) / sub
        fy = (np.arange(nb * sub) + rng.uniform(0, 1, nb * sub)) / sub
        mx, my = np.meshgrid(ex[0] + fx * bx, ey[0] + fy * by, indexing="ij")
        q = np.zeros((mx.size, 7))
        q[:, 0], q[:, 1], q[:, 2], q[:, 3], q[:, 4] = x, y, S[0, 0], S[0, 1], S[1, 1]
        q[:, 5], q[:, 6] = mx.ravel(), my.ravel()
        D, *_ = oracle_mod.pndf(st, q, kernel=2)
        Dm = D.reshape(nb, sub, nb, sub).mean(axis=(1, 3)) * bx * by
        return np.abs(Dm - hist).sum() / hist.sum()

    small, big = l1(250_000, 1, 8), l1(4_000_000, 2, 48)
    assert big < 0.01, (small, big)
    assert big < 0.5 * small
