"""Pins for the Jacobian clamp of Eq. 6 and for P-NDF sampling (Sec. 3).

Expected values by other routes than the oracle's: the kernel mass recovered
by integrating D over the normal plane (the clamp keeps the mass of
zero-area triangles, which the exact P-NDF drops), per-triangle sample
frequencies against this file's own quadrature of the kernel over each uv
triangle, sampled normals lying in their triangle's normal image (or its
equilateral replacement), and the binned samples matching D.
"""

import math

import numpy as np
import pytest

from test_oracle_pins import gauss

EPS = 1e-6
N0 = np.array([0.125, -0.0625])
M = np.array([[0.02, 0.004], [-0.006, 0.018]])


def plateau_ramp(N=40, edge=16):
    """Flat at N0 for i <= edge, then linear: n = N0 + M (i - edge, j - j0)
    continuing from the plateau (zero-area triangles on the flat half)."""
    st = np.zeros((N, N, 2))
    for j in range(N):
        for i in range(N):
            d = np.array([max(i - edge, 0), 0.0]) if i <= edge else np.array([i - edge, (j - N / 2) * 0.5])
            st[j, i] = N0 + M @ d if i > edge else N0
    return st


def test_clamp_keeps_the_mass_of_flat_triangles(oracle_mod):
    """With the clamp every triangle, flat ones included, maps its uv area
    onto the normal plane with Jacobian max(|cross|, eps): D integrates to
    the kernel mass 1 - e^-8; without it the flat half's mass is lost."""
    st = plateau_ramp()
    x, y, s2 = 16.5, 20.25, 4.0
    rng = np.random.default_rng(1)

    def grid(lo, hi, res, skip=None):
        off = rng.uniform(0, 1, 2)
        h = (hi - lo) / res
        mx, my = np.meshgrid(lo[0] + (np.arange(res) + off[0]) * h[0], lo[1] + (np.arange(res) + off[1]) * h[1])
        mx, my = mx.ravel(), my.ravel()
        if skip is not None:
            keep = ~((mx >= skip[0][0]) & (mx < skip[1][0]) & (my >= skip[0][1]) & (my < skip[1][1]))
            mx, my = mx[keep], my[keep]
        q = np.zeros((mx.size, 7))
        q[:, 0], q[:, 1], q[:, 2], q[:, 4], q[:, 5], q[:, 6] = x, y, s2, s2, mx, my
        return q, h[0] * h[1]

    # the flat triangles' replacements all sit on N0 (radius about 6.2e-4): a
    # fine grid there, a coarse one elsewhere
    spike = (N0 - 8e-4, N0 + 8e-4)
    lo = st.reshape(-1, 2).min(0) - 2e-3
    hi = st[12:30, 8:26].reshape(-1, 2).max(0) + 2e-3
    qc, ac = grid(lo, hi, 1000, skip=spike)
    qf, af = grid(spike[0], spike[1], 500)
    mass = {}
    for name, eps in (("clamp", EPS), ("exact", 0.0)):
        mass[name] = oracle_mod.pndf(st, qc, jac_eps=eps)[0].sum() * ac + oracle_mod.pndf(st, qf, jac_eps=eps)[0].sum() * af
    mass_c, mass_e = mass["clamp"], mass["exact"]
    target = 1.0 - math.exp(-8.0)
    assert abs(mass_c - target) < 0.01 * target, (mass_c, mass_e)
    assert mass_e < 0.7 * target  # the plateau's mass is gone without the clamp


def test_clamp_only_touches_small_jacobians(oracle_mod):
    """On a map whose triangles all have |cross| >= eps the clamp changes nothing."""
    from paper_2505_08985_gb300 import synth
    st = synth.normals_from_height(synth.bumps_height(32, 5, seed=5, noise=0.0, sig=(3.0, 8.0))).double().numpy()
    q = synth.make_queries(synth.bumps_map(n=32, n_bumps=5, seed=5), 400, synth.QueryMix(sigma=(1.0, 3.0)), 2)
    q = q.double().numpy()
    q[:, 0:2] = np.clip(q[:, 0:2], 12, 19)
    D0, f0, h0, hh0 = oracle_mod.pndf(st, q)
    D1, f1, h1, hh1 = oracle_mod.pndf(st, q, jac_eps=1e-12)
    np.testing.assert_array_equal(D0, D1)
    assert np.array_equal(hh0, hh1)


def _tri_masses(st, x, y, S, K=24):
    """This file's own quadrature of the 4-sigma-cut Gaussian over every uv
    triangle near the footprint (K^2 sub-triangle centroids per triangle)."""
    N = st.shape[0]
    a = np.arange(K)
    pts = []
    for i in range(K):
        for j in range(K - i):
            pts.append(((i + 1 / 3) / K, (j + 1 / 3) / K))
            if i + j <= K - 2:
                pts.append(((i + 2 / 3) / K, (j + 2 / 3) / K))
    P = np.asarray(pts)
    w = 1.0 / (2 * K * K)
    out = {}
    r = 4 * math.sqrt(max(S[0], S[2]))
    for j in range(max(0, int(y - r) - 1), min(N - 2, int(y + r) + 1) + 1):
        for i in range(max(0, int(x - r) - 1), min(N - 2, int(x + r) + 1) + 1):
            for tri in range(2):
                u, v = (P[:, 0], P[:, 1]) if tri == 0 else (1 - P[:, 0], 1 - P[:, 1])
                g, _ = gauss(i + u - x, j + v - y, S[0], S[1], S[2])
                mass = g.sum() * w
                if mass > 0:
                    out[2 * (j * (N - 1) + i) + tri] = mass
    return out


def test_sample_frequencies_follow_the_kernel(oracle_mod):
    """Samples fall in each uv triangle with probability (kernel mass over
    the triangle) / (total mass): chi-square against an independent
    quadrature, for a correlated S."""
    from paper_2505_08985_gb300 import synth
    st = synth.normals_from_height(synth.bumps_height(32, 5, seed=5, noise=0.0, sig=(3.0, 8.0))).double().numpy()
    x, y, S = 15.3, 16.1, (2.0, 0.7, 1.2)
    n = 400_000
    q = np.tile([x, y, S[0], S[1], S[2], 0.0, 0.0], (n, 1))
    U = np.random.default_rng(7).uniform(size=(n, 2))
    m, tri, flags = oracle_mod.sample(st, q, U)
    assert (flags & oracle_mod.F_OUTSIDE).sum() == 0
    masses = _tri_masses(st, x, y, S)
    total = sum(masses.values())
    ids, counts = np.unique(tri, return_counts=True)
    got = dict(zip(ids.tolist(), counts.tolist()))
    assert set(got) <= set(masses)
    exp = np.array([n * masses[t] / total for t in masses])
    obs = np.array([got.get(t, 0) for t in masses])
    keep = exp > 20
    chi2 = (((obs - exp) ** 2) / exp)[keep].sum()
    dof = keep.sum() - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof), (chi2, dof)


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_samples_lie_on_their_triangles(oracle_mod, kernel):
    """Each sampled m lies in the closed normal triangle it came from (or its
    equilateral replacement)."""
    st = plateau_ramp()
    n = 20000
    q = np.tile([20.0, 20.5, 5.0, 1.0, 3.0, 0.0, 0.0], (n, 1))
    U = np.random.default_rng(kernel).uniform(size=(n, 2))
    m, tri, flags = oracle_mod.sample(st, q, U, kernel=kernel, jac_eps=EPS)
    assert (tri >= 0).all()
    N = st.shape[0]
    side = math.sqrt(2 * EPS / math.sqrt(3))
    for k in range(0, n, 7):
        t = tri[k]
        qd, which = divmod(int(t), 2)
        j, i = divmod(qd, N - 1)
        vs = [(i, j), (i + 1, j), (i, j + 1)] if which == 0 else [(i + 1, j + 1), (i, j + 1), (i + 1, j)]
        nv = np.array([st[b, a] for a, b in vs])
        cr = (nv[1, 0] - nv[0, 0]) * (nv[2, 1] - nv[0, 1]) - (nv[1, 1] - nv[0, 1]) * (nv[2, 0] - nv[0, 0])
        if abs(cr) < EPS:  # the replacement: within its circumradius of the centroid
            assert np.linalg.norm(m[k] - nv.mean(0)) <= side / math.sqrt(3) * (1 + 1e-9)
        else:  # barycentric coordinates of m in n(T) are all >= 0
            lam = np.linalg.solve(np.vstack([nv.T, np.ones(3)]), np.append(m[k], 1.0))
            assert lam.min() >= -1e-9, lam


def test_binned_samples_match_clamped_pndf(oracle_mod):
    """Histogram of sampled normals (plateau + ramp map, clamp on) converges
    to the bin-integrated clamped D / kernel mass: sampling and evaluation
    are consistent, including the replaced flat triangles."""
    st = plateau_ramp()
    x, y, s2 = 17.5, 20.25, 2.25
    target = 1.0 - math.exp(-8.0)

    def l1(n, seed, sub):
        q = np.tile([x, y, s2, 0.0, s2, 0.0, 0.0], (n, 1))
        U = np.random.default_rng(seed).uniform(size=(n, 2))
        m, tri, flags = oracle_mod.sample(st, q, U, jac_eps=EPS)
        lo, hi = m.min(0) - 1e-6, m.max(0) + 1e-6
        nb = 12
        ex, ey = np.linspace(lo[0], hi[0], nb + 1), np.linspace(lo[1], hi[1], nb + 1)
        hist, _, _ = np.histogram2d(m[:, 0], m[:, 1], bins=[ex, ey])
        hist /= n
        bx, by = ex[1] - ex[0], ey[1] - ey[0]
        rng = np.random.default_rng(seed + 1)
        fx = (np.arange(nb * sub) + rng.uniform(0, 1, nb * sub)) / sub
        fy = (np.arange(nb * sub) + rng.uniform(0, 1, nb * sub)) / sub
        mx, my = np.meshgrid(ex[0] + fx * bx, ey[0] + fy * by, indexing="ij")
        qq = np.zeros((mx.size, 7))
        qq[:, 0], qq[:, 1], qq[:, 2], qq[:, 4], qq[:, 5], qq[:, 6] = x, y, s2, s2, mx.ravel(), my.ravel()
        D, *_ = oracle_mod.pndf(st, qq, jac_eps=EPS)
        Dm = D.reshape(nb, sub, nb, sub).mean(axis=(1, 3)) * bx * by / target
        return np.abs(Dm - hist).sum()

    small, big = l1(40_000, 1, 24), l1(1_000_000, 2, 96)
    assert big < 0.02, (small, big)
    assert big < 0.6 * small
