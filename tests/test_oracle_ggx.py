"""Pins for the GGX projected-area fit per mip node (Eq. 12) and the
shadow-masking term (Sec. 4.3).

Independent routes: a fit fed projected areas of a known GGX Omega returns
it; a flat map has P(w) = w_z and Omega = 0; a node's box-filtered P equals
uv-space quadrature of Eq. 13 (sub-triangle centroids of the Eq. 3
interpolation); Lambda for a uniform isotropic Omega = alpha^2 I equals the
textbook GGX Smith Lambda (-1 + sqrt(1 + alpha^2 tan^2 theta)) / 2;
interpolation properties (constants and linear fields reproduced, level
blends between the two levels' values); G = 1 for a flat, fully lit surface.
"""

import math

import numpy as np
import pytest

from paper_2505_08985_gb300 import synth
from test_oracle_pins import interp_normal


def layout(N):
    import oracle
    return oracle.ClusterFits(N)


def unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def test_fit_recovers_a_ggx_omega(oracle_mod):
    """P sampled from P'(w) = (w_z + sqrt(w_z^2 + w^T Omega w)) / 2 of a known
    anisotropic, rotated Omega: the least-squares fit returns Omega."""
    dirs = oracle_mod.ggx_dirs()
    O0 = np.array([0.09, -0.025, 0.04])
    q = O0[0] * dirs[:, 0] ** 2 + 2 * O0[1] * dirs[:, 0] * dirs[:, 1] + O0[2] * dirs[:, 1] ** 2
    P = 0.5 * (dirs[:, 2] + np.sqrt(dirs[:, 2] ** 2 + q))
    np.testing.assert_allclose(oracle_mod.ggx_fit(P, dirs), O0, rtol=0, atol=1e-13)


def test_flat_map_has_zero_omega(oracle_mod):
    """All normals vertical: P(w) = w_z for every node, Omega = 0."""
    st = np.zeros((33, 33, 2))
    O = oracle_mod.ggx_fits(st)
    ok = np.isfinite(O[:, 0])
    assert ok.sum() > 0
    np.testing.assert_allclose(O[ok], 0.0, atol=1e-14)
    P = oracle_mod.ggx_node_P(st, 3, 1, 2)
    np.testing.assert_allclose(P, oracle_mod.ggx_dirs()[:, 2], rtol=1e-14)


def _uv_quadrature_P(st, l, I, J, w, K):
    """4^-l times the integral over the node's uv square of max(n~.w, 0)/n~_z
    (Eq. 13 with the box filter), K^2 sub-triangle centroids per triangle."""
    pts = []
    for a in range(K):
        for b in range(K - a):
            pts.append(((a + 1 / 3) / K, (b + 1 / 3) / K))
            if a + b <= K - 2:
                pts.append(((a + 2 / 3) / K, (b + 2 / 3) / K))
    P = np.asarray(pts)
    s = 1 << l
    tot = 0.0
    for j in range(s * J, s * J + s):
        for i in range(s * I, s * I + s):
            for tri in range(2):
                u, v = (P[:, 0], P[:, 1]) if tri == 0 else (1 - P[:, 0], 1 - P[:, 1])
                n = interp_normal(st, i + u, j + v)
                nz = np.sqrt(1 - (n ** 2).sum(1))
                tot += (np.maximum(n[:, 0] * w[0] + n[:, 1] * w[1] + nz * w[2], 0) / nz).sum() / (2 * K * K)
    return tot / (s * s)


@pytest.mark.parametrize("wz", [0.3, 0.08])
def test_node_P_matches_uv_quadrature(oracle_mod, wz):
    """The box-filtered projected area of a node (Eq. 9-11 per triangle,
    including partly shadowed triangles at grazing light) equals uv-space
    quadrature of Eq. 13; the gap shrinks as the quadrature is refined."""
    st = synth.normals_from_height(synth.bumps_height(40, 6, seed=13, noise=0.0, sig=(3.0, 8.0))).double().numpy()
    dirs = unit([[math.sqrt(1 - wz * wz) * math.cos(p), math.sqrt(1 - wz * wz) * math.sin(p), wz]
                 for p in (0.3, 2.1, 4.0)])
    P = oracle_mod.ggx_node_P(st, 2, 3, 5, dirs)
    e = []
    for K in (6, 24):
        Q = np.array([_uv_quadrature_P(st, 2, 3, 5, w, K) for w in dirs])
        e.append(np.abs(Q - P).max() / P.max())
    assert e[1] < 2e-3 and e[1] < 0.5 * e[0], e


def test_lambda_is_ggx_smith_for_isotropic_omega(oracle_mod):
    """With Omega = alpha^2 I at every node, Lambda'(w) is the GGX Smith
    Lambda, (-1 + sqrt(1 + alpha^2 tan^2 theta)) / 2, at any footprint."""
    N = 65
    lay = layout(N)
    a2 = 0.07
    O = np.zeros((lay.c.shape[0], 3))
    O[:, 0] = O[:, 2] = a2
    rng = np.random.default_rng(3)
    n = 500
    th = rng.uniform(0.05, 1.45, n)
    ph = rng.uniform(0, 2 * np.pi, n)
    w = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    q = np.zeros((n, 7))
    q[:, 0:2] = rng.uniform(0, N - 1, (n, 2))
    q[:, 2] = q[:, 4] = rng.uniform(0.5, 20.0, n) ** 2
    lam = oracle_mod.ggx_lambda(O, N, q, w)
    expect = 0.5 * (-1 + np.sqrt(1 + a2 * np.tan(th) ** 2))
    np.testing.assert_allclose(lam, expect, rtol=1e-12, atol=1e-14)


def test_interpolation_properties(oracle_mod):
    """A field linear in the node centre at every level is reproduced inside
    the map; a footprint between two levels gets Omega between theirs."""
    N = 129
    lay = layout(N)
    O = np.full((lay.c.shape[0], 3), np.nan)
    for l in range(2, lay.L + 1):
        S = 1 << (lay.L - l)
        a = 1 << l
        J, I = np.meshgrid(np.arange(S), np.arange(S), indexing="ij")
        cx, cy = (I + 0.5) * a, (J + 0.5) * a
        o = lay.offsets[l]
        O[o:o + S * S, 0] = (0.01 + 1e-4 * cx + 2e-4 * cy).ravel()
        O[o:o + S * S, 1] = 0.0
        O[o:o + S * S, 2] = (0.02 + 0.003 * l) * np.ones(S * S)
    w = unit([[0.6, 0.0, 0.8]])
    for x, y, sig in ((40.3, 51.7, 1.6), (70.0, 33.0, 3.0), (64.0, 64.0, 5.5)):
        q = np.array([[x, y, sig * sig, 0.0, sig * sig, 0.0, 0.0]])
        lam = oracle_mod.ggx_lambda(O, N, q, w)[0]
        Oxx = 0.01 + 1e-4 * x + 2e-4 * y
        P = 0.5 * (w[0, 2] + math.sqrt(w[0, 2] ** 2 + Oxx * w[0, 0] ** 2))
        assert abs(lam - (P / w[0, 2] - 1)) < 1e-12  # O_yy does not enter along x
    # level blend: along y only O_yy (level-dependent) enters
    wy = unit([[0.0, 0.6, 0.8]])
    lams = []
    for sig in (1.2, 1.5, 2.5, 4.0, 7.0):
        q = np.array([[64.0, 64.0, sig * sig, 0.0, sig * sig, 0.0, 0.0]])
        lams.append(oracle_mod.ggx_lambda(O, N, q, wy)[0])
    assert np.all(np.diff(lams) > 0)  # larger footprints use higher (rougher) levels, blended continuously


def test_shadow_masking_flat_and_backfacing(oracle_mod):
    N = 33
    lay = layout(N)
    O = np.zeros((lay.c.shape[0], 3))
    q = np.array([[16.0, 16.0, 4.0, 0.0, 4.0, 0.05, -0.02]] * 3)
    wi = unit([[0.3, 0.1, 0.9], [0.3, 0.1, 0.9], [-0.999, 0.0, 0.02]])
    wo = unit([[-0.2, 0.4, 0.8], [0.1, -0.2, 0.95], [0.0, 0.0, 1.0]])
    G = oracle_mod.shadow_masking(O, N, q, wi, wo)
    np.testing.assert_allclose(G[:2], 1.0, rtol=1e-14)
    assert G[2] == 0.0  # light below the facet normal
