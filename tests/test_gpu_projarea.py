"""GPU parity of pndf_diffuse_projected_area against the FP64 oracle (Eq. 10-11, Alg. 1)."""

import math

import numpy as np
import pytest
import torch

import oracle
from paper_2505_08985_gb300 import synth
from parity import rel_err

pytestmark = pytest.mark.gpu
DEV = "cuda"
RTOL = 1e-4


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_08985_gb300 import pndf
    return pndf


def dirs(nq, seed, grazing=False):
    rng = np.random.default_rng(seed)
    th = rng.uniform(1.2, 1.5695, nq) if grazing else np.arccos(rng.uniform(1e-3, 1.0, nq))
    ph = rng.uniform(0, 2 * np.pi, nq)
    w = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    return torch.from_numpy(w.astype(np.float32))


def grazing_dirs(nq, seed, wz=(0.01, 0.1)):
    """Unit directions with w_z uniform in wz (light near the horizon)."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(wz[0], wz[1], nq)
    ph = rng.uniform(0, 2 * np.pi, nq)
    r = np.sqrt(1 - z * z)
    return torch.from_numpy(np.stack([r * np.cos(ph), r * np.sin(ph), z], 1).astype(np.float32))


def general_path_fraction(st, q, w):
    """Share of the footprint triangles (uv centroid inside the 4-sigma
    ellipse) that are partly visible (some vertex sees w, another does not)
    or whose normals collapsed onto a segment (|cross| < 1e-12), over all
    requests: the triangles that take the general FP64 path."""
    st = np.asarray(st, np.float64)
    q = np.asarray(q, np.float64)
    w = np.asarray(w, np.float64)
    w = w / np.linalg.norm(w, axis=1, keepdims=True)
    N = st.shape[0]
    tot = slow = 0
    for k in range(q.shape[0]):
        x, y, sxx, sxy, syy = q[k, :5]
        det = sxx * syy - sxy * sxy
        i0, i1 = max(int(np.floor(x - 4 * np.sqrt(sxx))) - 1, 0), min(int(np.ceil(x + 4 * np.sqrt(sxx))), N - 2)
        j0, j1 = max(int(np.floor(y - 4 * np.sqrt(syy))) - 1, 0), min(int(np.ceil(y + 4 * np.sqrt(syy))), N - 2)
        if i0 > i1 or j0 > j1:
            continue
        J, I = np.meshgrid(np.arange(j0, j1 + 1), np.arange(i0, i1 + 1), indexing="ij")
        n0, n1, n2, n3 = st[J, I], st[J, I + 1], st[J + 1, I], st[J + 1, I + 1]
        for a, b, c, off in ((n0, n1, n2, 1 / 3), (n3, n2, n1, 2 / 3)):
            dx, dy = I + off - x, J + off - y
            inside = (syy * dx * dx - 2 * sxy * dx * dy + sxx * dy * dy) / det <= 16
            cr = (b[..., 0] - a[..., 0]) * (c[..., 1] - a[..., 1]) - (b[..., 1] - a[..., 1]) * (c[..., 0] - a[..., 0])

            def sees(n):
                return n[..., 0] * w[k, 0] + n[..., 1] * w[k, 1] + np.sqrt(1 - (n ** 2).sum(-1)) * w[k, 2] >= 0

            nv = sees(a).astype(int) + sees(b) + sees(c)
            gen = (np.abs(cr) < 1e-12) | ((nv > 0) & (nv < 3))
            tot += int(inside.sum())
            slow += int((gen & inside).sum())
    return slow / max(tot, 1)


def run(P, st, q, w):
    h = P.pndf_build_hierarchy(st.to(DEV))
    Pv = P.pndf_diffuse_projected_area(h, q.to(DEV), w.to(DEV)).cpu().double().numpy()
    h.free()
    return Pv


@pytest.mark.parametrize("grazing", [False, True])
def test_bumps256(P, grazing):
    st = synth.bumps_map(n=256, n_bumps=64, seed=1)
    q = synth.make_queries(st, 1500, synth.QueryMix(sigma=(1.0, 8.0), aspect=(1.0, 3.0)), 21)
    w = dirs(1500, 3, grazing)
    got = run(P, st, q, w)
    ref = oracle.projarea(st, q, w)
    r = rel_err(got, ref)
    assert r.max() <= RTOL, (r.max(), int(np.argmax(r)))


def test_scratch_fp16_map_and_borders(P):
    """Binary16 map with steep grooves (many partially visible triangles at
    grazing light), footprints over the border."""
    st = synth.scratch_map(n=300, n_grooves=80, seed=6).half()
    mix = synth.QueryMix(sigma=(0.6, 24.0), aspect=(1.0, 4.0), centre_margin=-20)
    q = synth.make_queries(st.float(), 800, mix, 6)
    w = torch.cat([dirs(400, 4, False), dirs(400, 5, True)])
    got = run(P, st, q, w)
    ref = oracle.projarea(st.float(), q, w)
    r = rel_err(got, ref)
    assert r.max() <= RTOL, (r.max(), int(np.argmax(r)))


@pytest.mark.parametrize("fmt", ["f32", "f16"])
def test_general_path_heavy_noise(P, fmt):
    """Light near the horizon (w_z in [0.01, 0.1]) over a map of independent
    per-texel normals N(0, 0.3^2) clamped to |s|, |t| <= 0.4: more than half
    of the footprint triangles are partly visible or collapsed, so the
    general FP64 path (clip, corner fan, chord and arc excesses, collapsed
    segments) carries most of P."""
    rng = np.random.default_rng(11)
    st = torch.from_numpy(np.clip(rng.normal(0.0, 0.3, (96, 96, 2)), -0.4, 0.4).astype(np.float32))
    if fmt == "f16":
        st = st.half()
    stf = st.float()
    q = synth.make_queries(stf, 300, synth.QueryMix(sigma=(0.8, 6.0), aspect=(1.0, 3.0)), 12)
    w = grazing_dirs(300, 13)
    assert general_path_fraction(stf.numpy(), q.numpy(), w.numpy()) > 0.5
    got = run(P, st, q, w)
    ref = oracle.projarea(stf, q, w)
    r = rel_err(got, ref)
    assert r.max() <= RTOL, (r.max(), int(np.argmax(r)))


def test_general_path_heavy_clamped_bumps(P):
    """Steep bumps clamped to |s|, |t| <= 0.4 (plateaus where whole quads
    collapse onto segments of the clamp boundary) under grazing light: more
    than half of the footprint triangles collapsed or partly visible."""
    h = synth.bumps_height(128, 200, seed=4, amp=(6.0, 12.0), sig=(1.5, 3.0), noise=0.05)
    st = synth.normals_from_height(h)
    q = synth.make_queries(st, 300, synth.QueryMix(sigma=(1.0, 8.0), aspect=(1.0, 3.0)), 14)
    w = grazing_dirs(300, 15, wz=(0.01, 0.2))
    assert general_path_fraction(st.numpy(), q.numpy(), w.numpy()) > 0.5
    got = run(P, st, q, w)
    ref = oracle.projarea(st, q, w)
    r = rel_err(got, ref)
    assert r.max() <= RTOL, (r.max(), int(np.argmax(r)))


def test_normal_incidence_equals_half_kernel_mass(P):
    """w = (0, 0, 1): P = sum_T k_r(T) / 2 (every triangle visible, integrand 1)."""
    st = synth.flake_normals(128, 60, seed=2)
    q = synth.make_queries(st, 200, synth.QueryMix(sigma=(1.0, 10.0), aspect=(1.0, 2.0)), 2)
    w = torch.tensor([[0.0, 0.0, 1.0]]).repeat(200, 1)
    got = run(P, st, q, w)
    ref = oracle.projarea(st, q, w)
    assert rel_err(got, ref).max() <= RTOL


def test_empty_and_invalid(P):
    st = synth.bumps_map(n=64, n_bumps=4, seed=2)
    h = P.pndf_build_hierarchy(st.to(DEV))
    out = P.pndf_diffuse_projected_area(h, torch.zeros(0, 8, device=DEV), torch.zeros(0, 3, device=DEV))
    assert out.shape == (0,)
    q = synth.make_queries(st, 4, synth.QueryMix(sigma=(3.0, 3.0)), 2)
    q[2, 4] = 0.0
    Pv = P.pndf_diffuse_projected_area(h, q.to(DEV), dirs(4, 1).to(DEV)).cpu().numpy()
    assert np.isnan(Pv[2]) and np.isfinite(Pv[[0, 1, 3]]).all()
    assert P.pndf_device_status() & P.PNDF_QF_INVALID
    h.free()


def test_mixed16384_fp16_sampled(P):
    """The 16384^2 binary16 mixed map: a sample of projected-area requests
    (sigma 1..1024 log-uniform, light uniform on the hemisphere) against the oracle."""
    cfg = synth.MIXED_16384
    st = synth.mixed_map(n=cfg["n"], seed=cfg["seed"], device=DEV).half()
    rng = np.random.default_rng(3)
    q = synth.make_queries(st.float(), 4096, cfg["mix"], cfg["seed"])
    sig = torch.sqrt(q[:, 2]).cpu().numpy()
    # the oracle is brute force: keep the sample's total footprint area bounded
    edges = np.exp(np.linspace(0, math.log(1024), 6))
    idx = []
    for a, b in zip(edges[:-1], edges[1:]):
        cand = np.flatnonzero((sig >= a) & (sig < b))
        idx.append(rng.choice(cand, size=min(8 if b > 200 else 20, cand.size), replace=False))
    idx = np.sort(np.concatenate(idx))
    w = synth.hemisphere_dirs(4096, seed=cfg["seed"])
    h = P.pndf_build_hierarchy(st)
    got = P.pndf_diffuse_projected_area(h, q, w.to(DEV)).cpu().double().numpy()
    h.free()
    ref = oracle.projarea(st.cpu().float(), q.cpu()[idx], w[idx])
    r = rel_err(got[idx], ref)
    assert r.max() <= RTOL, (r.max(), idx[int(np.argmax(r))])
    assert np.isfinite(got).all()
