"""GPU parity of the Jacobian clamp of Eq. 6 and of P-NDF sampling (Sec. 3)
with the FP64 oracle, through the C ABI.

Sampling is compared sample by sample on the same uniforms: the triangle each
uv point falls in, and the sampled normal to FP32 output precision (samples
whose uv point is within 1e-9 texel of a quad or diagonal edge, a tie, are
excluded and counted).  The clamped P-NDF is held to the per-query bar of the
exact path.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2505_08985_gb300 import synth
from parity import check_pndf
from test_oracle_sampling import plateau_ramp

pytestmark = pytest.mark.gpu
DEV = "cuda"
EPS = float(np.float32(1e-6))  # the value the GPU receives


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_08985_gb300 import pndf
    return pndf


def clamped_flakes():
    """Flakes whose normals are clamped to [-0.1, 0.1]^2 have whole cells of
    exactly equal texels: zero-area triangles next to normal ones."""
    st = synth.flake_normals(512, 1500, seed=31, texel_noise=0.0)
    return st.clamp(-0.1, 0.1)


@pytest.mark.parametrize("name", ["plateau_ramp", "clamped_flakes", "scratch512"])
def test_clamped_pndf_matches_oracle(P, name):
    st = {"plateau_ramp": lambda: torch.as_tensor(plateau_ramp(), dtype=torch.float32),
          "clamped_flakes": clamped_flakes,
          "scratch512": lambda: synth.scratch_map(n=512, n_grooves=120, seed=22)}[name]()
    n = st.shape[0]
    mix = synth.QueryMix(sigma=(0.8, min(12.0, n / 12)), aspect=(1.0, 3.0), frac_near=0.9,
                         centre_margin=min(14, n // 3))
    # half the normals within the replacements' radius (about 6.2e-4) of a texel normal
    q = torch.cat([synth.make_queries(st, 1500, mix, 3),
                   synth.make_queries(st, 1500, synth.QueryMix(sigma=mix.sigma, aspect=mix.aspect, frac_near=1.0,
                                                               near_noise=3e-4, centre_margin=mix.centre_margin), 4)])
    ref = oracle.pndf(st, q, jac_eps=EPS)
    for bf in (0, 1):
        h = P.pndf_build_hierarchy(st.to(DEV), bounds_fmt=bf)
        stt = torch.zeros(q.shape[0], P.STATS_FIELDS, dtype=torch.int32, device=DEV)
        D = P.pndf_eval_batch_ex(h, q.to(DEV), stats=stt, jac_eps=EPS).cpu().double().numpy()
        h.free()
        stt = stt.cpu().numpy().astype(np.int64)
        s = check_pndf(D, ref, hits_gpu=stt[:, 3], hash_gpu=stt[:, 4], label=f"{name} clamp b={bf}")
        assert s["excluded"] < 0.1 * q.shape[0], s
    if name != "scratch512":  # the clamp really changed something
        exact = oracle.pndf(st, q)[0]
        assert (np.abs(ref[0] - exact) > 1e-6 * np.abs(exact) + 1e-12).sum() > 50
    assert P.pndf_device_status() == 0


@pytest.mark.parametrize("kernel", [0, 1, 2])
@pytest.mark.parametrize("eps", [0.0, EPS])
def test_samples_match_oracle(P, kernel, eps):
    st = clamped_flakes()
    nq = 200_000
    rng = np.random.default_rng(kernel * 7 + int(eps > 0))
    centres = rng.uniform(-8, st.shape[0] + 7, (nq, 2))  # some footprints reach past the map
    s1, s2 = rng.uniform(0.5, 6.0, nq), rng.uniform(0.5, 6.0, nq)
    th = rng.uniform(0, np.pi, nq)
    c, s = np.cos(th), np.sin(th)
    q = np.zeros((nq, 8), np.float32)
    q[:, 0:2] = centres
    q[:, 2] = c * c * s1 * s1 + s * s * s2 * s2
    q[:, 3] = c * s * (s1 * s1 - s2 * s2)
    q[:, 4] = s * s * s1 * s1 + c * c * s2 * s2
    U = rng.uniform(0, 1, (nq, 2)).astype(np.float32)
    h = P.pndf_build_hierarchy(st.to(DEV), bounds_fmt=1)
    m, tri, fl = P.pndf_sample_normals(h, torch.as_tensor(q, device=DEV), torch.as_tensor(U, device=DEV),
                                       kernel=kernel, jac_eps=eps)
    h.free()
    m, tri, fl = m.cpu().double().numpy(), tri.cpu().numpy().astype(np.int64), fl.cpu().numpy()
    mo, trio, flo = oracle.sample(st, q, U, kernel=kernel, jac_eps=eps)
    outside = (flo & oracle.F_OUTSIDE) != 0
    assert np.array_equal(outside, (fl & P.PNDF_SF_OUTSIDE) != 0)
    assert outside.any() and (~outside).any()
    ok = ~outside & ((flo & oracle.F_NEAR_EDGE) == 0)
    assert ok.sum() > 0.99 * (~outside).sum()
    assert np.array_equal(tri[ok], trio[ok])
    np.testing.assert_allclose(m[ok], mo[ok], rtol=0, atol=2e-7)


def test_sampling_errors(P):
    st = synth.bumps_map(n=64, n_bumps=4, seed=1).to(DEV)
    q = synth.camera_queries(64, 10, seed=1, device=DEV)
    U = torch.rand(10, 2, device=DEV)
    h = P.pndf_build_hierarchy(st, bounds_fmt=1)
    for kw in ({"kernel": 5}, {"jac_eps": 1e-12}, {"jac_eps": -1.0}):
        with pytest.raises(P.PndfError) as ei:
            P.pndf_sample_normals(h, q, U, **kw)
        assert ei.value.code == 1
    with pytest.raises(P.PndfError) as ei:
        P.pndf_eval_batch_ex(h, q, jac_eps=1e-6, kernel=1)
    assert ei.value.code == 6  # the clamp is for the Gaussian path
    bad = q.clone()
    bad[3, 2] = -1.0
    m, tri, fl = P.pndf_sample_normals(h, bad, U)
    assert fl[3].item() == P.PNDF_SF_INVALID and tri[3].item() == -1
    h.free()
