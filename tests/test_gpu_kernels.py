"""GPU parity of the disk and box footprint kernels (the paper's kernel
ablation: (3 sigma)^2 footprints in place of the Gaussian's (6 sigma)^2)
with the FP64 oracle, through the C ABI."""

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


def run(P, h, q, kernel, mode=0, tau=0.0):
    qd = q.to(DEV)
    stt = torch.zeros(q.shape[0], P.STATS_FIELDS, dtype=torch.int32, device=DEV)
    D = P.pndf_eval_batch_ex(h, qd, stats=stt, kernel=kernel, mode=mode, tau=tau)
    torch.cuda.synchronize()
    return D.cpu().double().numpy(), stt.cpu().numpy().astype(np.int64)


def anisotropic(st, n, seed, sigma=(1.0, 24.0)):
    return synth.make_queries(st, n, synth.QueryMix(sigma=sigma, aspect=(1.0, 4.0), frac_near=0.8), seed)


@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("name", ["bumps256", "scratch512", "flakes512"])
def test_kernel_matches_oracle(P, kernel, name):
    st = {"bumps256": lambda: synth.bumps_map(n=256, n_bumps=40, seed=21),
          "scratch512": lambda: synth.scratch_map(n=512, n_grooves=120, seed=22),
          "flakes512": lambda: synth.flake_normals(512, 1500, seed=23)}[name]()
    q = anisotropic(st, 3000, 7)
    ref = oracle.pndf(st, q, kernel=kernel)
    for bf in (0, 1):
        h = P.pndf_build_hierarchy(st.to(DEV), bounds_fmt=bf)
        D, stt = run(P, h, q, kernel)
        h.free()
        s = check_pndf(D, ref, hits_gpu=stt[:, 3], hash_gpu=stt[:, 4], label=f"{name} kernel={kernel} b={bf}")
        assert s["excluded"] < 0.05 * q.shape[0], s
        assert s["nonzero"] > 0.2 * s["compared"], s  # smaller supports: more normals see no hit
    assert P.pndf_device_status() == 0


@pytest.mark.parametrize("kernel", [1, 2])
def test_kernel_hierarchy_prunes_only(P, kernel):
    """Pyramid and flat evaluation test the same contributing triangles: the
    pruning ellipse (q <= 2.25 disk, q <= 4.5 box) holds the support."""
    st = synth.bumps_map(n=200, n_bumps=40, seed=7)
    q = anisotropic(st, 3000, 8, sigma=(0.7, 12.0))
    h = P.pndf_build_hierarchy(st.to(DEV), bounds_fmt=1)
    Dh, sh = run(P, h, q, kernel, mode=0)
    Df, sf = run(P, h, q, kernel, mode=1)
    h.free()
    assert np.array_equal(sh[:, 3], sf[:, 3]) and np.array_equal(sh[:, 4], sf[:, 4])
    assert rel_err(Dh, Df).max() <= 1e-5


def test_smaller_footprints_test_fewer_triangles(P):
    """For the same footprints the disk and box kernels test far fewer
    triangles than the 4-sigma Gaussian (the source of the paper's speed-up)."""
    st = synth.scratch_map(n=1024, n_grooves=250, seed=4)
    q = anisotropic(st, 4000, 9, sigma=(2.0, 32.0))
    h = P.pndf_build_hierarchy(st.to(DEV), bounds_fmt=1)
    tests = [run(P, h, q, k)[1][:, 2].sum() for k in (0, 1, 2)]
    h.free()
    assert tests[1] < 0.5 * tests[0] and tests[2] < 0.5 * tests[0], tests


@pytest.mark.parametrize("kernel", [1, 2])
def test_kernel_with_cluster_cut(P, kernel):
    st = synth.bumps_map(n=256, n_bumps=40, seed=21)
    q = anisotropic(st, 1500, 5, sigma=(4.0, 48.0))
    fits = oracle.cluster_fits(st)
    ref = oracle.pndf_cluster(st, q, 1e-2, fits, kernel=kernel)
    h = P.pndf_build_hierarchy(st.to(DEV), bounds_fmt=1, clusters=True)
    D, stt = run(P, h, q, kernel, tau=1e-2)
    h.free()
    s = check_pndf(D, ref, hits_gpu=stt[:, 3], hash_gpu=stt[:, 4], label=f"cluster kernel={kernel}")
    assert s["excluded"] < 0.1 * q.shape[0], s
    assert stt[:, 9].sum() > 0


def test_invalid_kernel(P):
    st = synth.bumps_map(n=64, n_bumps=4, seed=1).to(DEV)
    q = synth.camera_queries(64, 10, seed=1, device=DEV)
    h = P.pndf_build_hierarchy(st, bounds_fmt=1)
    with pytest.raises(P.PndfError) as ei:
        P.pndf_eval_batch_ex(h, q, kernel=3)
    assert ei.value.code == 1
    h.free()
