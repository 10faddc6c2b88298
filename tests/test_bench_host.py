"""Host-side helpers of bench.py's per-kernel rooflines (CPU only): the
algorithmic byte counts of the pyramid, the choice of the binding resource,
and that ncu census counts are used only for the sources they were taken on."""

import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def bench():
    old = sys.argv
    sys.argv = ["bench.py"]
    try:
        import bench as b
    finally:
        sys.argv = old
    return b


def test_pyramid_counts(bench):
    from paper_2505_08985_gb300 import pndf
    for n in (5, 65, 100, 8192):
        L = pndf.top_level(n)
        assert (1 << L) >= n - 1 and (L == 2 or (1 << (L - 1)) < n - 1)
        nodes = 0
        for l in range(2, L + 1):
            side = 1 << (L - l)
            nodes += side * side
        assert bench.tree_nodes(n) == nodes
        assert bench.leaf_blocks(n) == (1 << (L - 2)) ** 2
        # map read + copy written (8 B per FP32 texel each) + level 0 and levels 2..L (8 B boxes)
        # + one 8 B capsule per quad
        assert bench.pyramid_bytes(n, 8, 8) == 16 * n * n + 8 * ((1 << L) ** 2 + nodes) + 8 * (1 << L) ** 2


def test_family_roofline_picks_the_binding_resource(bench):
    peaks = {"issue": 1000.0, "fp32": 80.0, "fp64": 1.25}
    # HBM only: 1e9 units x 10 B in 10 ms = 1000 GB/s of 5000
    r = bench.family_roofline("x", ["k"], 10.0, 1e9, "unit", 10, {}, peaks, 5000.0)
    assert r["bound"] == "hbm" and r["frac"] == pytest.approx(0.2)
    # with a census: 1e9 units x 5 warp inst in 10 ms = 500 G/s (0.5 of issue) beats HBM 0.2
    census = {"x": {"dram_bytes": 12.0, "warp_inst": 5.0, "fp32_flop": 100.0, "fp64_flop": 0.0}}
    r = bench.family_roofline("x", ["k"], 10.0, 1e9, "unit", 10, census, peaks, 5000.0)
    assert r["bound"] == "issue" and r["frac"] == pytest.approx(0.5)
    assert r["fracs"]["fp32"] == pytest.approx(10.0 / 80.0) and r["traffic"] == pytest.approx(12e9)
    # no byte model and no census: no roofline claimed
    r = bench.family_roofline("y", ["k"], 10.0, 1e9, "unit", None, census, peaks, 5000.0)
    assert r["bound"] is None and r["frac"] is None


def test_census_needs_matching_sources(bench, tmp_path, monkeypatch):
    p = tmp_path / "census.txt"
    line = "per_unit pyramid_build dram_bytes=24 warp_inst=0.5 fp32_flop=0 fp64_flop=0\n"
    p.write_text("sources_sha256_16: 0000000000000000\n" + line)
    monkeypatch.setattr(bench, "CENSUS_FILE", str(p))
    assert bench.committed_census() == {}
    p.write_text(f"sources_sha256_16: {bench.sources_hash(bench.CENSUS_SOURCES)}\n" + line)
    c = bench.committed_census()
    assert c["pyramid_build"]["dram_bytes"] == 24.0 and c["pyramid_build"]["warp_inst"] == 0.5


def test_source_hash_follows_code_not_comments(bench, tmp_path, monkeypatch):
    t = bench.code_text('int a = 1; // note\n/* block\n note */ const char *s = "x // y /* z */";\nchar q = \'"\';  b  =\n c;')
    assert t == 'int a = 1; const char *s = "x // y /* z */"; char q = \'"\'; b = c;'
    d = tmp_path / "paper_2505_08985_gb300" / "csrc"
    d.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (d / "k.cu").write_text("// kernel (Sec. 1)\n__global__ void k(float *x) { x[0] = 1.0f; }\n")
    h0 = bench.sources_hash(["k.cu"])
    (d / "k.cu").write_text("// kernel (Sec. 2), reworded\n__global__  void k(float *x)\n{\n    x[0] = 1.0f;  /* one */\n}\n")
    assert bench.sources_hash(["k.cu"]) == h0
    (d / "k.cu").write_text("// kernel (Sec. 2)\n__global__ void k(float *x) { x[0] = 2.0f; }\n")
    assert bench.sources_hash(["k.cu"]) != h0


def test_traversal_roofline_follows_the_path_byte_model(bench, monkeypatch):
    """roofline.frac is reproducible from the stats counts: HBM on nodes x 8 B
    + leaf blocks x 25 texels x 8 B + 36 B per query; with a committed
    instruction count the issue fraction is computed beside it and `bound`
    names the larger one."""
    monkeypatch.setattr(bench, "compute_peaks", lambda dev: {"issue": 1000.0, "fp32": 80.0, "fp64": 1.25,
                                                             "sms": 152, "sm_mhz": 2070.0})
    monkeypatch.setattr(bench, "hbm_peak", lambda: (6000.0, "measured"))
    monkeypatch.setattr(bench, "committed_traffic", lambda tag: None)
    monkeypatch.setattr(bench, "committed_ncu_pct", lambda tag: None)
    w = {"nodes": 1000, "leaf_blocks": 200, "bytes": 99999, "quads": 3200, "tri_tests": 50, "hits": 5}
    monkeypatch.setattr(bench, "committed_profile_value", lambda key: None)
    r = bench.traversal_roofline(None, w, nq=10, kernel_ms=2.0, world=1)
    nbytes = 1000 * 8 + 200 * 25 * 8 + 36 * 10
    assert r["hbm"]["algorithmic_bytes_per_launch"] == nbytes
    assert r["bound"] == "hbm" and r["issue"] is None
    assert abs(r["frac"] - nbytes / 2e-3 / 1e9 / 6000.0) < 1e-15
    assert r["builder_byte_model"]["bytes_per_launch"] == 99999
    monkeypatch.setattr(bench, "committed_profile_value", lambda key: 1e5 if key == "warp_inst_per_query_f16" else None)
    r = bench.traversal_roofline(None, w, nq=10, kernel_ms=2.0, world=1)
    assert r["bound"] == "alu" and r["unit"] == "G warp-instructions/s"
    assert abs(r["frac"] - 1e5 * 10 / 2e-3 / 1e9 / 1000.0) < 1e-12
    assert r["hbm"]["frac"] < r["frac"]


def test_sigma_strata_draws_per_octave(bench):
    import torch
    rng = np.random.default_rng(0)
    sig = np.exp(rng.uniform(0, np.log(64), 5000))
    q = torch.zeros(5000, 8)
    q[:, 2] = torch.from_numpy(sig ** 2)
    q[:, 4] = torch.from_numpy(sig ** 2)
    idx = bench.sigma_strata(q, np.exp2(np.arange(7)), [50] * 6, seed=1)
    assert idx.size == 300 and np.unique(idx).size == 300
    counts = np.histogram(np.sqrt(q[idx, 2].double().numpy()), bins=np.exp2(np.arange(7)))[0]
    assert (counts == 50).all()


def test_both_arms_name_the_same_workload(bench):
    a = bench.workload_config(8192, 1 << 22, 1)
    assert a["workload"] == bench.WORKLOAD and a["queries_per_gpu"] == 1 << 22
    assert set(a) == set(bench.workload_config(4096, 10, 2))
