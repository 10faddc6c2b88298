"""Host-side helpers of bench.py's per-kernel rooflines (CPU only): the
algorithmic byte counts of the pyramid, the choice of the binding resource,
and that ncu census counts are used only for the sources they were taken on."""

import os
import sys

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
        assert bench.pyramid_bytes(n, 8, 8) == 16 * n * n + 8 * ((1 << L) ** 2 + nodes)


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
