#!/usr/bin/env python
"""P-NDF throughput benchmark on the 8192^2 metallic-flake workload.

Workload: an 8192 x 8192 Voronoi flake normal map (about 200k cells, constant
cell normals ~ N(0, 0.15^2 I) plus N(0, 0.005^2) per texel, FP32 (s, t)) and
4,194,304 isotropic Gaussian-footprint queries (sigma log-uniform in 1..512
texels, centres uniform, 70% of normals drawn near the footprint's normals
and 30% uniform in [-0.4, 0.4]^2), all seeded and synthetic.

One step = the whole hot path over the batch: rebuild the min/max bound
pyramid from the texels, key and sort the queries, traverse and leaf-test,
reduce and write D in caller order.  `value` uses FP16 outward-rounded
bounds (leaf maths in FP32); the plain FP32-bounds path is timed beside it.
Texels (512 MiB) and queries (128 MiB) exceed the 129 MB L2 and are re-read
every step, so no explicit flush is needed.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs an independent replica on its own queries
(weak scaling); rank 0 prints one JSON line.
"""

from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2505_08985_gb300 import synth  # noqa: E402

METRIC = "P-NDF queries/sec @8192^2 map (FP16-bound served vs plain FP32), p50/p99 latency"
UNIT = "queries/s"
WORKLOAD = "flake8192_fp32map_4M_iso_sigma1-512"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--queries", type=int, default=synth.FLAKE_8192["queries"])
    ap.add_argument("--map-size", dest="n", type=int, default=synth.FLAKE_8192["n"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target oracle work for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the error against the FP64 oracle per workload")
    ap.add_argument("--strong", action="store_true",
                    help="under torchrun: shard one batch of --queries over the ranks (strong scaling) instead of "
                         "one batch per rank")
    ap.add_argument("--kernels", default="disk,box", help="footprint kernels to measure besides the Gaussian ('' = skip)")
    ap.add_argument("--no-clamp-sampling", action="store_true", help="skip the Eq. 6 clamp and sampling figures")
    ap.add_argument("--cluster-taus", default="1e-4,1e-3",
                    help="cluster cut thresholds to measure on the same workload ('' = skip)")
    ap.add_argument("--serve-batches", type=int, default=2000, help="serving workload size (0 = skip serving)")
    ap.add_argument("--serve-load", type=float, default=0.8, help="offered load, fraction of plain FP32 capacity")
    ap.add_argument("--serve-streams", type=int, default=2, help="streams the served steps alternate over")
    ap.add_argument("--serve-sweep", default="0.5,0.95",
                    help="further offered loads for the latency sweep ('' = skip)")
    ap.add_argument("--mixed-requests", type=int, default=4096,
                    help="projected-area + P-NDF sample on the 16384^2 FP16 map (0 = skip)")
    ap.add_argument("--mixed-stream-batches", type=int, default=256,
                    help="served glint + diffuse stream on the mixed map: batches, half P-NDF and half projected "
                         "area (0 = skip)")
    ap.add_argument("--mixed-map-size", type=int, default=synth.MIXED_16384["n"],
                    help="side of the mixed scratches + flakes map (cells and grooves scale with the area)")
    ap.add_argument("--kernel-census", action="store_true",
                    help="launch every kernel family except the traversal once on a small workload and print "
                         "the units each launch processed (the program the per-kernel ncu census profiles)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only: no data-path collective)
# ---------------------------------------------------------------------------

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() and args.impl == "gpu" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v: float) -> float:
    if world == 1:
        return v
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, v: float) -> float:
    if world == 1:
        return v
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.f is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.f.read())) if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# measured peaks and committed ncu traffic
# ---------------------------------------------------------------------------

def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash() -> str:
    return sources_hash(("eval.cu", "common.cuh"))


CENSUS_FILE = os.path.join(ROOT, "profiles", "kernels_census_flake4096_mixed4096.txt")
CENSUS_SOURCES = ("build.cu", "cluster.cu", "eval.cu", "projarea.cu", "sample.cu", "common.cuh", "ggx.cuh")


def code_text(src: str) -> str:
    """C/C++/CUDA source with its comments removed and each run of whitespace
    made one space (comment markers inside string and character literals are
    not comments), so that a source hash follows the code and not its
    commentary or layout."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def sources_hash(files) -> str:
    """Hash of the code (comments and layout aside) of the named kernel sources."""
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2505_08985_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(code_text(fh.read()).encode())
        h.update(b"\0")
    return h.hexdigest()[:16]


def committed_census() -> dict:
    """Per-unit counts of each kernel family (DRAM bytes, warp instructions,
    FP32 and FP64 FLOPs with an FMA as two) from the committed ncu census,
    if it was taken on the current sources; else {}."""
    if not os.path.exists(CENSUS_FILE):
        return {}
    src, out = None, {}
    with open(CENSUS_FILE) as f:
        for line in f:
            if line.startswith("sources_sha256_16:"):
                src = line.split(":", 1)[1].strip()
            elif line.startswith("per_unit "):
                parts = line.split()
                out[parts[1]] = {k: float(v) for k, v in (kv.split("=", 1) for kv in parts[2:])}
    return out if src == sources_hash(CENSUS_SOURCES) else {}


def compute_peaks(dev) -> dict:
    """Issue and arithmetic peaks from the unit counts and the maximum SM
    clock: 4 warp schedulers, 128 FP32 lanes and 2 FP64 lanes per SM per
    clock (the last gives the nominal 1.25 TFLOP/s FP64), an FMA as 2 FLOPs."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f)["sm_max_mhz"])
    except Exception:
        mhz = 2070.0
    clk = mhz * 1e6
    return {"issue": sms * 4 * clk / 1e9, "fp32": sms * 128 * 2 * clk / 1e12, "fp64": sms * 2 * 2 * clk / 1e12,
            "sms": sms, "sm_mhz": mhz}


def family_roofline(family, kernels, ms, units, unit, hbm_bytes_per_unit, census, peaks, hbm_pk):
    """Roofline of one kernel family from its live CUDA-event time: HBM on
    algorithmic bytes, and (with a census of the current sources) instruction
    issue, FP32 and FP64 FLOP/s from its per-unit counts; `bound` is the
    resource with the largest fraction."""
    sec = ms / 1e3
    out = {"kernels": kernels, "ms": ms, "units": units, "unit": unit}
    fr = {}
    if hbm_bytes_per_unit is not None:
        out["algorithmic_bytes"] = hbm_bytes_per_unit * units
        fr["hbm"] = (hbm_bytes_per_unit * units / sec / 1e9, hbm_pk, "GB/s")
    c = census.get(family)
    if c:
        fr["issue"] = (c["warp_inst"] * units / sec / 1e9, peaks["issue"], "G warp-inst/s")
        fr["fp32"] = (c["fp32_flop"] * units / sec / 1e12, peaks["fp32"], "TFLOP/s")
        fr["fp64"] = (c["fp64_flop"] * units / sec / 1e12, peaks["fp64"], "TFLOP/s")
        out["traffic"] = c["dram_bytes"] * units
    if not fr:
        out.update(bound=None, achieved=None, peak=None, frac=None)
        return out
    bound = max(fr, key=lambda k: fr[k][0] / fr[k][1])
    a, pk, u = fr[bound]
    out.update(bound=bound, achieved=a, peak=pk, unit_rate=u, frac=a / pk,
               fracs={k: v[0] / v[1] for k, v in fr.items()})
    return out


def committed_ncu_pct(bounds_tag: str):
    """ncu's DRAM, L2, L1 and issue throughput (% of peak) for the traversal
    kernel from the committed summary, if taken on the current source."""
    p = os.path.join(ROOT, "profiles", f"traverse_{WORKLOAD}.txt")
    if not os.path.exists(p):
        return None
    src, val = None, None
    with open(p) as f:
        for line in f:
            if line.startswith("kernel_source_sha256_16:"):
                src = line.split(":", 1)[1].strip()
            if line.startswith(f"ncu_pct_of_peak_{bounds_tag}:"):
                val = {k: float(v) for k, v in (kv.split("=") for kv in line.split(":", 1)[1].split())}
    return val if src == kernel_source_hash() else None


def committed_profile_value(key: str):
    """One number of the committed traversal profile summary ("key: value"),
    if the summary was taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", f"traverse_{WORKLOAD}.txt")
    if not os.path.exists(p):
        return None
    src, val = None, None
    with open(p) as f:
        for line in f:
            if line.startswith("kernel_source_sha256_16:"):
                src = line.split(":", 1)[1].strip()
            if line.startswith(f"{key}:"):
                val = float(line.split(":", 1)[1].split()[0])
    return val if src == kernel_source_hash() else None


def traversal_roofline(dev, work_f16: dict, nq: int, kernel_ms: float, world: int) -> dict:
    """Roofline of the dominant kernel (traversal + leaf test) per launch.

    HBM, on the path's byte model: every visited node's box
    (8 B in binary16) + every leaf block's (b + 1)^2 = 25 texels (8 B each,
    FP32) + the query's 32 B record and 4 B result.  Instruction issue, on the
    warp instructions per query of the committed ncu capture of the same
    kernel source (152 SMs x 4 schedulers x the maximum SM clock).  `bound` is
    the ceiling with the larger fraction; the other is kept beside it, and so
    is the builder's own byte model (every level-0 box tested, each tested
    triangle's three texels, 40 B per query), which counts texels of a leaf
    block once per triangle that reads them."""
    pk, pk_kind = hbm_peak()
    sec = kernel_ms / 1e3
    s8d = work_f16["nodes"] * 8 + work_f16["leaf_blocks"] * 25 * 8 + 36 * nq
    hbm = {"achieved": s8d / sec / 1e9, "peak": pk, "unit": "GB/s", "frac": s8d / sec / 1e9 / pk,
           "algorithmic_bytes_per_launch": s8d, "peak_source": f"{pk_kind} hbm_gbs",
           "byte_model": "nodes x 8 B + leaf blocks x 25 texels x 8 B + 36 B per query"}
    peaks = compute_peaks(dev)
    wipq = committed_profile_value("warp_inst_per_query_f16")
    issue = None
    if wipq is not None:
        ach = wipq * nq / sec / 1e9
        issue = {"achieved": ach, "peak": peaks["issue"], "unit": "G warp-instructions/s", "frac": ach / peaks["issue"],
                 "warp_instructions_per_query": wipq, "peak_source": f"{peaks['sms']} SMs x 4 x {peaks['sm_mhz']:.0f} MHz"}
    bound = "alu" if issue and issue["frac"] > hbm["frac"] else "hbm"
    top = issue if bound == "alu" else hbm
    out = {"bound": bound, "achieved": top["achieved"], "peak": top["peak"], "unit": top["unit"], "frac": top["frac"],
           "traffic": committed_traffic("f16"), "hbm": hbm, "issue": issue,
           "ncu_pct_of_peak": committed_ncu_pct("f16"),
           "builder_byte_model": {"bytes_per_launch": work_f16["bytes"],
                                  "achieved_gbs": work_f16["bytes"] / sec / 1e9,
                                  "frac_hbm": work_f16["bytes"] / sec / 1e9 / pk}}
    return out


def committed_traffic(bounds_tag: str):
    """DRAM bytes per launch of the traversal kernel from the committed ncu
    summary, if it was taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", f"traverse_{WORKLOAD}.txt")
    if not os.path.exists(p):
        return None
    src, val = None, None
    with open(p) as f:
        for line in f:
            if line.startswith("kernel_source_sha256_16:"):
                src = line.split(":", 1)[1].strip()
            if line.startswith(f"dram_bytes_per_launch_{bounds_tag}:"):
                val = float(line.split(":", 1)[1].split()[0])
    return val if src == kernel_source_hash() else None


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def workload_config(n: int, nq: int, world: int) -> dict:
    """The `config` object of both arms' JSON lines: the same workload keys."""
    return {"workload": WORKLOAD, "map": f"{n}^2 Voronoi flakes, fp32 (s,t)",
            "queries_per_gpu": nq, "sigma": "log-uniform 1..512 texels, isotropic",
            "bounds": "fp16 outward-rounded", "leaf_math": "fp32 (fp64 below 1e-10 area)",
            "l2": "inputs larger than L2 (512 MiB texels + 128 MiB queries re-read each step)",
            "step": "rebuild pyramid + key/sort + split plan + traverse/leaf + unpermute", "parallelism": f"replicas x{world}"}


def make_workload(args, device, rank):
    cfg = synth.FLAKE_8192
    st = synth.flake_map(n=args.n, seed=cfg["seed"], device=device)
    q = synth.make_queries(st, args.queries, cfg["mix"], cfg["seed"] + 1000 * rank)
    return st, q


def oracle_rate(st_cpu, q_cpu, seconds, seed):
    """Oracle queries/s on a random sample sized for about `seconds` of wall time."""
    import oracle
    rng = np.random.default_rng(seed)
    n_done, t_total, k = 0, 0.0, 64
    while t_total < seconds:
        idx = np.sort(rng.choice(q_cpu.shape[0], size=min(k, q_cpu.shape[0]), replace=False))
        t0 = time.perf_counter()
        oracle.pndf(st_cpu, q_cpu[idx])
        dt = time.perf_counter() - t0
        n_done += idx.size
        t_total += dt
        remaining = seconds - t_total
        if remaining <= 0.1 * seconds:
            break
        k = int(min(max(2 * k, (idx.size / dt) * remaining), 1 << 16))
    return n_done / t_total, n_done, t_total


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle
    oracle.build()
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    st, q = make_workload(args, dev, 0)
    st_cpu, q_cpu = st.cpu(), q.cpu()
    del st, q
    cores = oracle.default_threads()
    per_step = 256
    rng = np.random.default_rng(12345)
    times = []
    for step in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(q_cpu.shape[0], size=per_step, replace=False))
        t0 = time.perf_counter()
        oracle.pndf(st_cpu, q_cpu[idx])
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    total = sum(times)
    v = per_step * len(times) / total
    sample = f"{per_step} random queries of the {args.queries}-query workload per step"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.n, args.queries, args.gpus),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# glint + diffuse on the 16384^2 FP16 map: P-NDF and projected area
# ---------------------------------------------------------------------------

def footprint_triangles(q: torch.Tensor, n: int) -> int:
    """Triangles whose uv centroid lies in the 4-sigma ellipse and inside the
    map (the triangles one projected-area request integrates), counted per
    quad row from the ellipse's x-interval at the two centroid heights."""
    q = q.double().cpu()
    tot = 0
    for x, y, sxx, sxy, syy in q[:, :5].tolist():
        det = sxx * syy - sxy * sxy
        ia, ib, ic = syy / det, -sxy / det, sxx / det
        ry = 4.0 * math.sqrt(syy)
        j0, j1 = max(0, int(math.floor(y - ry)) - 1), min(n - 2, int(math.ceil(y + ry)))
        if j0 > j1:
            continue
        j = torch.arange(j0, j1 + 1, dtype=torch.float64)
        for off in (1.0 / 3.0, 2.0 / 3.0):
            dy = j + off - y
            disc = (ib * dy) ** 2 - ia * (ic * dy * dy - 16.0)
            ok = disc >= 0
            sq = torch.sqrt(torch.clamp(disc, min=0.0))
            lo = x + (-ib * dy - sq) / ia - off
            hi = x + (-ib * dy + sq) / ia - off
            i_lo = torch.clamp(torch.ceil(lo), min=0)
            i_hi = torch.clamp(torch.floor(hi), max=n - 2)
            cnt = torch.clamp(i_hi - i_lo + 1, min=0)
            tot += int(cnt[ok].sum())
    return tot


def mixed_map_scaled(n: int, dev) -> torch.Tensor:
    """The binary16 scratches + flakes map at side n, with cells and grooves
    scaled with the area so that they keep their size in texels."""
    cfg = synth.MIXED_16384
    a = (n / cfg["n"]) ** 2
    return synth.mixed_map(n=n, n_cells=max(1, round(800_000 * a)), n_grooves=max(1, round(8000 * a)),
                           seed=cfg["seed"], device=dev).half()


def leaf_blocks(n: int) -> int:
    """Leaf nodes (4 x 4 quads) of the pyramid over an n x n map."""
    from paper_2505_08985_gb300 import pndf
    return 4 ** (pndf.top_level(n) - 2)


def tree_nodes(n: int) -> int:
    """Nodes of levels 2..L of the pyramid over an n x n map."""
    from paper_2505_08985_gb300 import pndf
    L = pndf.top_level(n)
    return sum(4 ** (L - l) for l in range(2, L + 1))


def pyramid_bytes(n: int, texel_bytes: int, box_bytes: int) -> int:
    """Algorithmic bytes of one pyramid build: the map read once, the
    hierarchy's copy of it written once, every stored box written once
    (level 0 and levels 2..L, padded to 2^L quads per side) and every quad's
    8-byte capsule."""
    from paper_2505_08985_gb300 import pndf
    quads = 4 ** pndf.top_level(n)
    return 2 * n * n * texel_bytes + (quads + tree_nodes(n)) * box_bytes + 8 * quads


def run_census(dev):
    """Every kernel family but the traversal, each launched once in this
    order on a small workload: the pyramid build and query sort of a 4096^2
    FP32 flake map with 262,144 queries, sampling those footprints, the
    cluster build of the same map, then on a 4096^2 binary16 mixed map 1024
    projected-area requests, the GGX fit and Lambda' for 262,144 requests.
    This is the program the per-kernel ncu census profiles; it prints the
    units each family's launch processed."""
    from paper_2505_08985_gb300 import pndf
    n, nq = 4096, 1 << 18
    cfg = synth.FLAKE_8192
    st = synth.flake_map(n=n, n_cells=round(200_000 * (n / cfg["n"]) ** 2), seed=cfg["seed"], device=dev)
    q = synth.make_queries(st, nq, cfg["mix"], cfg["seed"])
    U = torch.rand(nq, 2, device=dev, generator=torch.Generator(device=dev).manual_seed(11))
    stm = mixed_map_scaled(n, dev)
    mcfg = synth.MIXED_16384
    qm = synth.make_queries(stm.float(), nq, mcfg["mix"], mcfg["seed"])
    w = synth.hemisphere_dirs(nq, seed=mcfg["seed"], device=dev)
    npa = 1024
    torch.cuda.synchronize()
    calls = []
    h = pndf.pndf_build_hierarchy(st, bounds_fmt=pndf.PNDF_BOUNDS_F16_OUTWARD)
    calls.append(("pyramid_build", n * n))
    pndf.pndf_sort_queries(h, q)
    calls.append(("query_sort", nq))
    pndf.pndf_sample_normals(h, q, U, jac_eps=1e-6)
    calls.append(("sampling", nq))
    torch.cuda.synchronize()
    h.free()
    hc = pndf.pndf_build_hierarchy(st, bounds_fmt=pndf.PNDF_BOUNDS_F16_OUTWARD, clusters=True)
    calls.append(("cluster_fit", leaf_blocks(n)))
    torch.cuda.synchronize()
    hc.free()
    hm = pndf.pndf_build_hierarchy(stm, bounds_fmt=pndf.PNDF_BOUNDS_F16_OUTWARD)
    calls.append(("mixed_pyramid_build", n * n))
    pndf.pndf_diffuse_projected_area(hm, qm[:npa].contiguous(), w[:npa].contiguous())
    calls.append(("projected_area", footprint_triangles(qm[:npa], n)))
    g = pndf.pndf_ggx_create(hm)
    calls.append(("ggx_fit", leaf_blocks(n)))
    pndf.pndf_ggx_lambda(g, qm, w)
    calls.append(("ggx_lambda", nq))
    torch.cuda.synchronize()
    g.free()
    hm.free()
    print(json.dumps({"census": calls, "device_status": pndf.pndf_device_status()}), flush=True)


def run_mixed(args, dev):
    from paper_2505_08985_gb300 import pndf

    cfg = synth.MIXED_16384
    st = mixed_map_scaled(args.mixed_map_size, dev)
    nq = args.mixed_requests
    q = synth.make_queries(st.float(), 2 * nq, cfg["mix"], cfg["seed"])
    qa, qp = q[:nq].contiguous(), q[nq:].contiguous()
    w = synth.hemisphere_dirs(nq, seed=cfg["seed"], device=dev)
    h = pndf.pndf_build_hierarchy(st, bounds_fmt=pndf.PNDF_BOUNDS_F16_OUTWARD)
    P = torch.empty(nq, dtype=torch.float32, device=dev)
    D = torch.empty(nq, dtype=torch.float32, device=dev)
    pndf.pndf_diffuse_projected_area(h, qa[:256], w[:256], out=P[:256])  # warm
    pndf.pndf_eval_batch(h, qp, out=D)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    pndf.pndf_diffuse_projected_area(h, qa, w, out=P)
    ev[1].record()
    pndf.pndf_eval_batch(h, qp, out=D)
    ev[2].record()
    torch.cuda.synchronize()
    pa_ms, pn_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    assert torch.isfinite(P).all() and torch.isfinite(D).all()
    # the same P-NDF batch with one warp per query (no division of large footprints)
    D1 = torch.empty_like(D)
    ev[0].record()
    pndf.pndf_eval_batch_ex(h, qp, out=D1, split=False)
    ev[1].record()
    torch.cuda.synchronize()
    pn_whole_ms = ev[0].elapsed_time(ev[1])
    assert torch.equal(D, D1)
    tris = footprint_triangles(qa, st.shape[0])
    acc = None
    if not args.no_accuracy:
        import oracle
        st_cpu = st.float().cpu()
        # P-NDF: octaves of sigma 1..1024, fewer of the costly large footprints
        idx = sigma_strata(qp, np.exp2(np.arange(11)), [600, 600, 600, 600, 400, 200, 80, 30, 12, 5], seed=17)
        qs = qp[torch.from_numpy(idx).to(dev)].contiguous()
        acc = {"mixed16384_pndf": oracle_errors(st_cpu, qs, gpu_results({"fp16_bounds": h}, qs),
                                                f"{idx.size} of {nq} queries, per octave of sigma (1..1024): "
                                                "600 below 16, then 400, 200, 80, 30, 12, 5")}
        ia = sigma_strata(qa, np.exp2(np.arange(11)), [20, 20, 20, 20, 12, 8, 5, 3, 2, 1], seed=19)
        Po = oracle.projarea(st_cpu, qa[torch.from_numpy(ia).to(dev)].cpu(), w[torch.from_numpy(ia).to(dev)].cpu())
        Pg = P[torch.from_numpy(ia).to(dev)].double().cpu().numpy()
        nzp = Po != 0  # a footprint can see nothing of the light: P = 0 exactly
        relp = np.abs(Pg[nzp] - Po[nzp]) / np.abs(Po[nzp])
        acc["mixed16384_projected_area"] = {
            "subset": f"{ia.size} of {nq} requests, per octave of sigma (1..1024): 20 below 16, then 12, 8, 5, 3, 2, 1",
            "compared": int(ia.size), "zero_P": int((~nzp).sum()), "zero_mismatches": int(((~nzp) & (Pg != 0)).sum()),
            "rel_err_max": float(relp.max()), "rel_err_p99": float(np.quantile(relp, 0.99)),
            "rel_err_median": float(np.median(relp))}
    # GGX fit of every mip node (Eq. 12): build time, Lambda' throughput, and
    # its projected area P' = w_z (1 + Lambda') against the analytic P above
    ev[0].record()
    g = pndf.pndf_ggx_create(h)
    ev[1].record()
    reps = max(1, (1 << 22) // nq)
    qb, wb = qa.repeat(reps, 1), w.repeat(reps, 1)
    lam = pndf.pndf_ggx_lambda(g, qb, wb)  # warm
    ev[2].record()
    lam = pndf.pndf_ggx_lambda(g, qb, wb)
    ev[3].record()
    torch.cuda.synchronize()
    fit_ms, lam_ms = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
    Pg = (w[:, 2] * (1.0 + lam[:nq])).double()
    rel = ((Pg - P.double()).abs() / P.double().clamp_min(1e-12)).cpu()
    covered = torch.isfinite(rel)  # footprints whose mip nodes all reach past the map border have no fit
    graz = (w[:, 2] < 0.2).cpu()
    ggx_acc = ggx_breakdown(h, g, st, qa, dev, with_nodes=not args.no_accuracy)
    g.free()
    stream_out = run_mixed_stream(args, st, h) if args.mixed_stream_batches > 0 else None
    h.free()

    def pct(x, p):
        x = x[torch.isfinite(x)]
        return float(torch.quantile(x, p)) if x.numel() else float("nan")

    out = {"workload": f"16384^2 binary16 mixed map (scratches + flakes); {nq} projected-area requests and {nq} "
                        "P-NDF queries, sigma log-U(1, 1024), light uniform on the hemisphere",
            "projected_area": {"requests_per_s": nq / (pa_ms / 1e3), "ms": pa_ms, "triangles": tris,
                               "triangles_per_s": tris / (pa_ms / 1e3)},
            "pndf": {"queries_per_s": nq / (pn_ms / 1e3), "ms": pn_ms, "ms_one_warp_per_query": pn_whole_ms,
                     "same_bits_one_warp_per_query": True},
            "map_n": st.shape[0],
            "ggx_fit": {"build_ms": fit_ms, "lambda_ms": lam_ms, "lambda_requests": qb.shape[0],
                        "lambda_per_s": qb.shape[0] / (lam_ms / 1e3),
                        "footprints_covered": float(covered.double().mean()),
                        "P_rel_diff_vs_analytic": {"median": pct(rel, 0.5), "p95": pct(rel, 0.95),
                                                   "median_grazing_wz<0.2": pct(rel[graz], 0.5),
                                                   "median_wz>=0.2": pct(rel[~graz], 0.5)},
                        "breakdown_by_wz": ggx_acc}}
    if acc is not None:
        out["accuracy"] = acc
    if stream_out is not None:
        out["served_stream"] = stream_out
    return out


GGX_WZ_BANDS = ((0.02, 0.1), (0.1, 0.2), (0.2, 0.4), (0.4, 0.7), (0.7, 1.0))


def ggx_breakdown(h, g, st, qa, dev, with_nodes=True, per_band=384, nodes_per_level=16, seed=41):
    """Where the GGX projected area P' = w_z (1 + Lambda') (Eq. 12) departs from
    the analytic P (Eq. 9-11), per band of w_z.  At query footprints (the fit
    interpolated between nodes and levels, Gaussian footprint): |P' - P| / P,
    the odd part |P(w) - P(w~)| / (P(w) + P(w~)) with w~ = (-w_x, -w_y, w_z)
    (no even model, GGX included, can represent it) and the even-part error
    |P' - (P(w) + P(w~)) / 2| / P.  At the fit's own footprint (a node's box,
    the exact P from the oracle at directions between the fit's azimuths):
    |P'_node - P_node| / P_node, levels 2, 4 and 6."""
    from paper_2505_08985_gb300 import pndf
    rng = np.random.default_rng(seed)
    n = min(per_band, qa.shape[0])
    q = qa[:n].contiguous()
    out = {"fit_directions": "16 azimuths at w_z = 0.3", "query_footprints": {}, "node_footprints": {}}
    for lo, hi in GGX_WZ_BANDS:
        wz = rng.uniform(lo, hi, n)
        ph = rng.uniform(0, 2 * np.pi, n)
        r = np.sqrt(1 - wz * wz)
        w = torch.tensor(np.stack([r * np.cos(ph), r * np.sin(ph), wz], 1), dtype=torch.float32, device=dev)
        wf = w.clone()
        wf[:, :2] = -wf[:, :2]
        P = pndf.pndf_diffuse_projected_area(h, q, w).double()
        Pf = pndf.pndf_diffuse_projected_area(h, q, wf).double()
        Pg = (w[:, 2] * (1.0 + pndf.pndf_ggx_lambda(g, q, w))).double()
        ok = torch.isfinite(Pg) & (P > 0) & (Pf > 0)
        P, Pf, Pg = P[ok], Pf[ok], Pg[ok]
        tot = ((Pg - P).abs() / P).cpu()
        odd = ((P - Pf).abs() / (P + Pf)).cpu()
        even = ((Pg - 0.5 * (P + Pf)).abs() / P).cpu()
        out["query_footprints"][f"{lo}-{hi}"] = {
            "n": int(ok.sum()), "rel_err_median": float(tot.median()), "rel_err_p95": float(torch.quantile(tot, 0.95)),
            "odd_part_median": float(odd.median()), "even_part_err_median": float(even.median())}
    if with_nodes:
        import oracle
        from concurrent.futures import ThreadPoolExecutor
        stc = st.float().cpu()
        L = pndf.top_level(st.shape[0])
        dirs = []
        for lo, hi in GGX_WZ_BANDS:
            wz = 0.5 * (lo + hi)
            ph = 2 * np.pi * (np.arange(8) + 0.5) / 8  # between the fit's 16 azimuths
            dirs.append(np.stack([np.sqrt(1 - wz * wz) * np.cos(ph), np.sqrt(1 - wz * wz) * np.sin(ph),
                                  np.full(8, wz)], 1))
        dirs = np.concatenate(dirs)
        jobs = []
        for l in (2, 4, 6):
            S = 1 << (L - l)
            Om = pndf.pndf_ggx_level(g, l).double().cpu().numpy()
            for _ in range(nodes_per_level):
                I, J = (int(v) for v in rng.integers(0, S - 1, 2))
                if np.isfinite(Om[J, I, 0]):
                    jobs.append((l, I, J, Om[J, I]))

        def run(job):
            l, I, J, O = job
            return job, oracle.ggx_node_P(stc, l, I, J, dirs)

        with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
            res = [r for r in ex.map(run, jobs) if r[1] is not None]
        for b, (lo, hi) in enumerate(GGX_WZ_BANDS):
            d = dirs[8 * b:8 * b + 8]
            errs = []
            for (l, I, J, O), Pn in res:
                qf = O[0] * d[:, 0] ** 2 + 2 * O[1] * d[:, 0] * d[:, 1] + O[2] * d[:, 1] ** 2
                Pp = 0.5 * (d[:, 2] + np.sqrt(np.maximum(d[:, 2] ** 2 + qf, 0.0)))
                Pn = Pn[8 * b:8 * b + 8]
                m = Pn > 0
                errs += list(np.abs(Pp[m] - Pn[m]) / Pn[m])
            e = np.asarray(errs)
            out["node_footprints"][f"wz={0.5 * (lo + hi):.2f}"] = {
                "n": int(e.size), "rel_err_median": float(np.median(e)) if e.size else float("nan"),
                "rel_err_p95": float(np.quantile(e, 0.95)) if e.size else float("nan")}
        out["node_sample"] = f"{len(res)} nodes of levels 2, 4, 6; 8 azimuths between the fit's per band"
    return out


def run_mixed_stream(args, st, h):
    """Glint + diffuse served as one stream on the binary16 mixed map: batches
    alternate between 1024 P-NDF queries and 16 projected-area requests
    (sigma log-U(1, 1024), light uniform on the hemisphere), Poisson arrivals
    at 0.8 of the served path's own saturated rate on this stream; the served
    path (continuous batching, both kinds in the same steps) against each
    batch launched alone in arrival order."""
    from paper_2505_08985_gb300 import pndf, serve
    dev = st.device
    cfg = synth.MIXED_16384
    nb = args.mixed_stream_batches
    npn, npa = 1024, 16
    A = pndf.PNDF_SEGMENT_PROJECTED_AREA
    qs = synth.make_queries(st.float(), nb * npn, cfg["mix"], cfg["seed"] + 7)
    ws = synth.hemisphere_dirs(nb * npa, seed=cfg["seed"] + 8, device=dev)

    def requests(arrivals):
        out = []
        for k, a in enumerate(arrivals):
            if k % 2:
                lo = npa * (k // 2)
                out.append(serve.Request(rid=k, map=0, queries=qs[lo:lo + npa].contiguous(), arrival=a, kind=A,
                                         omega=ws[lo:lo + npa].contiguous()))
            else:
                lo = npn * (k // 2)
                out.append(serve.Request(rid=k, map=0, queries=qs[lo:lo + npn].contiguous(), arrival=a))
        return out

    b = serve.ContinuousBatcher([h], step_queries=4096, max_area_requests=64, sort=True)
    b.run(requests([0.0] * nb), realtime=False)  # warm
    cap = b.run(requests([0.0] * nb), realtime=False)
    rate = 0.8 * nb / cap["span_s"]
    arr = serve.poisson_arrivals(nb, rate, seed=23)
    rs = requests(arr)
    sv = b.run(rs, realtime=True)
    b.close()
    rp = requests(arr)
    pl = serve.run_plain([h], rp, realtime=True, sort=pndf.PNDF_SORT_NONE)

    def by_kind(reqs, kind):
        lat = [1e3 * r.latency for r in reqs if r.kind == kind]
        return {"p50_ms": serve.percentile(lat, 0.5), "p99_ms": serve.percentile(lat, 0.99)}

    equal = all(torch.equal(a.D, b_.D) for a, b_ in zip(rs, rp))
    return {"stream": f"{nb} batches alternating {npn} P-NDF queries and {npa} projected-area requests "
                      f"({nb // 2 * npn} queries and {nb // 2 * npa} area requests, a bounded sample of the "
                      "8M-request mix); Poisson arrivals at 0.8 of the served saturated rate "
                      f"({rate:.1f} batches/s)",
            "served_capacity_batches_per_s": nb / cap["span_s"],
            "served": {"requests_per_s": (nb // 2) * (npn + npa) / sv["span_s"], "p50_ms": sv["p50_ms"],
                       "p99_ms": sv["p99_ms"], "pndf": by_kind(rs, pndf.PNDF_SEGMENT_PNDF), "projected_area": by_kind(rs, A)},
            "plain_per_batch": {"requests_per_s": (nb // 2) * (npn + npa) / pl["span_s"], "p50_ms": pl["p50_ms"],
                                "p99_ms": pl["p99_ms"], "pndf": by_kind(rp, pndf.PNDF_SEGMENT_PNDF),
                                "projected_area": by_kind(rp, A)},
            "served_equals_plain_bitwise": equal}


# ---------------------------------------------------------------------------
# serving: four resident maps, Poisson stream of camera batches
# ---------------------------------------------------------------------------

def run_serving(args, dev):
    """Served FP16 path (continuous batching over graph-replayed persistent
    steps) against the plain FP32 per-batch path, on the four-map camera
    stream and on the same stream with every batch on the 8192^2 flake map.
    The plain path runs both with the library's default per-batch sort and
    with each batch in arrival (pixel) order, at every offered load."""
    from paper_2505_08985_gb300 import pndf, serve

    sts = synth.serving_maps(device=dev)
    batches = synth.serving_batches(args.serve_batches, seed=9)
    n = len(batches)
    loads = [args.serve_load] + [float(x) for x in args.serve_sweep.split(",") if x.strip()]
    t0 = time.perf_counter()

    def stream(map_of, label):
        qs = [synth.camera_queries(sts[map_of(m)].shape[0], sz, seed=sd, device=dev) for (m, sz, sd) in batches]
        used = sorted({map_of(m) for (m, _, _) in batches})
        h16 = {i: pndf.pndf_build_hierarchy(sts[i], bounds_fmt=pndf.PNDF_BOUNDS_F16_OUTWARD) for i in used}
        h32 = {i: pndf.pndf_build_hierarchy(sts[i], bounds_fmt=pndf.PNDF_BOUNDS_F32) for i in used}
        slot = {i: k for k, i in enumerate(used)}
        l16 = [h16[i] for i in used]
        l32 = [h32[i] for i in used]
        torch.cuda.synchronize()

        def requests(arrivals):
            return [serve.Request(rid=k, map=slot[map_of(batches[k][0])], queries=qs[k], arrival=a)
                    for k, a in enumerate(arrivals)]

        total = sum(b[1] for b in batches)
        cap_sorted = serve.run_plain(l32, requests([0.0] * n), realtime=False)
        cap_unsorted = serve.run_plain(l32, requests([0.0] * n), realtime=False, sort=pndf.PNDF_SORT_NONE)
        rate = args.serve_load * cap_sorted["queries_per_s"] / (total / n)
        ns = min(n, 300)
        tune = serve.autotune(l16, requests([0.0] * ns), arrivals=serve.poisson_arrivals(ns, rate, seed=5),
                              streams=args.serve_streams, capacity_sample=requests([0.0] * n))
        batcher = serve.ContinuousBatcher(l16, step_queries=tune.step_queries, warps_per_cta=tune.warps_per_cta,
                                          ctas_per_sm=tune.ctas_per_sm, sort=tune.sort, streams=args.serve_streams)
        s0 = batcher.steps
        served_cap = batcher.run(requests([0.0] * n), realtime=False)
        served_steps = batcher.steps - s0
        keep = ("p50_ms", "p99_ms", "mean_ms", "queries_per_s")
        runs = []
        for load in loads:
            r = load * cap_sorted["queries_per_s"] / (total / n)
            arr = serve.poisson_arrivals(n, r, seed=17)
            sv = batcher.run(requests(arr), realtime=True)
            steps = batcher.steps
            pl = serve.run_plain(l32, requests(arr), realtime=True)
            pu = serve.run_plain(l32, requests(arr), realtime=True, sort=pndf.PNDF_SORT_NONE)
            runs.append({"load": load, "batches_per_s": r,
                         "served_fp16": {k: sv[k] for k in keep},
                         "plain_fp32_sorted": {k: pl[k] for k in keep},
                         "plain_fp32_unsorted": {k: pu[k] for k in keep}})
        batcher.close()
        # which part of the gap to the plain path is the bound format: the plain
        # path on the FP16 hierarchies, and the served path on the FP32 ones
        cap_unsorted16 = serve.run_plain(l16, requests([0.0] * n), realtime=False, sort=pndf.PNDF_SORT_NONE)
        b32 = serve.ContinuousBatcher(l32, step_queries=tune.step_queries, warps_per_cta=tune.warps_per_cta,
                                      ctas_per_sm=tune.ctas_per_sm, sort=tune.sort, streams=args.serve_streams)
        b32.run(requests([0.0] * min(n, 50)), realtime=False)  # warm
        served_cap32 = b32.run(requests([0.0] * n), realtime=False)
        b32.close()
        # and whether the host's per-step work bounds the served capacity: the
        # same path with steps four times larger
        b4 = serve.ContinuousBatcher(l16, step_queries=4 * tune.step_queries, warps_per_cta=tune.warps_per_cta,
                                     ctas_per_sm=tune.ctas_per_sm, sort=tune.sort, streams=args.serve_streams)
        b4.run(requests([0.0] * min(n, 50)), realtime=False)  # warm
        served_cap4 = b4.run(requests([0.0] * n), realtime=False)
        steps4 = b4.steps
        b4.close()
        for h in list(h16.values()) + list(h32.values()):
            h.free()
        caps = {"served_fp16": served_cap["queries_per_s"], "plain_fp32_sorted": cap_sorted["queries_per_s"],
                "plain_fp32_unsorted": cap_unsorted["queries_per_s"],
                "plain_fp16_unsorted": cap_unsorted16["queries_per_s"], "served_fp32": served_cap32["queries_per_s"],
                "served_fp16_steps_x4": served_cap4["queries_per_s"]}
        host = {"served_fp16": dict(served_cap["host"], steps=served_steps),
                "served_fp16_steps_x4": dict(served_cap4["host"], steps=steps4)}
        best_plain = max(caps["plain_fp32_sorted"], caps["plain_fp32_unsorted"])
        return {"workload": f"{label}; {n} camera batches, sizes log-U(1K, 1M), {total} queries; Poisson arrivals, "
                            "offered load as a fraction of the sorted plain FP32 capacity",
                "loads": runs,
                "capacity_queries_per_s": caps,
                "capacity_host_time_s": host,
                "served_over_best_plain_capacity": caps["served_fp16"] / best_plain,
                "autotune": {"objective": f"among candidates within 0.97 of the best saturated throughput (the "
                                          f"whole stream) and 1.05 of the lowest p99 (the first {ns} batches "
                                          f"at load {args.serve_load:g}), the highest saturated throughput",
                             "step_queries": tune.step_queries, "warps_per_cta": tune.warps_per_cta,
                             "ctas_per_sm": tune.ctas_per_sm, "sort": tune.sort,
                             "table [step, ctas_per_sm, warps, sort, p99_ms, q/s at the load, saturated q/s]": tune.table}}

    out = {"four_maps": stream(lambda m: m, "4 resident maps (1024^2 bumps, 2048^2 scratches, 4096^2 and 8192^2 "
                                            "flakes), each batch on a random one"),
           "flake8192_only": stream(lambda m: 3, "every batch on the 8192^2 flake map")}
    out["wall_s"] = time.perf_counter() - t0
    return out


# ---------------------------------------------------------------------------
# Cluster cut (Sec. 4.2, Eq. 7-8): the approximate variant on the same workload
# ---------------------------------------------------------------------------

def run_cluster_cut(args, world, st, q, D_exact, exact_kernel_ms):
    """Queries/s of the cluster cut for each tau on the bench workload (hierarchy
    with clusters built once; a step = key/sort + traversal with the cut +
    unpermute), the work it saves, the build cost of the cluster hierarchy, and
    how far its densities move from the exact ones (the surrogate map
    approximates the normal map)."""
    from paper_2505_08985_gb300 import pndf
    dev = q.device
    nq = q.shape[0]
    stream = torch.cuda.current_stream()
    D_ref = D_exact.clone()
    D = torch.empty_like(D_ref)
    h = pndf.pndf_build_hierarchy(st, bounds_fmt=pndf.PNDF_BOUNDS_F16_OUTWARD, clusters=True)
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pndf.pndf_update_hierarchy(h, st)
    b0.record(stream)
    for _ in range(3):
        pndf.pndf_update_hierarchy(h, st)
    b1.record(stream)
    torch.cuda.synchronize()
    out = {"workload": WORKLOAD, "bounds": "fp16 outward-rounded (widened to hold the cluster corners)",
           "hierarchy_bytes": h.nbytes, "build_ms": b0.elapsed_time(b1) / 3, "per_tau": {}}
    pos = D_ref > 0
    for tau in [float(t) for t in args.cluster_taus.split(",") if t.strip()]:
        stt = torch.zeros(nq, pndf.STATS_FIELDS, dtype=torch.int32, device=dev)
        pndf.pndf_eval_batch_ex(h, q, out=D, stats=stt, tau=tau)
        s = stt.to(torch.int64).sum(0).cpu().tolist()
        del stt
        for _ in range(args.warmup):
            pndf.pndf_eval_batch_ex(h, q, out=D, tau=tau)
        kb = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ke = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier(world)
        t0.record(stream)
        for k in range(args.steps):
            pndf.pndf_eval_batch_ex(h, q, out=D, tau=tau, ev_begin=kb[k], ev_end=ke[k])
        t1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(world, t0.elapsed_time(t1))
        kms = sum(a.elapsed_time(b) for a, b in zip(kb, ke)) / args.steps
        diff = (D - D_ref).abs()
        out["per_tau"][f"{tau:g}"] = {
            "value": sum_over_ranks(world, float(nq * args.steps)) / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms / args.steps, "traverse_kernel_ms": kms,
            "traversal_speedup_vs_exact": exact_kernel_ms / kms,
            "work_per_query": {"nodes": s[0] / nq, "quads": s[7] / nq, "tri_tests": s[2] / nq,
                               "cluster_checks": s[8] / nq, "clusters": s[9] / nq, "hits": s[3] / nq},
            "rel_l1_vs_exact": float(diff.sum() / D_ref.abs().sum()),
            "frac_queries_off_by_1pct": float((diff[pos] > 0.01 * D_ref[pos]).float().mean()),
        }
    h.free()
    return out


def run_kernels(args, world, st, q, gauss_kernel_ms, gauss_tri_tests):
    """The disk and box footprint kernels (the (3 sigma)^2 footprints the
    paper pairs with the Gaussian's (6 sigma)^2) on the bench workload: same
    map, same queries, FP16 bounds; a step = key/sort + traversal + unpermute."""
    from paper_2505_08985_gb300 import pndf
    dev = q.device
    nq = q.shape[0]
    stream = torch.cuda.current_stream()
    D = torch.empty(nq, dtype=torch.float32, device=dev)
    h = pndf.pndf_build_hierarchy(st, bounds_fmt=pndf.PNDF_BOUNDS_F16_OUTWARD)
    out = {"workload": WORKLOAD, "support": "disk q <= 1.5^2, box |L^-1 d|_inf <= 1.5 (S = L L^T); "
                                            "Gaussian cut at q <= 16", "per_kernel": {}}
    ids = {"disk": pndf.PNDF_KERNEL_DISK, "box": pndf.PNDF_KERNEL_BOX}
    for name in [k.strip() for k in args.kernels.split(",") if k.strip()]:
        kern = ids[name]
        stt = torch.zeros(nq, pndf.STATS_FIELDS, dtype=torch.int32, device=dev)
        pndf.pndf_eval_batch_ex(h, q, out=D, stats=stt, kernel=kern)
        s = stt.to(torch.int64).sum(0).cpu().tolist()
        del stt
        for _ in range(args.warmup):
            pndf.pndf_eval_batch_ex(h, q, out=D, kernel=kern)
        kb = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ke = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier(world)
        t0.record(stream)
        for k in range(args.steps):
            pndf.pndf_eval_batch_ex(h, q, out=D, kernel=kern, ev_begin=kb[k], ev_end=ke[k])
        t1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(world, t0.elapsed_time(t1))
        kms = sum(a.elapsed_time(b) for a, b in zip(kb, ke)) / args.steps
        out["per_kernel"][name] = {
            "value": sum_over_ranks(world, float(nq * args.steps)) / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms / args.steps, "traverse_kernel_ms": kms,
            "traversal_speedup_vs_gauss": gauss_kernel_ms / kms,
            "tri_tests_per_query": s[2] / nq, "tri_tests_vs_gauss": s[2] / max(gauss_tri_tests, 1),
            "hits_per_query": s[3] / nq}
    h.free()
    return out


def run_clamp_sampling(args, world, st, q, gauss_kernel_ms, D_exact):
    """The Jacobian clamp of Eq. 6 (eps = 1e-6) on the bench workload, and
    P-NDF sampling: one normal per query footprint from two uniforms each
    (a step = one call over all 4M footprints, uniforms resident)."""
    from paper_2505_08985_gb300 import pndf
    dev = q.device
    nq = q.shape[0]
    stream = torch.cuda.current_stream()
    eps = 1e-6
    D = torch.empty(nq, dtype=torch.float32, device=dev)
    h = pndf.pndf_build_hierarchy(st, bounds_fmt=pndf.PNDF_BOUNDS_F16_OUTWARD)
    out = {"workload": WORKLOAD, "jac_eps": eps}

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier(world)
        t0.record(stream)
        for _ in range(args.steps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(world, t0.elapsed_time(t1)) / args.steps

    ms = timed(lambda: pndf.pndf_eval_batch_ex(h, q, out=D, jac_eps=eps))
    diff = (D - D_exact).abs()
    out["clamped_pndf"] = {"value": sum_over_ranks(world, float(nq)) / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                           "queries_changed_by_clamp": float((diff > 1e-5 * D_exact.abs()).float().mean())}
    g = torch.Generator(device=dev).manual_seed(11)
    U = torch.rand(nq, 2, device=dev, generator=g)
    ms = timed(lambda: pndf.pndf_sample_normals(h, q, U, jac_eps=eps))
    out["sampling"] = {"value": sum_over_ranks(world, float(nq)) / (ms / 1e3), "unit": "samples/s", "ms_per_step": ms,
                       "note": "Gaussian footprints of the workload (sigma 1..512), FP64 position arithmetic"}
    h.free()
    return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args, world, rank, local):
    from paper_2505_08985_gb300 import pndf

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    st, q = make_workload(args, dev, rank)
    nq = q.shape[0]
    D = torch.empty(nq, dtype=torch.float32, device=dev)

    # algorithmic work per launch, from one untimed stats pass per bounds format
    work = {}
    for tag, bf in (("f16", pndf.PNDF_BOUNDS_F16_OUTWARD), ("f32", pndf.PNDF_BOUNDS_F32)):
        h = pndf.pndf_build_hierarchy(st, bounds_fmt=bf)
        stt = torch.zeros(nq, pndf.STATS_FIELDS, dtype=torch.int32, device=dev)
        pndf.pndf_eval_batch(h, q, out=D, stats=stt)
        s = stt.to(torch.int64).sum(0).cpu().tolist()
        h.free()
        node_b = 8 if tag == "f16" else 16
        texel_b = 8
        # per unit: a node or quad box (node_b), a tested triangle's three
        # vertices (3 texels), and per query its record, order slot and result
        work[tag] = {"nodes": s[0], "quads": s[7], "leaf_blocks": s[1], "tri_tests": s[2], "hits": s[3],
                     "bytes": (s[0] + s[7]) * node_b + s[2] * 3 * texel_b + nq * (32 + 4 + 4)}
        del stt
    torch.cuda.synchronize()

    def timed(bf, steps, warmup, clocks=False):
        h = pndf.pndf_build_hierarchy(st, bounds_fmt=bf)
        kb = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ke = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        for _ in range(warmup):
            pndf.pndf_update_hierarchy(h, st)
            pndf.pndf_eval_batch_ex(h, q, out=D)
        torch.cuda.synchronize()
        barrier(world)
        sampler = ClockSampler(dev.index) if clocks else None
        if sampler:
            sampler.__enter__()
        l0 = pndf.pndf_launch_count()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t_start.record(stream)
        for k in range(steps):
            pndf.pndf_update_hierarchy(h, st)
            pndf.pndf_eval_batch_ex(h, q, out=D, ev_begin=kb[k], ev_end=ke[k])
        t_end.record(stream)
        torch.cuda.synchronize()
        launches = pndf.pndf_launch_count() - l0
        barrier(world)
        if sampler:
            sampler.__exit__(None, None, None)
        ms = t_start.elapsed_time(t_end)
        kms = [a.elapsed_time(b) for a, b in zip(kb, ke)]
        h.free()
        return ms, kms, launches, (sampler.summary() if sampler else None)

    ms16, kms16, launches, clocks = timed(pndf.PNDF_BOUNDS_F16_OUTWARD, args.steps, args.warmup, clocks=True)
    ms32, kms32, _, _ = timed(pndf.PNDF_BOUNDS_F32, args.steps, args.warmup)
    ms16_max = max_over_ranks(world, ms16)
    ms32_max = max_over_ranks(world, ms32)
    total_q = sum_over_ranks(world, float(nq * args.steps))
    value = total_q / (ms16_max / 1e3)
    value32 = total_q / (ms32_max / 1e3)

    # end to end through the public API from host buffers: every step the
    # pyramid is rebuilt from the texels in pinned host memory (the build
    # kernel reads them over the host link itself), the queries are copied in
    # from pinned host memory and D goes back to pinned host memory
    st_h = st.cpu().pin_memory()
    q_h = q.cpu().pin_memory()
    D_h = torch.empty(nq, dtype=torch.float32).pin_memory()
    h = pndf.pndf_build_hierarchy(st, bounds_fmt=pndf.PNDF_BOUNDS_F16_OUTWARD)
    for _ in range(max(1, args.warmup)):
        pndf.pndf_update_hierarchy(h, st_h)
        pndf.pndf_eval_batch_host(h, q_h, D_h)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pndf.pndf_update_hierarchy(h, st_h)
        pndf.pndf_eval_batch_host(h, q_h, D_h)  # synchronises the stream after the copy-back
    e2e_s = time.perf_counter() - t0
    h.free()
    e2e_s = max_over_ranks(world, e2e_s)
    e2e_value = total_q / e2e_s
    assert torch.isfinite(D_h).all()

    # error against the FP64 oracle on a sigma-stratified 10k subset (untimed)
    acc = None
    if rank == 0 and world == 1 and not args.no_accuracy:
        idx = sigma_strata(q, np.exp2(np.arange(10)), [1112] * 9, seed=13)
        qs = q[torch.from_numpy(idx).to(dev)].contiguous()
        hs = {"fp32_bounds": pndf.pndf_build_hierarchy(st, bounds_fmt=pndf.PNDF_BOUNDS_F32),
              "fp16_bounds": pndf.pndf_build_hierarchy(st, bounds_fmt=pndf.PNDF_BOUNDS_F16_OUTWARD)}
        acc = {"flake8192": oracle_errors(st.cpu(), qs, gpu_results(hs, qs),
                                          f"{idx.size} of {nq} queries, equal counts per octave of sigma (1..512)")}
        for h in hs.values():
            h.free()

    # roofline of the dominant kernel (traversal + leaf test), per launch
    kavg16 = sum(kms16) / len(kms16)
    cluster = run_cluster_cut(args, world, st, q, D, kavg16) if args.cluster_taus else None
    kernels = run_kernels(args, world, st, q, kavg16, work["f16"]["tri_tests"]) if args.kernels else None
    clamp = None if args.no_clamp_sampling else run_clamp_sampling(args, world, st, q, kavg16, D)
    peak, peak_kind = hbm_peak()
    traffic = committed_traffic("f16")
    stage_ms = time_build_and_sort(args, world, st, q)
    flop_model = traversal_flops(dev, work["f16"], kavg16, world, peak)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms16_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args.n, nq, world),
        "fp32_bounds_plain": {"value": value32, "unit": UNIT, "ms_per_step": ms32_max / args.steps,
                              "traverse_kernel_ms": sum(kms32) / len(kms32)},
        "traverse_kernel_ms": kavg16,
        "leaf_triangle_tests_per_s": work["f16"]["tri_tests"] * world / (kavg16 / 1e3),
        "traversal_flops": flop_model,
        "roofline": traversal_roofline(dev, work["f16"], nq, kavg16, world),
        "work_per_launch": work,
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": int(st.numel() * 4 + q.numel() * 4), "d2h_bytes_per_step": int(nq * 4)},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if acc is not None:
        acc.update(accuracy_small(dev))
        line["accuracy_vs_fp64_oracle"] = acc
    if cluster:
        line["cluster_cut"] = cluster
    if kernels:
        line["footprint_kernels"] = kernels
    if clamp:
        line["jacobian_clamp_and_sampling"] = clamp

    if args.serve_batches > 0 or args.mixed_requests > 0:
        del st, q, D, st_h, q_h, D_h
        torch.cuda.empty_cache()
    if args.mixed_requests > 0:
        line["glint_diffuse_16384"] = run_mixed(args, dev)
        if "accuracy_vs_fp64_oracle" in line and "accuracy" in line["glint_diffuse_16384"]:
            line["accuracy_vs_fp64_oracle"].update(line["glint_diffuse_16384"].pop("accuracy"))
        torch.cuda.empty_cache()
    if args.serve_batches > 0:
        line["serving"] = run_serving(args, dev)
        line["serving"]["note"] = "per GPU (each rank serves its own replica of the stream)"
    line["kernel_rooflines"] = kernel_rooflines(dev, args.n, nq, stage_ms, kavg16, line["roofline"], cluster, clamp,
                                                line.get("glint_diffuse_16384"))
    if (args.serve_batches > 0 or args.mixed_requests > 0) and rank == 0 and world == 1 and not args.no_cpu_baseline:
        st, q = make_workload(args, dev, rank)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        st_cpu, q_cpu = st.cpu(), q.cpu()
        rate, n_done, secs = oracle_rate(st_cpu, q_cpu, args.cpu_seconds, seed=7)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": oracle.default_threads(), "kind": "oracle",
                                "sample": f"{n_done} random queries of the same workload, {secs:.1f} s wall"}
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# error against the FP64 oracle, per workload (outside every timed region)
# ---------------------------------------------------------------------------

def sigma_strata(q: torch.Tensor, edges, per_bin, seed: int) -> np.ndarray:
    """Indices of a sigma-stratified subset: up to per_bin[k] queries drawn at
    random from bin [edges[k], edges[k+1]) of the footprint's major sigma."""
    qq = q[:, 2:5].double().cpu().numpy()
    tr, det = qq[:, 0] + qq[:, 2], qq[:, 0] * qq[:, 2] - qq[:, 1] ** 2
    sig = np.sqrt(0.5 * tr + np.sqrt(np.maximum(0.25 * tr * tr - det, 0.0)))
    rng = np.random.default_rng(seed)
    out = []
    for k, (a, b) in enumerate(zip(edges[:-1], edges[1:])):
        cand = np.flatnonzero((sig >= a) & (sig < b))
        if cand.size:
            out.append(rng.choice(cand, size=min(per_bin[k], cand.size), replace=False))
    return np.sort(np.concatenate(out)) if out else np.zeros(0, np.int64)


def oracle_errors(st_cpu, q_sub: torch.Tensor, gpu: dict, subset: str) -> dict:
    """Per-query relative error of each GPU result against the FP64 oracle on
    the same queries: max / p99 / median over the compared queries (those the
    oracle flags as ties are excluded and counted by reason), exact-zero
    mismatches, and how many queries took the FP64 leaf branch."""
    import oracle
    Do, fo, _, _ = oracle.pndf(st_cpu, q_sub.cpu())
    ok = (fo & oracle.F_EXCLUDE) == 0
    out = {"subset": subset, "queries": int(len(Do)), "compared": int(ok.sum()),
           "excluded": {"near_edge": int(((fo & oracle.F_NEAR_EDGE) != 0).sum()),
                        "near_cut": int(((fo & oracle.F_NEAR_CUT) != 0).sum()),
                        "degenerate": int(((fo & oracle.F_DEGENERATE) != 0).sum()),
                        "invalid": int(((fo & oracle.F_INVALID) != 0).sum())},
           "oracle_tiny_area_hits": int(((fo & oracle.F_TINY) != 0).sum()), "results": {}}
    for name, (D, fl) in gpu.items():
        D = D.double().cpu().numpy()
        nz = ok & (Do != 0)
        rel = np.abs(D[nz] - Do[nz]) / np.abs(Do[nz])
        out["results"][name] = {
            "rel_err_max": float(rel.max()) if rel.size else 0.0,
            "rel_err_p99": float(np.quantile(rel, 0.99)) if rel.size else 0.0,
            "rel_err_median": float(np.median(rel)) if rel.size else 0.0,
            "zero_mismatches": int((ok & (Do == 0) & (D != 0)).sum()),
            "fp64_branch_queries": int(((fl.cpu().numpy() & 1) != 0).sum())}
    return out


def gpu_results(h_by_name: dict, q_sub: torch.Tensor) -> dict:
    from paper_2505_08985_gb300 import pndf
    out = {}
    for name, h in h_by_name.items():
        fl = torch.zeros(q_sub.shape[0], dtype=torch.int32, device=q_sub.device)
        D = pndf.pndf_eval_batch(h, q_sub, flags=fl)
        out[name] = (D, fl)
    return out


def accuracy_small(dev) -> dict:
    """The bumps (all 4096 queries) and scratch (10k of 1M, sigma-stratified)
    workloads against the oracle, FP32 and FP16 bounds."""
    from paper_2505_08985_gb300 import pndf
    res = {}
    for key, cfg, make, strata in (
            ("bumps256", synth.BUMPS_256, lambda c: synth.bumps_map(n=c["n"], seed=c["seed"], device=dev), None),
            ("scratch2048", synth.SCRATCH_2048, lambda c: synth.scratch_map(n=c["n"], seed=c["seed"], device=dev),
             (np.exp2(np.arange(7)), [1667] * 6))):
        st = make(cfg)
        q = synth.make_queries(st, cfg["queries"], cfg["mix"], cfg["seed"])
        if strata is None:
            idx, subset = np.arange(q.shape[0]), f"all {q.shape[0]} queries"
        else:
            idx = sigma_strata(q, strata[0], strata[1], seed=11)
            subset = f"{idx.size} of {q.shape[0]} queries, equal counts per octave of major sigma"
        qs = q[torch.from_numpy(idx).to(dev)].contiguous()
        hs = {"fp32_bounds": pndf.pndf_build_hierarchy(st, bounds_fmt=pndf.PNDF_BOUNDS_F32),
              "fp16_bounds": pndf.pndf_build_hierarchy(st, bounds_fmt=pndf.PNDF_BOUNDS_F16_OUTWARD)}
        res[key] = oracle_errors(st.cpu(), qs, gpu_results(hs, qs), subset)
        for h in hs.values():
            h.free()
        del st, q
    return res



def traversal_flops(dev, w, kernel_ms, world, hbm_pk):
    """The traversal's arithmetic against the FP32 roofline, on the counted
    work of the stats pass: about 20 FLOPs per node test, 20 per triangle
    test and 40 per hit (plus one exp per hit), and leaf triangle tests per
    second against both the FP32 and the HBM ceilings (24 B of texels per
    test), at the maximum SM clock and at the clock measured under a
    power-capped dense load."""
    peaks = compute_peaks(dev)
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            loaded = float(json.load(f)["clocks_under_load"]["sm_mhz_median"])
    except Exception:
        loaded = 1455.0
    sec = kernel_ms / 1e3
    flops = 20 * w["nodes"] + 20 * w["tri_tests"] + 40 * w["hits"]
    tf = flops / sec / 1e12
    clocks = {f"{peaks['sm_mhz']:.0f}_mhz": peaks["fp32"], f"{loaded:.0f}_mhz": peaks["fp32"] * loaded / peaks["sm_mhz"]}
    tests = w["tri_tests"] / sec
    return {"model": "20 FLOPs per node test + 20 per triangle test + 40 per hit (+1 exp per hit)",
            "flops_per_launch": flops, "achieved_tflops": tf * world,
            "fp32_peak_tflops": clocks, "frac_fp32": {k: tf / v for k, v in clocks.items()},
            "leaf_triangle_tests": {"value": tests * world, "unit": "tests/s", "flops_per_test": 20,
                                    "frac_fp32": {k: tests * 20 / 1e12 / v for k, v in clocks.items()},
                                    "frac_hbm_24B_per_test": tests * 24 / 1e9 / hbm_pk}}


def time_build_and_sort(args, world, st, q):
    """CUDA-event time of the pyramid build (FP16 outward bounds) and of the
    query sort alone, each averaged over the bench's step count after warm-up."""
    from paper_2505_08985_gb300 import pndf
    stream = torch.cuda.current_stream()
    h = pndf.pndf_build_hierarchy(st, bounds_fmt=pndf.PNDF_BOUNDS_F16_OUTWARD)
    order = torch.empty(q.shape[0], dtype=torch.int32, device=q.device)
    out = {}
    for name, fn in (("pyramid_build", lambda: pndf.pndf_update_hierarchy(h, st)),
                     ("query_sort", lambda: pndf.pndf_sort_queries(h, q, order))):
        for _ in range(args.warmup):
            fn()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        for _ in range(args.steps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize()
        out[name] = max_over_ranks(world, t0.elapsed_time(t1)) / args.steps
    h.free()
    return out


def kernel_rooflines(dev, n, nq, stage_ms, traverse_ms, traverse_roof, cluster, clamp, mixed):
    """Roofline of every kernel family, from the CUDA-event times measured
    in this run.  Algorithmic bytes per unit: pyramid build, the FP32 map
    read and its copy written (8 B each per texel) plus every FP16 box written
    (8 B); query sort, the 32 B record read, the key written and read back
    and the order slot written (4 B each); traversal, as in `roofline` (the
    path's byte model, and instruction issue from the committed capture);
    sampling, record, uniforms, four texels and the outputs (88 B); Lambda',
    record, direction and result (48 B) plus the 12 B Omega of the eight
    nodes it blends (96 B); cluster fit, the map read (8 B per texel) and the
    cluster records and residuals written (36 B per node); projected area,
    two binary16 texels (8 B) per triangle; GGX fit, the binary16 map read
    (4 B per texel) and Omega written (12 B per node).  Issue and FLOP rates
    use the per-unit instruction counts of the committed ncu census, when it
    was taken on the current sources."""
    census = committed_census()
    peaks = compute_peaks(dev)
    pk, _ = hbm_peak()
    out = {"peaks": {"hbm_gbs": pk, "issue_g_warp_inst_per_s": peaks["issue"], "fp32_tflops": peaks["fp32"],
                     "fp64_tflops": peaks["fp64"],
                     "derived_from": f"{peaks['sms']} SMs at {peaks['sm_mhz']:.0f} MHz; HBM measured copy"},
           "census": "profiles/" + os.path.basename(CENSUS_FILE) if census else None}
    fams = {}
    fams["pyramid_build"] = family_roofline("pyramid_build", ["build_tiles", "build_up"], stage_ms["pyramid_build"],
                                            n * n, "texel", pyramid_bytes(n, 8, 8) / (n * n), census, peaks, pk)
    fams["query_sort"] = family_roofline("query_sort", ["key_hist", "key_scan", "key_place"], stage_ms["query_sort"],
                                         nq, "query", 44, census, peaks, pk)
    tr = family_roofline("traverse", ["traverse_kernel"], traverse_ms, nq, "query",
                         traverse_roof["hbm"]["algorithmic_bytes_per_launch"] / nq, {}, peaks, pk)
    if traverse_roof["issue"]:
        tr["fracs"]["issue"] = traverse_roof["issue"]["frac"]
        if traverse_roof["bound"] == "alu":
            iss = traverse_roof["issue"]
            tr.update(bound="issue", achieved=iss["achieved"], peak=iss["peak"], unit_rate=iss["unit"],
                      frac=iss["frac"])
    tr["traffic"] = traverse_roof["traffic"]
    fams["traverse"] = tr
    if cluster:
        ms = cluster["build_ms"] - stage_ms["pyramid_build"]
        fams["cluster_fit"] = family_roofline("cluster_fit", ["cluster_tiles", "cluster_up"], ms, leaf_blocks(n),
                                              "leaf block", (8 * n * n + 36 * tree_nodes(n)) / leaf_blocks(n),
                                              census, peaks, pk)
        fams["cluster_fit"]["note"] = "cluster build minus the pyramid build it includes"
    if clamp:
        fams["sampling"] = family_roofline("sampling", ["sample_kernel"], clamp["sampling"]["ms_per_step"], nq,
                                           "sample", 88, census, peaks, pk)
    if mixed:
        m = mixed["map_n"]
        pa = mixed["projected_area"]
        fams["projected_area"] = family_roofline("projected_area", ["pa_bands", "pa_scan", "pa_items", "pa_reduce"], pa["ms"],
                                                 pa["triangles"], "triangle", 8, census, peaks, pk)
        gf = mixed["ggx_fit"]
        fams["ggx_fit"] = family_roofline("ggx_fit", ["ggx_leaf", "ggx_up"], gf["build_ms"], leaf_blocks(m),
                                          "leaf block", (4 * m * m + 12 * tree_nodes(m)) / leaf_blocks(m), census, peaks, pk)
        fams["ggx_fit"]["note"] = "includes the fit's allocation"
        fams["ggx_lambda"] = family_roofline("ggx_lambda", ["ggx_eval"], gf["lambda_ms"], gf["lambda_requests"],
                                             "request", 144, census, peaks, pk)
    out["families"] = fams
    return out


def run_strong(args, world, rank, local):
    """Strong scaling: one batch of --queries sharded over the ranks.  Every
    rank holds a replica of the hierarchy and the same seeded batch; per step
    rank 0 sorts the batch, splits the order into contiguous ranges of equal
    estimated work and broadcasts the order and the bounds; each rank gathers
    and evaluates its range in that order; the shards are all-gathered and
    rank 0 scatters them into caller order.  The timed step includes all of
    it; value = the batch's queries / the step time (max over ranks)."""
    import torch.distributed as dist
    from paper_2505_08985_gb300 import pndf, shard

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    st, q = make_workload(args, dev, 0)  # the same batch on every rank
    nq = q.shape[0]
    h = pndf.pndf_build_hierarchy(st, bounds_fmt=pndf.PNDF_BOUNDS_F16_OUTWARD)
    out = torch.empty(nq, dtype=torch.float32, device=dev)
    order = torch.empty(nq, dtype=torch.int32, device=dev)
    block = shard.work_block(nq, world)

    def step():
        bounds_t = torch.zeros(world + 1, dtype=torch.int64, device=dev)
        if rank == 0:
            pndf.pndf_sort_queries(h, q, order)
            parts = pndf.pndf_shard_work(q, order, block=block).cpu().tolist()
            bounds_t.copy_(torch.tensor(shard.split_by_work(parts, world, nq, block)))
        dist.broadcast(order, 0)
        dist.broadcast(bounds_t, 0)
        bounds = bounds_t.cpu().tolist()
        a, b = bounds[rank], bounds[rank + 1]
        qi = pndf.pndf_gather_queries(q, order, a, b - a)
        Di = pndf.pndf_eval_batch_ex(h, qi, sort=pndf.PNDF_SORT_NONE)
        allD = shard.gather_shards(Di, bounds, rank, world)
        if rank == 0:
            for i in range(world):
                pndf.pndf_scatter_results(allD[bounds[i] - bounds[0]:bounds[i + 1] - bounds[0]].contiguous(), order,
                                          bounds[i], out)
        return bounds

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        bounds = step()
    t1.record()
    torch.cuda.synchronize()
    ms = max_over_ranks(world, t0.elapsed_time(t1)) / args.steps
    if rank == 0:
        ref = pndf.pndf_eval_batch(h, q)
        assert torch.equal(ref, out), "sharded result differs from one batch"
        cfg = workload_config(args.n, nq, world)
        cfg["parallelism"] = f"one batch sharded over {world} replicas"
        print(json.dumps({"metric": METRIC, "value": nq / (ms / 1e3), "unit": UNIT, "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                          "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                          "config": cfg, "shard_bounds": bounds}), flush=True)
    h.free()


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    try:
        if args.impl == "reference":
            run_reference(args, world, rank)
        elif args.kernel_census:
            if not torch.cuda.is_available():
                raise SystemExit("bench.py: no CUDA device (the GPU arm has no CPU fallback)")
            run_census(torch.device("cuda:0"))
        else:
            if not torch.cuda.is_available():
                raise SystemExit("bench.py: no CUDA device (the GPU arm has no CPU fallback)")
            if args.strong and world > 1:
                run_strong(args, world, rank, local)
            else:
                run_gpu(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
