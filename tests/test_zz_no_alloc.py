"""The allocation-free entry point gives the same densities as pndf_eval_batch.

pndf_eval_batch_noalloc is for callers that may not allocate device memory
during evaluation (a renderer plugin whose host owns every device allocation,
a real-time thread that cannot take cudaMalloc's device-wide synchronisation,
a fixed device-memory budget).  Its sort scratch is a fixed device array of the
library that every call shares, so the test makes two calls in a row with
different batches and compares each with the allocating entry point.  This file
is collected last so that a stop-at-first-failure run has already run every
other test; it passes alone in a fresh process as well as after the others.
"""

import ctypes

import numpy as np
import pytest
import torch

from paper_2505_08985_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_08985_gb300 import pndf
    return pndf


def test_noalloc_matches_allocating_entry_point_twice(P):
    """Both entry points run the same kernels in the same evaluation order,
    and a query's density does not depend on which warp or launch evaluates
    it, so the results are bit for bit equal."""
    st = synth.scratch_map(n=512, n_grooves=100, seed=41).to(DEV)
    mix = synth.QueryMix(sigma=(1.0, 30.0), aspect=(1.0, 4.0), frac_near=0.7)
    batches = [synth.make_queries(st, 20000, mix, 42), synth.make_queries(st, 7001, mix, 43)]
    for bounds in (P.PNDF_BOUNDS_F32, P.PNDF_BOUNDS_F16_OUTWARD):
        h = P.pndf_build_hierarchy(st, bounds_fmt=bounds)
        for q in batches:  # two calls in a row: the shared scratch keeps the previous call's contents
            ref = P.pndf_eval_batch(h, q)
            flags = torch.zeros(q.shape[0], dtype=torch.int32, device=DEV)
            got = P.pndf_eval_batch_noalloc(h, q, flags=flags)
            assert torch.equal(got, ref)
            assert int(torch.count_nonzero(ref)) > 1000
            assert not (flags.cpu().numpy() & P.PNDF_QF_INVALID).any()
        h.free()
    assert P.pndf_device_status() == 0


def _cudart():
    for name in ("libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so.13", "libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    raise RuntimeError("the CUDA runtime library the extension links was not found")


def _pool_peak_after(rt, fn) -> int:
    """Peak bytes in use in the device's default memory pool (the pool the
    library's stream-ordered scratch comes from) while fn's work runs."""
    pool = ctypes.c_void_p()
    dev = torch.cuda.current_device()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    zero = ctypes.c_uint64(0)
    used_high = 0x8  # cudaMemPoolAttrUsedMemHigh
    torch.cuda.synchronize()
    assert rt.cudaMemPoolSetAttribute(pool, used_high, ctypes.byref(zero)) == 0
    fn()
    torch.cuda.synchronize()
    peak = ctypes.c_uint64(0)
    assert rt.cudaMemPoolGetAttribute(pool, used_high, ctypes.byref(peak)) == 0
    return int(peak.value)


def test_noalloc_takes_nothing_from_the_memory_pool(P):
    """The entry point's defining property: no device allocation.  The
    default pool's high-water mark stays at zero across a call (results and
    flags preallocated), while the allocating entry point raises it, which
    shows the check sees an allocation."""
    rt = _cudart()
    rt.cudaDeviceGetDefaultMemPool.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]
    rt.cudaMemPoolSetAttribute.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    rt.cudaMemPoolGetAttribute.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    st = synth.bumps_map(n=256, n_bumps=16, seed=5).to(DEV)
    h = P.pndf_build_hierarchy(st)
    q = synth.make_queries(st, 50000, synth.QueryMix(sigma=(1.0, 12.0)), 6)
    out = torch.empty(q.shape[0], dtype=torch.float32, device=DEV)
    flags = torch.empty(q.shape[0], dtype=torch.int32, device=DEV)
    P.pndf_eval_batch_noalloc(h, q, out=out, flags=flags)  # first call on the device: address lookup
    assert _pool_peak_after(rt, lambda: P.pndf_eval_batch_noalloc(h, q, out=out, flags=flags)) == 0
    assert _pool_peak_after(rt, lambda: P.pndf_eval_batch_ex(h, q, out=out, flags=flags)) > 0
    assert torch.equal(out, P.pndf_eval_batch_noalloc(h, q))
    h.free()


def test_noalloc_rejects_batches_over_its_limit(P):
    st = synth.bumps_map(n=32, n_bumps=3, seed=1).to(DEV)
    h = P.pndf_build_hierarchy(st)
    limit = P.pndf_eval_noalloc_max_queries()
    assert limit == 1 << 20
    q = torch.zeros(limit + 1, 8, dtype=torch.float32, device=DEV)
    with pytest.raises(P.PndfError) as ei:
        P.pndf_eval_batch_noalloc(h, q)
    assert ei.value.code == 5  # PNDF_ERR_CAPACITY
    h.free()
