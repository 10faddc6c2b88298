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

import numpy as np
import pytest
import torch

from paper_2505_08985_gb300 import synth
from parity import RTOL, rel_err

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_08985_gb300 import pndf
    return pndf


def test_noalloc_matches_allocating_entry_point_twice(P):
    st = synth.scratch_map(n=512, n_grooves=100, seed=41).to(DEV)
    mix = synth.QueryMix(sigma=(1.0, 30.0), aspect=(1.0, 4.0), frac_near=0.7)
    batches = [synth.make_queries(st, 20000, mix, 42), synth.make_queries(st, 7001, mix, 43)]
    for bounds in (P.PNDF_BOUNDS_F32, P.PNDF_BOUNDS_F16_OUTWARD):
        h = P.pndf_build_hierarchy(st, bounds_fmt=bounds)
        for q in batches:  # two calls in a row: the shared scratch keeps the previous call's contents
            ref = P.pndf_eval_batch(h, q).cpu().double().numpy()
            flags = torch.zeros(q.shape[0], dtype=torch.int32, device=DEV)
            got = P.pndf_eval_batch_noalloc(h, q, flags=flags).cpu().double().numpy()
            assert rel_err(got, ref).max() <= RTOL
            assert np.count_nonzero(ref) > 1000
            assert not (flags.cpu().numpy() & P.PNDF_QF_INVALID).any()
        h.free()
    assert P.pndf_device_status() == 0


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
