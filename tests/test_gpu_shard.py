"""One batch sharded over hierarchy replicas (contiguous ranges of the
evaluation order with equal estimated work, gathered back into caller
order): the result equals one pndf_eval_batch bit for bit, since a query's
density depends only on the query and the read-only map (Eq. 5).  Several
replicas share the one GPU here; the data movement is the same as across
devices."""

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


@pytest.mark.parametrize("nshards", [2, 3])
def test_sharded_equals_one_batch(P, nshards):
    from paper_2505_08985_gb300 import shard
    st = synth.flake_normals(1024, 3000, seed=12).to(DEV)
    mix = synth.QueryMix(sigma=(1.0, 100.0), frac_near=0.7)
    q = synth.make_queries(st, 50000, mix, 12)
    h = P.pndf_build_hierarchy(st, bounds_fmt=P.PNDF_BOUNDS_F16_OUTWARD)
    replicas = [h] + [P.pndf_build_hierarchy(st, bounds_fmt=P.PNDF_BOUNDS_F16_OUTWARD) for _ in range(nshards - 1)]
    ref = P.pndf_eval_batch(h, q)
    D, bounds = shard.eval_sharded(replicas, q)
    torch.cuda.synchronize()
    assert torch.equal(D, ref)
    assert len(bounds) == nshards + 1 and bounds[0] == 0 and bounds[-1] == q.shape[0]
    assert all(b > a for a, b in zip(bounds, bounds[1:]))  # every replica gets work
    # the estimated work is balanced: each range within 15% of an equal share
    order = P.pndf_sort_queries(h, q)
    w = P.pndf_shard_work(q, order, block=256).cpu().numpy()
    cum = np.concatenate([[0.0], np.cumsum(w)])
    shares = [(cum[(b + 255) // 256] - cum[a // 256]) / cum[-1] for a, b in zip(bounds, bounds[1:])]
    assert max(abs(s - 1.0 / nshards) for s in shares) < 0.15, shares
    for r in replicas:
        r.free()


def test_gather_and_scatter_are_inverse(P):
    st = synth.bumps_map(n=128, n_bumps=10, seed=3).to(DEV)
    q = synth.make_queries(st, 3001, synth.QueryMix(sigma=(1.0, 9.0)), 3)
    h = P.pndf_build_hierarchy(st)
    order = P.pndf_sort_queries(h, q)
    g = P.pndf_gather_queries(q, order, 1000, 1500)
    assert torch.equal(g, q[order[1000:2500].long()])
    out = torch.full((3001,), -1.0, device=DEV)
    P.pndf_scatter_results(torch.arange(1500, dtype=torch.float32, device=DEV), order, 1000, out)
    idx = order[1000:2500].long()
    assert torch.equal(out[idx], torch.arange(1500, dtype=torch.float32, device=DEV))
    rest = torch.ones(3001, dtype=torch.bool, device=DEV)
    rest[idx] = False
    assert (out[rest] == -1.0).all()
    h.free()
