"""One batch sharded over hierarchy replicas.

The P-NDF of each query depends only on the query and the (read-only) map
(Sec. 4.2, Eq. 5), so a batch splits over replicas of the hierarchy without
any exchange but the final gather.  The batch is put in evaluation order once
(the library's key sort: entry level, largest footprints first, then
footprint tile), the order is cut into contiguous ranges of about equal
estimated work (so each replica gets a spatially coherent part of the map and
a fair share of the large footprints' work), each range is gathered into a
contiguous batch and evaluated on its replica in that order, and the results
are scattered back into caller order on the home device.  Replicas may sit
on different devices (copies between devices are plain device-to-device
copies; no kernel reads another device's memory) or several on one device.
"""

from __future__ import annotations

import torch

from . import pndf

WORK_BLOCK = 4096  # positions of the evaluation order per work sum


def split_by_work(partials, nshards: int, nq: int, block: int = WORK_BLOCK) -> list[int]:
    """Boundaries 0 = b_0 <= b_1 <= ... <= b_n = nq of n contiguous ranges of
    the evaluation order with about equal estimated work: b_i is the block
    boundary whose cumulative work is nearest to i/n of the total (host logic
    on the per-block sums of pndf_shard_work)."""
    if nshards < 1:
        raise ValueError("nshards must be >= 1")
    sums = [float(x) for x in partials]
    total = sum(sums)
    bounds = [0]
    acc, b = 0.0, 0
    for i in range(1, nshards):
        target = total * i / nshards
        while b < len(sums) and acc + sums[b] <= target:
            acc += sums[b]
            b += 1
        if b < len(sums) and (acc + sums[b]) - target < target - acc:
            acc += sums[b]
            b += 1
        bounds.append(min(nq, max(bounds[-1], b * block)))
    bounds.append(nq)
    return bounds


def work_block(nq: int, nshards: int) -> int:
    """Positions per work sum: about 64 sums per shard, 256 to 4096 (large
    footprints cluster at the front of the order, so small batches need
    fine blocks to balance)."""
    b = nq // (64 * max(nshards, 1))
    return int(min(WORK_BLOCK, max(256, b)))


def eval_sharded(hierarchies, queries: torch.Tensor, out: torch.Tensor | None = None, block: int | None = None):
    """D for `queries` (on the first hierarchy's device) evaluated over all
    `hierarchies` (replicas of one map, any devices), in caller order on the
    queries' device.  Returns (D, bounds): bounds are the ranges of the
    evaluation order each replica evaluated."""
    home = queries.device
    h0 = hierarchies[0]
    if h0.device != home:
        raise ValueError("queries must be on the first hierarchy's device")
    nq = queries.shape[0]
    if out is None:
        out = torch.empty(nq, dtype=torch.float32, device=home)
    if nq == 0:
        return out, [0] * (len(hierarchies) + 1)
    block = block or work_block(nq, len(hierarchies))
    order = pndf.pndf_sort_queries(h0, queries)
    partials = pndf.pndf_shard_work(queries, order, block=block).cpu().tolist()
    bounds = split_by_work(partials, len(hierarchies), nq, block)
    home_stream = torch.cuda.current_stream(home)
    pieces = []
    for i, h in enumerate(hierarchies):
        a, b = bounds[i], bounds[i + 1]
        if b == a:
            continue
        qi = pndf.pndf_gather_queries(queries, order, a, b - a)
        if h.device != home:
            s = torch.cuda.current_stream(h.device)
            s.wait_stream(home_stream)
            with torch.cuda.device(h.device):
                qi = qi.to(h.device, non_blocking=True)
        Di = pndf.pndf_eval_batch_ex(h, qi, sort=pndf.PNDF_SORT_NONE)
        pieces.append((a, Di))
    for a, Di in pieces:
        if Di.device != home:
            home_stream.wait_stream(torch.cuda.current_stream(Di.device))
            Di = Di.to(home, non_blocking=True)
        pndf.pndf_scatter_results(Di, order, a, out)
    return out, bounds


def gather_shards(D_local: torch.Tensor, bounds: list[int], rank: int, world: int):
    """Across ranks (torch.distributed, one shard per rank): every rank holds
    the results of its range [bounds[rank], bounds[rank + 1]) of the
    evaluation order; rank 0 receives all of them concatenated in evaluation
    order (None on the other ranks).  Shards differ in length, so each is
    padded to the longest before the all-gather and cut back after."""
    import torch.distributed as dist
    counts = [bounds[i + 1] - bounds[i] for i in range(world)]
    if D_local.numel() != counts[rank]:
        raise ValueError("the local results do not match this rank's range")
    width = max(max(counts), 1)
    buf = torch.zeros(width, dtype=D_local.dtype, device=D_local.device)
    buf[:counts[rank]] = D_local
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    if rank != 0:
        return None
    return torch.cat([p[:c] for p, c in zip(parts, counts)])
