"""Sharding one amplitude estimate over several ranks (one GPU each).

Samples are independent and the Philox stream is counter-based, so rank r of
W takes the contiguous sample range ``shard_range(n_mc, r, W)`` with
``su_options.sample0`` at its start and ``n_blocks`` blocks of its own; the
union of the ranks' blocks is exactly the blocks of one run over all samples
(same samples, same per-block reductions).  The only exchange is the gather of
the per-block log-sum-exp tuples (4 doubles each) after the sampling, which
``gather_block_tuples`` does with torch.distributed (NCCL or gloo).
"""
from __future__ import annotations

import numpy as np


def shard_range(n_mc, rank, world):
    """(sample0, n) of rank's contiguous share of n_mc samples."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank out of range")
    lo = rank * n_mc // world
    hi = (rank + 1) * n_mc // world
    return lo, hi - lo


def gather_block_tuples(local, group=None):
    """All-gather every rank's (n_blocks_r, levels, 4) tuple array and return
    them concatenated in rank order (the block order of the whole run)."""
    import torch
    import torch.distributed as dist

    local = np.ascontiguousarray(local, dtype=np.float64)
    world = dist.get_world_size(group)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    shape = torch.tensor(list(local.shape), dtype=torch.int64, device=dev)
    shapes = [torch.zeros_like(shape) for _ in range(world)]
    dist.all_gather(shapes, shape, group=group)
    rows = [int(s[0]) for s in shapes]
    width = int(np.prod(local.shape[1:]))
    mx = max(rows)
    buf = torch.zeros((mx, width), dtype=torch.float64, device=dev)
    buf[:local.shape[0]] = torch.from_numpy(local.reshape(local.shape[0], width)).to(dev)
    parts = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    out = [p[:r].cpu().numpy() for p, r in zip(parts, rows)]
    return np.concatenate(out, axis=0).reshape((-1,) + local.shape[1:])
