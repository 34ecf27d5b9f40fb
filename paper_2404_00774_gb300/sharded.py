"""Row-sharded search over several GPUs (one process per GPU).

Every rank holds the rows of one contiguous block of datapoints, indexed
under the same codebook C (so every shard ranks the partitions alike and
probes the same ones, Section 2.2).  A search runs on every shard, the
per-shard top-k lists are gathered (the only exchange step) and merged into
the global top k, a point counting once (Section 3.5).  This module only
sequences calls: the searches and the merge are the library's kernels
(soar_search, soar_merge_topk); torch.distributed carries the lists.
"""
from __future__ import annotations

import torch

from . import binding as sb


def shard_bounds(n: int, rank: int, world: int) -> tuple[int, int]:
    """Rows [lo, hi) of rank `rank`: contiguous blocks whose sizes differ by at most one."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def all_shard_offsets(n: int, world: int, device) -> torch.Tensor:
    """First global row of every rank's shard, int64 [world]."""
    return torch.tensor([shard_bounds(n, r, world)[0] for r in range(world)], dtype=torch.int64, device=device)


def gather_lists(ids: torch.Tensor, scores: torch.Tensor, group=None):
    """Every rank's [nq][k] lists stacked as [nq][world][k] (all-gather)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    gi = [torch.empty_like(ids) for _ in range(world)]
    gs = [torch.empty_like(scores) for _ in range(world)]
    dist.all_gather(gi, ids.contiguous(), group=group)
    dist.all_gather(gs, scores.contiguous(), group=group)
    return torch.stack(gi, dim=1).contiguous(), torch.stack(gs, dim=1).contiguous()


def sharded_search(index, Q: torch.Tensor, k: int, t: int, n_total: int, group=None, search=None, merge=None):
    """Global top k of the queries Q over all shards; every rank returns the
    same [nq][k] ids (global row ids) and scores.

    ``search(index, Q, k, t)`` and ``merge(ids, scores, k, offsets)`` default to
    the library's soar_search and soar_merge_topk; they are parameters so that
    the sharding and gathering logic can be exercised on the host."""
    import torch.distributed as dist
    search = search or (lambda ix, q, kk, tt: sb.soar_search(ix, q, kk, tt))
    merge = merge or (lambda i, s, kk, off: sb.soar_merge_topk(i, s, kk, off))
    ids, scores = search(index, Q, k, t)
    gi, gs = gather_lists(ids, scores, group)
    offsets = all_shard_offsets(n_total, dist.get_world_size(group), gi.device)
    return merge(gi, gs, k, offsets)
