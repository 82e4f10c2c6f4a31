"""Host-side sharding of a scan across ranks (one process per GPU).

The scan splits by SNP with no exchange on the data path (section "Data
slicing": a slice starting at a given marker is an independent job).  A rank
scans SNP rows [begin, end) of its shard; hit lists concatenate and the
permutation minima merge by element-wise minimum.  The only collectives are the
timing barrier and max, and the optional gathers below.
"""
from __future__ import annotations

import numpy as np


def shard_bounds(S, rank, world):
    """SNP rows [begin, end) of `rank` when S rows are split into `world` nearly
    equal contiguous shards (the first S % world shards get one extra row)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank / world")
    base, extra = divmod(int(S), int(world))
    begin = rank * base + min(rank, extra)
    end = begin + base + (1 if rank < extra else 0)
    return begin, end


def merge_hits(parts):
    """Concatenates per-shard hit lists (each an int array [k, 4] of trait, snp,
    d0, d1 with global SNP indices) plus their H, p; returns them sorted by
    (snp, trait)."""
    hits = np.concatenate([p[0] for p in parts], axis=0) if parts else np.zeros((0, 4), np.int64)
    H = np.concatenate([p[1] for p in parts]) if parts else np.zeros(0)
    P = np.concatenate([p[2] for p in parts]) if parts else np.zeros(0)
    order = np.lexsort((hits[:, 0], hits[:, 1])) if hits.size else np.zeros(0, np.int64)
    return hits[order], H[order], P[order]


def merge_minp(parts):
    """Element-wise minimum of per-shard [P, T] minimum-p tables."""
    out = np.array(parts[0], dtype=np.float64, copy=True)
    for p in parts[1:]:
        np.minimum(out, p, out=out)
    return out


def max_over_ranks(x, device=None):
    """Maximum of a float over all ranks of the default process group (x itself
    when torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_objects(obj):
    """All ranks' `obj` in rank order (a one-element list without a process group)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return [obj]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, obj)
    return out
