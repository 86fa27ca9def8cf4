"""Contiguous shards of a triple store, one per GPU.

Section 3 (after Algorithm 1) spreads the search over several GPUs by giving
each GPU its own chunk of the triples, running the search kernel on every GPU
and aggregating the results.  Here a shard is the triple range
``[base, base + n_local)`` of the store's columns, loaded as a borrowed view
(``tid_load`` with ``copy=0``); ``tid_match`` on it returns LOCAL ascending
indices, and ``base + local`` are the store's own indices.  Because the shards
are contiguous and in rank order, the global answer of a search is the
concatenation, in rank order, of every shard's list offset by its base: the
only exchange is a count per rank and the lists themselves.

Any store the int32 index type allows (at most 2^31 - 1 triples, 26 GB) fits
one GB300, so shards buy speed, not room: N GPUs each scan n/N triples of the
same query.  The benchmark instead runs independent queries on each GPU
(replicas), which needs no exchange at all.
"""
from __future__ import annotations

import numpy as np

ALIGN = 4  # triples: 16 bytes of int32, so every shard of an aligned store keeps 16-byte loads


def shard_range(n: int, world: int, rank: int, align: int = ALIGN) -> tuple[int, int]:
    """(base, n_local) of rank's shard: near-equal contiguous ranges in rank order,
    every inner boundary a multiple of `align`, together covering [0, n)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} of world {world}")
    if n < 0 or align < 1:
        raise ValueError("n >= 0 and align >= 1")

    def cut(r):
        return n if r == world else (n * r // world) // align * align

    lo, hi = cut(rank), cut(rank + 1)
    return lo, max(0, hi - lo)


def load_shard(ctx, s, p, o, world: int, rank: int):
    """Borrow rank's shard of device columns s, p, o (torch CUDA tensors, which
    must outlive the store).  Returns (store, base)."""
    from . import binding
    base, m = shard_range(int(s.shape[0]), world, rank)
    store = binding.tid_load(ctx, s[base:base + m], p[base:base + m], o[base:base + m], copy=0)
    return store, base


def global_indices(local: np.ndarray, base: int) -> np.ndarray:
    """A shard's local index list as the store's indices (int32: n < 2^31)."""
    return np.asarray(local, dtype=np.int32) + np.int32(base)


def gather_global(local: np.ndarray, base: int, group=None) -> np.ndarray:
    """Every rank's local list (host int32) in, the whole store's ascending list
    out, on every rank: one all-gather of the counts, one of the lists padded to
    the longest.  Tensors live on the CPU for gloo and on the current CUDA device
    for nccl."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" \
        else torch.device("cpu")
    mine = torch.from_numpy(global_indices(local, base)).to(dev)
    cnt = torch.tensor([mine.numel()], dtype=torch.int64, device=dev)
    counts = [torch.zeros_like(cnt) for _ in range(world)]
    dist.all_gather(counts, cnt, group=group)
    counts = [int(c.item()) for c in counts]
    width = max(counts + [1])
    padded = torch.zeros(width, dtype=torch.int32, device=dev)
    padded[:mine.numel()] = mine
    parts = [torch.zeros_like(padded) for _ in range(world)]
    dist.all_gather(parts, padded, group=group)
    return np.concatenate([t[:c].cpu().numpy() for t, c in zip(parts, counts)]).astype(np.int32)
