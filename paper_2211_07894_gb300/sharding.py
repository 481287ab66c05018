"""Partitioning of the Gateaux-derivative work over ranks (one GPU per rank).

Two partitions are natural (independent units, no data-path collective for
the derivatives themselves):

* by system: each rank owns whole systems (what ``bench.py --gpus N`` runs);
* by direction: each rank evaluates a contiguous slice of the K directions of
  one system on its own replica of Psi.  The least-squares step (Eq. plowrank)
  then needs all K derivatives, which is the one real exchange: an all-gather
  of the slices of v and f (K x nspin x N_g each), after which every rank can
  run the K x K step locally.
"""

from __future__ import annotations


def shard_bounds(K: int, world: int, rank: int):
    """[start, stop) of the directions owned by `rank` (balanced, contiguous)."""
    if world < 1 or not (0 <= rank < world) or K < 0:
        raise ValueError("bad shard arguments")
    base, rem = divmod(K, world)
    start = rank * base + min(rank, rem)
    return start, start + base + (1 if rank < rem else 0)


def gather_directions(local, K: int, group=None):
    """All-gather the per-rank slices (leading dimension = directions) of a
    direction-sharded array into the full (K, ...) array on every rank.
    Slices are padded to the largest slice for the collective."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    sizes = [shard_bounds(K, world, r) for r in range(world)]
    width = max(b - a for a, b in sizes)
    pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[: b - a] for p, (a, b) in zip(parts, sizes)], dim=0)
