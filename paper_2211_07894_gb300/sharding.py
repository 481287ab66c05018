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


def sharded_step(ctx, V, R, alpha, rho=None, sys=0, group=None, coeff=None, s_rel=None):
    """One least-squares preconditioning step (Eqs. plowrank, quasinewton)
    over the K directions V of system `sys`, with the Gateaux derivatives
    evaluated direction-sharded over the ranks of `group`.

    Every rank holds its own context (its replica of the subspace) and passes
    the same V ([K][nspin][N_g]) and R ([nspin][N_g]).  Rank r evaluates its
    contiguous slice of the directions (shard_bounds) through ctx.gateaux (the
    other systems of the context get no directions); the slices of f are
    all-gathered, the one exchange; then every rank runs ctx.apply over all K
    derivatives, so the coefficients, s_rel and the updated density rho are
    the same on every rank (coeff / s_rel: optional output tensors).  Returns
    (F, coeff, s_rel), F the gathered (K, nspin, N_g) derivatives.
    """
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        world, rank = dist.get_world_size(group), dist.get_rank(group)
    else:
        world, rank = 1, 0                   # no process group: one rank owns every direction
    K = int(V.shape[0])
    a, b = shard_bounds(K, world, rank)
    Vs = [None] * int(getattr(ctx, "nsys", 1))
    Vs[sys] = V[a:b].contiguous()
    F_parts, _ = ctx.gateaux(Vs)
    F = gather_directions(F_parts[sys], K, group) if world > 1 else F_parts[sys]
    if coeff is None and s_rel is None:
        coeff, s_rel = ctx.apply(sys, R, V, F, alpha, rho=rho)
    else:
        coeff, s_rel = ctx.apply(sys, R, V, F, alpha, rho=rho, coeff=coeff, s_rel=s_rel)
    return F, coeff, s_rel
