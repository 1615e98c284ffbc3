"""Population sharding across ranks for the GA fitness batch.

The (parameter set, configuration) evaluations are independent (Sec. III.C), so P parameter sets
split across ranks with the configurations replicated: each rank builds the same neighbour lists
and geometry and evaluates its contiguous slice of the population. The only exchange per
generation is the gather of the fitness values Z[P] (8 bytes per parameter set), plus a broadcast
of the next population from the rank that breeds it.

These helpers work with any torch.distributed backend (gloo on CPU tensors, NCCL on CUDA tensors).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def population_shard(P: int, world_size: int, rank: int) -> tuple[int, int]:
    """[start, stop) of rank's slice of P parameter sets: contiguous, sizes differing by at most one,
    the larger slices first. A rank may get an empty slice when P < world_size."""
    if P < 0 or world_size < 1 or not 0 <= rank < world_size:
        raise ValueError(f"bad shard request P={P} world_size={world_size} rank={rank}")
    base, extra = divmod(P, world_size)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def gather_population_values(local: torch.Tensor, P: int, group=None) -> torch.Tensor:
    """All-gather each rank's per-parameter-set values (shape [n_rank, ...], rows in the order of its
    slice) into the full [P, ...] tensor on every rank, in population order."""
    ws = dist.get_world_size(group)
    rank = dist.get_rank(group)
    s0, s1 = population_shard(P, ws, rank)
    if local.shape[0] != s1 - s0:
        raise ValueError(f"rank {rank} holds {local.shape[0]} rows, its slice has {s1 - s0}")
    rows = population_shard(P, ws, 0)[1]                # the largest slice
    pad = torch.zeros((rows,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: s1 - s0] = local
    parts = [torch.empty_like(pad) for _ in range(ws)]
    dist.all_gather(parts, pad, group=group)
    out = [parts[r][: population_shard(P, ws, r)[1] - population_shard(P, ws, r)[0]] for r in range(ws)]
    return torch.cat(out, dim=0)


def broadcast_population(params: torch.Tensor, src: int = 0, group=None) -> torch.Tensor:
    """Broadcast the [P][6] population from rank src to every rank (in place) and return it."""
    dist.broadcast(params, src=src, group=group)
    return params
