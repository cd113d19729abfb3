"""Sharding of independent graphs across ranks (one process per GPU).

Batches of independent graphs shard without any exchange on the data path:
rank r of N runs seeds [r * per_rank, (r + 1) * per_rank) and numbers its
graphs from graph_id_base = r * graphs_per_rank, so the RnBP Philox streams
(keyed by graph id) of different ranks never coincide and the union over ranks
equals one run over all graphs. One given batch splits into contiguous graph
ranges balanced by directed edges (balanced_ranges). The only collectives are
the timing and counter reductions after the timed region.
"""
from __future__ import annotations


def shard_seeds(rank: int, world: int, per_rank: int) -> range:
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return range(rank * per_rank, (rank + 1) * per_rank)


def graph_id_base(rank: int, graphs_per_rank: int) -> int:
    return rank * graphs_per_rank


def balanced_ranges(edge_counts, world: int) -> list[range]:
    """Contiguous ranges of a batch's graphs, one per rank, balanced by
    directed edges (the per-round work of the update and selection kernels):
    rank r ends its range where the running edge sum first reaches
    (r + 1) / world of the total. With contiguous ranges a rank passes its
    range's start as bp_options.graph_id_base, so every graph keeps its
    batch-wide id and the sharded runs draw the same RnBP random streams as one
    run over the whole batch. A rank's load exceeds the ideal share by less
    than its largest graph."""
    import numpy as np
    m = np.asarray(edge_counts, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    total = int(m.sum())
    cum = np.cumsum(m)
    out, start = [], 0
    for r in range(world):
        if r == world - 1:
            end = len(m)
        else:
            target = (r + 1) * total / world
            end = int(np.searchsorted(cum, target, side="left")) + 1 if total > 0 else start
            end = max(start, min(end, len(m)))
        out.append(range(start, end))
        start = end
    return out


def reduce_step_stats(dist, device, total_ms: float, counters: list[float]):
    """Max of the timed milliseconds and sum of the counters over all ranks
    (dist = torch.distributed, initialised; device = tensor device for the
    backend). Returns (max_ms, summed counters)."""
    import torch
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor(list(counters), dtype=torch.float64, device=device)
    dist.all_reduce(c)
    return float(t.item()), [float(x) for x in c.tolist()]
