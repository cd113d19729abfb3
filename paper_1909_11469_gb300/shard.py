"""Sharding of independent graphs across ranks (one process per GPU).

Batches of independent graphs shard without any exchange on the data path:
rank r of N runs seeds [r * per_rank, (r + 1) * per_rank) and numbers its
graphs from graph_id_base = r * graphs_per_rank, so the RnBP Philox streams
(keyed by graph id) of different ranks never coincide and the union over ranks
equals one run over all graphs. The only collectives are the timing and
counter reductions after the timed region.
"""
from __future__ import annotations


def shard_seeds(rank: int, world: int, per_rank: int) -> range:
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return range(rank * per_rank, (rank + 1) * per_rank)


def graph_id_base(rank: int, graphs_per_rank: int) -> int:
    return rank * graphs_per_rank


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
