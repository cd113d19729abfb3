"""The N > 1 host logic on CPU: two gloo ranks shard the seeds of a batch
without overlap, number their graphs so the RnBP random streams differ, and
reduce the timing (max) and counters (sum) as bench.py does."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1909_11469_gb300 import shard, synth


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = list(shard.shard_seeds(rank, world, 5))
        batch = synth.ising_grid_batch(6, 1.0, seeds)
        base = shard.graph_id_base(rank, batch.n_graphs)
        # fake per-rank timing and counters
        ms, (committed, n) = shard.reduce_step_stats(dist, "cpu", 10.0 + rank, [100.0 * (rank + 1), 1.0])
        gathered = [None] * world
        dist.all_gather_object(gathered, {"seeds": seeds, "base": base,
                                          "first_unary": batch.unary_log[:4].tolist()})
        if rank == 0:
            out.put({"ms": ms, "committed": committed, "n": n, "ranks": gathered})
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_and_reductions():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res["ms"] == 11.0 and res["committed"] == 300.0 and res["n"] == 2.0
    s0, s1 = res["ranks"][0]["seeds"], res["ranks"][1]["seeds"]
    assert set(s0).isdisjoint(s1) and sorted(s0 + s1) == list(range(10))
    assert res["ranks"][0]["base"] == 0 and res["ranks"][1]["base"] == 5
    # rank 1's graph 0 is seed 5: the same inputs a single run over all ten seeds gives
    single = synth.ising_grid(6, 1.0, 5)
    assert np.allclose(res["ranks"][1]["first_unary"], single.unary_log[:4])


def test_philox_streams_differ_across_ranks():
    """Graph g of rank r draws with graph id r * G + g: the oracle's RnBP frontier
    of the same graph under the two ids differs (so ranks never share draws),
    and each equals the one-process run with that id."""
    import oracle
    prob = synth.ising_grid(8, 2.0, 3)
    a = oracle.run(prob, "rnbp", parallelism=0.5, high_p=0.5, eps=1e-9, max_rounds=1, trace_cap=1,
                   graph_id=shard.graph_id_base(0, 5))
    b = oracle.run(prob, "rnbp", parallelism=0.5, high_p=0.5, eps=1e-9, max_rounds=1, trace_cap=1,
                   graph_id=shard.graph_id_base(1, 5))
    assert not np.array_equal(a["trace"], b["trace"])


def test_shard_rejects_bad_rank():
    with pytest.raises(ValueError):
        shard.shard_seeds(2, 2, 5)


def test_balanced_ranges_cover_and_balance():
    batch = synth.er_batch(300, 7, n_max=3000)
    m = np.diff(batch.row_ptr[batch.graph_var_offsets])
    for world in (1, 2, 3, 8):
        rs = shard.balanced_ranges(m, world)
        assert len(rs) == world
        assert [g for r in rs for g in r] == list(range(batch.n_graphs))
        loads = [int(m[list(r)].sum()) for r in rs]
        assert max(loads) - m.sum() / world < m.max() + 1


def _worker_ranges(rank, world, port, out):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        batch = synth.er_batch(40, 3, n_max=300)
        m = np.diff(batch.row_ptr[batch.graph_var_offsets])
        mine = shard.balanced_ranges(m, world)[rank]
        # the rank's first graph under its batch-wide id replays the one-process run
        g0 = mine.start
        res = oracle.run(batch.graph(g0), "rnbp", parallelism=0.5, eps=1e-6, max_rounds=30, seed=2,
                         graph_id=mine.start + 0)
        load = int(m[list(mine)].sum())
        gathered = [None] * world
        dist.all_gather_object(gathered, {"range": [mine.start, mine.stop], "load": load,
                                          "committed": res["committed_updates"]})
        if rank == 0:
            out.put(gathered)
    finally:
        dist.destroy_process_group()


def test_two_rank_balanced_batch():
    """Each rank takes its balanced range of one batch and numbers its graphs
    from the range start: the rank's graphs replay the one-process run."""
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 30500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker_ranges, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (a0, b0), (a1, b1) = res[0]["range"], res[1]["range"]
    assert a0 == 0 and b0 == a1 and b1 == 40
    batch = synth.er_batch(40, 3, n_max=300)
    ref = oracle.run(batch.graph(a1), "rnbp", parallelism=0.5, eps=1e-6, max_rounds=30, seed=2, graph_id=a1)
    assert res[1]["committed"] == ref["committed_updates"]
