"""Partition of one graph across ranks (paper_1909_11469_gb300.partition), on
CPU: the plans reproduce the CSR, the exchange lists pair up, and gloo ranks
that run LBP and RnBP on their blocks -- one exchange of cut messages and one
(max, count) all-reduce per round -- reproduce the one-process FP64 oracle
run: the same rounds, beliefs within 1e-12."""
import os

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1909_11469_gb300 import partition, synth


def _check_plans(prob, owner):
    plans = partition.build_plans(prob.row_ptr, prob.col, prob.rev, owner)
    n, m = prob.n, prob.m
    seen_v = np.concatenate([p.vertices[:p.n_owned] for p in plans])
    assert np.array_equal(np.sort(seen_v), np.arange(n))
    seen_e = np.concatenate([p.edges for p in plans])
    assert np.array_equal(np.sort(seen_e), np.arange(m))
    for p in plans:
        owned = p.vertices[:p.n_owned]
        assert np.all(np.diff(owned) > 0)
        # the local rows are the global rows of the owned vertices
        assert np.array_equal(np.diff(p.row_ptr), np.diff(prob.row_ptr)[owned])
        assert np.array_equal(p.vertices[p.col], prob.col[p.edges])
        glob = np.concatenate([p.edges, p.halo_edges])
        assert np.array_equal(glob[p.rev], prob.rev[p.edges])
        # halo slots hold exactly the reverses of the cut out-edges
        cut = p.edges[owner[prob.col[p.edges]] != p.rank]
        assert np.array_equal(np.sort(prob.rev[cut]), p.halo_edges)
        for q, (ids, slots) in p.send.items():
            rids, rslots = plans[q].recv[p.rank]
            assert np.array_equal(ids, rids)
            assert np.array_equal(glob[slots], ids)
            qglob = np.concatenate([plans[q].edges, plans[q].halo_edges])
            assert np.array_equal(qglob[rslots], ids)
        assert sum(len(ids) for ids, _ in p.recv.values()) == p.n_halo_slots
    return plans


def test_grid_blocks_cover_the_csr():
    rows, cols, pr, pc = 12, 10, 2, 3
    prob = synth.ising_grid(rows, 1.0, seed=0, cols=cols)
    owner = partition.grid_blocks(rows, cols, pr, pc)
    assert sorted(np.unique(owner).tolist()) == list(range(pr * pc))
    plans = _check_plans(prob, owner)
    # cut of a block partition: (pc - 1) column cuts over all rows, (pr - 1) row
    # cuts over all columns, each undirected edge two messages
    assert partition.cut_messages(plans) == 2 * (rows * (pc - 1) + cols * (pr - 1))


@pytest.mark.parametrize("world", [2, 3, 5])
def test_contiguous_ranges_cover_the_csr(world):
    prob = synth.er_batch(1, seed=3, n_min=400, n_max=400)
    owner = partition.contiguous_ranges(prob.row_ptr, world)
    assert np.all(np.diff(owner) >= 0) and owner.max() == world - 1
    loads = np.bincount(owner, weights=np.diff(prob.row_ptr), minlength=world)
    assert loads.max() - prob.m / world <= np.diff(prob.row_ptr).max()
    _check_plans(prob, owner)


# ------------------------------------------------------------------ distributed replay
def _ising_candidates(plan, unary, beta_local, msg):
    """Eq. 2 for the binary Ising layout, probability domain, on the owned
    out-edges: msg[slot, x] over local edges and halo slots."""
    n_own = plan.n_owned
    out = np.empty((plan.n_local_edges, 2))
    s = np.array([-1.0, 1.0])
    for i in range(n_own):
        b, e = plan.row_ptr[i], plan.row_ptr[i + 1]
        inc = msg[plan.rev[b:e]]                   # messages into i, one per out-edge
        for t in range(b, e):
            w = np.exp(unary[i]) * np.prod(np.delete(inc, t - b, axis=0), axis=0)
            psi = np.exp(beta_local[t] * np.outer(s, s))   # [x_i, x_j]
            c = w @ psi
            out[t] = c / c.sum()
    return out


def _replay_worker(rank, world, port, sched, par, owner, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch

    import oracle
    try:
        prob = synth.ising_grid(12, 1.5, seed=4, cols=11)
        plan = partition.build_plans(prob.row_ptr, prob.col, prob.rev, owner)[rank]
        unary = prob.unary_log.reshape(-1, 2).astype(np.float64)[plan.vertices[:plan.n_owned]]
        beta = prob.pair_log.astype(np.float64)[plan.edges]
        msg = np.full((plan.n_local_edges + plan.n_halo_slots, 2), 0.5)
        eps, high_p, thr_ratio, max_rounds = 1e-6, 1.0, 0.9, 500
        t, n_prev, converged = 0, 0, False
        while True:
            cand = _ising_candidates(plan, unary, beta, msg)
            r = np.abs(cand - msg[:plan.n_local_edges]).max(axis=1)
            red = torch.tensor([float(r.max(initial=0.0)), float((r >= eps).sum())], dtype=torch.float64)
            mx = red[:1].clone()
            cnt = red[1:].clone()
            dist.all_reduce(mx, op=dist.ReduceOp.MAX)      # the per-round all-reduce (max, count)
            dist.all_reduce(cnt)
            rmax, n_t = float(mx.item()), int(cnt.item())
            if rmax < eps:
                converged = True
                break
            if t == max_rounds:
                break
            t += 1
            if sched == "lbp":
                pick = np.ones(plan.n_local_edges, bool)
            else:
                p = high_p if t == 1 else (par if n_t / n_prev > thr_ratio else high_p)
                thr = int(p * 65536.0)
                pick = np.zeros(plan.n_local_edges, bool)
                for le, ge in enumerate(plan.edges):
                    if r[le] >= eps:
                        w = int(oracle.philox4x32_10([int(ge) // 8, t, 0, 0], [0, 0])[(int(ge) % 8) // 2])
                        u = (w >> 16) if int(ge) % 2 else (w & 0xFFFF)
                        pick[le] = p >= 1.0 or u < thr
            n_prev = n_t
            msg[:plan.n_local_edges][pick] = cand[pick]
            # one exchange: cut messages to the rank owning their destination
            reqs = []
            bufs = {}
            for q, (ids, slots) in plan.send.items():
                reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(msg[slots])), dst=q))
            for q, (ids, slots) in plan.recv.items():
                bufs[q] = torch.empty((len(ids), 2), dtype=torch.float64)
                reqs.append(dist.irecv(bufs[q], src=q))
            for rq in reqs:
                rq.wait()
            for q, (ids, slots) in plan.recv.items():
                msg[slots] = bufs[q].numpy()
        # beliefs of the owned vertices (Eq. 3)
        bel = np.empty((plan.n_owned, 2))
        for i in range(plan.n_owned):
            b, e = plan.row_ptr[i], plan.row_ptr[i + 1]
            w = np.exp(unary[i]) * np.prod(msg[plan.rev[b:e]], axis=0)
            bel[i] = w / w.sum()
        gathered = [None] * world
        dist.all_gather_object(gathered, (plan.vertices[:plan.n_owned].tolist(), bel.tolist(), t, converged))
        if rank == 0:
            out.put(gathered)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("sched,par", [("lbp", 1.0), ("rnbp", 0.5)])
@pytest.mark.parametrize("world,layout", [(2, (1, 2)), (4, (2, 2))])
def test_partitioned_run_equals_one_process(sched, par, world, layout):
    import oracle
    prob = synth.ising_grid(12, 1.5, seed=4, cols=11)
    owner = partition.grid_blocks(12, 11, *layout)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29600 + (os.getpid() % 500) + 7 * world
    procs = [ctx.Process(target=_replay_worker, args=(r, world, port, sched, par, owner, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = oracle.run(prob, sched, parallelism=par, eps=1e-6, max_rounds=500, seed=0, graph_id=0)
    bel = np.empty((prob.n, 2))
    for verts, b, t, conv in res:
        bel[verts] = np.array(b)
        assert t == ref["rounds"] and conv == ref["converged"]
    assert np.abs(bel - ref["beliefs"]).max() < 1e-12
