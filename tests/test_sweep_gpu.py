"""The Residual Splash sweeps (binary messages): one launch per sub-step over
batch-wide per-level vertex lists, the commit of a level fused with the
evaluation of the next (the splash of Section III-C with the level order h,
..., 0, ..., h). FP64 runs replay the oracle exactly, and the lists built by
the cluster selection and by the grid-wide kernels give the same bits in
every storage format. (Two other sweep forms -- a commit and an evaluation
entry per thread, and every sub-step in one cluster kernel -- measured slower
and are retired: bp_options.splash_sweep 2 and 3 are rejected.)"""
import math

import numpy as np
import pytest

import oracle
from paper_1909_11469_gb300 import bp, synth

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-10


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def uneven_batch():
    members = [synth.ising_grid(9, 1.0, seed=1), synth.ising_chain(300, 2.0, seed=2),
               synth.ising_grid(20, 2.0, seed=3, cols=7), synth.ising_tree(50, 1.5, seed=4),
               synth.ising_grid(3, 0.0, seed=5)]
    members += [synth.er_batch(1, seed=s, n_min=30, n_max=400).graph(0) for s in range(5)]
    return members, synth.concat_batch(members)


def run(prob, dtype, sweep, depth=2, par=0.1, rounds=40, eps=1e-5, profile=0, **opts):
    """RS run; profile = 1 launches the rounds directly, 0 replays captured rounds."""
    with bp.Graph(prob) as g:
        st = g.run("rs", par, eps=eps, max_rounds=rounds, msg_dtype=dtype, splash_sweep=sweep,
                   splash_depth=depth, profile=profile, **opts)
        return (st, g.beliefs(), g.messages(), [(x["converged"], x["rounds"], x["committed_updates"])
                                                 for x in g.graph_stats()], g.profile())


@pytest.mark.parametrize("depth", [0, 1, 2, 3])
@pytest.mark.parametrize("select_path", [1, 2])
def test_fp64_batch_replays_oracle(select_path, depth):
    """Every graph of an uneven batch matches the oracle run of that graph
    alone over 40 rounds: rounds, convergence, committed updates, beliefs.
    (The horizon is short: the 156-vertex ER member is not contracting -- the
    k-th largest vertex residual stays near 0.5 for 170 rounds -- so the
    rounding differences of two FP64 implementations grow from round to round
    until one of them takes other splash roots, although the smallest relative
    gap at the k-th root in the oracle's 214 rounds is 1.2e-6, at round 132.)"""
    members, batch = uneven_batch()
    T = 40
    st, bel, msg, gst, prof = run(batch, "f64", 1, depth=depth, par=0.05, rounds=T, select_path=select_path)
    assert prof["sweep_ctas"] == 0 and prof["sweep_form"] == 0
    for gi, m in enumerate(members):
        ref = oracle.run(m, "rs", parallelism=0.05, eps=1e-5, max_rounds=T, splash_depth=depth,
                         graph_id=gi)
        assert gst[gi][1] == ref["rounds"], gi
        assert bool(gst[gi][0]) == ref["converged"], gi
        assert gst[gi][2] == ref["committed_updates"], gi
        v0, v1 = batch.graph_var_offsets[gi], batch.graph_var_offsets[gi + 1]
        assert np.abs(bel[v0:v1] - ref["beliefs"]).max() < 1e-9, gi


def selection_safe_rounds(m, depth, p, T, gid):
    """Rounds of the oracle's RS run (at most T) before the first root
    selection that rounding decides: the k-th largest vertex residual is below
    1e-12 or within 1e-9 (relative) of the next. On trees a deep splash makes
    messages exact, so many vertex residuals fall to rounding level (exact 0
    in one FP64 implementation, 1e-16 in the other) while k roots are still
    chosen among them; from that round on the two runs may splash other
    vertices."""
    kv = min(max(math.ceil(p * len(m.col)), 1), m.n)
    row_ptr, rev = np.asarray(m.row_ptr), np.asarray(m.rev)
    for r in range(T):
        o = oracle.run(m, "rs", parallelism=p, eps=1e-5, max_rounds=r, splash_depth=depth, graph_id=gid)
        if o["converged"]:
            return T
        _, res = oracle.evaluate(m, o["messages"])
        vres = np.array([res[rev[row_ptr[v]:row_ptr[v + 1]]].max() if row_ptr[v + 1] > row_ptr[v] else 0.0
                         for v in range(m.n)])
        s = np.sort(vres)[::-1]
        kth, nxt = s[kv - 1], (s[kv] if kv < m.n else -1.0)
        if kth < 1e-12 or kth - nxt <= 1e-9 * kth:
            return r
    return T


@pytest.mark.parametrize("depth", [4, 7, 16])
def test_deep_splash_fp64_replays_oracle(depth):
    """Splashes deeper than the level lists hold (h > 3) sweep by scanning the
    level array: the uneven batch matches the oracle graph by graph for as many
    rounds (at most 40) as every graph's root selection stays clear of rounding
    (the 300-vertex chain: 9 rounds at h = 7, 6 at h = 16; at h = 7 and 16 its
    run over 40 rounds did differ from the oracle's after that point)."""
    members, batch = uneven_batch()
    T = min(selection_safe_rounds(m, depth, 0.05, 40, gi) for gi, m in enumerate(members))
    assert T >= 5
    st, bel, msg, gst, prof = run(batch, "f64", 0, depth=depth, par=0.05, rounds=T)
    assert prof["sweep_ctas"] == 0
    for gi, m in enumerate(members):
        ref = oracle.run(m, "rs", parallelism=0.05, eps=1e-5, max_rounds=T, splash_depth=depth,
                         graph_id=gi)
        assert gst[gi][1] == ref["rounds"], gi
        assert bool(gst[gi][0]) == ref["converged"], gi
        assert gst[gi][2] == ref["committed_updates"], gi
        v0, v1 = batch.graph_var_offsets[gi], batch.graph_var_offsets[gi + 1]
        assert np.abs(bel[v0:v1] - ref["beliefs"]).max() < 1e-9, gi


@pytest.mark.parametrize("kind", ["tree", "chain"])
def test_one_deep_splash_is_exact_on_a_tree(kind):
    """One root (p tiny) and a splash as deep as the tree: one round is a
    collect-distribute pass, so the beliefs are the exact marginals."""
    from tests import _exact
    if kind == "tree":
        prob = synth.ising_tree(12, 2.0, seed=11)
        exact = _exact.brute_force_marginals(prob)
    else:
        prob = synth.paper_ising(1, 17, C=6.0, seed=3)
        exact = _exact.chain_marginals(prob)
    with bp.Graph(prob) as g:
        st = g.run("rs", 1e-9, eps=1e-300, max_rounds=1, msg_dtype="f64", splash_depth=prob.n - 1)
        assert st["rounds"] == 1
        assert np.abs(g.beliefs() - exact).max() < 1e-12


@pytest.mark.parametrize("sweep", [0, 1])
def test_fp64_trace_replay(sweep):
    """Same splash roots every round and the same state after 60 rounds of a
    ragged 13 x 11 grid."""
    prob = synth.ising_grid(13, 2.0, seed=4, cols=11)
    T = 60
    ref = oracle.run(prob, "rs", parallelism=0.1, eps=1e-7, max_rounds=T, trace_cap=T)
    with bp.Graph(prob) as g:
        st = g.run("rs", 0.1, eps=1e-7, max_rounds=T, msg_dtype="f64", splash_sweep=sweep,
                   record_trace=1, trace_capacity=T)
        tr = g.trace("rs")
        assert st["rounds"] == ref["rounds"]
        assert np.array_equal(tr, ref["trace"][:ref["rounds"]])
        assert st["committed_updates"] == ref["committed_updates"]
        assert np.abs(g.beliefs() - ref["beliefs"]).max() < TOL_F64
        assert np.abs(g.messages() - ref["messages"]).max() < TOL_F64


@pytest.mark.parametrize("name", ["uneven", "er", "grids"])
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "q16"])
@pytest.mark.parametrize("depth", [2, 3])
def test_selection_paths_bit_identical(name, dtype, depth):
    """The level lists come from the cluster selection (BFS inside the
    cluster) or from the grid-wide kernels (separate BFS launches): the sweeps
    over them give the same bits, captured or launched directly."""
    if name == "uneven":
        prob = uneven_batch()[1]
    elif name == "er":
        prob = synth.er_batch(60, 7, n_max=1500)
    else:
        prob = synth.ising_grid_batch(40, 2.5, range(6))
    a = run(prob, dtype, 1, depth=depth, select_path=1)
    b = run(prob, dtype, 1, depth=depth, select_path=2, profile=1 if depth == 3 else 0)
    keys = ("rounds", "committed_updates", "candidate_evals", "converged")
    assert [a[0][k] for k in keys] == [b[0][k] for k in keys]
    assert a[3] == b[3]
    assert np.array_equal(a[1], b[1]), float(np.abs(a[1] - b[1]).max())
    assert np.array_equal(a[2], b[2])


def test_bad_splash_sweep_rejected():
    prob = synth.ising_grid(5, 1.0, seed=0)
    with bp.Graph(prob) as g:
        for bad in (2, 3, 4):
            with pytest.raises(bp.BPError) as ei:
                g.run("rs", 0.1, splash_sweep=bad)
            assert ei.value.code == bp.BP_ERR_INVALID_ARG
