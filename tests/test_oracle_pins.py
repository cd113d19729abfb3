"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test targets a plausible mistake: a dropped or extra factor in Eq. 2 (closed
form, brute force), a wrong cavity index (closed form), a transposed pairwise
table (asymmetric tables on trees), a wrong residual or convergence test
(invariants, special cases), a wrong schedule (identities, serial RBP), a wrong
random stream (Philox known answers), a wrong selection (top-k, BFS).
"""
import os

import numpy as np
import pytest
import scipy.sparse
import scipy.sparse.csgraph

from paper_1909_11469_gb300 import synth
from tests import _exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- Philox
def test_philox_known_answers(orc):
    rows = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        out = orc.philox4x32_10(w[:4], w[4:6])
        assert [int(x) for x in out] == w[6:]
        rows += 1
    assert rows == 3


def test_rnbp_random_filter_fraction(orc):
    """With every message above eps and p = HighP = 0.3 in round 1, the committed
    fraction is Binomial(M, 0.3): within 5 sigma."""
    prob = synth.ising_grid(60, 1.0, seed=3)
    res = orc.run(prob, "rnbp", parallelism=0.3, high_p=0.3, eps=1e-12, max_rounds=1,
                  trace_cap=1)
    m = prob.m
    picked = int(np.unpackbits(res["trace"][0].view(np.uint8)).sum())
    assert res["committed_updates"] == picked
    sd = np.sqrt(m * 0.3 * 0.7)
    assert abs(picked - 0.3 * m) < 5 * sd


def test_rnbp_random_filter_independent(orc):
    """The random filter's picks are independent Bernoulli(p) draws: for two
    messages that share a Philox block (adjacent ids: the two halves of one
    word, or neighbouring words) and for one message in two graphs of a batch
    (graph ids 0 and 1), both are picked with probability p^2 (within 5 sigma;
    round 1, where every message is eligible). A draw reused across the halves
    of a word, across the words of a block or across graphs would give p
    instead."""
    prob = synth.ising_grid(60, 1.0, seed=3)
    p = 0.3
    m = prob.m
    picks = []
    for gid in (0, 1):
        res = orc.run(prob, "rnbp", parallelism=p, high_p=p, eps=1e-12, max_rounds=1, trace_cap=1, graph_id=gid)
        picks.append(np.unpackbits(res["trace"][0].view(np.uint8), bitorder="little")[:m].astype(bool))
    r1, r1b = picks

    def near_p2(both, n):
        sd = np.sqrt(n * p * p * (1 - p * p))
        assert abs(both - p * p * n) < 5 * sd, (both, p * p * n, sd)

    m8 = m - m % 8
    near_p2(int((r1[0:m8:2] & r1[1:m8:2]).sum()), m8 // 2)        # halves of one word
    near_p2(int((r1[0:m8:8] & r1[2:m8:8]).sum()), m8 // 8)        # words 0 and 1 of a block
    near_p2(int((r1[0:m8:8] & r1[7:m8:8]).sum()), m8 // 8)        # first and last message of a block
    near_p2(int((r1 & r1b).sum()), m)                             # one message in two graphs


# --------------------------------------------------------------------------- Eq. 2
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ising_message_closed_form(orc, seed):
    """Every candidate of a random message state equals the atanh closed form."""
    prob = synth.ising_grid(6, 2.5, seed=seed)
    rng = np.random.default_rng(100 + seed)
    p1 = rng.uniform(0.05, 0.95, size=prob.m)
    msg = np.stack([1 - p1, p1], axis=1)
    cand, r = orc.evaluate(prob, msg)
    for e in range(prob.m):
        u = 0.5 * np.log(cand[e, 1] / cand[e, 0])
        assert abs(u - _exact.ising_closed_form(prob, msg, e)) < 1e-13
        assert abs(r[e] - np.abs(cand[e] - msg[e]).max()) < 1e-15
    assert np.allclose(cand.sum(axis=1), 1.0, atol=1e-14)


def test_table_message_direct_eq2(orc):
    """Asymmetric tables, k = 3: every candidate equals a direct transcription of
    Eq. 2 (catches a transposed table or a wrong cavity)."""
    prob = synth.random_table_graph(7, 3, extra_edges=3, seed=5)
    rng = np.random.default_rng(9)
    msg = rng.uniform(0.1, 1.0, size=(prob.m, 3))
    msg /= msg.sum(axis=1, keepdims=True)
    cand, _ = orc.evaluate(prob, msg)
    for e in range(prob.m):
        np.testing.assert_allclose(cand[e], _exact.message_eq2(prob, msg, e), rtol=0, atol=1e-14)


# --------------------------------------------------------------------------- trees
@pytest.mark.parametrize("schedule,par", [("lbp", 1.0), ("rbp", 0.1), ("rs", 0.05), ("rnbp", 0.5)])
def test_tree_exact_brute_force(orc, schedule, par):
    """BP is exact on trees: every schedule converges to the brute-force marginals."""
    prob = synth.ising_tree(12, 2.0, seed=11)
    res = orc.run(prob, schedule, parallelism=par, eps=1e-13, max_rounds=5000, seed=7)
    assert res["converged"]
    exact = _exact.brute_force_marginals(prob)
    assert np.abs(res["beliefs"] - exact).max() < 1e-12


@pytest.mark.parametrize("kind", ["ising_tree", "chain", "table_tree"])
def test_rs_one_deep_splash_is_exact_on_a_tree(orc, kind):
    """Residual Splash with a single root and a splash as deep as the tree
    sweeps the levels from the leaves to the root and back out (Section III-A),
    which on a tree is one exact collect-distribute pass: after ONE round every
    belief equals the exact marginal. A sweep in the wrong order, a sub-step
    that reads stale messages or a missing commit leaves it inexact, and so
    does a splash too shallow to reach the leaves (checked as the control)."""
    if kind == "ising_tree":
        prob, exact = synth.ising_tree(12, 2.0, seed=11), None
    elif kind == "chain":
        prob = synth.paper_ising(1, 40, C=6.0, seed=3)
        exact = _exact.chain_marginals(prob)
    else:
        prob, exact = synth.random_table_graph(9, 3, extra_edges=0, seed=4), None
    if exact is None:
        exact = _exact.brute_force_marginals(prob)
    p_one_root = 1e-9   # k_v = clamp(ceil(p M), 1, n) = 1
    deep = orc.run(prob, "rs", parallelism=p_one_root, eps=1e-300, max_rounds=1, splash_depth=prob.n - 1)
    assert deep["rounds"] == 1
    assert np.abs(deep["beliefs"] - exact).max() < 1e-12
    shallow = orc.run(prob, "rs", parallelism=p_one_root, eps=1e-300, max_rounds=1, splash_depth=1)
    assert np.abs(shallow["beliefs"] - exact).max() > 1e-6


def test_tree_exact_tables_k3(orc):
    prob = synth.random_table_graph(9, 3, extra_edges=0, seed=4)
    res = orc.run(prob, "lbp", eps=1e-14, max_rounds=100)
    assert res["converged"]
    assert np.abs(res["beliefs"] - _exact.brute_force_marginals(prob)).max() < 1e-12


def test_lbp_tree_rounds_bounded_by_diameter(orc):
    """On a tree LBP messages are exact after diameter rounds, so the residuals are
    exactly zero at the next evaluation."""
    prob = synth.ising_chain(40, 2.0, seed=2)
    res = orc.run(prob, "lbp", eps=1e-300, max_rounds=1000)
    assert res["converged"] and res["final_max_residual"] == 0.0
    assert res["rounds"] <= 39


def test_chain_forward_backward(orc):
    prob = synth.paper_ising(1, 300, C=10.0, seed=1)
    res = orc.run(prob, "lbp", eps=1e-14, max_rounds=1000)
    assert res["converged"]
    assert np.abs(res["beliefs"] - _exact.chain_marginals(prob)).max() < 1e-11


# --------------------------------------------------------------------------- special cases
def test_zero_field_symmetric_beliefs(orc):
    """lambda = 0: the model is symmetric under x -> -x, so beliefs are (1/2, 1/2)."""
    prob = synth.ising_grid(8, 2.0, seed=4, lam_max=0.0)
    res = orc.run(prob, "lbp", eps=1e-4, max_rounds=50)
    assert np.abs(res["beliefs"] - 0.5).max() < 1e-15


def test_zero_coupling_converges_immediately(orc):
    """beta = 0: every candidate is uniform, so the uniform start is already a fixed
    point: rounds = 0 and beliefs are the normalised unaries."""
    prob = synth.ising_grid(7, 0.0, seed=4)
    res = orc.run(prob, "lbp", eps=1e-12, max_rounds=50)
    assert res["converged"] and res["rounds"] == 0
    un = np.exp(prob.unary_log.astype(np.float64).reshape(-1, 2))
    assert np.abs(res["beliefs"] - un / un.sum(axis=1, keepdims=True)).max() < 1e-15


def test_single_edge_one_round(orc):
    """Two vertices, one edge: the first round commits the exact messages; the
    next evaluation finds zero residuals."""
    row_ptr, col, rev = synth.csr_from_undirected(2, np.array([0]), np.array([1]))
    prob = synth.Problem(2, 2, row_ptr, col, rev, np.array([-0.3, 0.3, 0.7, -0.7], np.float32),
                         synth.PAIR_ISING_BETA, np.array([1.1, 1.1], np.float32),
                         np.array([0, 2], np.int64))
    res = orc.run(prob, "lbp", eps=1e-15, max_rounds=10)
    assert res["converged"] and res["rounds"] == 1
    assert np.abs(res["beliefs"] - _exact.brute_force_marginals(prob)).max() < 1e-15


def test_isolated_vertices(orc):
    """A vertex without neighbours keeps its normalised unary as belief."""
    row_ptr, col, rev = synth.csr_from_undirected(4, np.array([0]), np.array([2]))
    un = np.array([0.1, -0.2, 0.5, 0.4, -1.0, 1.0, 0.0, 0.3], np.float32)
    prob = synth.Problem(4, 2, row_ptr, col, rev, un, synth.PAIR_ISING_BETA,
                         np.array([0.8, 0.8], np.float32), np.array([0, 4], np.int64))
    res = orc.run(prob, "lbp", eps=1e-15, max_rounds=10)
    e = np.exp(un.astype(np.float64).reshape(4, 2))
    for v in (1, 3):
        assert np.abs(res["beliefs"][v] - e[v] / e[v].sum()).max() < 1e-15
    assert np.abs(res["beliefs"] - _exact.brute_force_marginals(prob)).max() < 1e-15


def test_empty_graph(orc):
    row_ptr, col, rev = synth.csr_from_undirected(3, np.zeros(0, np.int64), np.zeros(0, np.int64))
    prob = synth.Problem(3, 2, row_ptr, col, rev, np.zeros(6, np.float32),
                         synth.PAIR_ISING_BETA, np.zeros(0, np.float32), np.array([0, 3], np.int64))
    res = orc.run(prob, "rnbp", parallelism=0.5)
    assert res["converged"] and res["rounds"] == 0
    assert np.all(res["beliefs"] == 0.5)


# --------------------------------------------------------------------------- invariants
@pytest.mark.parametrize("schedule,par", [("lbp", 1.0), ("rbp", 0.05), ("rs", 0.01), ("rnbp", 0.5)])
def test_loopy_invariants(orc, schedule, par):
    """Messages stay normalised; a converged state is an eps fixed point of Eq. 2
    (re-evaluated by a direct transcription); beliefs follow Eq. 3."""
    prob = synth.ising_grid(8, 1.0, seed=21)
    eps = 1e-6
    res = orc.run(prob, schedule, parallelism=par, eps=eps, max_rounds=20000, seed=3)
    msg = res["messages"]
    assert np.abs(msg.sum(axis=1) - 1.0).max() < 1e-12
    assert res["converged"]
    worst = max(np.abs(_exact.message_eq2(prob, msg, e) - msg[e]).max() for e in range(prob.m))
    assert worst < eps
    assert np.abs(res["beliefs"] - _exact.beliefs_eq3(prob, msg)).max() < 1e-14
    assert np.all(res["beliefs"] >= 0) and np.allclose(res["beliefs"].sum(axis=1), 1.0)


# --------------------------------------------------------------------------- schedules
def test_rbp_full_frontier_equals_lbp(orc):
    prob = synth.ising_grid(9, 1.5, seed=8)
    a = orc.run(prob, "lbp", eps=1e-6, max_rounds=300)
    b = orc.run(prob, "rbp", parallelism=1.0, eps=1e-6, max_rounds=300)
    assert a["rounds"] == b["rounds"] and a["converged"] == b["converged"]
    assert np.array_equal(a["beliefs"], b["beliefs"])


def test_rs_all_roots_equals_lbp(orc):
    """With every vertex a root, the splash is one simultaneous sub-step over all
    out-messages: exactly an LBP round."""
    prob = synth.ising_grid(7, 1.5, seed=9)
    a = orc.run(prob, "lbp", eps=1e-6, max_rounds=300)
    b = orc.run(prob, "rs", parallelism=1.0, rs_roots_mode=1, eps=1e-6, max_rounds=300)
    assert a["rounds"] == b["rounds"]
    assert np.array_equal(a["beliefs"], b["beliefs"])


@pytest.mark.parametrize("seed", [0, 1])
def test_rbp_k1_equals_serial_heap_rbp(orc, seed):
    """RBP with a frontier of one message is serial residual BP driven by a
    priority queue (the paper's SRBP comparator)."""
    prob = synth.ising_grid(4, 1.5, seed=seed)
    eps = 1e-8
    res = orc.run(prob, "rbp", parallelism=1e-9, eps=eps, max_rounds=4000)
    upd, conv, msg = _exact.serial_rbp(prob, eps, 4000)
    assert res["converged"] == conv
    assert res["rounds"] == upd
    assert np.abs(res["messages"] - msg).max() < 1e-12


def test_rnbp_full_p_commits_exactly_unconverged(orc):
    """LowP = HighP = 1: the frontier of every round is exactly {r >= eps}."""
    prob = synth.ising_grid(6, 2.0, seed=2)
    eps = 1e-3
    res = orc.run(prob, "rnbp", parallelism=1.0, high_p=1.0, eps=eps, max_rounds=3, trace_cap=3)
    msg = np.full((prob.m, 2), 0.5)
    for t in range(res["rounds"]):
        cand = np.array([_exact.message_eq2(prob, msg, e) for e in range(prob.m)])
        r = np.abs(cand - msg).max(axis=1)
        bits = np.unpackbits(res["trace"][t].view(np.uint8), bitorder="little")[:prob.m]
        assert np.array_equal(bits.astype(bool), r >= eps)
        msg[r >= eps] = cand[r >= eps]


def _residuals_eq2_eq4(prob, msg):
    cand = np.array([_exact.message_eq2(prob, msg, e) for e in range(prob.m)])
    return cand, np.abs(cand - msg).max(axis=1)


def _top_k_ids(key, k):
    """Ids of the k largest keys, ties to the smaller id (numpy lexsort)."""
    order = np.lexsort((np.arange(key.shape[0]), -key))
    top, rest = key[order[k - 1]], (key[order[k]] if k < key.shape[0] else -1.0)
    assert top - rest > 1e-12 * max(top, 1e-300)   # the pin needs a clear k-th key
    return np.sort(order[:k])


def test_rbp_frontier_is_top_k_of_eq4_residuals(orc):
    """RBP (Section III-A, reading R4): every round commits exactly the
    k = ceil(p M) messages of largest Eq. 4 residual, ties to the smaller id;
    residuals re-derived here from a direct Eq. 2 transcription."""
    prob = synth.ising_grid(6, 2.0, seed=12)
    p, T = 0.13, 4   # p M = 15.6: ceil and floor differ
    k = int(np.ceil(p * prob.m))
    res = orc.run(prob, "rbp", parallelism=p, eps=1e-9, max_rounds=T, trace_cap=T)
    assert res["rounds"] == T and res["committed_updates"] == k * T
    msg = np.full((prob.m, 2), 0.5)
    for t in range(T):
        cand, r = _residuals_eq2_eq4(prob, msg)
        bits = np.unpackbits(res["trace"][t].view(np.uint8), bitorder="little")[:prob.m]
        assert np.array_equal(np.flatnonzero(bits), _top_k_ids(r, k)), t
        msg[bits.astype(bool)] = cand[bits.astype(bool)]
    assert np.abs(res["messages"] - msg).max() < 1e-12


def test_rs_roots_are_top_k_vertex_residuals(orc):
    """Residual Splash (Section III-A, reading R5): the roots of round t + 1 are
    the k_v = clamp(ceil(p M), 1, n) vertices of largest vertex residual (the
    largest Eq. 4 residual of an incoming message) in the state after t
    rounds, ties to the smaller id."""
    prob = synth.ising_grid(7, 2.0, seed=13)
    p, T = 0.05, 4
    kv = min(max(int(np.ceil(p * prob.m)), 1), prob.n)
    res = orc.run(prob, "rs", parallelism=p, eps=1e-9, max_rounds=T, trace_cap=T)
    assert res["rounds"] == T
    rev = np.asarray(prob.rev)
    for t in range(T):
        state = orc.run(prob, "rs", parallelism=p, eps=1e-9, max_rounds=t)["messages"]
        _, r = _residuals_eq2_eq4(prob, state)
        vres = np.array([r[rev[prob.row_ptr[v]:prob.row_ptr[v + 1]]].max() for v in range(prob.n)])
        bits = np.unpackbits(res["trace"][t].view(np.uint8), bitorder="little")[:prob.n]
        assert np.array_equal(np.flatnonzero(bits), _top_k_ids(vres, kv)), t


def test_rnbp_edge_ratio_switch(orc):
    """p follows EdgeRatio: replay the frontier sizes from the trace with the
    Philox stream and check LowP is used exactly when N_t / N_{t-1} > 0.9."""
    prob = synth.ising_grid(10, 2.5, seed=6)
    eps, low = 1e-4, 0.3
    T = 40
    res = orc.run(prob, "rnbp", parallelism=low, eps=eps, max_rounds=T, seed=99, trace_cap=T)
    msg = np.full((prob.m, 2), 0.5)
    n_prev = None
    used_low = 0
    for t in range(1, res["rounds"] + 1):
        cand = np.array([_exact.message_eq2(prob, msg, e) for e in range(prob.m)])
        r = np.abs(cand - msg).max(axis=1)
        n_t = int((r >= eps).sum())
        p = 1.0 if t == 1 else (low if n_t / n_prev > 0.9 else 1.0)
        sel = np.zeros(prob.m, bool)
        for e in np.nonzero(r >= eps)[0]:
            word = int(orc.philox4x32_10([e // 8, t, 0, 0], [99, 0])[(e % 8) // 2])
            u = (word >> 16) if e % 2 else (word & 0xFFFF)
            sel[e] = p >= 1.0 or u < int(p * 2 ** 16)
        bits = np.unpackbits(res["trace"][t - 1].view(np.uint8), bitorder="little")[:prob.m]
        assert np.array_equal(bits.astype(bool), sel), t
        used_low += p < 1
        msg[sel] = cand[sel]
        n_prev = n_t
    assert used_low > 0


# --------------------------------------------------------------------------- selection
def test_top_k_matches_sort(orc):
    rng = np.random.default_rng(0)
    key = np.round(rng.random(5000), 2)        # many ties
    for k in (1, 7, 100, 4999, 5000):
        chosen = orc.top_k(key, k)
        order = np.lexsort((np.arange(key.size), -key))
        expect = np.zeros(key.size, bool)
        expect[order[:k]] = True
        assert np.array_equal(chosen, expect)


def test_splash_levels_textbook_bfs(orc):
    prob = synth.ising_grid(15, 1.0, seed=0)
    rng = np.random.default_rng(1)
    roots = np.zeros(prob.n, np.uint8)
    roots[rng.choice(prob.n, 6, replace=False)] = 1
    A = scipy.sparse.csr_matrix((np.ones(prob.m), prob.col, prob.row_ptr), shape=(prob.n, prob.n))
    d = scipy.sparse.csgraph.shortest_path(A, unweighted=True, indices=np.nonzero(roots)[0]).min(axis=0)
    for h in (0, 1, 2, 3):
        lv = orc.splash_levels(prob, roots, h)
        expect = np.where(d <= h, d, -1).astype(np.int32)
        assert np.array_equal(lv, expect)


def test_trace_follow_reproduces_run(orc):
    """Following its own recorded frontiers, the oracle lands on the same state."""
    prob = synth.ising_grid(8, 2.0, seed=5)
    for sched, par in (("rnbp", 0.4), ("rbp", 0.05), ("rs", 0.02)):
        a = orc.run(prob, sched, parallelism=par, eps=1e-5, max_rounds=60, seed=1, trace_cap=60)
        b = orc.run(prob, sched, eps=1e-5, trace_in=a["trace"], trace_rounds=a["rounds"])
        assert b["rounds"] == a["rounds"]
        assert np.array_equal(a["beliefs"], b["beliefs"])
        assert a["committed_updates"] == b["committed_updates"]


# --------------------------------------------------------------------------- storage emulation
def _bf16_exact(x):
    f = np.asarray(x, dtype=np.float32)
    return np.all(f.astype(np.float64) == np.asarray(x)) and np.all((f.view(np.uint32) & 0xFFFF) == 0)


def _bf16_scale(prob):
    """The library's BF16 code scale: the smallest power of two >= 2 max|beta| / 250."""
    return float(2.0 ** np.ceil(np.log2(2 * float(np.abs(prob.pair_log).max()) / 250)))


def test_bf16_storage_values_are_bf16(orc):
    """Under BF16 storage every stored Ising word w = 2^(|u| / b - 125) is a
    bfloat16 value, under plain BF16 every stored log-odds is one, and every
    stored k-state log is one too."""
    prob = synth.ising_grid(6, 1.5, seed=1)
    b = _bf16_scale(prob)
    res = orc.run(prob, "rnbp", parallelism=0.5, eps=1e-4, max_rounds=30, storage="bf16", storage_scale=b)
    u = np.log(res["messages"][:, 1]) - np.log(res["messages"][:, 0])
    w = np.exp2(np.abs(u) / b - 125.0)
    wb = np.float32(w)
    assert _bf16_exact(wb) and np.abs(wb / w - 1).max() < 1e-9
    res = orc.run(prob, "rnbp", parallelism=0.5, eps=1e-4, max_rounds=30, storage="bf16_plain")
    u = np.log(res["messages"][:, 1]) - np.log(res["messages"][:, 0])
    assert _bf16_exact(np.float32(u)) and np.abs(np.float32(u) - u).max() < 1e-12
    prob = synth.potts_grid(4, 5, seed=1)
    res = orc.run(prob, "lbp", eps=1e-4, max_rounds=10, storage="bf16")
    lg = np.log(res["messages"])
    assert _bf16_exact(np.float32(lg)) and np.abs(np.float32(lg) - lg).max() < 1e-12


def test_q16_storage_grid_and_bound(orc):
    """Q16 log-odds are integer multiples of the step, |q| <= 32767, and the
    rounding moves beliefs by far less than the step bound 4 * step / 4 per vertex
    would allow for a contracting run."""
    prob = synth.ising_grid(6, 1.5, seed=2)
    beta_max = float(np.abs(prob.pair_log).max())
    step = float(np.float32(2 * beta_max / 32767))
    res = orc.run(prob, "lbp", eps=1e-6, max_rounds=40, storage="q16", storage_scale=step)
    u = np.log(res["messages"][:, 1]) - np.log(res["messages"][:, 0])
    q = u / step
    assert np.abs(q - np.round(q)).max() < 1e-6 and np.abs(q).max() <= 32767
    exact = orc.run(prob, "lbp", eps=1e-6, max_rounds=40)
    assert np.abs(res["beliefs"] - exact["beliefs"]).max() < 2e-3


def test_rounded_storage_residual_zero_when_unchanged(orc):
    """With rounded storage a converged state is a fixed point of rounding: every
    candidate rounds back to the stored word, so the final residual is exactly 0
    or below eps (bf16 limit cycles aside, reported as not converged)."""
    prob = synth.ising_tree(12, 1.0, seed=2)
    for storage, scale in (("bf16", _bf16_scale(prob)), ("bf16_plain", 0.0)):
        res = orc.run(prob, "lbp", eps=1e-12, max_rounds=200, storage=storage, storage_scale=scale)
        assert res["converged"] and res["final_max_residual"] == 0.0


# --------------------------------------------------------------------------- storage rounding pins
# Known answers derived by hand from the formats' definitions (not from the
# oracle). bfloat16 keeps 8 significant bits: in the binade [2^e, 2^(e+1)) the
# spacing is 2^(e-7), and a value halfway between two neighbours goes to the one
# whose last kept mantissa bit is 0 (round to nearest, ties to even).
#   1 + 2^-8          halfway between 1 (mantissa 0, even) and 1 + 2^-7 (1, odd)  -> 1
#   1 + 3*2^-8        halfway between 1 + 2^-7 (1, odd) and 1 + 2^-6 (2, even)    -> 1 + 2^-6
#   1 + 2^-8 + 2^-20  just above the first tie                                    -> 1 + 2^-7
#   2 - 2^-8          halfway between 1 + 127/128 (127, odd) and 2 (carry into
#                     the exponent, mantissa 0)                                   -> 2
#   3 + 2^-7          in [2, 4) the spacing is 2^-6; halfway between 3 (mantissa
#                     64, even) and 3 + 2^-6 (65, odd)                            -> 3
#   0.3               float32(0.3) = 0.300000011920929; in [0.25, 0.5) the
#                     spacing is 2^-9, 0.3 / 2^-9 = 153.6 -> 154 * 2^-9           -> 0.30078125
# Negative values mirror. A truncating rounding fails the 2nd, 3rd, 4th and 6th
# rows; rounding ties away from zero fails the 1st and 5th.
BF16_KNOWN = [
    (1 + 2.0 ** -8, 1.0),
    (1 + 3 * 2.0 ** -8, 1 + 2.0 ** -6),
    (1 + 2.0 ** -8 + 2.0 ** -20, 1 + 2.0 ** -7),
    (2 - 2.0 ** -8, 2.0),
    (3 + 2.0 ** -7, 3.0),
    (float(np.float32(0.3)), 154 * 2.0 ** -9),
]
# Q16 with step s = 2^-12: the stored value is s * (nearest integer to u / s,
# ties to even), clamped to +-32767 steps.
#   2.5 s -> 2 s (tie, even)      3.5 s -> 4 s (tie, even)     2.75 s -> 3 s
#   2.25 s -> 2 s                 40000 s -> 32767 s (clamp)
# A truncating quantiser fails 3.5 s and 2.75 s; ties away from zero fails 2.5 s.
Q16_STEP = 2.0 ** -12
Q16_KNOWN = [(2.5, 2), (3.5, 4), (2.75, 3), (2.25, 2), (40000.0, 32767)]


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_bf16_rounding_known_answers(orc, sign):
    for u, want in BF16_KNOWN:
        assert orc.stored_logodds("bf16_plain", sign * u) == sign * want, (u, want)


# The BF16 exponent code of an Ising log-odds u with scale b: the word is the
# bfloat16 value nearest to w = 2^(|u| / b - 125) (sign of u), read back as
# |u| = (log2 |w| + 125) b. Hand-derived cases:
#   b = 1, u = 0:     w = 2^-125 exactly                       -> 0
#   b = 0.1, u = 3.3: |u| / b - 125 = -92, w = 2^-92 exactly    -> 3.3
#   b = 1, u = 0.3:   w = 2^-125 * 2^0.3, 2^0.3 = 1.2311444...; the 8-bit
#                     significand is 1.2311444 * 128 = 157.586 -> 158 / 128
#                     -> log2(158 / 128) = 0.3037807...  (truncation: 157 / 128,
#                     0.2946...)
#   b = 2, u = 0.6:   the same word (|u| / b = 0.3)            -> 2 log2(158 / 128)
#   b = 1, u = 0.5:   2^0.5 * 128 = 181.02 -> 181 / 128        -> log2(181 / 128)
BF16X_KNOWN = [(1.0, 0.0, 0.0), (0.1, 3.3, 3.3), (1.0, 0.3, np.log2(158 / 128)),
               (2.0, 0.6, 2 * np.log2(158 / 128)), (1.0, 0.5, np.log2(181 / 128))]


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_bf16_exponent_code_known_answers(orc, sign):
    for b, u, want in BF16X_KNOWN:
        got = orc.stored_logodds("bf16", sign * u, b)
        assert abs(got - sign * want) < 1e-12, (b, u, want, got)


def test_bf16_exponent_code_through_a_run(orc):
    """The exponent code is what a run stores: the single copying edge carries
    t = 0.3 and -0.5 (scale 1) as log2(158 / 128) and -log2(181 / 128)."""
    res = orc.run(_copy_edge(0.3, -0.5), "lbp", eps=1e-15, max_rounds=5, storage="bf16", storage_scale=1.0)
    assert res["converged"] and res["rounds"] == 1
    got = _stored_u(res)
    assert abs(got[0] - np.log2(158 / 128)) < 1e-12 and abs(got[1] + np.log2(181 / 128)) < 1e-12, got


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_q16_rounding_known_answers(orc, sign):
    for steps, want in Q16_KNOWN:
        got = orc.stored_logodds("q16", sign * steps * Q16_STEP, Q16_STEP)
        assert got == sign * want * Q16_STEP, (steps, want, got / Q16_STEP)


def _copy_edge(t0: float, t1: float):
    """Two vertices joined by one edge whose coupling beta = 30 makes each
    message copy its source's field: with unary log-potentials (0, t) the
    message's log-odds is log[(e^{-b} + e^{b+t}) / (e^{b} + e^{t-b})]
    = t + O(e^{-2b + |t|}), i.e. t to far below FP64 resolution for |t| <= 10."""
    row_ptr, col, rev = synth.csr_from_undirected(2, np.array([0]), np.array([1]))
    return synth.Problem(2, 2, row_ptr, col, rev, np.array([0.0, t0, 0.0, t1], np.float32),
                         synth.PAIR_ISING_BETA, np.array([30.0, 30.0], np.float32),
                         np.array([0, 2], np.int64))


def _stored_u(res):
    m = res["messages"]
    return np.log(m[:, 1]) - np.log(m[:, 0])


def test_bf16_plain_rounding_through_a_run(orc):
    """The rounding pinned above is the one a run stores: message 0 -> 1 carries
    t = vertex 0's field, message 1 -> 0 carries vertex 1's. Round 1 commits the
    rounded values, round 2 finds them unchanged (residual 0)."""
    for u, want in BF16_KNOWN:
        assert float(np.float32(u)) == u
        res = orc.run(_copy_edge(u, -u), "lbp", eps=1e-15, max_rounds=5, storage="bf16_plain")
        assert res["converged"] and res["rounds"] == 1
        got = _stored_u(res)
        # edge 0 is 0 -> 1 (CSR row 0), edge 1 is 1 -> 0
        assert abs(got[0] - want) < 1e-12 and abs(got[1] + want) < 1e-12, (u, want, got)


def test_q16_storage_rounding_through_a_run(orc):
    """Q16 through a run, on values clear of ties (a tie through a run is decided
    by the FP64 rounding of the computed log-odds): 2.75 s -> 3 s, 2.25 s -> 2 s,
    the clamp at 32767 s, and the mirrored negatives."""
    for steps, want in [(2.75, 3), (2.25, 2), (3.6, 4), (40000.0, 32767)]:
        t = steps * Q16_STEP
        res = orc.run(_copy_edge(t, -t), "lbp", eps=1e-15, max_rounds=5, storage="q16",
                      storage_scale=Q16_STEP)
        assert res["converged"] and res["rounds"] == 1
        got = _stored_u(res) / Q16_STEP
        assert abs(got[0] - want) < 1e-6 and abs(got[1] + want) < 1e-6, (steps, want, got)


def test_bf16_storage_of_k_state_logs(orc):
    """k-state layout: each normalised log m(x) is rounded on its own (no
    renormalisation). With a copying 3x3 table (log-potential 0 on the diagonal,
    -200 elsewhere) and equal unaries the message is uniform, log m(x) = -ln 3 =
    -1.0986...; in [1, 2) the bfloat16 spacing is 2^-7 and 1.0986 / 2^-7 = 140.6,
    so the stored log is -141 / 128 (truncation would give -140 / 128)."""
    k = 3
    row_ptr, col, rev = synth.csr_from_undirected(2, np.array([0]), np.array([1]))
    tab = np.full((2, k, k), -200.0, np.float32)
    tab[:, np.arange(k), np.arange(k)] = 0.0
    prob = synth.Problem(2, k, row_ptr, col, rev, np.full(2 * k, 0.25, np.float32),
                         synth.PAIR_TABLE, tab.reshape(-1), np.array([0, 2], np.int64))
    res = orc.run(prob, "lbp", eps=1e-15, max_rounds=5, storage="bf16")
    assert np.abs(np.log(res["messages"]) + 141.0 / 128.0).max() < 1e-12


def test_bf16_formats_against_the_exact_oracle(orc):
    """The belief tolerance 2e-3 of BF16 storage, on a converging loopy grid
    (37x29, beta ~ U[-1, 1], LBP, eps = 1e-4), three seeds. Plain bfloat16
    log-odds have a relative step of 2^-7: one step of a log-odds near 2 is
    2^-6, and such steps keep the stored messages cycling between neighbours
    (never below eps) with belief errors above 2e-3. The exponent code's step is
    at most b / 128 <= 2 max|beta| / 16000 in log-odds: those runs converge and
    stay an order of magnitude inside the tolerance."""
    for seed in (7, 1, 2):
        prob = synth.ising_grid(37, 1.0, seed=seed, cols=29)
        exact = orc.run(prob, "lbp", eps=1e-4, max_rounds=2000)
        code = orc.run(prob, "lbp", eps=1e-4, max_rounds=2000, storage="bf16", storage_scale=_bf16_scale(prob))
        plain = orc.run(prob, "lbp", eps=1e-4, max_rounds=2000, storage="bf16_plain")
        assert exact["converged"] and code["converged"] and not plain["converged"]
        assert np.abs(code["beliefs"] - exact["beliefs"]).max() < 2e-4
        assert np.abs(plain["beliefs"] - exact["beliefs"]).max() > 2e-3


# --------------------------------------------------------------------------- dynamic p for RBP / RS
def _frontier_sizes(res):
    return [int(np.unpackbits(row.view(np.uint8)).sum()) for row in res["trace"][:res["rounds"]]]


@pytest.mark.parametrize("sched", ["rbp", "rs"])
def test_dynamic_p_with_equal_fractions_is_the_fixed_schedule(orc, sched):
    """LowP = HighP = p: the EdgeRatio switch picks p either way, so the run is
    the fixed-p run, frontier for frontier."""
    prob = synth.ising_grid(9, 2.0, seed=4)
    a = orc.run(prob, sched, parallelism=0.05, eps=1e-6, max_rounds=60, trace_cap=60)
    b = orc.run(prob, sched, parallelism=0.05, high_p=0.05, eps=1e-6, max_rounds=60, trace_cap=60, dynamic_p=1)
    assert a["rounds"] == b["rounds"] and np.array_equal(a["trace"], b["trace"])
    assert np.array_equal(a["beliefs"], b["beliefs"])


def test_dynamic_p_never_low_is_lbp(orc):
    """A threshold no EdgeRatio exceeds keeps HighP = 1: every round commits the
    whole frontier, which is LBP's trajectory (RBP with p = 1 is LBP)."""
    prob = synth.ising_grid(9, 1.5, seed=2)
    lbp = orc.run(prob, "lbp", eps=1e-6, max_rounds=500)
    dyn = orc.run(prob, "rbp", parallelism=0.01, high_p=1.0, ratio_threshold=1e300, eps=1e-6,
                  max_rounds=500, dynamic_p=1)
    assert lbp["converged"] and dyn["rounds"] == lbp["rounds"]
    assert np.abs(dyn["beliefs"] - lbp["beliefs"]).max() < 1e-15


@pytest.mark.parametrize("sched", ["rbp", "rs"])
def test_dynamic_p_frontier_sizes_follow_edge_ratio(orc, sched):
    """Round 1 uses HighP; round t > 1 uses LowP exactly when N_t / N_{t-1} > 0.9,
    N_t = messages with residual >= eps at the evaluation before round t (read
    from runs stopped after t - 1 rounds). RBP commits ceil(p M) messages, RS
    picks ceil(p M) roots (clamped to n)."""
    prob = synth.ising_grid(8, 2.5, seed=6)
    lo, hi, T = 0.02, 0.3, 25
    res = orc.run(prob, sched, parallelism=lo, high_p=hi, eps=1e-5, max_rounds=T, trace_cap=T, dynamic_p=1)
    n_t = [orc.run(prob, sched, parallelism=lo, high_p=hi, eps=1e-5, max_rounds=t, dynamic_p=1)["final_unconverged"]
           for t in range(T + 1)]
    sizes = _frontier_sizes(res)
    m, n = prob.m, prob.n
    switched = 0
    for t in range(1, res["rounds"] + 1):
        p = hi if t == 1 else (lo if n_t[t - 1] / n_t[t - 2] > 0.9 else hi)
        switched += p == lo
        want = min(int(np.ceil(p * m)), m if sched == "rbp" else n)
        if sched == "rbp":
            assert sizes[t - 1] == want, (t, sizes[t - 1], want)
        else:
            assert sizes[t - 1] == want, (t, sizes[t - 1], want)
    assert 0 < switched < res["rounds"] - 1


# --------------------------------------------------------------------------- exact grid marginals, KL (Fig. 5)
@pytest.mark.parametrize("rows,cols,seed", [(4, 4, 0), (3, 5, 1), (5, 3, 2), (4, 5, 3)])
def test_grid_transfer_matrix_equals_brute_force(rows, cols, seed):
    """The row transfer-matrix elimination used for 10x10 grids equals
    enumeration of all 2^n assignments on grids small enough to enumerate."""
    prob = synth.ising_grid(rows, 2.0, seed=seed, cols=cols)
    assert np.abs(_exact.grid_marginals(prob, rows, cols) - _exact.brute_force_marginals(prob)).max() < 1e-13


def test_kl_vs_exact_10x10_rnbp_matches_serial_rbp(orc):
    """Section IV-E / Fig. 5: on the paper's 10x10 Ising set at C = 2, exact
    marginals by elimination, KL(exact || beliefs) per graph for RnBP (LowP
    0.7) and serial residual BP (RBP with one message per round). The paper
    reports the same quality for both; here each KL is within 2% of the other
    on every seed (observed at most 0.7%), and both are fixed points within
    4 * 10 eps of each other (R18)."""
    for seed in range(10):
        prob = synth.paper_ising(10, 10, 2.0, seed=seed)
        exact = _exact.grid_marginals(prob, 10, 10)
        rn = orc.run(prob, "rnbp", parallelism=0.7, eps=1e-4, max_rounds=10000, seed=seed)
        sr = orc.run(prob, "rbp", parallelism=1e-9, eps=1e-4, max_rounds=200000)
        assert rn["converged"] and sr["converged"]
        k_rn = _exact.kl_divergence(exact, rn["beliefs"]).sum()
        k_sr = _exact.kl_divergence(exact, sr["beliefs"]).sum()
        assert 0 < k_rn < 0.5 and abs(k_rn - k_sr) <= 0.02 * k_sr, (seed, k_rn, k_sr)
        assert np.abs(rn["beliefs"] - sr["beliefs"]).max() < 4 * 10 * 1e-4


# --------------------------------------------------------------------------- variable state counts
def _pad_states(prob, k_to, seed=0):
    """The same MRF with k_to states per vertex: the added states get unary
    log-potential -inf (absent) and arbitrary pairwise entries."""
    rng = np.random.default_rng(seed)
    k = prob.k
    un = np.full((prob.n, k_to), -np.inf, np.float32)
    un[:, :k] = prob.unary_log.reshape(prob.n, k)
    tab = rng.normal(0.0, 3.0, size=(prob.m, k_to, k_to)).astype(np.float32)
    for e in range(prob.m):
        r = prob.rev[e]
        if r < e:
            tab[e] = tab[r].T
    tab[:, :k, :k] = prob.pair_log.reshape(prob.m, k, k)
    return synth.Problem(prob.n, k_to, prob.row_ptr, prob.col, prob.rev, un.ravel(), synth.PAIR_TABLE,
                         tab.ravel(), prob.graph_var_offsets)


@pytest.mark.parametrize("sched,par", [("lbp", 1.0), ("rnbp", 0.4), ("rbp", 0.1), ("rs", 0.1)])
def test_absent_states_equal_the_smaller_state_space(orc, sched, par):
    """A 3-state MRF laid out with 5 states, the 2 extra ones absent (unary
    -inf, arbitrary pairwise entries): every schedule takes the same frontiers
    and rounds, and the present states' beliefs and messages equal the 3-state
    run (absent states carry no mass)."""
    prob = synth.random_table_graph(30, 3, extra_edges=15, seed=5, pair_std=0.6)
    big = _pad_states(prob, 5)
    a = orc.run(prob, sched, parallelism=par, high_p=0.9, eps=1e-6, max_rounds=300, seed=2, trace_cap=300)
    b = orc.run(big, sched, parallelism=par, high_p=0.9, eps=1e-6, max_rounds=300, seed=2, trace_cap=300)
    assert a["rounds"] == b["rounds"] and a["converged"] == b["converged"]
    assert np.array_equal(a["trace"], b["trace"])
    assert np.abs(b["beliefs"][:, :3] - a["beliefs"]).max() < 1e-14 and np.all(b["beliefs"][:, 3:] == 0)
    assert np.abs(b["messages"][:, :3] - a["messages"]).max() < 1e-14 and np.all(b["messages"][:, 3:] == 0)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_variable_state_counts_tree_exact(orc, seed):
    """Irregular trees whose vertices have 2 to 6 states: BP is exact on trees,
    so every schedule's converged beliefs equal enumeration over the ragged
    state spaces (absent states have zero probability)."""
    prob = synth.protein_like(8, seed=seed, k_min=2, k_max=6, tree=True)
    exact = _exact.brute_force_marginals(prob)
    for sched, par in (("lbp", 1.0), ("rnbp", 0.5), ("rs", 0.2)):
        res = orc.run(prob, sched, parallelism=par, eps=1e-12, max_rounds=2000, seed=seed)
        assert res["converged"]
        assert np.abs(res["beliefs"] - exact).max() < 1e-12
