"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Protocol (see the parity readings in the design notes):
  * FP64 messages: exact replay. GPU and oracle select on their own; frontiers,
    round counts and convergence must agree, beliefs within 1e-10.
  * FP32 / BF16 / Q16 messages: trace-follow. The GPU records its frontier every
    round; the oracle commits exactly those frontiers with its own FP64
    arithmetic for the same number of rounds. Max |belief error| <= 1e-5 (FP32
    vs the exact oracle), <= 2e-3 (BF16 vs the oracle emulating BF16 storage;
    Q16 vs the exact oracle).
"""
import numpy as np
import pytest

import oracle
from paper_1909_11469_gb300 import bp, synth
from tests import _exact

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-10
TOL_F32 = 1e-5
TOL_BF16 = 2e-3


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def gpu_run(prob, sched, par=1.0, eps=1e-4, max_rounds=1000, dtype="f32", trace=0, **opts):
    with bp.Graph(prob) as g:
        st = g.run(sched, par, eps=eps, max_rounds=max_rounds, msg_dtype=dtype,
                   record_trace=1 if trace else 0, trace_capacity=trace, **opts)
        out = {"stats": st, "beliefs": g.beliefs(), "messages": g.messages(),
               "graph_stats": g.graph_stats()}
        if dtype in ("q16", "bf16") and prob.k == 2 and prob.pair_kind == synth.PAIR_ISING_BETA:
            out["storage_scale"] = g.storage_scale(dtype)
        if trace:
            out["trace"] = g.trace(sched)
    return out


def _trace_bits(trace, lo, hi):
    """Bits [lo, hi) of every row of a batch trace, repacked from bit 0."""
    words = (hi - lo + 31) // 32
    out = np.zeros((len(trace), words), np.uint32)
    for t, row in enumerate(trace):
        b = np.unpackbits(row.view(np.uint8), bitorder="little")[lo:hi]
        pad = np.zeros(words * 32, np.uint8)
        pad[:hi - lo] = b
        out[t] = np.packbits(pad, bitorder="little").view(np.uint32)
    return out


def all_ones_trace(count, rounds):
    words = (count + 31) // 32
    t = np.zeros((rounds, words), dtype=np.uint32)
    bits = np.zeros(words * 32, dtype=np.uint8)
    bits[:count] = 1
    t[:] = np.packbits(bits, bitorder="little").view(np.uint32)
    return t


def follow(prob, sched, res, eps, storage="f64"):
    """Oracle run that commits the GPU's recorded frontiers."""
    rounds = res["stats"]["rounds"]
    kw = dict(eps=eps, storage=storage,
              storage_scale=res.get("storage_scale", 0.0) if storage in ("q16", "bf16") else 0.0)
    if sched == "lbp":
        tr = all_ones_trace(prob.m, rounds)
        return oracle.run(prob, "lbp", trace_in=tr, trace_rounds=rounds, **kw)
    assert res["trace"].shape[0] == rounds
    return oracle.run(prob, sched, trace_in=res["trace"], trace_rounds=rounds, **kw)


# ------------------------------------------------------------ FP64 exact replay
@pytest.mark.parametrize("variant", [1, 3])
@pytest.mark.parametrize("sched,par", [("lbp", 1.0), ("rnbp", 0.5)])
def test_ising10_fp64_exact_replay(sched, par, variant):
    """10x10 Ising, beta ~ U[-2, 2], seeds 0..9, eps 1e-4, max 1000 rounds."""
    for seed in range(10):
        prob = synth.ising_grid(10, 2.0, seed=seed)
        ref = oracle.run(prob, sched, parallelism=par, eps=1e-4, max_rounds=1000, seed=seed)
        res = gpu_run(prob, sched, par, 1e-4, 1000, "f64", seed=seed, kernel_variant=variant)
        assert res["stats"]["converged"] == ref["converged"], seed
        assert res["stats"]["rounds"] == ref["rounds"], seed
        if ref["converged"]:
            assert res["stats"]["committed_updates"] == ref["committed_updates"]
            assert np.abs(res["beliefs"] - ref["beliefs"]).max() < TOL_F64, seed


# kernel_variant 1: per-round kernels; 3: persistent batch kernel (one cluster per graph)
VARIANTS = [1, 3]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("sched,par", [("lbp", 1.0), ("rnbp", 0.5), ("rnbp", 0.1), ("rbp", 0.05),
                                       ("rbp", 1e-3), ("rs", 0.02), ("rs", 0.2)])
def test_fp64_exact_replay_trace(sched, par, variant):
    """Same frontier every round, same state after 60 rounds (ragged 13x11 grid)."""
    prob = synth.ising_grid(13, 2.0, seed=4, cols=11)
    T = 60
    ref = oracle.run(prob, sched, parallelism=par, eps=1e-7, max_rounds=T, seed=5, trace_cap=T)
    res = gpu_run(prob, sched, par, 1e-7, T, "f64", trace=T if sched != "lbp" else 0, seed=5,
                  kernel_variant=variant)
    assert res["stats"]["rounds"] == ref["rounds"]
    if sched != "lbp":
        assert np.array_equal(res["trace"], ref["trace"][:ref["rounds"]])
    assert res["stats"]["committed_updates"] == ref["committed_updates"]
    assert np.abs(res["beliefs"] - ref["beliefs"]).max() < TOL_F64
    assert np.abs(res["messages"] - ref["messages"]).max() < TOL_F64


@pytest.mark.parametrize("sched,par", [("rbp", 0.1), ("rs", 0.1)])
def test_ising10_fp64_converging_seeds_rbp_rs(sched, par):
    for seed in (0, 5):
        prob = synth.ising_grid(10, 2.0, seed=seed)
        ref = oracle.run(prob, sched, parallelism=par, eps=1e-4, max_rounds=10000)
        res = gpu_run(prob, sched, par, 1e-4, 10000, "f64")
        assert ref["converged"] and res["stats"]["converged"]
        assert res["stats"]["rounds"] == ref["rounds"]
        assert np.abs(res["beliefs"] - ref["beliefs"]).max() < TOL_F64


# ------------------------------------------------------------ trees: exactness
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", TOL_F32)])
@pytest.mark.parametrize("sched,par", [("lbp", 1.0), ("rnbp", 0.6), ("rbp", 0.2), ("rs", 0.05)])
def test_tree_exact_marginals(dtype, tol, sched, par):
    prob = synth.ising_tree(14, 2.0, seed=3)
    res = gpu_run(prob, sched, par, 1e-9 if dtype == "f64" else 1e-6, 5000, dtype)
    assert res["stats"]["converged"]
    assert np.abs(res["beliefs"] - _exact.brute_force_marginals(prob)).max() < tol


def test_chain_forward_backward_fp32():
    prob = synth.paper_ising(1, 2000, C=10.0, seed=2)
    res = gpu_run(prob, "lbp", 1.0, 1e-6, 5000, "f32")
    assert res["stats"]["converged"]
    assert np.abs(res["beliefs"] - _exact.chain_marginals(prob)).max() < TOL_F32


# ------------------------------------------------------------ FP32 / BF16 trace-follow
# (dtype, oracle storage, beta_max, rounds, tolerance). beta <= 1.2 is a
# contracting case run to convergence; beta <= 2.5 is a hard case over a short
# horizon (on a non-contracting trajectory rounding differences grow with the
# rounds, so long horizons there measure the dynamics, not the kernel).
# 16-bit storage against the exact oracle is held to the 2e-3 BF16 tolerance;
# against the oracle that emulates the same format, a candidate within the
# FP32-vs-FP64 difference of a rounding boundary can land one step apart on the
# two sides (a step of at most 2 max|beta| / 16000 in log-odds for the BF16
# exponent code, 2 max|beta| / 32767 for Q16): 2e-4 on the contracting case.
TRACE_CASES = [
    ("f32", "f64", 1.2, 2000, TOL_F32), ("f32", "f64", 2.5, 25, TOL_F32),
    ("q16", "f64", 1.2, 2000, TOL_BF16), ("q16", "q16", 1.2, 2000, 2e-4),
    ("q16", "q16", 2.5, 25, TOL_BF16),
    ("bf16", "f64", 1.2, 2000, TOL_BF16), ("bf16", "bf16", 1.2, 2000, 2e-4),
    ("bf16", "bf16", 2.5, 25, TOL_BF16),
]


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("dtype,oracle_storage,beta_max,T,tol", TRACE_CASES)
@pytest.mark.parametrize("sched,par", [("lbp", 1.0), ("rnbp", 0.5), ("rnbp", 0.1),
                                       ("rbp", 0.01), ("rs", 0.01)])
def test_trace_follow_ising(dtype, oracle_storage, beta_max, T, tol, sched, par, variant):
    """37x29 grid (ragged over 256-vertex blocks). A Residual Splash round sweeps
    2h + 1 = 5 levels, so its short horizon is 5 times fewer rounds."""
    prob = synth.ising_grid(37, beta_max, seed=7, cols=29)
    if T < 100 and sched == "rs":
        T = T // 5
    res = gpu_run(prob, sched, par, 1e-4, T, dtype, trace=T, seed=3, kernel_variant=variant)
    if T > 100:
        assert res["stats"]["converged"]
    ref = follow(prob, sched, res, 1e-4, oracle_storage)
    assert ref["rounds"] == res["stats"]["rounds"]
    err = np.abs(res["beliefs"] - ref["beliefs"]).max()
    assert err < tol, err


@pytest.mark.parametrize("seed", [7, 1, 2])
def test_bf16_storage_error_vs_exact_oracle(seed):
    """BF16 (exponent-coded log-odds) and Q16 storage converge on this loopy
    grid and stay inside 2e-3 of the exact FP64 oracle run independently to
    its own convergence (not trace-following: the GPU selects on its own)."""
    prob = synth.ising_grid(37, 1.0, seed=seed, cols=29)
    exact = oracle.run(prob, "lbp", eps=1e-4, max_rounds=2000)
    for dtype in ("bf16", "q16"):
        res = gpu_run(prob, "lbp", 1.0, 1e-4, 2000, dtype)
        err = np.abs(res["beliefs"] - exact["beliefs"]).max()
        print(f"{dtype} vs exact {err:.3e} (converged {res['stats']['converged']}, rounds "
              f"{res['stats']['rounds']} vs {exact['rounds']})")
        assert res["stats"]["converged"] and exact["converged"]
        assert err < TOL_BF16


def test_messages_normalised_and_beliefs_consistent():
    prob = synth.ising_grid(40, 2.5, seed=1)
    res = gpu_run(prob, "rnbp", 0.5, 1e-4, 300, "f32", seed=2)
    msg = res["messages"]
    assert np.abs(msg.sum(axis=1) - 1).max() < 1e-6
    assert np.abs(res["beliefs"] - _exact.beliefs_eq3(prob, msg)).max() < 1e-6


# ------------------------------------------------------------ k-state tables
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", TOL_F32)])
def test_table_tree_k3_exact(dtype, tol):
    prob = synth.random_table_graph(9, 3, extra_edges=0, seed=4)
    res = gpu_run(prob, "lbp", 1.0, 1e-10 if dtype == "f64" else 1e-7, 200, dtype)
    assert res["stats"]["converged"]
    assert np.abs(res["beliefs"] - _exact.brute_force_marginals(prob)).max() < tol


@pytest.mark.parametrize("k", [3, 5, 8, 13, 32])
def test_table_loopy_fp64_replay(k):
    prob = synth.random_table_graph(40, k, extra_edges=25, seed=k, pair_std=0.5)
    ref = oracle.run(prob, "rnbp", parallelism=0.5, eps=1e-6, max_rounds=50, seed=1, trace_cap=50)
    res = gpu_run(prob, "rnbp", 0.5, 1e-6, 50, "f64", trace=50, seed=1)
    assert res["stats"]["rounds"] == ref["rounds"]
    assert np.array_equal(res["trace"], ref["trace"][:ref["rounds"]])
    assert np.abs(res["beliefs"] - ref["beliefs"]).max() < TOL_F64


@pytest.mark.parametrize("k", [3, 8])
@pytest.mark.parametrize("sched,par", [("rbp", 0.1), ("rs", 0.1)])
def test_table_frontier_schedules_fp64_replay(k, sched, par):
    """k-state tables under RBP (k values copied per committed message) and
    Residual Splash (k-state splash evaluation and commit per level)."""
    prob = synth.random_table_graph(40, k, extra_edges=25, seed=k, pair_std=0.5)
    ref = oracle.run(prob, sched, parallelism=par, eps=1e-6, max_rounds=30, trace_cap=30)
    res = gpu_run(prob, sched, par, 1e-6, 30, "f64", trace=30)
    assert res["stats"]["rounds"] == ref["rounds"]
    assert np.array_equal(res["trace"], ref["trace"][:ref["rounds"]])
    assert res["stats"]["committed_updates"] == ref["committed_updates"]
    assert np.abs(res["beliefs"] - ref["beliefs"]).max() < TOL_F64
    assert np.abs(res["messages"] - ref["messages"]).max() < TOL_F64


@pytest.mark.parametrize("dtype,tol", [("f32", TOL_F32), ("bf16", TOL_BF16)])
@pytest.mark.parametrize("sched,par", [("lbp", 1.0), ("rnbp", 0.5)])
def test_potts_trace_follow(dtype, tol, sched, par):
    prob = synth.potts_grid(12, 32, seed=2)
    res = gpu_run(prob, sched, par, 1e-4, 60, dtype, trace=60, seed=4)
    ref = follow(prob, sched, res, 1e-4, "bf16" if dtype == "bf16" else "f64")
    err = np.abs(res["beliefs"] - ref["beliefs"]).max()
    assert err < tol, err


# ------------------------------------------------------------ batches
@pytest.mark.parametrize("variant", [1, 3, 4])
@pytest.mark.parametrize("sched,par", [("lbp", 1.0), ("rnbp", 0.5), ("rbp", 0.05), ("rs", 0.05)])
def test_batch_equals_independent_runs(sched, par, variant):
    """A batch of uneven graphs: every graph converges or stops on its own and
    matches the oracle run of that graph alone (graph id = its batch index)."""
    members = [synth.ising_grid(9, 1.0, seed=1), synth.ising_chain(300, 2.0, seed=2),
               synth.ising_grid(20, 2.0, seed=3, cols=7), synth.ising_tree(50, 1.5, seed=4),
               synth.ising_grid(3, 0.0, seed=5)]
    members += [synth.er_batch(1, seed=s, n_min=30, n_max=200).graph(0) for s in range(5)]
    batch = synth.concat_batch(members)
    res = gpu_run(batch, sched, par, 1e-5, 500, "f64", seed=9, kernel_variant=variant)
    gstats = res["graph_stats"]
    for gi, m in enumerate(members):
        ref = oracle.run(m, sched, parallelism=par, eps=1e-5, max_rounds=500, seed=9, graph_id=gi)
        assert gstats[gi]["rounds"] == ref["rounds"], gi
        assert bool(gstats[gi]["converged"]) == ref["converged"], gi
        v0, v1 = batch.graph_var_offsets[gi], batch.graph_var_offsets[gi + 1]
        if ref["converged"] or ref["rounds"] < 100:
            assert np.abs(res["beliefs"][v0:v1] - ref["beliefs"]).max() < 1e-9, gi


# ------------------------------------------------------------ edge cases
def test_edge_cases():
    # no edges at all
    row_ptr, col, rev = synth.csr_from_undirected(5, np.zeros(0, np.int64), np.zeros(0, np.int64))
    un = np.random.default_rng(0).normal(size=10).astype(np.float32)
    prob = synth.Problem(5, 2, row_ptr, col, rev, un, synth.PAIR_ISING_BETA,
                         np.zeros(0, np.float32), np.array([0, 5], np.int64))
    res = gpu_run(prob, "rnbp", 0.5, 1e-4, 10, "f32")
    e = np.exp(un.astype(np.float64).reshape(5, 2))
    assert res["stats"]["converged"] and res["stats"]["rounds"] == 0
    assert np.abs(res["beliefs"] - e / e.sum(1, keepdims=True)).max() < 1e-6
    # max_rounds = 0: beliefs from uniform messages
    prob = synth.ising_grid(6, 1.0, seed=1)
    res = gpu_run(prob, "lbp", 1.0, 1e-4, 0, "f64")
    ref = oracle.run(prob, "lbp", eps=1e-4, max_rounds=0)
    assert res["stats"]["rounds"] == 0 and not res["stats"]["converged"]
    assert np.abs(res["beliefs"] - ref["beliefs"]).max() < 1e-12
    # beta = 0: converged at round 0
    prob = synth.ising_grid(6, 0.0, seed=1)
    res = gpu_run(prob, "rbp", 0.1, 1e-4, 10, "f32")
    assert res["stats"]["converged"] and res["stats"]["rounds"] == 0
    # single edge: one round
    row_ptr, col, rev = synth.csr_from_undirected(2, np.array([0]), np.array([1]))
    prob = synth.Problem(2, 2, row_ptr, col, rev, np.array([-0.3, 0.3, 0.7, -0.7], np.float32),
                         synth.PAIR_ISING_BETA, np.array([1.1, 1.1], np.float32),
                         np.array([0, 2], np.int64))
    res = gpu_run(prob, "lbp", 1.0, 1e-12, 10, "f64")
    assert res["stats"]["converged"] and res["stats"]["rounds"] == 1
    assert np.abs(res["beliefs"] - _exact.brute_force_marginals(prob)).max() < 1e-14


def test_errors_on_device():
    prob = synth.ising_grid(4, 1.0, seed=0)
    h = bp.bp_create_graph(prob.n, 2, prob.row_ptr, prob.col, prob.rev)
    try:
        with pytest.raises(bp.BPError) as ei:
            bp.bp_run(h, "lbp", 1.0, 1e-4, 10)
        assert ei.value.code == bp.BP_ERR_NO_POTENTIALS
        with pytest.raises(bp.BPError) as ei:
            bp.bp_get_beliefs(h)
        assert ei.value.code == bp.BP_ERR_NO_RESULT
        tprob = synth.random_table_graph(6, 3, 2, seed=0)
        with bp.Graph(tprob) as tg:
            with pytest.raises(bp.BPError) as ei:
                tg.run("lbp", 1.0, msg_dtype="q16")
            assert ei.value.code == bp.BP_ERR_UNSUPPORTED
        bad = prob.pair_log.copy()
        bad[0] += 1.0
        with pytest.raises(bp.BPError) as ei:
            bp.bp_set_potentials(h, prob.unary_log, 0, bad)
        assert ei.value.code == bp.BP_ERR_NONFINITE
        un = prob.unary_log.copy()
        un[3] = np.nan
        with pytest.raises(bp.BPError) as ei:
            bp.bp_set_potentials(h, un, 0, prob.pair_log)
        assert ei.value.code == bp.BP_ERR_NONFINITE
        bp.bp_set_potentials(h, prob.unary_log, 0, prob.pair_log)
        for args in ((7, 1.0, 1e-4, 10), ("rbp", 0.0, 1e-4, 10), ("lbp", 1.0, 0.0, 10),
                     ("lbp", 1.0, 1e-4, -1)):
            with pytest.raises(bp.BPError) as ei:
                bp.bp_run(h, *args)
            assert ei.value.code == bp.BP_ERR_INVALID_ARG
        st = bp.bp_run(h, "lbp", 1.0, 1e-4, 10)
        assert st["status"] == 0
    finally:
        bp.bp_destroy_graph(h)


@pytest.mark.parametrize("variant", [1, 3])
def test_time_budget_stops_cleanly(variant):
    prob = synth.ising_grid(60, 3.0, seed=1)
    with bp.Graph(prob) as g:
        st = g.run("rbp", 1e-4, eps=1e-12, max_rounds=10_000_000, time_budget_ms=50.0,
                   kernel_variant=variant)
        assert st["status"] == bp.BP_ERR_TIMEOUT and not st["converged"]
        b = g.beliefs()
        assert np.all(np.isfinite(b)) and np.allclose(b.sum(1), 1.0)
        st2 = g.run("lbp", 1.0, eps=1e-4, max_rounds=5)
        assert st2["status"] == 0 and st2["rounds"] == 5


# ------------------------------------------------------------ Potts update paths
@pytest.mark.parametrize("path,dtype,tol", [(1, "f32", TOL_F32), (3, "f32", TOL_F32),
                                            (2, "f32", TOL_BF16), (3, "bf16", 1.6e-2),
                                            (2, "bf16", 1.6e-2)])
@pytest.mark.parametrize("sched,par", [("lbp", 1.0), ("rnbp", 0.5)])
def test_potts_update_paths(path, dtype, tol, sched, par):
    """Shared k = 32 table on a 20x20 grid: CUDA cores (1), tensor cores BF16 (2)
    and tensor cores with the BF16 residual products (3), against the oracle
    following the GPU frontiers (BF16 storage: the BF16-emulating oracle).
    Tensor-core BF16 products keep 8 significant bits per factor, so path 2 is
    held to the BF16 tolerance. With BF16 storage (plain per-state logs) a
    candidate within the FP32-vs-FP64 difference of a bfloat16 boundary stores
    one step apart on the two sides (a step of a log near 2-4 is 2^-6), so both
    tensor-core paths get the k-state BF16 flip bound (1.6e-2; observed up to
    3.9e-3 with path 3)."""
    prob = synth.potts_grid(20, 32, seed=5)
    res = gpu_run(prob, sched, par, 1e-4, 25, dtype, trace=25, seed=4, potts_path=path)
    ref = follow(prob, sched, res, 1e-4, "bf16" if dtype == "bf16" else "f64")
    err = np.abs(res["beliefs"] - ref["beliefs"]).max()
    print(f"potts path {path} {dtype} {sched}: {err:.3e}")
    assert err < tol, err


@pytest.mark.gpu
def test_potts_tensor_core_ragged_tiles():
    """k = 20 (states padded to 32) on an irregular graph whose tiles hold
    uneven vertex and edge counts."""
    row_ptr, col, rev = synth.csr_from_undirected(*_random_graph(300, 700, seed=2))
    rng = np.random.default_rng(3)
    k = 20
    theta = np.eye(k) + np.triu(rng.normal(0, 0.3, (k, k)))
    theta = np.triu(theta) + np.triu(theta, 1).T
    prob = synth.Problem(300, k, row_ptr, col, rev, rng.standard_normal(300 * k).astype(np.float32),
                         synth.PAIR_SHARED, theta.astype(np.float32).ravel(), np.array([0, 300], np.int64))
    res = gpu_run(prob, "lbp", 1.0, 1e-4, 20, "f32", potts_path=3)
    ref = oracle.run(prob, "lbp", eps=1e-4, trace_in=all_ones_trace(prob.m, res["stats"]["rounds"]),
                     trace_rounds=res["stats"]["rounds"])
    assert np.abs(res["beliefs"] - ref["beliefs"]).max() < TOL_F32


def _potts_members_shared_table():
    """k = 32 members of one shared table: two grids, a chain (a tree: exact
    after its diameter) and a pair of vertices, so tensor-core tiles span
    graph boundaries and graphs stop at different rounds."""
    members = [synth.potts_grid(7, 32, seed=1), synth.potts_grid(13, 32, seed=3, cols=5),
               synth.potts_grid(1, 32, seed=4, cols=40), synth.potts_grid(1, 32, seed=5, cols=2)]
    for mbr in members[1:]:
        mbr.pair_log = members[0].pair_log.copy()
    return members


@pytest.mark.parametrize("path,dtype,tol", [(3, "f32", TOL_F32), (2, "f32", TOL_BF16), (3, "bf16", 1.6e-2)])
@pytest.mark.parametrize("sched,par", [("lbp", 1.0), ("rnbp", 0.5)])
def test_potts_tensor_core_batch(path, dtype, tol, sched, par):
    """A batch of k = 32 graphs on the tensor-core paths: every graph matches
    the oracle run of that graph alone that follows the graph's own recorded
    frontiers for its own rounds (BF16 storage: the BF16-emulating oracle)."""
    members = _potts_members_shared_table()
    batch = synth.concat_batch(members)
    res = gpu_run(batch, sched, par, 1e-4, 60, dtype, trace=61, seed=4, potts_path=path)
    rounds = [x["rounds"] for x in res["graph_stats"]]
    assert len(set(rounds)) > 1, rounds
    storage = "bf16" if dtype == "bf16" else "f64"
    for gi, mbr in enumerate(members):
        v0, v1 = batch.graph_var_offsets[gi], batch.graph_var_offsets[gi + 1]
        e0, e1 = batch.row_ptr[v0], batch.row_ptr[v1]
        r = rounds[gi]
        if sched == "lbp":
            tr = all_ones_trace(mbr.m, r)
        else:
            tr = _trace_bits(res["trace"][:r], int(e0), int(e1))
        ref = oracle.run(mbr, sched, eps=1e-4, storage=storage, trace_in=tr, trace_rounds=r)
        err = np.abs(res["beliefs"][v0:v1] - ref["beliefs"]).max()
        assert err < tol, (gi, err)


def _random_graph(n, m, seed):
    rng = np.random.default_rng(seed)
    seen = set()
    ei, ej = [], []
    while len(seen) < m:
        a, b = (int(x) for x in rng.integers(0, n, 2))
        if a != b and (min(a, b), max(a, b)) not in seen:
            seen.add((min(a, b), max(a, b)))
            ei.append(a)
            ej.append(b)
    return n, np.array(ei), np.array(ej)


# ------------------------------------------------------------ dynamic p for RBP / RS
def _rs_clear_rounds(prob, ref, lo, hi, gid, T):
    """Leading rounds of an oracle RS run (dynamic p) whose root choice is
    clear of rounding: the k-th and (k+1)-th largest vertex residuals (Eq. 4,
    max over incoming messages, from the oracle's state before the round)
    differ by more than 1e-12. Once few vertices are unconverged, many vertex
    residuals are exactly 0 in the oracle's probability arithmetic and ~1e-17
    in the GPU's log-odds arithmetic, and the roots among them are picked by
    rounding."""
    rounds = ref["rounds"]
    for t in range(rounds):
        st = oracle.run(prob, "rs", parallelism=lo, high_p=hi, eps=1e-4, max_rounds=t, graph_id=gid, dynamic_p=1)
        _, r = oracle.evaluate(prob, st["messages"])
        vres = np.zeros(prob.n)
        np.maximum.at(vres, prob.col, r)
        k = int(np.unpackbits(ref["trace"][t].view(np.uint8), bitorder="little")[:prob.n].sum())
        srt = np.sort(vres)[::-1]
        if k < prob.n and srt[k - 1] - srt[k] <= 1e-12:
            return t
    return rounds



@pytest.mark.parametrize("variant", [1, 3])
@pytest.mark.parametrize("sched,lo,hi", [("rbp", 0.02, 0.3), ("rs", 0.02, 0.3), ("rbp", 0.1, 1.0),
                                         ("rs", 0.01, 0.2)])
def test_dynamic_p_fp64_exact_replay(sched, lo, hi, variant):
    """RBP / RS with the EdgeRatio switch of their frontier fraction (LowP =
    parallelism, HighP = high_p): FP64 messages replay the oracle frontier for
    frontier on 10x10 grids (5 seeds, one batch) and on uneven ER graphs."""
    # 120 rounds: on a run that never contracts, ~1e-16 differences per step
    # grow until two near-tied RS root residuals swap (seen after 100-400 rounds)
    for prob, T in ((synth.ising_grid_batch(10, 2.0, range(5)), 120), (synth.er_batch(12, 5, n_max=300), 60)):
        res = gpu_run(prob, sched, lo, 1e-4, T, "f64", trace=T, kernel_variant=variant, high_p=hi, dynamic_p=1)
        gst = res["graph_stats"]
        for gi in range(prob.n_graphs):
            one = prob.graph(gi)
            ref = oracle.run(one, sched, parallelism=lo, high_p=hi, eps=1e-4, max_rounds=T, graph_id=gi,
                             trace_cap=T, dynamic_p=1)
            v0, v1 = prob.graph_var_offsets[gi], prob.graph_var_offsets[gi + 1]
            lo_b, hi_b = (v0, v1) if sched == "rs" else (prob.row_ptr[v0], prob.row_ptr[v1])
            rounds = ref["rounds"]
            clear = _rs_clear_rounds(one, ref, lo, hi, gi, T) if sched == "rs" else rounds
            got = _trace_bits(res["trace"][:rounds], lo_b, hi_b)
            assert np.array_equal(got[:clear], ref["trace"][:clear]), gi
            if clear < rounds:
                continue   # a root choice decided by rounding (see _rs_clear_rounds)
            assert gst[gi]["rounds"] == ref["rounds"], gi
            assert bool(gst[gi]["converged"]) == ref["converged"], gi
            assert np.array_equal(got, ref["trace"][:rounds]), gi
            # the same frontiers every round; the log-odds (GPU) and probability
            # (oracle) arithmetic round apart by ~1e-16 per step, which a
            # trajectory that never contracts (a graph that runs to its cap)
            # grows to ~1e-7
            tol = 1e-8 if ref["converged"] else 1e-5
            assert np.abs(res["beliefs"][v0:v1] - ref["beliefs"]).max() < tol, gi


@pytest.mark.parametrize("sched", ["rbp", "rs"])
def test_dynamic_p_fp32_trace_follow(sched):
    prob = synth.ising_grid(37, 1.2, seed=7, cols=29)
    res = gpu_run(prob, sched, 0.01, 1e-4, 400, "f32", trace=400, high_p=0.2, dynamic_p=1)
    ref = follow(prob, sched, res, 1e-4, "f64")
    assert ref["rounds"] == res["stats"]["rounds"]
    assert np.abs(res["beliefs"] - ref["beliefs"]).max() < TOL_F32


# ------------------------------------------------------------ KL against exact marginals (Fig. 5)
def test_kl_vs_exact_10x10_gpu():
    """Section IV-E / Fig. 5 on the GPU: the paper's 10x10 Ising set at C = 2
    (10 seeds as one batch), RnBP with LowP 0.7 in FP32 messages. Per graph,
    KL(exact || GPU beliefs), exact by row elimination, is within 2% of the
    KL of the FP64 oracle's serial residual BP (RBP with one message per round)."""
    seeds = range(10)
    batch = synth.concat_batch([synth.paper_ising(10, 10, 2.0, seed=s) for s in seeds])
    res = gpu_run(batch, "rnbp", 0.7, 1e-4, 10000, "f32", seed=0)
    for gi in seeds:
        one = batch.graph(gi)
        exact = _exact.grid_marginals(one, 10, 10)
        sr = oracle.run(one, "rbp", parallelism=1e-9, eps=1e-4, max_rounds=200000)
        assert res["graph_stats"][gi]["converged"] and sr["converged"]
        v0, v1 = batch.graph_var_offsets[gi], batch.graph_var_offsets[gi + 1]
        k_gpu = _exact.kl_divergence(exact, res["beliefs"][v0:v1]).sum()
        k_sr = _exact.kl_divergence(exact, sr["beliefs"]).sum()
        print(f"seed {gi}: KL(exact || GPU RnBP) {k_gpu:.5f}, KL(exact || serial RBP) {k_sr:.5f}")
        assert abs(k_gpu - k_sr) <= 0.02 * k_sr, (gi, k_gpu, k_sr)


# ------------------------------------------------------------ variable state counts (absent states)
@pytest.mark.parametrize("sched,par", [("lbp", 1.0), ("rnbp", 0.4), ("rbp", 0.1), ("rs", 0.1)])
def test_variable_states_fp64_exact_replay(sched, par):
    """Irregular graph with 2 to 32 states per vertex (the protein-folding
    shape of Section IV-E, synthetic): FP64 messages replay the oracle's
    frontiers, rounds and beliefs; absent states get no belief."""
    prob = synth.protein_like(200, seed=1)
    T = 40
    ref = oracle.run(prob, sched, parallelism=par, high_p=0.9, eps=1e-4, max_rounds=T, seed=2, trace_cap=T)
    res = gpu_run(prob, sched, par, 1e-4, T, "f64", trace=T, seed=2, high_p=0.9)
    assert res["stats"]["rounds"] == ref["rounds"]
    if sched != "lbp":
        assert np.array_equal(res["trace"], ref["trace"][:ref["rounds"]])
    assert np.abs(res["beliefs"] - ref["beliefs"]).max() < TOL_F64
    absent = np.isinf(prob.unary_log.reshape(prob.n, prob.k))
    assert np.all(res["beliefs"][absent] == 0)


@pytest.mark.parametrize("dtype,tol", [("f32", TOL_F32), ("bf16", 1.6e-2)])
def test_variable_states_trace_follow(dtype, tol):
    """The paper's protein setting (RnBP, LowP 0.4, HighP 0.9) on a 400-vertex
    irregular graph with 2 to 32 states per vertex, 60 rounds, against the
    oracle following the GPU frontiers (BF16: the oracle emulating it)."""
    prob = synth.protein_like(400, seed=2)
    res = gpu_run(prob, "rnbp", 0.4, 1e-4, 60, dtype, trace=60, seed=1, high_p=0.9)
    ref = follow(prob, "rnbp", res, 1e-4, "bf16" if dtype == "bf16" else "f64")
    assert np.abs(res["beliefs"] - ref["beliefs"]).max() < tol


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", TOL_F32)])
def test_variable_states_tree_exact(dtype, tol):
    prob = synth.protein_like(8, seed=3, k_min=2, k_max=6, tree=True)
    res = gpu_run(prob, "lbp", 1.0, 1e-12 if dtype == "f64" else 1e-7, 500, dtype)
    assert res["stats"]["converged"]
    assert np.abs(res["beliefs"] - _exact.brute_force_marginals(prob)).max() < tol


@pytest.mark.parametrize("sched,par", [("lbp", 1.0), ("rnbp", 0.4)])
def test_wide_states_fp64_exact_replay(sched, par):
    """Up to 81 states per vertex (the protein-folding range of Section IV-E;
    the layout has 81 states, a warp per vertex with 3 states per lane): FP64
    messages replay the oracle's frontiers, rounds and beliefs; absent states
    get no belief."""
    prob = synth.protein_like(60, seed=4, k_min=2, k_max=81)
    assert prob.k == 81
    T = 30
    ref = oracle.run(prob, sched, parallelism=par, high_p=0.9, eps=1e-4, max_rounds=T, seed=2, trace_cap=T)
    res = gpu_run(prob, sched, par, 1e-4, T, "f64", trace=T, seed=2, high_p=0.9)
    assert res["stats"]["rounds"] == ref["rounds"]
    if sched != "lbp":
        assert np.array_equal(res["trace"], ref["trace"][:ref["rounds"]])
    assert np.abs(res["beliefs"] - ref["beliefs"]).max() < TOL_F64
    absent = np.isinf(prob.unary_log.reshape(prob.n, prob.k))
    assert np.all(res["beliefs"][absent] == 0)


@pytest.mark.parametrize("dtype,tol", [("f32", TOL_F32), ("bf16", 1.6e-2)])
@pytest.mark.parametrize("sched,par", [("rnbp", 0.4), ("rs", 0.2)])
def test_wide_states_trace_follow(dtype, tol, sched, par):
    """81 states per vertex at most, FP32 / BF16 storage, RnBP and Residual
    Splash (the k-state splash runs the same kernel per level), against the
    oracle following the GPU frontiers."""
    prob = synth.protein_like(120, seed=5, k_min=2, k_max=81)
    res = gpu_run(prob, sched, par, 1e-4, 25, dtype, trace=25, seed=1, high_p=0.9)
    ref = follow(prob, sched, res, 1e-4, "bf16" if dtype == "bf16" else "f64")
    assert np.abs(res["beliefs"] - ref["beliefs"]).max() < tol


@pytest.mark.parametrize("k", [40, 128])
def test_wide_shared_table(k):
    """A shared k x k table with k > 32 (no tensor-core tiles: the warp-per-
    vertex kernel reads the table through the read-only cache): FP32 LBP on a
    grid against the oracle for the same rounds."""
    prob = synth.potts_grid(8, k, seed=3)
    res = gpu_run(prob, "lbp", 1.0, 1e-4, 15, "f32")
    ref = oracle.run(prob, "lbp", eps=1e-4, trace_in=all_ones_trace(prob.m, res["stats"]["rounds"]),
                     trace_rounds=res["stats"]["rounds"])
    assert np.abs(res["beliefs"] - ref["beliefs"]).max() < TOL_F32
    with bp.Graph(prob) as g:
        with pytest.raises(bp.BPError) as ei:
            g.run("lbp", 1.0, max_rounds=2, potts_path=3)
        assert ei.value.code == bp.BP_ERR_UNSUPPORTED


def test_absent_states_need_tables():
    prob = synth.potts_grid(4, 5, seed=0)
    un = prob.unary_log.copy()
    un[3] = -np.inf
    with bp.Graph(synth.potts_grid(4, 5, seed=0)) as g:
        with pytest.raises(bp.BPError) as ei:
            bp.bp_set_potentials(g.handle, un, prob.pair_kind, prob.pair_log)
        assert ei.value.code == bp.BP_ERR_UNSUPPORTED
        un2 = prob.unary_log.copy()
        un2[:5] = -np.inf
        tab = synth.random_table_graph(16, 5, 0, seed=1)
        with pytest.raises(bp.BPError) as ei:
            bp.bp_set_potentials(g.handle, un2, synth.PAIR_SHARED, prob.pair_log)
        assert ei.value.code in (bp.BP_ERR_NONFINITE, bp.BP_ERR_UNSUPPORTED)
