"""The binary update mappings (thread per vertex, the persistent cluster
kernel, the prefetching thread-per-vertex form, the streamed warp tiles)
compute the same arithmetic in the same order, so every
schedule and storage format gives bit-identical beliefs, rounds and counters
whichever mapping runs."""
import numpy as np
import pytest

from paper_1909_11469_gb300 import bp, synth

pytestmark = pytest.mark.gpu

VARIANTS = [1, 3, 4, 6]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("name", ["grid", "er"])
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "q16"])
@pytest.mark.parametrize("sched,par", [("lbp", 1.0), ("rnbp", 0.5), ("rbp", 0.1), ("rs", 0.1)])
def test_mappings_bit_identical(name, dtype, sched, par):
    prob = synth.ising_grid_batch(37, 2.5, range(5)) if name == "grid" else synth.er_batch(40, 3, n_max=800)
    results = {}
    variants = [v for v in VARIANTS if not (v == 6 and dtype == "f64")]   # 6: FP32 arithmetic only
    for v in variants:
        with bp.Graph(prob) as g:
            st = g.run(sched, par, eps=1e-4, max_rounds=30, msg_dtype=dtype, seed=3, kernel_variant=v)
            results[v] = ((st["rounds"], st["committed_updates"], st["candidate_evals"]), g.beliefs(),
                          [(x["converged"], x["rounds"]) for x in g.graph_stats()])
    key0, bel0, gs0 = results[variants[0]]
    for v in variants[1:]:
        key, bel, gs = results[v]
        assert key == key0, (v, key, key0)
        assert gs == gs0, v
        assert np.array_equal(bel, bel0), (v, float(np.abs(bel - bel0).max()))


@pytest.mark.parametrize("dtype", ["f32", "bf16", "q16"])
def test_rnbp_state_bit_identical(dtype):
    """RnBP on the streamed mapping (warp-tile commit) and on the thread-per-
    vertex mapping (vertex-tile commit): the stored messages, the final
    residuals, the per-round commit trace and the per-graph counters are the
    same bits, on a batch whose graphs stop at different rounds."""
    prob = synth.concat_batch([synth.er_batch(30, 5, n_max=600), synth.ising_grid(12, 0.3, seed=4),
                               synth.ising_chain(50, 0.2, seed=2)])
    out = {}
    for v in (1, 6):
        with bp.Graph(prob) as g:
            st = g.run("rnbp", 0.5, eps=1e-4, max_rounds=60, msg_dtype=dtype, seed=7, kernel_variant=v,
                       record_trace=1, trace_capacity=61)
            out[v] = (st["rounds"], st["committed_updates"], g.messages(), g.residuals(), g.trace("rnbp"),
                      [(x["converged"], x["rounds"], x["committed_updates"]) for x in g.graph_stats()])
    assert out[1][0] == out[6][0] and out[1][1] == out[6][1]
    assert out[1][5] == out[6][5]
    assert len({r for _, r, _ in out[6][5]}) > 1          # graphs stopped at different rounds
    for i in (2, 3, 4):
        assert np.array_equal(out[1][i], out[6][i]), i
    # without a trace the streamed mapping commits inside the update (both
    # EdgeRatio outcomes written, three message buffers): the same state again
    with bp.Graph(prob) as g:
        st = g.run("rnbp", 0.5, eps=1e-4, max_rounds=60, msg_dtype=dtype, seed=7, kernel_variant=6)
        assert g.profile()["fused_commit"] == 1
        fused = (st["rounds"], st["committed_updates"], g.messages(), g.residuals(),
                 [(x["converged"], x["rounds"], x["committed_updates"]) for x in g.graph_stats()])
    assert fused[0] == out[1][0] and fused[1] == out[1][1] and fused[4] == out[1][5]
    for i in (2, 3):
        assert np.array_equal(fused[i], out[1][i]), i


def test_rnbp_time_budget_stop_equals_round_cap():
    """A run stopped by its wall-clock budget ends after a whole round (the
    round's commit included): its messages equal those of a run of the other
    mapping stopped by max_rounds at the same committed round."""
    prob = synth.ising_grid(60, 3.0, seed=1)
    with bp.Graph(prob) as g:
        st = g.run("rnbp", 0.5, eps=1e-12, max_rounds=10_000_000, time_budget_ms=50.0, kernel_variant=6,
                   seed=2)
        assert st["status"] == bp.BP_ERR_TIMEOUT and not st["converged"]
        rounds, committed, msg = st["rounds"], st["committed_updates"], g.messages()
    assert rounds > 1
    with bp.Graph(prob) as g:
        st1 = g.run("rnbp", 0.5, eps=1e-12, max_rounds=rounds, kernel_variant=1, seed=2)
        assert st1["rounds"] == rounds and st1["committed_updates"] == committed
        assert np.array_equal(g.messages(), msg)


def _star_batch(leaves_list, seed=0):
    """Stars (one hub joined to `leaves` vertices) followed by isolated
    vertices, as one batch: hubs at the tile edge limit, tiles cut by the
    vertex limit, and runs of edgeless vertices between tiles."""
    rng = np.random.default_rng(seed)
    probs = []
    for leaves in leaves_list:
        n = leaves + 1 + 40
        ei = np.zeros(leaves, np.int64)
        ej = np.arange(1, leaves + 1, dtype=np.int64)
        row_ptr, col, rev = synth.csr_from_undirected(n, ei, ej)
        un = rng.uniform(-1, 1, n).astype(np.float32)
        unary = np.stack([-un, un], 1).reshape(-1).astype(np.float32)
        beta = np.zeros(col.shape[0], np.float32)
        pos = synth._undirected_positions(row_ptr, col)
        b = rng.uniform(-1.5, 1.5, pos.shape[0]).astype(np.float32)
        beta[pos] = b
        beta[rev[pos]] = b
        probs.append(synth.Problem(n, 2, row_ptr, col, rev, unary, synth.PAIR_ISING_BETA, beta,
                                   np.array([0, n], np.int64)))
    return synth.concat_batch(probs)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "q16"])
def test_streamed_tiles_edge_cases(dtype):
    """The streamed warp tiles at their limits (a vertex with 128 out-edges
    fills a tile; 127 and 1 edges share none), with edgeless vertices between
    tiles and graphs without edges, give mapping 1's bits."""
    prob = synth.concat_batch([_star_batch([128, 127, 1, 64]), synth.ising_grid(9, 1.0, seed=2),
                               _star_batch([0, 3], seed=1)])
    out = {}
    for v in (1, 6):
        with bp.Graph(prob) as g:
            st = g.run("rnbp", 0.5, eps=1e-6, max_rounds=50, msg_dtype=dtype, seed=1, kernel_variant=v)
            out[v] = (st["rounds"], st["committed_updates"], g.beliefs())
    assert out[1][:2] == out[6][:2]
    assert np.array_equal(out[1][2], out[6][2])


def test_streamed_tiles_reject_high_degree():
    """A vertex with more than 128 out-edges does not fit a warp tile: the
    streamed mapping is refused, the automatic choice still runs."""
    prob = _star_batch([129])
    with bp.Graph(prob) as g:
        with pytest.raises(bp.BPError) as ei:
            g.run("lbp", 1.0, eps=1e-4, max_rounds=5, kernel_variant=6)
        assert ei.value.code == bp.BP_ERR_UNSUPPORTED
        g.run("lbp", 1.0, eps=1e-4, max_rounds=5)
    with bp.Graph(synth.ising_grid(6, 1.0, seed=0)) as g:
        with pytest.raises(bp.BPError) as ei:
            g.run("lbp", 1.0, eps=1e-4, max_rounds=5, kernel_variant=6, msg_dtype="f64")
        assert ei.value.code == bp.BP_ERR_UNSUPPORTED
