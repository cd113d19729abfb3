"""The binary update mappings (thread per vertex, tiled edge quads, the
persistent cluster kernel, the prefetching thread-per-vertex forms) compute
the same arithmetic in the same order, so every schedule and storage format
gives bit-identical beliefs, rounds and counters whichever mapping runs."""
import numpy as np
import pytest

from paper_1909_11469_gb300 import bp, synth

pytestmark = pytest.mark.gpu

VARIANTS = [1, 2, 3, 4, 5]


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
    for v in VARIANTS:
        with bp.Graph(prob) as g:
            st = g.run(sched, par, eps=1e-4, max_rounds=30, msg_dtype=dtype, seed=3, kernel_variant=v)
            results[v] = ((st["rounds"], st["committed_updates"], st["candidate_evals"]), g.beliefs(),
                          [(x["converged"], x["rounds"]) for x in g.graph_stats()])
    key0, bel0, gs0 = results[VARIANTS[0]]
    for v in VARIANTS[1:]:
        key, bel, gs = results[v]
        assert key == key0, (v, key, key0)
        assert gs == gs0, v
        assert np.array_equal(bel, bel0), (v, float(np.abs(bel - bel0).max()))
