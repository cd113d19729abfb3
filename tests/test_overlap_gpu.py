"""Programmatic dependent launches (bp_options.overlap_launches, on by
default): the per-round update, decision and RnBP commit grids may be
scheduled while the previous kernel drains and wait for it before reading run
state, so every result is bit-identical to ordinary launches (2 = off), in
captured rounds and in directly launched (profiled) rounds, and FP64 runs
still replay the oracle."""
import numpy as np
import pytest

import oracle
from paper_1909_11469_gb300 import bp, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def run(prob, sched, par, dtype, overlap, variant=0, rounds=40, profile=0, **opts):
    with bp.Graph(prob) as g:
        st = g.run(sched, par, eps=1e-5, max_rounds=rounds, msg_dtype=dtype, seed=3,
                   overlap_launches=overlap, kernel_variant=variant, profile=profile, **opts)
        return (st, g.beliefs(), g.messages(),
                [(x["converged"], x["rounds"], x["committed_updates"]) for x in g.graph_stats()],
                g.profile())


@pytest.mark.parametrize("name", ["grids", "er"])
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "q16"])
@pytest.mark.parametrize("sched,par", [("lbp", 1.0), ("rnbp", 0.5), ("rbp", 0.1), ("rs", 0.1)])
def test_overlap_bit_identical(name, dtype, sched, par):
    prob = synth.ising_grid_batch(37, 2.5, range(5)) if name == "grids" else synth.er_batch(40, 3, n_max=800)
    a = run(prob, sched, par, dtype, 2)
    assert a[4]["overlap_launches"] == 0
    for overlap, variant, profile in ((1, 0, 0), (1, 1, 0), (1, 0, 1), (0, 0, 0)):
        b = run(prob, sched, par, dtype, overlap, variant=variant, profile=profile)
        assert b[4]["overlap_launches"] == 1
        keys = ("rounds", "committed_updates", "candidate_evals", "converged")
        assert [a[0][k] for k in keys] == [b[0][k] for k in keys], (variant, profile)
        assert a[3] == b[3], (variant, profile)
        assert np.array_equal(a[1], b[1]), (variant, profile, float(np.abs(a[1] - b[1]).max()))
        assert np.array_equal(a[2], b[2]), (variant, profile)


@pytest.mark.parametrize("sched,par", [("lbp", 1.0), ("rnbp", 0.5), ("rbp", 0.05), ("rs", 0.1)])
def test_overlap_fp64_replays_oracle(sched, par):
    """Ragged 13 x 11 grid, 60 rounds: the same frontier every round and the
    same state as the oracle."""
    prob = synth.ising_grid(13, 2.0, seed=4, cols=11)
    T = 60
    ref = oracle.run(prob, sched, parallelism=par, eps=1e-7, max_rounds=T, seed=5, trace_cap=T)
    with bp.Graph(prob) as g:
        st = g.run(sched, par, eps=1e-7, max_rounds=T, msg_dtype="f64", seed=5, overlap_launches=1,
                   record_trace=1 if sched != "lbp" else 0, trace_capacity=T if sched != "lbp" else 0)
        assert st["rounds"] == ref["rounds"]
        if sched != "lbp":
            assert np.array_equal(g.trace(sched), ref["trace"][:ref["rounds"]])
        assert st["committed_updates"] == ref["committed_updates"]
        assert np.abs(g.beliefs() - ref["beliefs"]).max() < 1e-10
        assert np.abs(g.messages() - ref["messages"]).max() < 1e-10


def test_overlap_default_batch_few_rounds():
    """The benchmark's batch shape (50 Ising 100 x 100 grids), a few rounds of
    every schedule, with and without overlapped launches."""
    prob = synth.ising_grid_batch(100, 2.5, range(50))
    for sched, par in (("lbp", 1.0), ("rnbp", 0.5), ("rbp", 0.1), ("rs", 0.1)):
        a = run(prob, sched, par, "f32", 2, rounds=6)
        b = run(prob, sched, par, "f32", 1, rounds=6)
        assert a[0]["committed_updates"] == b[0]["committed_updates"], sched
        assert np.array_equal(a[1], b[1]), sched


def test_bad_overlap_rejected():
    prob = synth.ising_grid(5, 1.0, seed=0)
    with bp.Graph(prob) as g:
        with pytest.raises(bp.BPError):
            g.run("lbp", 1.0, overlap_launches=3)
