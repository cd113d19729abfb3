"""Parity at the workload sizes the benchmark and the configurations use.

Whole-trajectory oracle runs are affordable for a few rounds even at a million
vertices, so these tests follow the GPU's frontiers for a short horizon and
compare every belief (or a sample of graphs of a batch) against the FP64 oracle.
The GPU runs use the benchmark's launch configuration: a batch handle, FP32
messages, the caller's torch stream.
"""
import numpy as np
import pytest

import oracle
from paper_1909_11469_gb300 import bp, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _bits(trace, lo, hi):
    """Bits [lo, hi) of every row of a union trace, repacked from bit 0."""
    rows = []
    for row in trace:
        b = np.unpackbits(row.view(np.uint8), bitorder="little")[lo:hi]
        pad = np.zeros(((hi - lo + 31) // 32) * 32, np.uint8)
        pad[:hi - lo] = b
        rows.append(np.packbits(pad, bitorder="little").view(np.uint32))
    return np.array(rows, dtype=np.uint32).reshape(len(rows), -1)


def _ones(count, rounds):
    words = (count + 31) // 32
    bits = np.zeros(words * 32, np.uint8)
    bits[:count] = 1
    return np.tile(np.packbits(bits, bitorder="little").view(np.uint32), (rounds, 1))


def _stream_opts():
    import torch
    return {"cuda_stream": torch.cuda.current_stream().cuda_stream}


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("sched,par", [("lbp", 1.0), ("rnbp", 0.5), ("rbp", 0.1), ("rs", 0.1)])
def test_bench_batch_sampled_graphs(sched, par, variant):
    """50 seeds of the 100x100, beta ~ U[-2.5, 2.5] grid as one batch (the bench
    workload); graphs 0, 17 and 49 followed by the oracle for 12 rounds (3 for
    Residual Splash, whose rounds sweep 2h + 1 = 5 levels each)."""
    batch = synth.ising_grid_batch(100, 2.5, range(50))
    T = 3 if sched == "rs" else 12
    with bp.Graph(batch) as g:
        st = g.run(sched, par, eps=1e-4, max_rounds=T, msg_dtype="f32", record_trace=1,
                   trace_capacity=T, seed=0, kernel_variant=variant, **_stream_opts())
        bel = g.beliefs()
        tr = g.trace(sched)
        gst = g.graph_stats()
    assert st["rounds"] == T
    for gi in (0, 17, 49):
        one = batch.graph(gi)
        v0, v1 = batch.graph_var_offsets[gi], batch.graph_var_offsets[gi + 1]
        if sched == "lbp":
            tin = _ones(one.m, T)
        elif sched == "rs":
            tin = _bits(tr, v0, v1)
        else:
            e0, e1 = batch.row_ptr[v0], batch.row_ptr[v1]
            tin = _bits(tr, e0, e1)
        ref = oracle.run(one, sched, eps=1e-4, trace_in=tin, trace_rounds=gst[gi]["rounds"])
        assert np.abs(bel[v0:v1] - ref["beliefs"]).max() < 1e-5, gi


@pytest.mark.parametrize("sched,dtype,tol", [("lbp", "f32", 1e-5), ("rnbp", "f32", 1e-5),
                                             ("rnbp", "q16", 2e-3), ("lbp", "bf16", 2e-3),
                                             ("rnbp", "bf16", 2e-3)])
def test_ising1000_full_grid(sched, dtype, tol):
    """1000x1000 Ising, beta ~ U[-3, 3] (4M messages): 4 rounds, every belief
    against the oracle following the GPU frontiers."""
    prob = synth.ising_grid(1000, 3.0, seed=0)
    T = 4
    with bp.Graph(prob) as g:
        st = g.run(sched, 0.5, eps=1e-4, max_rounds=T, msg_dtype=dtype, record_trace=1,
                   trace_capacity=T, seed=1, **_stream_opts())
        bel = g.beliefs()
        tr = g.trace(sched) if sched != "lbp" else _ones(prob.m, T)
    assert st["rounds"] == T
    ref = oracle.run(prob, sched, eps=1e-4, trace_in=tr, trace_rounds=T,
                     storage="f64", seed=1)
    assert np.abs(bel - ref["beliefs"]).max() < tol


@pytest.mark.parametrize("variant", [0, 1])
def test_er_batch_4096_sampled(variant):
    """4096 Erdos-Renyi graphs (n log-uniform in [50, 5000], mean degree 4,
    beta ~ U[-3, 3]): every graph converges or stops on its own; sampled graphs
    match oracle runs of the same length."""
    batch = synth.er_batch(4096, seed=0)
    T = 40
    with bp.Graph(batch) as g:
        g.run("rnbp", 0.5, eps=1e-4, max_rounds=T, msg_dtype="f64", seed=2, kernel_variant=variant,
              **_stream_opts())
        bel = g.beliefs()
        gst = g.graph_stats()
    rng = np.random.default_rng(0)
    for gi in rng.choice(4096, 6, replace=False):
        one = batch.graph(int(gi))
        ref = oracle.run(one, "rnbp", parallelism=0.5, eps=1e-4, max_rounds=T, seed=2,
                         graph_id=int(gi))
        assert gst[gi]["rounds"] == ref["rounds"], gi
        assert bool(gst[gi]["converged"]) == ref["converged"], gi
        v0, v1 = batch.graph_var_offsets[gi], batch.graph_var_offsets[gi + 1]
        assert np.abs(bel[v0:v1] - ref["beliefs"]).max() < 1e-9, gi


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_er_batch_4096_fused_commit_equals_commit_kernel(dtype):
    """The benchmark's workload as the bench runs it (RnBP on the streamed
    update without a trace: the commit inside the update, both EdgeRatio
    outcomes written) against the same run with a recorded trace (the commit
    kernel after the update, whose frontiers the trace-follow test below checks
    against the oracle): the same messages, residuals and per-graph counters,
    bit for bit, after 30 rounds."""
    batch = synth.er_batch(4096, seed=0)
    out = []
    for trace in (0, 1):
        with bp.Graph(batch) as g:
            st = g.run("rnbp", 0.5, eps=1e-4, max_rounds=30, msg_dtype=dtype, record_trace=trace,
                       trace_capacity=30 if trace else 0, seed=3, kernel_variant=6, **_stream_opts())
            assert g.profile()["fused_commit"] == (0 if trace else 1)
            out.append((st["rounds"], st["committed_updates"], g.messages(), g.residuals(),
                        [(x["converged"], x["rounds"], x["committed_updates"]) for x in g.graph_stats()]))
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1] and out[0][4] == out[1][4]
    assert np.array_equal(out[0][2], out[1][2]) and np.array_equal(out[0][3], out[1][3])


@pytest.mark.parametrize("dtype,tol,T", [("f32", 1e-5, 20), ("bf16", 2e-3, 6)])
@pytest.mark.parametrize("variant", [0, 6])
def test_er_batch_4096_trace_follow(dtype, tol, T, variant):
    """The benchmark's workload (4096 Erdos-Renyi graphs, 17.9M messages,
    beta ~ U[-3, 3]): T RnBP rounds (LowP 0.5) with the automatic and the
    streamed update mapping; on sampled graphs the exact FP64 oracle commits
    the GPU's recorded frontiers of that graph. (beta up to 3 is far from
    contracting, so BF16's rounding is followed for a shorter horizon.)"""
    batch = synth.er_batch(4096, seed=0)
    with bp.Graph(batch) as g:
        g.run("rnbp", 0.5, eps=1e-4, max_rounds=T, msg_dtype=dtype, record_trace=1, trace_capacity=T,
              seed=3, kernel_variant=variant, **_stream_opts())
        bel = g.beliefs()
        gst = g.graph_stats()
        tr = g.trace("rnbp")
    rng = np.random.default_rng(1)
    for gi in rng.choice(4096, 8, replace=False):
        gi = int(gi)
        one = batch.graph(gi)
        v0, v1 = batch.graph_var_offsets[gi], batch.graph_var_offsets[gi + 1]
        e0, e1 = batch.row_ptr[v0], batch.row_ptr[v1]
        rounds = gst[gi]["rounds"]
        ref = oracle.run(one, "rnbp", eps=1e-4, trace_in=_bits(tr[:rounds], e0, e1), trace_rounds=rounds)
        assert np.abs(bel[v0:v1] - ref["beliefs"]).max() < tol, gi


def test_potts256_k32():
    """Potts 256x256, k = 32, shared table: 3 RnBP rounds (LowP 0.5), every
    belief against the oracle following the GPU frontiers."""
    prob = synth.potts_grid(256, 32, seed=0)
    T = 3
    with bp.Graph(prob) as g:
        g.run("rnbp", 0.5, eps=1e-4, max_rounds=T, msg_dtype="f32", record_trace=1,
              trace_capacity=T, seed=0, **_stream_opts())
        bel = g.beliefs()
        tr = g.trace("rnbp")
    ref = oracle.run(prob, "rnbp", eps=1e-4, trace_in=tr, trace_rounds=T)
    assert np.abs(bel - ref["beliefs"]).max() < 1e-5
