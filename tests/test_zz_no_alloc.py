"""The allocation-free LBP entry point (bp_lbp_run_noalloc).

It exists for callers that cannot allocate device memory themselves or
through the library: code under another framework's caching allocator that
already holds the GPU's memory, latency-critical paths where cudaMalloc or
cudaFree would synchronise the device, plug-ins that must leave the allocation
state untouched. Its scratch is a static device array inside the library, so
its results must equal bp_run's, call after call, and a call after the first
one on a device must not change the device's free memory. This file is
collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# The largest graph the static scratch holds, and the first-call set-up bound:
# the 5 MiB array plus the entry point's device code, in the driver's pages.
NA_MAX_EDGES = 1 << 18
NA_MAX_VARS = 1 << 17
FIRST_CALL_MAX_BYTES = 64 << 20


def _dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def _device_arrays(torch, prob):
    return (_dev(torch, prob.row_ptr, np.int32), _dev(torch, prob.col, np.int32),
            _dev(torch, prob.rev, np.int32), _dev(torch, prob.unary_log, np.float32),
            _dev(torch, prob.pair_log, np.float32))


def _noalloc(torch, bp, prob, arrays, eps, max_rounds, stream=None):
    out = torch.empty(prob.n * 2, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    rounds, conv = bp.bp_lbp_run_noalloc(prob.n, prob.m, *arrays, eps, max_rounds, out, stream)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    return rounds, conv, out.cpu().numpy().reshape(-1, 2), free_before - free_after


def test_noalloc_matches_bp_run_two_calls_in_a_row():
    """Two calls in a row on different graphs: each equals bp_run with the
    same mapping bit for bit (and the automatic mapping within 1e-5); the
    first call on the device may only load the entry point (bounded), the
    second allocates nothing."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1909_11469_gb300 import bp, synth

    stream = torch.cuda.current_stream().cuda_stream
    for call, seed in enumerate((0, 1)):
        prob = synth.ising_grid(64, 1.0, seed=seed, cols=48)
        arrays = _device_arrays(torch, prob)
        rounds, conv, bel, used = _noalloc(torch, bp, prob, arrays, 1e-4, 500, stream)
        with bp.Graph(prob) as g:
            st = g.run("lbp", 1.0, eps=1e-4, max_rounds=500, msg_dtype="f32", kernel_variant=1)
            same_mapping = g.beliefs()
            st_auto = g.run("lbp", 1.0, eps=1e-4, max_rounds=500, msg_dtype="f32")
            auto = g.beliefs()
        assert rounds == st["rounds"] and conv == bool(st["converged"])
        assert np.array_equal(bel, same_mapping)
        assert rounds == st_auto["rounds"] and np.abs(bel - auto).max() < 1e-5
        if call == 0:
            assert used <= FIRST_CALL_MAX_BYTES, used
        else:
            assert used == 0, used


def test_noalloc_at_the_edge_capacity():
    """A 256x256 grid (65,536 vertices, 261,120 directed edges: the largest
    square grid the scratch holds) equals bp_run, twice in a row, with no
    allocation."""
    import torch

    from paper_1909_11469_gb300 import bp, synth

    prob = synth.ising_grid(256, 1.0, seed=3)
    assert prob.m <= NA_MAX_EDGES and prob.m > NA_MAX_EDGES - 4096
    arrays = _device_arrays(torch, prob)
    with bp.Graph(prob) as g:
        st = g.run("lbp", 1.0, eps=1e-4, max_rounds=300, msg_dtype="f32", kernel_variant=1)
        ref = g.beliefs()
    for _ in range(2):
        rounds, conv, bel, used = _noalloc(torch, bp, prob, arrays, 1e-4, 300)
        assert rounds == st["rounds"] and conv == bool(st["converged"])
        assert np.array_equal(bel, ref)
        assert used == 0, used


def test_noalloc_rejects_oversize_and_bad_graph():
    import torch

    from paper_1909_11469_gb300 import bp, synth

    prob = synth.ising_grid(8, 1.0, seed=0)
    arrays = _device_arrays(torch, prob)
    out = torch.empty(prob.n * 2, dtype=torch.float64, device="cuda")
    # both limits, each exceeded by one with the other one valid (rejected on
    # the host, before any device array is read)
    for n, m in ((NA_MAX_VARS + 1, prob.m), (prob.n, NA_MAX_EDGES + 1), (1 << 20, prob.m)):
        with pytest.raises(bp.BPError) as ei:
            bp.bp_lbp_run_noalloc(n, m, *arrays, 1e-4, 10, out)
        assert ei.value.code == bp.BP_ERR_UNSUPPORTED
    bad = prob.rev.copy()
    bad[0], bad[1] = bad[1], bad[0]
    rp, col, _, un, beta = arrays
    with pytest.raises(bp.BPError) as ei:
        bp.bp_lbp_run_noalloc(prob.n, prob.m, rp, col, _dev(torch, bad, np.int32), un, beta, 1e-4, 10, out)
    assert ei.value.code == bp.BP_ERR_BAD_GRAPH
    rounds, _ = bp.bp_lbp_run_noalloc(prob.n, prob.m, *arrays, 1e-4, 10, out)
    assert rounds <= 10
