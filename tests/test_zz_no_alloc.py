"""The allocation-free LBP entry point (bp_lbp_run_noalloc).

It exists for callers that cannot allocate device memory themselves or
through the library: code under another framework's caching allocator that
already holds the GPU's memory, latency-critical paths where cudaMalloc or
cudaFree would synchronise the device, plug-ins that must leave the allocation
state untouched. Its scratch is a static device array inside the library, so
its results must equal bp_run's, call after call, and a call must not change
the device's free memory. This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def test_noalloc_matches_bp_run_two_calls_in_a_row():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1909_11469_gb300 import bp, synth

    stream = torch.cuda.current_stream().cuda_stream
    for call, seed in enumerate((0, 1)):
        prob = synth.ising_grid(64, 1.0, seed=seed, cols=48)
        rp = _dev(torch, prob.row_ptr, np.int32)
        col = _dev(torch, prob.col, np.int32)
        rev = _dev(torch, prob.rev, np.int32)
        un = _dev(torch, prob.unary_log, np.float32)
        beta = _dev(torch, prob.pair_log, np.float32)
        out = torch.empty(prob.n * 2, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rounds, conv = bp.bp_lbp_run_noalloc(prob.n, prob.m, rp, col, rev, un, beta, 1e-4, 500, out,
                                             stream)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        with bp.Graph(prob) as g:
            st = g.run("lbp", 1.0, eps=1e-4, max_rounds=500, msg_dtype="f32")
            ref = g.beliefs()
        assert rounds == st["rounds"] and conv == bool(st["converged"])
        assert np.abs(out.cpu().numpy().reshape(-1, 2) - ref).max() < 1e-5
        if call == 1:   # the first call on a device may load the module
            assert free_after == free_before


def test_noalloc_rejects_oversize_and_bad_graph():
    import torch

    from paper_1909_11469_gb300 import bp, synth

    prob = synth.ising_grid(8, 1.0, seed=0)
    rp = _dev(torch, prob.row_ptr, np.int32)
    col = _dev(torch, prob.col, np.int32)
    rev = _dev(torch, prob.rev, np.int32)
    un = _dev(torch, prob.unary_log, np.float32)
    beta = _dev(torch, prob.pair_log, np.float32)
    out = torch.empty(prob.n * 2, dtype=torch.float64, device="cuda")
    with pytest.raises(bp.BPError) as ei:
        bp.bp_lbp_run_noalloc(1 << 20, prob.m, rp, col, rev, un, beta, 1e-4, 10, out)
    assert ei.value.code == bp.BP_ERR_UNSUPPORTED
    bad = prob.rev.copy()
    bad[0], bad[1] = bad[1], bad[0]
    with pytest.raises(bp.BPError) as ei:
        bp.bp_lbp_run_noalloc(prob.n, prob.m, rp, col, _dev(torch, bad, np.int32), un, beta, 1e-4, 10, out)
    assert ei.value.code == bp.BP_ERR_BAD_GRAPH
    rounds, _ = bp.bp_lbp_run_noalloc(prob.n, prob.m, rp, col, rev, un, beta, 1e-4, 10, out)
    assert rounds <= 10
