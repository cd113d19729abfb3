"""Host-side checks of the C ABI (no GPU): the library loads, exports every
function include/bp_gb300.h declares, its structs match the binding's layout,
and invalid graphs are rejected before any device work."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1909_11469_gb300 import bp, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bp_gb300.h")


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    return bp.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bp_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(bp._SIGNATURES)


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stddef.h>
#include <stdio.h>
#include "bp_gb300.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(bp_options), sizeof(bp_run_stats),
         offsetof(bp_options, cuda_stream), offsetof(bp_options, kernel_variant),
         offsetof(bp_run_stats, device_ms), offsetof(bp_run_stats, status),
         sizeof(bp_profile), offsetof(bp_profile, kernel_variant),
         sizeof(bp_tune_result), offsetof(bp_tune_result, ms_per_round_select),
         offsetof(bp_options, overlap_launches), offsetof(bp_profile, overlap_launches));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    vals = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert vals == [ctypes.sizeof(bp.bp_options), ctypes.sizeof(bp.bp_run_stats),
                    bp.bp_options.cuda_stream.offset, bp.bp_options.kernel_variant.offset,
                    bp.bp_run_stats.device_ms.offset, bp.bp_run_stats.status.offset,
                    ctypes.sizeof(bp.bp_profile), bp.bp_profile.kernel_variant.offset,
                    ctypes.sizeof(bp.bp_tune_result), bp.bp_tune_result.ms_per_round_select.offset,
                    bp.bp_options.overlap_launches.offset, bp.bp_profile.overlap_launches.offset]


def test_status_strings(L):
    for code in range(0, -10, -1):
        assert bp.bp_status_string(code) not in ("", "unknown status")
    assert bp.bp_status_string(-77) == "unknown status"


def test_default_options(L):
    o = bp.bp_default_options()
    assert o.high_p == 1.0 and o.ratio_threshold == 0.9 and o.splash_depth == 2
    assert o.msg_dtype == bp.BP_F32 and o.cuda_stream is None
    # automatic choices: update mapping, selection path, sweep form, launch overlap
    assert o.kernel_variant == 0 and o.select_path == 0 and o.splash_sweep == 0 and o.overlap_launches == 0
    assert bp.bp_default_options(splash_sweep=1, overlap_launches=2).splash_sweep == 1


def _expect(code, fn):
    with pytest.raises(bp.BPError) as ei:
        fn()
    assert ei.value.code == code, str(ei.value)


def test_invalid_graphs_rejected_on_host(L):
    p = synth.ising_grid(3, 1.0, seed=0)
    rp, col, rev = p.row_ptr.copy(), p.col.copy(), p.rev.copy()
    bad_rev = rev.copy()
    bad_rev[0], bad_rev[1] = bad_rev[1], bad_rev[0]
    _expect(bp.BP_ERR_BAD_GRAPH, lambda: bp.bp_create_graph(p.n, 2, rp, col, bad_rev))
    bad_col = col.copy()
    bad_col[3] = p.n
    _expect(bp.BP_ERR_BAD_GRAPH, lambda: bp.bp_create_graph(p.n, 2, rp, bad_col, rev))
    bad_rp = rp.copy()
    bad_rp[2], bad_rp[3] = bad_rp[3], bad_rp[2]
    _expect(bp.BP_ERR_BAD_GRAPH, lambda: bp.bp_create_graph(p.n, 2, bad_rp, col, rev))
    big_rp = rp.copy()
    big_rp[1] = p.m + 5
    _expect(bp.BP_ERR_BAD_GRAPH, lambda: bp.bp_create_graph(p.n, 2, big_rp, col, rev))
    # self-loop: 2 vertices, edge 0->0 with rev = itself
    _expect(bp.BP_ERR_BAD_GRAPH, lambda: bp.bp_create_graph(
        2, 2, np.array([0, 1, 1]), np.array([0], np.int32), np.array([0], np.int32)))
    _expect(bp.BP_ERR_UNSUPPORTED, lambda: bp.bp_create_graph(p.n, 129, rp, col, rev))
    _expect(bp.BP_ERR_UNSUPPORTED, lambda: bp.bp_create_graph(p.n, 1, rp, col, rev))
    # a batch whose edge crosses from graph 0 into graph 1
    _expect(bp.BP_ERR_BAD_GRAPH, lambda: bp.bp_create_batch(
        np.array([0, 4, p.n]), 2, rp, col, rev))
    _expect(bp.BP_ERR_BAD_GRAPH, lambda: bp.bp_create_batch(
        np.array([0, 5, 4, p.n]), 2, rp, col, rev))


def test_tuning_entry_points_reject_bad_arguments(L):
    out = bp.bp_tune_result()
    assert L.bp_autotune(None, 0, 1.0, 1e-4, None, 4, ctypes.byref(out)) == bp.BP_ERR_INVALID_ARG
    assert L.bp_set_graph_parallelism(None, None) == bp.BP_ERR_INVALID_ARG
    cand = np.array([0.5])
    assert L.bp_autotune_parallelism(None, bp.BP_RNBP, cand.ctypes.data, 1, 1e-4, 10, None,
                                     None) == bp.BP_ERR_INVALID_ARG
