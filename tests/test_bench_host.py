"""Host-side arithmetic of bench.py (no GPU): the algorithmic byte counts per
message, the round caps, and the roofline figures computed from a profiled
step. A profiled step is a list of (schedule, p, run stats, profile, per-graph
stats) as bench.py collects it from bp_run / bp_get_profile."""
import math

import pytest

import bench


def test_bytes_per_message():
    # binary Ising: rev 4 + q 4 + incoming, old and new message (3 s) + residual in frontier modes
    assert bench.bytes_per_msg("lbp", "f32") == 20
    assert bench.bytes_per_msg("rnbp", "f32") == 24
    assert bench.bytes_per_msg("rbp", "bf16") == 18
    assert bench.bytes_per_msg("lbp", "q16") == 14
    assert bench.bytes_per_msg("rs", "f64") == 8 + 24 + 8
    # k-state: rev 4 + 3 k s + residual 4
    assert bench.bytes_per_msg("rnbp", "f32", k=32) == 4 + 3 * 32 * 4 + 4
    assert bench.bytes_per_vertex() == 12 and bench.bytes_per_vertex(32) == 8 + 128
    # RnBP with the commit inside the streamed update: + the second outcome (s)
    assert bench.bytes_per_msg("rnbp", "f32", fused=True) == 28
    assert bench.bytes_per_msg("rnbp", "bf16", fused=True) == 20


def test_eval_roofline_counts_the_fused_outcome():
    """A profiled RnBP step whose rounds committed inside the update counts the
    second outcome's bytes; the same step without it does not."""
    plain = _step("rnbp", full_evals=1000, vertices=250, eval_ms=1.0)
    fused = _step("rnbp", full_evals=1000, vertices=250, eval_ms=1.0, extra={"fused_commit": 1})
    a, _ = bench.eval_roofline([plain], "f32", 1000.0, "measured")
    b, _ = bench.eval_roofline([fused], "f32", 1000.0, "measured")
    assert a["bytes_per_launch"] == (24 * 1000 + 12 * 250) / 10
    assert b["bytes_per_launch"] == (28 * 1000 + 12 * 250) / 10


def test_round_caps():
    assert bench.round_cap("lbp", 1.0) == 1000
    assert bench.round_cap("rnbp", 0.5) == 2000
    assert bench.round_cap("rbp", 0.1) == 10000
    assert bench.round_cap("rs", 0.3) == math.ceil(1000 / 0.3)


def _step(sched="lbp", full_evals=1000, vertices=250, eval_ms=2.0, launches=10, extra=None, st=None):
    pr = {"full_evals": full_evals, "active_vertices": vertices, "eval_ms": eval_ms, "eval_launches": launches,
          "decide_ms": 0.5, "frontier_ms": 1.0, "select_ms": 0.4, "sweep_ms": 0.6, "sweep_launches": 0,
          "kernel_variant": 4, "sweep_form": 0}
    pr.update(extra or {})
    stats = {"committed_updates": 500}
    stats.update(st or {})
    return (sched, 1.0, stats, pr, [])


def test_eval_roofline_in_step_and_isolated():
    step = [_step("lbp", full_evals=1000, vertices=250, eval_ms=2.0, launches=10)]
    out, phase = bench.eval_roofline(step, "f32", 1000.0, "measured")
    alg = 20 * 1000 + 12 * 250
    assert out["achieved"] == pytest.approx(alg / 2e-3 / 1e9)
    assert out["frac"] == pytest.approx(out["achieved"] / 1000.0)
    assert out["bytes_per_launch"] == pytest.approx(alg / 10)
    assert phase == {"eval_ms": 2.0, "decide_ms": 0.5, "frontier_ms": 1.0}
    # kernel alone: per-launch bytes of the whole graph (m messages, n vertices) / isolated ms
    out2, _ = bench.eval_roofline(step, "f32", 1000.0, "measured", isolated={"lbp": 0.01}, n=400, m=1600)
    per_launch = 20 * 1600 + 12 * 400
    assert out2["achieved"] == pytest.approx(per_launch / 1e-5 / 1e9)
    assert out2["in_step"]["achieved"] == pytest.approx(out["achieved"])


def test_sweep_roofline_bytes():
    assert bench.sweep_roofline([_step("lbp")], "f32", 100, 400, 1000.0, "m") is None
    rs = _step("rs", extra={"sweep_ms": 4.0, "sweep_launches": 60}, st={"committed_updates": 10000})
    out = bench.sweep_roofline([rs], "f32", 100, 400, 1000.0, "m")
    dbar = 400 / 100
    b = 10000 * (13 + 8 + 16 / dbar) + 10000 * (8 + 12 / dbar)
    assert out["achieved"] == pytest.approx(b / 4e-3 / 1e9)
    assert out["kernel"].startswith("k_splash_list_step") and out["sweep_form"] == "per_sub_step"
    assert out["avg_launch_us"] == pytest.approx(4e3 / 60)


def test_select_roofline():
    rbp = _step("rbp", full_evals=4000, launches=5, st={"committed_updates": 400})
    out = bench.select_roofline([rbp], "f32", 100, 400, 1000.0, "m", "rbp")
    b = 4 * 4000 + 2 * 4 * 400
    assert out["launches"] == 4   # the last evaluation selects nothing
    assert out["achieved"] == pytest.approx(b / 0.4e-3 / 1e9)
    rs = _step("rs", full_evals=4000, vertices=1000, launches=5)
    out = bench.select_roofline([rs], "f32", 100, 400, 1000.0, "m", "rs")
    assert out["achieved"] == pytest.approx((8 * 4000 + 5 * 1000) / 0.4e-3 / 1e9)
    assert bench.select_roofline([rs], "f32", 100, 400, 1000.0, "m", "rbp") is None


def test_mcnemar_exact_known_values():
    """The statistics tests' paired test: two-sided exact McNemar p-values,
    against Binomial(n, 1/2) tails worked by hand (8 pairs all on one side:
    2 / 2^8; 5 against 1: 2 (1 + 6) / 2^6)."""
    from tests._stats import mcnemar_exact
    assert mcnemar_exact(0, 0) == 1.0
    assert mcnemar_exact(8, 0) == 2 / 2 ** 8
    assert mcnemar_exact(0, 8) == 2 / 2 ** 8
    assert mcnemar_exact(5, 1) == 2 * 7 / 2 ** 6
    assert mcnemar_exact(3, 3) == 1.0
