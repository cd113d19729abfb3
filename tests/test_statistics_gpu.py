"""Independent statistics over 50 seeds: the GPU (FP32 messages) and the FP64
oracle each select their own frontiers. The converged fraction may differ by
at most one seed (a threshold flip), except under RnBP, whose random frontiers
(Section IV-A) make convergence within the cap a matter of the random stream
on a marginal seed (on the 100x100 seeds at LowP 0.5 the oracle's own
converged count varies between 45 and 47 over random streams 0 to 3): there
the seeds converged on one side only must not lean to one side beyond chance,
by the exact two-sided McNemar test at level 0.01 (with all of them on one
side that takes 8 such seeds). Converged beliefs agree within 10 eps
per incoming message (both are eps fixed points of the same map and a belief
combines up to d_max = 4 incoming messages, so the bound is 4 * 10 eps).
Rounds: LBP is deterministic, so every seed's round count agrees within 10%;
the frontier schedules (RnBP's eps filter and random draws, RBP/RS ties and
top-k) follow a different frontier sequence after the first FP32-vs-FP64
threshold flip, which on a marginal seed moves its convergence time a lot, so
for them the median round count agrees within 10% (the share of seeds within
10% each and the mean log ratio of the round counts are printed: 0.5 to 0.9
of the seeds; a single marginal seed, 1448 against 374 rounds, moves the mean
log ratio of 8 seeds by 0.17). The per-seed statement holds exactly for FP64
messages: there GPU and oracle select the same frontiers every round, so
converged flags and round counts are identical on all 50 seeds."""
import multiprocessing as mp

import numpy as np
import pytest

from paper_1909_11469_gb300 import bp, synth
from tests._stats import mcnemar_exact

pytestmark = pytest.mark.gpu

EPS = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _oracle_one(args):
    side, beta_max, seed, gid, sched, par, cap = args
    import oracle
    prob = synth.ising_grid(side, beta_max, seed)
    r = oracle.run(prob, sched, parallelism=par, eps=EPS, max_rounds=cap, seed=0, graph_id=gid)
    return r["converged"], r["rounds"], r["beliefs"]


def _compare(side, beta_max, sched, par, cap, n_seeds=50):
    batch = synth.ising_grid_batch(side, beta_max, range(n_seeds))
    with bp.Graph(batch) as g:
        g.run(sched, par, eps=EPS, max_rounds=cap, msg_dtype="f32", seed=0)
        gst = g.graph_stats()
        bel = g.beliefs()
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, mp.cpu_count())) as pool:
        ref = pool.map(_oracle_one, [(side, beta_max, s, s, sched, par, cap) for s in range(n_seeds)])
    conv_g = np.array([x["converged"] for x in gst], bool)
    conv_o = np.array([r[0] for r in ref], bool)
    if sched == "rnbp":
        b = int((conv_g & ~conv_o).sum())
        c = int((conv_o & ~conv_g).sum())
        pv = mcnemar_exact(b, c)
        print(f"\n  converged on the GPU only: {b}, on the oracle only: {c} (exact McNemar p = {pv:.3f})")
        assert pv >= 0.01, (b, c, pv)
    else:
        assert abs(int(conv_g.sum()) - int(conv_o.sum())) <= 1, (conv_g.sum(), conv_o.sum())
    both = [s for s in range(n_seeds) if conv_g[s] and conv_o[s]]
    rg = np.array([gst[s]["rounds"] for s in both], float)
    ro = np.array([ref[s][1] for s in both], float)
    close = np.abs(rg - ro) <= np.maximum(1, 0.1 * ro)
    worst = 0.0
    for s in both:
        v0, v1 = batch.graph_var_offsets[s], batch.graph_var_offsets[s + 1]
        err = float(np.abs(bel[v0:v1] - ref[s][2]).max())
        worst = max(worst, err)
        assert err < 4 * 10 * EPS, (s, err)
    off = [(s, int(a), int(b)) for s, a, b, c in zip(both, rg, ro, close) if not c]
    flips = [s for s in range(n_seeds) if conv_g[s] != conv_o[s]]
    print(f"\n  seeds outside 10% (seed, GPU rounds, oracle rounds): {off}; converged on one side only: {flips}; "
          f"max belief difference on seeds converged on both sides: {worst:.2e}")
    if both:
        if sched == "lbp":
            assert close.all(), list(zip(both, rg, ro))
        else:
            assert abs(np.median(rg) - np.median(ro)) <= max(1, 0.1 * np.median(ro)), (np.median(rg), np.median(ro))
            bias = float(np.mean(np.log(np.maximum(rg, 1) / np.maximum(ro, 1))))
            print(f"  seeds within 10%: {close.mean():.2f}, mean log round ratio {bias:+.3f}")
    return conv_g.mean(), conv_o.mean(), (float(np.median(rg)) if both else None), \
        (float(np.median(ro)) if both else None), (float(close.mean()) if both else None), len(both)


@pytest.mark.parametrize("beta_max", [1.0, 2.5])
@pytest.mark.parametrize("sched,par,cap", [("lbp", 1.0, 1000), ("rnbp", 0.5, 2000)])
def test_statistics_100x100(beta_max, sched, par, cap):
    """At beta <= 2.5 (the configuration's couplings, C = 5 in the paper's
    terms) no seed converges within the caps on either side; the test then
    checks only that both sides agree on that (the printed line says so)."""
    fg, fo, mg, mo, cl, nb = _compare(100, beta_max, sched, par, cap)
    print(f"100x100 beta<={beta_max} {sched}: converged GPU {fg:.2f} oracle {fo:.2f}, "
          f"median rounds {mg} / {mo}, seeds within 10%: {cl}"
          + ("" if nb else " (no seed converged on either side within the cap)"))
    if beta_max <= 1.0:
        assert nb > 0


# The paper's Ising sets use C = 2.5 (beta = lambda C, lambda ~ U[-0.5, 0.5], so
# |beta| <= 1.25): at that coupling the 100x100 seeds converge (all of them
# under RnBP at LowP 0.1 and 0.5, some under LBP, RBP and RS), so rounds and
# beliefs are compared on a non-empty set of seeds.
PAPER_C_BETA = 1.25


@pytest.mark.parametrize("sched,par,cap,n_seeds", [
    ("lbp", 1.0, 1000, 50), ("rnbp", 0.1, 10000, 50), ("rnbp", 0.5, 2000, 50), ("rnbp", 0.9, 1112, 50),
    ("rbp", 0.1, 10000, 16), ("rs", 0.1, 10000, 16)])
def test_statistics_100x100_paper_c(sched, par, cap, n_seeds):
    """100x100, beta ~ U[-1.25, 1.25]: RnBP at LowP 0.1, 0.5, 0.9, LBP, RBP and RS
    at p = 0.1 (16 seeds: a non-converging seed costs the FP64 oracle its full
    cap of rounds, each a full evaluation of 39,600 messages)."""
    fg, fo, mg, mo, cl, nb = _compare(100, PAPER_C_BETA, sched, par, cap, n_seeds)
    print(f"100x100 beta<={PAPER_C_BETA} {sched} p={par}: converged GPU {fg:.2f} oracle {fo:.2f}, "
          f"median rounds {mg} / {mo}, seeds within 10%: {cl}, converged on both sides: {nb}")
    if sched in ("rbp", "rs") and nb == 0:
        # about one seed in six converges within the cap at p = 0.1; when none of
        # the 16 does, both sides agree on that and the line above records it
        assert fg == 0 and fo == 0
    else:
        assert nb > 0


@pytest.mark.parametrize("sched,par,cap", [("rbp", 1e-2, 20000), ("rs", 1e-2, 20000),
                                           ("rbp", 1e-3, 40000), ("rs", 1e-3, 40000)])
def test_statistics_small_p(sched, par, cap):
    """RBP and RS at p = 1e-2 and 1e-3 (the configuration's lower parallelism
    settings), 50 seeds at the paper's coupling. On 100x100 these need 10^4 to
    10^5 rounds per seed, each a full FP64 evaluation of 39,600 messages in the
    oracle (~6 ms), beyond a test's time; a 30x30 grid (3,480 messages, at
    least ceil(p M) = 4 per round) converges on every seed."""
    fg, fo, mg, mo, cl, nb = _compare(30, PAPER_C_BETA, sched, par, cap)
    print(f"30x30 beta<={PAPER_C_BETA} {sched} p={par}: converged GPU {fg:.2f} oracle {fo:.2f}, "
          f"median rounds {mg} / {mo}, seeds within 10%: {cl}, converged on both sides: {nb}")
    assert nb > 0


@pytest.mark.parametrize("sched,par,cap", [("rbp", 0.1, 10000), ("rs", 0.1, 10000), ("rnbp", 0.1, 10000)])
def test_statistics_10x10(sched, par, cap):
    fg, fo, mg, mo, cl, nb = _compare(10, 2.0, sched, par, cap)
    print(f"10x10 beta<=2 {sched}: converged GPU {fg:.2f} oracle {fo:.2f}, "
          f"median rounds {mg} / {mo}, seeds within 10%: {cl}")


@pytest.mark.parametrize("sched,par,cap", [("lbp", 1.0, 1000), ("rnbp", 0.5, 2000), ("rbp", 0.1, 10000),
                                           ("rs", 0.1, 10000)])
def test_statistics_10x10_fp64_per_seed(sched, par, cap):
    """FP64 messages: 50 seeds, converged flag and rounds identical per seed."""
    n_seeds = 50
    batch = synth.ising_grid_batch(10, 2.0, range(n_seeds))
    with bp.Graph(batch) as g:
        g.run(sched, par, eps=EPS, max_rounds=cap, msg_dtype="f64", seed=0)
        gst = g.graph_stats()
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, mp.cpu_count())) as pool:
        ref = pool.map(_oracle_one, [(10, 2.0, s, s, sched, par, cap) for s in range(n_seeds)])
    got = [(bool(x["converged"]), int(x["rounds"])) for x in gst]
    want = [(bool(r[0]), int(r[1])) for r in ref]
    assert got == want
    print(f"10x10 beta<=2 {sched} FP64: converged {sum(c for c, _ in got)}/50 on both sides, rounds identical")
