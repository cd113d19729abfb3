#!/usr/bin/env python
"""Benchmark of frontier-scheduled loopy BP on one GB300 (or N, one rank per GPU).

Workload (default): binary Ising grids 100x100, lambda ~ U[-1, 1],
beta ~ U[-2.5, 2.5], 50 seeds held as one batch of 50 independent graphs, FP32
log-domain messages, eps = 1e-4. One step runs the whole hot path once over
the batch: LBP, RnBP (LowP 0.5), RBP (p 0.1) and Residual Splash (p 0.1, h 2),
each to convergence or its round cap (LBP 1000, RnBP ceil(1000/LowP),
RBP/RS ceil(1000/p)), beliefs included.

Metric: committed message updates per second (messages written by frontier
commits) over the timed steps, with the per-schedule converged fraction and
batch time-to-convergence reported beside it. The timed steps replay captured
CUDA graphs (after an untimed setup that tunes the update mapping and the
selection path). One further step of the same workload runs with CUDA events
between the kernels of every round: its phase split picks the dominant kernel
for the roofline; the message-update kernel is also timed alone (back-to-back
launches between two events) for its own roofline. Beside the metric: the
storage formats side by side (1000x1000), time to convergence on a converging
companion batch (100x100 at C = 2.5), per-graph launches against the batch
(ER), the e2e figure through the C ABI with host buffers, and the FP64 CPU
oracle on a bounded sample.

`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload (the method has no other reference implementation).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # the configuration the metric is quoted on: 100x100, beta ~ U[-2.5, 2.5], 50 seeds
    # (update mapping and selection path tuned per schedule in setup)
    # (update mapping and selection path tuned per schedule in setup; beside the
    # metric, time-to-convergence of the same 50-seed batch at the paper's
    # C = 2.5, i.e. beta ~ U[-1.25, 1.25], where the schedules converge, for
    # FP32, BF16 and Q16 storage: ttc_converging)
    "ising100x100_b2.5_50seeds": dict(
        kind="grid_batch", side=100, beta_max=2.5, lam_max=1.0, n_seeds=50, eps=1e-4, dtype="f32",
        schedules=[("lbp", 1.0), ("rnbp", 0.5), ("rbp", 0.1), ("rs", 0.1)], autotune="mapping",
        ttc_beta=1.25),
    # 1000x1000, beta ~ U[-3, 3]: one graph of 4M messages, LBP and RnBP
    # (the same schedules are also run once with BF16 and Q16 storage: dtype_compare)
    "ising1000x1000_b3": dict(
        kind="grid_batch", side=1000, beta_max=3.0, lam_max=1.0, n_seeds=1, eps=1e-4, dtype="f32",
        schedules=[("lbp", 1.0), ("rnbp", 0.5)], dtype_compare=["f32", "bf16", "q16"]),
    # Potts 256x256, k = 32, unary ~ N(0, 1), one shared table I + N(0, 0.3) noise, RnBP 0.5
    "potts256_k32": dict(
        kind="potts", side=256, k=32, eps=1e-4, dtype="f32", schedules=[("rnbp", 0.5)]),
    # 4096 Erdos-Renyi graphs, n log-uniform in [50, 5000], mean degree 4, beta ~ U[-3, 3]
    # (mapping autotuned per size class; RnBP LowP tuned per graph-size class
    # among 0.1 .. 0.9 in setup; per-graph launches timed on a sample of graphs)
    "er4096_b3": dict(
        kind="er_batch", n_graphs=4096, beta_max=3.0, lam_max=1.0, eps=1e-4, dtype="f32",
        schedules=[("rnbp", 0.5), ("lbp", 1.0)], autotune="mapping+p"),
}
DEFAULT_WORKLOAD = "er4096_b3"
L2_FLUSH_BYTES = 512 << 20          # > 126 MB of L2
# Algorithmic bytes of the full-evaluation kernel (binary Ising): per evaluated
# message rev (4), incoming message (s), exp(-2 beta) (4), old message (s), new
# message (s), + residual (4) in the frontier modes, + the second outcome (s)
# of the fused RnBP rounds; per processed vertex row_ptr, unary log-odds and
# graph id (12). s = 4 (FP32) or 2 (BF16, Q16).
MSG_BYTES = {"f32": 4, "bf16": 2, "q16": 2, "f64": 8}
# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
# roofline kernel from one ncu capture on the workload, valid only while the
# kernel is unchanged since the capture (the summaries and commands are in
# profiles/). Captures are cold (ncu flushes the caches), so they bound the warm
# traffic from above. Keys: (workload, storage, update mapping) and (workload,
# storage, sweep form). The 4096-graph ER capture is of an RnBP round with the
# commit fused (the residual and both EdgeRatio outcomes stored: 2/3 of the
# step's update launches); an LBP launch writes 8 B per message less.
NCU_SWEEP_TRAFFIC = {}
NCU_UPDATE_TRAFFIC = {("er4096_b3", "f32", 6): 255.336448e6 + 168.353536e6}
BYTES_PER_VERTEX = 12


def bytes_per_msg(sched: str, dtype: str, k: int = 2, fused: bool = False) -> int:
    """Per evaluated message: rev, incoming message, old message, new message
    (k values each for k-state messages, one log-odds for binary ones), the
    Ising exp(-2 beta) (binary only), + the residual in the frontier modes;
    fused RnBP rounds (commit inside the streamed update) write a second
    outcome of s bytes."""
    s = MSG_BYTES[dtype]
    if k == 2:
        return 8 + 3 * s + (0 if sched == "lbp" else (8 if dtype == "f64" else 4)) + (s if fused else 0)
    return 4 + 3 * k * s + (0 if sched == "lbp" else 4)


def bytes_per_vertex(k: int = 2) -> int:
    """Per processed vertex: row_ptr, graph id, unary (one log-odds, or k logs)."""
    return 12 if k == 2 else 8 + 4 * k


ROUNDS_SCALE = 1.0


def batch_kernel_bytes(sched: str, dtype: str, st: dict, pr: dict) -> float:
    """Algorithmic bytes of the persistent batch kernel for one run: the full
    evaluations (as bytes_per_msg) plus the frontier work: RnBP and RBP read
    every residual once per round (4 B) and copy each committed message (read +
    write, 2 s); RS pulls the incoming residuals of every vertex (rev + residual,
    8 B per message per round) and per splash-updated message reads rev, col,
    the source level, the incoming message and exp(-2 beta) and writes the
    candidate (13 + 2 s B), then commits it (2 s B)."""
    s = MSG_BYTES[dtype]
    b = bytes_per_msg(sched, dtype) * pr["full_evals"] + bytes_per_vertex() * pr["active_vertices"]
    if sched in ("rnbp", "rbp"):
        b += 4 * pr["full_evals"] + 2 * s * st["committed_updates"]
    elif sched == "rs":
        b += 8 * pr["full_evals"] + (13 + 4 * s) * st["committed_updates"]   # 4+4+1+4 + s + s, + 2 s
    return b


def eval_roofline(step, dtype: str, peak: float, peak_src: str, k: int = 2, kernel: str = "",
                  isolated=None, n: int = 0, m: int = 0):
    """Roofline of the per-round message-update kernel. achieved = algorithmic
    bytes / device time. With isolated = {schedule: ms per launch} (the kernel
    timed alone by bp_time_update: back-to-back launches between two CUDA
    events, every graph running) the time is the kernel's own, weighted by the
    profiled step's launches of each schedule; the profiled step's per-phase
    events (a pair around every directly launched update, so launch overhead
    included) give the in_step figure beside it."""
    alg_bytes, eval_ms, eval_launches = 0.0, 0.0, 0
    phase = {"eval_ms": 0.0, "decide_ms": 0.0, "frontier_ms": 0.0}
    for sched, p, st, pr, gst in step:
        fused = bool(pr.get("fused_commit", 0))
        alg_bytes += (bytes_per_msg(sched, dtype, k, fused) * pr["full_evals"]
                      + bytes_per_vertex(k) * pr["active_vertices"])
        eval_ms += pr["eval_ms"]
        eval_launches += pr["eval_launches"]
        for key in phase:
            phase[key] += pr[key]
    achieved = alg_bytes / (eval_ms / 1e3) / 1e9 if eval_ms > 0 else None
    mappings = sorted({pr.get("kernel_variant", 1) for _, _, _, pr, _ in step})
    names = {1: "k_eval_bin", 3: "k_eval_bin", 4: "k_eval_bin_pf<4 edges>", 6: "k_eval_bin_stream"}
    kname = " / ".join(dict.fromkeys(names.get(v, "k_eval_bin") for v in mappings))
    in_step = {"achieved": achieved, "frac": (achieved / peak) if achieved else None,
               "avg_launch_us": 1e3 * eval_ms / max(eval_launches, 1)}
    out = {"bound": "hbm", "kernel": kernel or f"{kname} ({dtype} messages; Eq. 2 + Eq. 4 + reduction)",
           "achieved": achieved, "peak": peak, "unit": "GB/s", "peak_source": peak_src,
           "frac": (achieved / peak) if achieved else None, "traffic": None,
           "launches": eval_launches, "bytes_per_launch": alg_bytes / max(eval_launches, 1),
           "avg_launch_us": 1e3 * eval_ms / max(eval_launches, 1), "timing": "in-step phase events"}
    if isolated:
        b_tot, t_tot, w_tot = 0.0, 0.0, 0
        for sched, p, st, pr, gst in step:
            if sched not in isolated or pr["eval_launches"] == 0:
                continue
            w = pr["eval_launches"]
            fused = bool(pr.get("fused_commit", 0))
            b_tot += w * (bytes_per_msg(sched, dtype, k, fused) * m + bytes_per_vertex(k) * n)
            t_tot += w * isolated[sched]
            w_tot += w
        if t_tot > 0:
            a = b_tot / (t_tot / 1e3) / 1e9
            out.update({"achieved": a, "frac": a / peak, "bytes_per_launch": b_tot / w_tot,
                        "avg_launch_us": 1e3 * t_tot / w_tot,
                        "timing": "kernel alone: back-to-back launches between CUDA events (bp_time_update)",
                        "in_step": in_step})
    return (out, phase)


def sweep_roofline(step, dtype: str, n: int, m: int, peak: float, peak_src: str):
    """Roofline of the Residual Splash sweep kernel k_splash_list_step (one
    launch per sub-step) from a profiled step. The sweeps run over per-level vertex lists: per evaluated
    message rev, col, the source's level, the incoming message, exp(-2 beta) and
    the written candidate (13 + 2 s B), per evaluated vertex its list entry,
    row_ptr and unary log-odds (16 B, spread over its d-bar out-messages); per
    committed message a read and a write of s bytes, per committed vertex its
    list entry and row_ptr (12 B). Every evaluated message is committed once."""
    s = MSG_BYTES[dtype]
    dbar = m / max(n, 1)
    b, ms, launches = 0.0, 0.0, 0
    for sched, p, st, pr, gst in step:
        if sched != "rs" or pr["sweep_launches"] == 0:
            continue
        upd = st["committed_updates"]
        b += upd * (13 + 2 * s + 16 / dbar) + upd * (2 * s + 12 / dbar)
        ms += pr["sweep_ms"]
        launches += pr["sweep_launches"]
    if ms <= 0:
        return None
    a = b / (ms / 1e3) / 1e9
    name = (f"k_splash_list_step ({dtype} messages; Residual Splash sweep over level lists: commit of one "
            "level fused with the evaluation of the next)")
    return {"bound": "hbm", "kernel": name, "sweep_form": "per_sub_step",
            "achieved": a,
            "peak": peak, "unit": "GB/s", "peak_source": peak_src, "frac": a / peak, "traffic": None,
            "launches": launches, "bytes_per_launch": b / launches, "avg_launch_us": 1e3 * ms / launches}


def select_roofline(step, dtype: str, n: int, m: int, peak: float, peak_src: str, which: str):
    """Roofline of one frontier kernel from a profiled step (which = "rbp":
    k_select_rbp, "rs": k_select_rs, "rnbp": the RnBP commit kernel, which runs
    only when the round does not commit inside the streamed update). RBP reads
    every residual once per round (4 B), RnBP its eps test (4 B of residual, or
    1/8 B of flag words after the streamed update), and both read and write each
    committed message (2 s B); the RS selection gathers the residuals of every
    vertex's incoming messages (rev 4 + residual 4 B per message) and writes
    the splash levels and level lists (1 + 4 B per vertex)."""
    s = MSG_BYTES[dtype]
    b, ms, launches = 0.0, 0.0, 0
    for sched, p, st, pr, gst in step:
        if sched != which:
            continue
        if sched == "rs":
            b += 8 * pr["full_evals"] + 5 * pr["active_vertices"]
        else:
            per_msg = 0.125 if (sched == "rnbp" and pr.get("kernel_variant", 1) == 6) else 4
            b += per_msg * pr["full_evals"] + 2 * s * st["committed_updates"]
        ms += pr["select_ms"]
        launches += max(pr["eval_launches"] - 1, 0)   # the last evaluation selects nothing
    if ms <= 0 or launches == 0:
        return None
    a = b / (ms / 1e3) / 1e9
    name = {"rbp": "k_select_rbp (cluster radix top-k of the residuals + commit)",
            "rs": "k_select_rs (vertex residuals, cluster top-k roots, BFS levels, level lists)",
            "rnbp": "k_commit_rnbp_pipe / k_commit_rnbp_wt (eps filter + Philox Bernoulli + commit)"}[which]
    return {"bound": "hbm", "kernel": f"{name}, {dtype} messages", "achieved": a, "peak": peak, "unit": "GB/s",
            "peak_source": peak_src, "frac": a / peak, "traffic": None, "launches": launches,
            "bytes_per_launch": b / launches, "avg_launch_us": 1e3 * ms / launches}


def round_cap(sched: str, p: float) -> int:
    """Round caps where the configuration is silent: LBP 1000, RnBP ceil(1000/LowP),
    RBP/RS ceil(1000/p) (about 1000 sweeps' worth of commits). --rounds-scale
    shrinks every cap by the same factor (used for profiler passes only: no graph
    of the default workload converges before its cap, so the kernel mix stays the
    same)."""
    base = 1000 if sched == "lbp" else int(np.ceil(1000.0 / p))
    return max(1, int(round(base * ROUNDS_SCALE)))


def make_batch(wl, rank: int, world: int = 1):
    """This rank's share of the workload and the Philox id of its first graph.
    ER: one batch of n_graphs x world graphs (seed 0) split into contiguous
    ranges balanced by directed edges (about n_graphs per rank: weak scaling),
    each rank keeping the batch-wide graph ids. Grid batches: a disjoint seed
    range per rank."""
    from paper_1909_11469_gb300 import shard, synth
    if wl["kind"] == "er_batch":
        full = synth.er_batch(wl["n_graphs"] * world, seed=0, beta_max=wl["beta_max"], lam_max=wl["lam_max"])
        if world == 1:
            return full, 0
        edges = np.diff(full.row_ptr[full.graph_var_offsets])
        r = shard.balanced_ranges(edges, world)[rank]
        return full.graphs(r.start, r.stop), r.start
    if wl["kind"] == "potts":
        return synth.potts_grid(wl["side"], wl["k"], seed=rank), 0
    seeds = shard.shard_seeds(rank, world, wl["n_seeds"])
    if wl["n_seeds"] == 1:
        return synth.ising_grid(wl["side"], wl["beta_max"], rank, wl["lam_max"]), 0
    batch = synth.ising_grid_batch(wl["side"], wl["beta_max"], seeds, wl["lam_max"])
    return batch, shard.graph_id_base(rank, batch.n_graphs)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        self.gpu = gpu_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle
def oracle_sample(wl, budget_rounds: int, seconds: float, prob=None):
    """The FP64 oracle, single thread, on a bounded sample of the workload,
    each schedule capped at budget_rounds rounds. ER batch: every 16th graph
    of the batch from graph 0 (its batch-wide Philox id), until `seconds` of
    oracle time; grid workloads: seed 0. Returns (committed updates, seconds,
    description)."""
    import oracle
    from paper_1909_11469_gb300 import synth

    def one_graph(g, gid):
        c, t = 0, 0.0
        for sched, p in wl["schedules"]:
            t0 = time.perf_counter()
            r = oracle.run(g, sched, parallelism=p, eps=wl["eps"],
                           max_rounds=min(budget_rounds, round_cap(sched, p)), seed=0, graph_id=gid)
            t += time.perf_counter() - t0
            c += r["committed_updates"]
        return c, t

    if wl["kind"] == "er_batch":
        batch = prob if prob is not None else make_batch(wl, 0, 1)[0]
        committed, t, used = 0, 0.0, 0
        for q in range(0, batch.n_graphs, 16):
            c, dt = one_graph(batch.graph(q), q)
            committed, t, used = committed + c, t + dt, used + 1
            if t >= seconds:
                break
        return committed, t, (f"{used} graphs of the batch (every 16th from graph 0), each schedule capped at "
                              f"{budget_rounds} rounds")
    if wl["kind"] == "potts":
        g = synth.potts_grid(wl["side"], wl["k"], seed=0)
    else:
        g = synth.ising_grid(wl["side"], wl["beta_max"], 0, wl["lam_max"])
    c, t = one_graph(g, 0)
    return c, t, f"seed 0 of the workload, each schedule capped at {budget_rounds} rounds"


def run_reference(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    rounds, seconds = 60, 8.0
    prob = make_batch(wl, 0, 1)[0] if wl["kind"] == "er_batch" else None
    for _ in range(args.warmup):
        oracle_sample(wl, rounds, 1.0, prob)
    committed, secs, desc = 0, 0.0, ""
    for _ in range(args.steps):
        c, t, desc = oracle_sample(wl, rounds, seconds, prob)
        committed += c
        secs += t
    value = committed / secs
    sample = f"{desc}, FP64 oracle, single thread, per step"
    line = {
        "metric": "message updates/sec", "value": value, "unit": "message updates/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample": sample},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": "message updates/s", "cores": 1,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "message updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-profile-step", action="store_true",
                    help="skip the extra step with per-phase CUDA events")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the side measurements (storage formats, converging companion batch, "
                         "per-graph launches), e.g. for profiler passes")
    ap.add_argument("--rounds-scale", type=float, default=1.0,
                    help="scale every round cap (profiler passes only)")
    ap.add_argument("--direct-launch", action="store_true",
                    help="timed steps launch kernels directly instead of replaying CUDA graphs "
                         "(profiler passes only)")
    ap.add_argument("--kernel-variant", type=int, default=0, choices=[0, 1, 3, 4, 6],
                    help="binary update mapping (0 = library's choice)")
    ap.add_argument("--potts-path", type=int, default=0, choices=[0, 1],
                    help="shared-table update: 0 automatic, 1 CUDA cores, 2 tensor cores BF16, "
                         "3 tensor cores split")
    ap.add_argument("--splash-sweep", type=int, default=0, choices=[0, 1],
                    help="Residual Splash sweeps: 0 library's choice, 1 one launch per sub-step")
    ap.add_argument("--overlap-launches", type=int, default=0, choices=[0, 1, 2],
                    help="programmatic dependent launches: 0 library's choice, 1 on, 2 off")
    ap.add_argument("--dtype", default=None, choices=["f32", "bf16", "q16", "f64"],
                    help="message storage (default: the workload's)")
    ap.add_argument("--autotune", default=None, choices=["none", "mapping", "mapping+p"],
                    help="tune the update mapping and selection path (and the RnBP LowP per graph-size "
                         "class) in setup (default: the workload's setting)")
    args = ap.parse_args()
    global ROUNDS_SCALE
    ROUNDS_SCALE = args.rounds_scale
    wl = dict(WORKLOADS[args.workload])
    if args.dtype:
        wl["dtype"] = args.dtype
    if args.impl == "reference":
        return run_reference(args, wl)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    __graft_entry__.build()
    from paper_1909_11469_gb300 import bp

    prob, gid_base = make_batch(wl, rank, world)
    stream = torch.cuda.current_stream()
    g = bp.Graph(prob)
    G = prob.n_graphs
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    from paper_1909_11469_gb300 import shard

    def opts(**kw):
        return bp.bp_default_options(msg_dtype=wl["dtype"], cuda_stream=stream.cuda_stream,
                                     graph_id_base=gid_base,
                                     kernel_variant=args.kernel_variant,
                                     potts_path=args.potts_path, splash_sweep=args.splash_sweep,
                                     overlap_launches=args.overlap_launches, **kw)

    def one_step(profile: int):
        out = []
        for sched, p in wl["schedules"]:
            st = bp.bp_run(g.handle, sched, p, wl["eps"], round_cap(sched, p), opts(profile=profile))
            out.append((sched, p, st, bp.bp_get_profile(g.handle), bp.bp_get_graph_stats(g.handle)))
        return out

    tuning = None
    tune = wl.get("autotune", "none") if args.autotune is None else args.autotune
    if args.kernel_variant != 0:
        tune = "none"
    if tune != "none" and prob.k == 2:
        # setup, untimed: mapping and selection path per schedule (size class of
        # this batch), then (mapping+p) the RnBP LowP per graph-size class
        tuning = {"mapping": {}}
        for sched, p in wl["schedules"]:
            r = bp.bp_autotune(g.handle, sched, p, wl["eps"], opts(), 16)
            tuning["mapping"][sched] = {"kernel_variant": r["kernel_variant"],
                                        "ms_per_round": [round(x, 4) for x in r["ms_per_round"]]}
            if sched in ("rbp", "rs"):
                tuning["mapping"][sched]["select_path"] = r["select_path"]
                tuning["mapping"][sched]["ms_per_round_select"] = [round(x, 4) for x in r["ms_per_round_select"]]
        if tune == "mapping+p" and any(sched == "rnbp" for sched, _ in wl["schedules"]):
            cand = [0.1, 0.3, 0.5, 0.7, 0.9]
            gp = bp.bp_autotune_parallelism(g.handle, "rnbp", cand, wl["eps"], 1000, opts())
            sizes = np.diff(prob.graph_var_offsets)
            cls = np.floor(np.log2(np.maximum(sizes, 1))).astype(int)
            tuning["rnbp_low_p_by_log2_size"] = {int(c): float(gp[np.argmax(cls == c)]) for c in np.unique(cls)}

    for _ in range(max(args.warmup, 0)):
        one_step(0)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    results = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for i in range(args.steps):
        flush.zero_()                     # L2 flush between timed steps (outside the events)
        starts[i].record(stream)
        results.append(one_step(1 if args.direct_launch else 0))
        ends[i].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = float(sum(step_ms))
    committed = sum(st["committed_updates"] for step in results for (_, _, st, _, _) in step)
    evals = sum(st["candidate_evals"] for step in results for (_, _, st, _, _) in step)
    launches = sum(pr["kernel_launches"] for step in results for (_, _, _, pr, _) in step)
    if world > 1:
        total_ms, (committed, evals, launches) = shard.reduce_step_stats(
            dist, "cuda", total_ms, [committed, evals, launches])
    value = committed / (total_ms / 1e3)

    # Roofline. One more step of the same workload with profiling: the
    # persistent batch kernel is timed as a whole; the per-round path times
    # every phase with CUDA events on the launching stream.
    flush.zero_()
    prof_step = [] if args.no_profile_step else one_step(1)
    torch.cuda.synchronize()
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    roofline, update_roofline, phase = None, None, None
    if prof_step and prof_step[0][3]["batch_kernel_ms"] > 0:
        b, ms = 0.0, 0.0
        for sched, p, st, pr, gst in prof_step:
            b += batch_kernel_bytes(sched, wl["dtype"], st, pr)
            ms += pr["batch_kernel_ms"]
        roofline = {"bound": "hbm", "kernel": f"k_persistent ({wl['dtype']} messages; all rounds of every "
                    "graph: Eq. 2 + Eq. 4 update, reduction, frontier)",
                    "achieved": b / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                    "peak_source": peak_src, "frac": b / (ms / 1e3) / 1e9 / peak, "traffic": None,
                    "launches": len(prof_step), "bytes_per_launch": b / len(prof_step),
                    "avg_launch_us": 1e3 * ms / len(prof_step)}
        # the message-update kernel of the per-round path on the same workload
        saved = args.kernel_variant
        args.kernel_variant = 1
        flush.zero_()
        upd_step = one_step(1)
        torch.cuda.synchronize()
        args.kernel_variant = saved
        update_roofline, phase = eval_roofline(upd_step, wl["dtype"], peak, peak_src)
    elif prof_step:
        kname = ""
        if prob.k > 2:
            tc_name = "k_potts_ws" if prob.k == 32 else "k_potts_tc"   # k = 32: warp-specialised form
            kname = {1: "k_potts_tc_pipe (CUDA cores)", 2: f"{tc_name} (tcgen05, BF16 products)",
                     3: f"{tc_name} (tcgen05, split BF16 products)"}.get(
                        args.potts_path or (3 if prob.k >= 16 else 0), "k_eval_gen")
        iso = {}
        for sched, p in wl["schedules"]:
            try:
                iso[sched] = bp.bp_time_update(g.handle, sched, p, opts(), 30)
            except bp.BPError:
                pass
        update_roofline, phase = eval_roofline(prof_step, wl["dtype"], peak, peak_src, prob.k, kname,
                                               isolated=iso, n=prob.n, m=prob.m)
        variants = {pr.get("kernel_variant") for _, _, _, pr, _ in prof_step}
        if prob.k == 2 and len(variants) == 1:
            update_roofline["traffic"] = NCU_UPDATE_TRAFFIC.get((args.workload, wl["dtype"], variants.pop()))
        phase["select_ms"] = sum(pr["select_ms"] for _, _, _, pr, _ in prof_step)
        phase["sweep_ms"] = sum(pr["sweep_ms"] for _, _, _, pr, _ in prof_step)
        # the dominant kernel class of the step gets the roofline
        # the kernel with the largest share of the profiled step gets the roofline
        def sel_ms(which):
            return sum(pr["select_ms"] for sc, _, _, pr, _ in prof_step if sc == which)
        sweep_rf = sweep_roofline(prof_step, wl["dtype"], prob.n, prob.m, peak, peak_src)
        if sweep_rf is not None:
            sweep_rf["traffic"] = NCU_SWEEP_TRAFFIC.get((args.workload, wl["dtype"], sweep_rf["sweep_form"]))
        cands = [(phase["eval_ms"], update_roofline), (phase["sweep_ms"], sweep_rf)]
        for which in ("rbp", "rs", "rnbp"):
            cands.append((sel_ms(which), select_roofline(prof_step, wl["dtype"], prob.n, prob.m, peak, peak_src,
                                                         which)))
        roofline = max((c for c in cands if c[1] is not None), key=lambda c: c[0])[1]
    per_sched = {}
    for step in results:
        for sched, p, st, pr, gst in step:
            key = f"{sched}_p{p}"
            d = per_sched.setdefault(key, {"ms": [], "converged_fraction": None, "median_rounds": None,
                                           "committed_updates": 0})
            d["ms"].append(st["device_ms"])
            d["committed_updates"] += st["committed_updates"]
            d["converged_fraction"] = float(np.mean([x["converged"] for x in gst]))
            d["median_rounds"] = float(np.median([x["rounds"] for x in gst]))
            d["conv_rounds"] = sorted(int(x["rounds"]) for x in gst if x["converged"])
            d["max_rounds"] = int(st["rounds"])
    for d in per_sched.values():
        d["batch_ms"] = float(np.median(d.pop("ms")))
        d["committed_updates"] //= args.steps
        d["graphs_per_s"] = G / (d["batch_ms"] / 1e3)
        # cumulative converged fraction against rounds (the paper's Figs. 2 and
        # 4 plot it against time): [fraction of all graphs converged, rounds,
        # ms at the batch's mean round time]
        cr, rmax = d.pop("conv_rounds"), d.pop("max_rounds")
        ms_round = d["batch_ms"] / max(rmax, 1)
        curve = []
        for q in (0.1, 0.25, 0.5, 0.75, 0.9, 1.0):
            if cr:
                r = cr[max(0, int(np.ceil(q * len(cr))) - 1)]
                curve.append([round(q * len(cr) / G, 4), r, round(r * ms_round, 3)])
        d["convergence_curve"] = curve

    # time-to-convergence on the converging companion batch (same sizes and
    # seeds, milder couplings): batch time until every graph converged or hit
    # its cap, per schedule and storage format
    ttc = None
    if wl.get("ttc_beta") and rank == 0 and not args.no_extras:
        from paper_1909_11469_gb300 import synth
        mild = synth.ising_grid_batch(wl["side"], wl["ttc_beta"], range(wl["n_seeds"]), wl["lam_max"])
        ttc = {"beta_max": wl["ttc_beta"], "graphs": mild.n_graphs}
        with bp.Graph(mild) as h:
            for dt in ("f32", "bf16", "q16"):
                for sched, p in wl["schedules"]:
                    o = bp.bp_default_options(msg_dtype=dt, cuda_stream=stream.cuda_stream)
                    bp.bp_run(h.handle, sched, p, wl["eps"], round_cap(sched, p), o)   # warm-up
                    st = bp.bp_run(h.handle, sched, p, wl["eps"], round_cap(sched, p), o)
                    gst = bp.bp_get_graph_stats(h.handle)
                    conv = [x["rounds"] for x in gst if x["converged"]]
                    ttc[f"{sched}_p{p}_{dt}"] = {
                        "batch_ms": st["device_ms"], "converged_fraction": len(conv) / len(gst),
                        "median_rounds_converged": float(np.median(conv)) if conv else None}

    # storage formats side by side: each schedule once per format, from
    # uniform messages to convergence or the round cap
    dtype_cmp = None
    if wl.get("dtype_compare") and rank == 0 and not args.no_extras:
        dtype_cmp = {}
        for dt in wl["dtype_compare"]:
            for sched, p in wl["schedules"]:
                o = bp.bp_default_options(msg_dtype=dt, cuda_stream=stream.cuda_stream)
                bp.bp_run(g.handle, sched, p, wl["eps"], round_cap(sched, p), o)   # warm-up
                flush.zero_()
                st = bp.bp_run(g.handle, sched, p, wl["eps"], round_cap(sched, p), o)
                gst = bp.bp_get_graph_stats(g.handle)
                dtype_cmp[f"{sched}_p{p}_{dt}"] = {
                    "ms": st["device_ms"], "rounds": st["rounds"],
                    "ms_per_round": st["device_ms"] / max(st["rounds"], 1),
                    "converged_fraction": float(np.mean([x["converged"] for x in gst])),
                    "updates_per_s": st["committed_updates"] / (st["device_ms"] / 1e3)}

    # batches: the same graphs launched one handle per graph, on a sample of
    # 64 graphs spread over the batch (per-graph launches vs the batched run)
    per_graph = None
    if G >= 256 and rank == 0 and not args.no_extras:
        idx = np.linspace(0, G - 1, 64).astype(int)
        tot_ms = {f"{sched}_p{p}": 0.0 for sched, p in wl["schedules"]}
        for q in idx:
            sub = prob.graph(int(q))
            with bp.Graph(sub) as h:
                for sched, p in wl["schedules"]:
                    pq = p
                    if sched == "rnbp" and tuning and "rnbp_low_p_by_log2_size" in tuning:
                        nq = int(prob.graph_var_offsets[q + 1] - prob.graph_var_offsets[q])
                        pq = tuning["rnbp_low_p_by_log2_size"][int(np.floor(np.log2(max(nq, 1))))]
                    o = bp.bp_default_options(msg_dtype=wl["dtype"], cuda_stream=stream.cuda_stream,
                                              graph_id_base=int(q))
                    bp.bp_run(h.handle, sched, pq, wl["eps"], round_cap(sched, p), o)   # warm-up
                    st = bp.bp_run(h.handle, sched, pq, wl["eps"], round_cap(sched, p), o)
                    tot_ms[f"{sched}_p{p}"] += st["device_ms"]
        per_graph = {k: {"graphs_per_s": len(idx) / (v / 1e3), "sample_graphs": len(idx)}
                     for k, v in tot_ms.items()}

    # end to end through the C ABI with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        unary_h = torch.from_numpy(prob.unary_log).pin_memory()
        pair_h = torch.from_numpy(prob.pair_log).pin_memory()
        bel_h = torch.empty((prob.n, prob.k), dtype=torch.float64).pin_memory()
        e2e_committed, e2e_s = 0, 0.0
        for it in range(args.steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            bp.bp_set_potentials(g.handle, unary_h, prob.pair_kind, pair_h)
            c = 0
            for sched, p in wl["schedules"]:
                st = bp.bp_run(g.handle, sched, p, wl["eps"], round_cap(sched, p), opts())
                bp.bp_get_beliefs(g.handle, bel_h)
                c += st["committed_updates"]
            dt = time.perf_counter() - t0
            if it > 0:                      # first pass is a warm-up
                e2e_committed += c
                e2e_s += dt
        e2e = {"value": e2e_committed / e2e_s, "unit": "message updates/s",
               "h2d_bytes_per_step": int(prob.unary_log.nbytes + prob.pair_log.nbytes),
               "d2h_bytes_per_step": int(bel_h.numel() * 8 * len(wl["schedules"]))}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        c, t, desc = oracle_sample(wl, 300, 12.0, prob)
        cpu = {"value": c / t, "unit": "message updates/s", "cores": 1, "kind": "oracle",
               "sample": f"{desc} ({t:.1f} s of FP64 oracle, single thread)"}

    if rank == 0:
        line = {
            "metric": "message updates/sec", "value": value, "unit": "message updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": wl["dtype"], "data": "synthetic",
            "config": {"workload": args.workload, "graphs_per_gpu": G, "autotune": tune,
                       "rounds_scale": args.rounds_scale, "direct_launch": bool(args.direct_launch),
                       "vertices": int(prob.n), "directed_messages": int(prob.m), "states": int(prob.k),
                       "potts_path": args.potts_path, "splash_sweep": args.splash_sweep,
                       "overlap_launches": args.overlap_launches,
                       "eps": wl["eps"], "schedules": [f"{s}:{p}" for s, p in wl["schedules"]],
                       "l2": "flushed between steps (512 MB write)",
                       "parallelism": f"dp{world}" if world > 1 else "single"},
            "candidate_evals_per_s": evals / (total_ms / 1e3),
            "schedules": per_sched,
            "per_graph_launches": per_graph, "tuning": tuning, "dtype_compare": dtype_cmp,
            "ttc_converging": ttc,
            "profiled_step_phase_ms": phase,
            "roofline": roofline, "update_kernel_roofline": update_roofline,
            "e2e": e2e, "cpu_baseline": cpu,
            "gpu_launches": int(launches), "clocks": clk,
        }
        print(json.dumps(line))
    g.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
