"""FP64 CPU oracle for frontier-based loopy belief propagation (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of
the benchmark may import this package; the product path never does. The C
source (bp_oracle.c) is plain FP64 C written from Eq. 1-4 and Algorithm 1 of the
paper; it shares no code with the CUDA library.

Parity status: every oracle function is pinned by a test in tests/test_oracle_pins.py
(brute-force enumeration, tree exactness, the Ising closed form, Philox
known-answer vectors, textbook top-k / BFS, schedule identities).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libbporacle.so")

LBP, RBP, RS, RNBP = 0, 1, 2, 3
SCHEDULES = {"lbp": LBP, "rbp": RBP, "rs": RS, "rnbp": RNBP}
STORAGE = {"f64": 0, "bf16": 1, "q16": 2, "bf16_plain": 3}


class OrcProblem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("k", ctypes.c_int32), ("m", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("rev", ctypes.c_void_p),
                ("unary_log", ctypes.c_void_p), ("pair_kind", ctypes.c_int32),
                ("pair_log", ctypes.c_void_p)]


class OrcParams(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int32), ("parallelism", ctypes.c_double),
                ("eps", ctypes.c_double), ("max_rounds", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("graph_id", ctypes.c_uint32),
                ("high_p", ctypes.c_double), ("ratio_threshold", ctypes.c_double),
                ("splash_depth", ctypes.c_int32), ("rs_roots_mode", ctypes.c_int32),
                ("trace_in", ctypes.c_void_p), ("trace_rounds", ctypes.c_int32),
                ("trace_out", ctypes.c_void_p), ("trace_cap", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("storage_scale", ctypes.c_double),
                ("dynamic_p", ctypes.c_int32)]


class OrcStats(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("committed_updates", ctypes.c_int64), ("candidate_evals", ctypes.c_int64),
                ("final_max_residual", ctypes.c_double), ("final_unconverged", ctypes.c_int64)]


_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile bp_oracle.c into a shared library next to it (plain gcc, -O2)."""
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.orc_run.argtypes = [ctypes.POINTER(OrcProblem), ctypes.POINTER(OrcParams),
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(OrcStats)]
            L.orc_run.restype = ctypes.c_int
            L.orc_evaluate.argtypes = [ctypes.POINTER(OrcProblem), ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]
            L.orc_evaluate.restype = ctypes.c_int
            L.orc_beliefs.argtypes = [ctypes.POINTER(OrcProblem), ctypes.c_void_p, ctypes.c_void_p]
            L.orc_beliefs.restype = ctypes.c_int
            L.orc_splash_levels.argtypes = [ctypes.POINTER(OrcProblem), ctypes.c_void_p,
                                            ctypes.c_int32, ctypes.c_void_p]
            L.orc_splash_levels.restype = ctypes.c_int
            L.orc_top_k.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
            L.orc_top_k.restype = ctypes.c_int
            L.orc_philox4x32_10.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            L.orc_philox4x32_10.restype = None
            L.orc_stored_logodds.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double]
            L.orc_stored_logodds.restype = ctypes.c_double
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class _Bound:
    """Keeps the contiguous arrays alive while the C structure points at them."""

    def __init__(self, prob):
        self.row_ptr = np.ascontiguousarray(prob.row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(prob.col, dtype=np.int32)
        self.rev = np.ascontiguousarray(prob.rev, dtype=np.int32)
        self.unary = np.ascontiguousarray(prob.unary_log, dtype=np.float32)
        self.pair = np.ascontiguousarray(prob.pair_log, dtype=np.float32)
        self.s = OrcProblem(int(prob.n), int(prob.k), int(self.col.shape[0]),
                            _ptr(self.row_ptr), _ptr(self.col), _ptr(self.rev),
                            _ptr(self.unary), int(prob.pair_kind), _ptr(self.pair))


def run(prob, schedule="lbp", parallelism=1.0, eps=1e-4, max_rounds=1000, seed=0,
        graph_id=0, high_p=1.0, ratio_threshold=0.9, splash_depth=2, rs_roots_mode=0,
        trace_in=None, trace_rounds=0, trace_cap=0, storage="f64", storage_scale=0.0, dynamic_p=0):
    """Run one graph (prob must hold a single graph). Returns a dict with beliefs
    [n, k], messages [M, k] (probability domain), stats and the selected trace.
    storage: "f64" (exact), "bf16", "q16" or "bf16_plain" (emulated 16-bit message
    storage; storage_scale is the library's scale of that format, bp_storage_scale)."""
    sched = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
    b = _Bound(prob)
    n, k, m = int(prob.n), int(prob.k), int(b.col.shape[0])
    words = ((n if sched == RS else m) + 31) // 32
    tin = None
    if trace_in is not None:
        tin = np.ascontiguousarray(trace_in, dtype=np.uint32).reshape(-1)
        if tin.shape[0] < trace_rounds * words:
            raise ValueError("trace_in too short")
    tout = np.zeros(max(trace_cap, 0) * words + 1, dtype=np.uint32)
    params = OrcParams(sched, float(parallelism), float(eps), int(max_rounds), int(seed),
                       int(graph_id), float(high_p), float(ratio_threshold), int(splash_depth),
                       int(rs_roots_mode), _ptr(tin) if tin is not None else None,
                       int(trace_rounds), _ptr(tout) if trace_cap > 0 else None, int(trace_cap),
                       STORAGE[storage], float(storage_scale), int(dynamic_p))
    beliefs = np.zeros(n * k + 1, dtype=np.float64)
    msgs = np.zeros(m * k + 1, dtype=np.float64)
    st = OrcStats()
    rc = lib().orc_run(ctypes.byref(b.s), ctypes.byref(params), _ptr(beliefs), _ptr(msgs),
                       ctypes.byref(st))
    if rc != 0:
        raise RuntimeError(f"orc_run failed with {rc}")
    return {
        "beliefs": beliefs[:n * k].reshape(n, k),
        "messages": msgs[:m * k].reshape(m, k),
        "converged": bool(st.converged), "rounds": int(st.rounds),
        "committed_updates": int(st.committed_updates),
        "candidate_evals": int(st.candidate_evals),
        "final_max_residual": float(st.final_max_residual),
        "final_unconverged": int(st.final_unconverged),
        "trace": tout[:max(trace_cap, 0) * words].reshape(max(trace_cap, 0), words),
    }


def evaluate(prob, messages: np.ndarray):
    """Candidates [M, k] and residuals [M] of every message from the given messages."""
    b = _Bound(prob)
    m, k = int(b.col.shape[0]), int(prob.k)
    msg = np.ascontiguousarray(messages, dtype=np.float64).reshape(-1)
    cand = np.zeros(m * k + 1)
    r = np.zeros(m + 1)
    if lib().orc_evaluate(ctypes.byref(b.s), _ptr(msg), _ptr(cand), _ptr(r)) != 0:
        raise RuntimeError("orc_evaluate failed")
    return cand[:m * k].reshape(m, k), r[:m]


def beliefs(prob, messages: np.ndarray):
    b = _Bound(prob)
    n, k = int(prob.n), int(prob.k)
    msg = np.ascontiguousarray(messages, dtype=np.float64).reshape(-1)
    out = np.zeros(n * k + 1)
    if lib().orc_beliefs(ctypes.byref(b.s), _ptr(msg), _ptr(out)) != 0:
        raise RuntimeError("orc_beliefs failed")
    return out[:n * k].reshape(n, k)


def splash_levels(prob, roots: np.ndarray, depth: int):
    b = _Bound(prob)
    root = np.ascontiguousarray(roots, dtype=np.uint8)
    level = np.zeros(int(prob.n) + 1, dtype=np.int32)
    if lib().orc_splash_levels(ctypes.byref(b.s), _ptr(root), int(depth), _ptr(level)) != 0:
        raise RuntimeError("orc_splash_levels failed")
    return level[:int(prob.n)]


def top_k(key: np.ndarray, k: int):
    key = np.ascontiguousarray(key, dtype=np.float64)
    chosen = np.zeros(key.shape[0] + 1, dtype=np.uint8)
    if lib().orc_top_k(_ptr(key), int(key.shape[0]), int(k), _ptr(chosen)) != 0:
        raise RuntimeError("orc_top_k failed")
    return chosen[:key.shape[0]].astype(bool)


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    kk = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(kk), _ptr(out))
    return out


def stored_logodds(storage: str, u: float, scale: float = 0.0) -> float:
    """The value an Ising log-odds u is stored as under the given storage mode."""
    return float(lib().orc_stored_logodds(STORAGE[storage], float(u), float(scale)))


def run_batch(prob, **kw):
    """Run every graph of a batch independently (graph g gets graph_id = g)."""
    res = []
    for g in range(prob.n_graphs):
        res.append(run(prob.graph(g), graph_id=g, **kw))
    return res
