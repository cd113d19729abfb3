"""Thin ctypes binding of libbp_gb300 (include/bp_gb300.h).

Functions carry the C names and only marshal arguments: NumPy arrays (or
pinned torch CPU tensors) become host pointers, results are copied into
caller-provided or freshly allocated NumPy arrays. Every step of belief
propagation runs in the CUDA library; there is no fallback path. If the
library is missing the first call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libbp_gb300.so")

BP_OK = 0
BP_ERR_INVALID_ARG = -1
BP_ERR_BAD_GRAPH = -2
BP_ERR_NO_POTENTIALS = -3
BP_ERR_NONFINITE = -4
BP_ERR_CUDA = -5
BP_ERR_TIMEOUT = -6
BP_ERR_OOM = -7
BP_ERR_UNSUPPORTED = -8
BP_ERR_NO_RESULT = -9
BP_ERR_INTERNAL = -10

BP_LBP, BP_RBP, BP_RS, BP_RNBP = 0, 1, 2, 3
SCHEDULES = {"lbp": BP_LBP, "rbp": BP_RBP, "rs": BP_RS, "rnbp": BP_RNBP}
BP_F64, BP_F32, BP_BF16, BP_Q16 = 0, 1, 2, 3
DTYPES = {"f64": BP_F64, "f32": BP_F32, "bf16": BP_BF16, "q16": BP_Q16}

BP_PAIR_ISING_BETA, BP_PAIR_TABLE, BP_PAIR_SHARED = 0, 1, 2


class bp_run_stats(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("committed_updates", ctypes.c_int64), ("candidate_evals", ctypes.c_int64),
                ("final_max_residual", ctypes.c_double), ("final_unconverged", ctypes.c_int64),
                ("status", ctypes.c_int32), ("n_graphs", ctypes.c_int32),
                ("device_ms", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class bp_options(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("high_p", ctypes.c_double),
                ("ratio_threshold", ctypes.c_double), ("splash_depth", ctypes.c_int32),
                ("rs_roots_mode", ctypes.c_int32), ("msg_dtype", ctypes.c_int32),
                ("record_trace", ctypes.c_int32), ("trace_capacity", ctypes.c_int32),
                ("rounds_per_launch", ctypes.c_int32), ("cuda_stream", ctypes.c_void_p),
                ("time_budget_ms", ctypes.c_double), ("graph_id_base", ctypes.c_uint32),
                ("kernel_variant", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("potts_path", ctypes.c_int32), ("select_path", ctypes.c_int32),
                ("splash_sweep", ctypes.c_int32), ("overlap_launches", ctypes.c_int32),
                ("dynamic_p", ctypes.c_int32)]


class bp_profile(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("eval_launches", ctypes.c_int64),
                ("full_evals", ctypes.c_int64), ("active_vertices", ctypes.c_int64),
                ("eval_ms", ctypes.c_double), ("decide_ms", ctypes.c_double),
                ("frontier_ms", ctypes.c_double), ("batch_kernel_ms", ctypes.c_double),
                ("select_ms", ctypes.c_double), ("sweep_ms", ctypes.c_double),
                ("sweep_launches", ctypes.c_int64), ("select_ctas", ctypes.c_int32 * 2),
                ("kernel_variant", ctypes.c_int32), ("sweep_ctas", ctypes.c_int32),
                ("sweep_form", ctypes.c_int32), ("overlap_launches", ctypes.c_int32),
                ("fused_commit", ctypes.c_int32)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["select_ctas"] = list(self.select_ctas)
        return d


class bp_tune_result(ctypes.Structure):
    _fields_ = [("kernel_variant", ctypes.c_int32), ("size_class", ctypes.c_int32),
                ("ms_per_round", ctypes.c_double * 8), ("select_path", ctypes.c_int32),
                ("ms_per_round_select", ctypes.c_double * 3)]

    def as_dict(self):
        return {"kernel_variant": self.kernel_variant, "size_class": self.size_class,
                "ms_per_round": list(self.ms_per_round), "select_path": self.select_path,
                "ms_per_round_select": list(self.ms_per_round_select)}


_P = ctypes.c_void_p
_SIGNATURES = {
    "bp_default_options": (None, [_P]),
    "bp_create_graph": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _P, _P, _P, _P]),
    "bp_create_batch": (ctypes.c_int, [ctypes.c_int32, _P, ctypes.c_int32, ctypes.c_int64, _P, _P, _P, _P]),
    "bp_set_potentials": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P]),
    "bp_run": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int32, _P, _P]),
    "bp_get_beliefs": (ctypes.c_int, [_P, _P]),
    "bp_get_messages": (ctypes.c_int, [_P, _P]),
    "bp_get_graph_stats": (ctypes.c_int, [_P, _P]),
    "bp_get_residuals": (ctypes.c_int, [_P, _P]),
    "bp_get_trace": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P]),
    "bp_get_profile": (ctypes.c_int, [_P, _P]),
    "bp_autotune": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double, ctypes.c_double, _P, ctypes.c_int32,
                                   _P]),
    "bp_set_graph_parallelism": (ctypes.c_int, [_P, _P]),
    "bp_time_update": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double, _P, ctypes.c_int32, _P]),
    "bp_autotune_parallelism": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32, ctypes.c_double,
                                               ctypes.c_int32, _P, _P]),
    "bp_lbp_run_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _P, _P, _P, _P, _P,
                                          ctypes.c_double, ctypes.c_int32, _P, _P, _P, _P]),
    "bp_storage_scale": (ctypes.c_int, [_P, ctypes.c_int32, _P]),
    "bp_graph_info": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "bp_destroy_graph": (None, [_P]),
    "bp_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "bp_last_error": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """The loaded CUDA library. Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class BPError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().bp_last_error().decode(errors="replace")
        super().__init__(f"{where}: {bp_status_string(code)} ({code}): {msg}")
        self.code = code


def _check(code: int, where: str) -> int:
    if code != BP_OK:
        raise BPError(code, where)
    return code


def _ptr(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()   # torch tensor (host memory, contiguous)


def _host(a, dtype):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=dtype)
    return a   # torch CPU tensor, already of the right dtype and contiguous


# ---------------------------------------------------------------- C functions
def bp_status_string(code: int) -> str:
    return lib().bp_status_string(int(code)).decode()


def bp_last_error() -> str:
    return lib().bp_last_error().decode(errors="replace")


def bp_default_options(**overrides) -> bp_options:
    o = bp_options()
    lib().bp_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if k == "msg_dtype" and isinstance(v, str):
            v = DTYPES[v]
        setattr(o, k, v)
    return o


def bp_create_graph(n_vars, n_states, row_ptr, col, rev) -> int:
    rp, c, r = _host(row_ptr, np.int64), _host(col, np.int32), _host(rev, np.int32)
    h = ctypes.c_void_p()
    m = int(c.shape[0]) if hasattr(c, "shape") else int(c.numel())
    _check(lib().bp_create_graph(int(n_vars), int(n_states), m, _ptr(rp), _ptr(c), _ptr(r),
                                 ctypes.byref(h)), "bp_create_graph")
    return h.value


def bp_create_batch(graph_var_offsets, n_states, row_ptr, col, rev) -> int:
    go = _host(graph_var_offsets, np.int64)
    rp, c, r = _host(row_ptr, np.int64), _host(col, np.int32), _host(rev, np.int32)
    h = ctypes.c_void_p()
    _check(lib().bp_create_batch(int(go.shape[0] - 1), _ptr(go), int(n_states), int(c.shape[0]),
                                 _ptr(rp), _ptr(c), _ptr(r), ctypes.byref(h)), "bp_create_batch")
    return h.value


def bp_set_potentials(handle, unary_log, pair_kind, pair_log) -> None:
    u, p = _host(unary_log, np.float32), _host(pair_log, np.float32)
    _check(lib().bp_set_potentials(handle, _ptr(u), int(pair_kind), _ptr(p)), "bp_set_potentials")


def bp_run(handle, schedule, parallelism, eps, max_rounds, options: bp_options | None = None):
    sched = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
    st = bp_run_stats()
    rc = lib().bp_run(handle, sched, float(parallelism), float(eps), int(max_rounds),
                      ctypes.byref(options) if options is not None else None, ctypes.byref(st))
    if rc not in (BP_OK, BP_ERR_TIMEOUT):
        raise BPError(rc, "bp_run")
    return st.as_dict()


def _info(handle):
    n, k, m, G = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
    _check(lib().bp_graph_info(handle, ctypes.byref(n), ctypes.byref(k), ctypes.byref(m),
                               ctypes.byref(G)), "bp_graph_info")
    return n.value, k.value, m.value, G.value


def bp_graph_info(handle):
    return dict(zip(("n_vars", "n_states", "n_dir_edges", "n_graphs"), _info(handle)))


def bp_get_beliefs(handle, out=None) -> np.ndarray:
    n, k, _, _ = _info(handle)
    if out is None:
        out = np.empty((n, k), dtype=np.float64)
    _check(lib().bp_get_beliefs(handle, _ptr(out)), "bp_get_beliefs")
    return out


def bp_get_messages(handle) -> np.ndarray:
    _, k, m, _ = _info(handle)
    out = np.empty((m, k), dtype=np.float64)
    _check(lib().bp_get_messages(handle, _ptr(out)), "bp_get_messages")
    return out


def bp_get_graph_stats(handle) -> list[dict]:
    _, _, _, G = _info(handle)
    arr = (bp_run_stats * G)()
    _check(lib().bp_get_graph_stats(handle, ctypes.cast(arr, ctypes.c_void_p)), "bp_get_graph_stats")
    return [a.as_dict() for a in arr]


def bp_get_trace(handle, count: int) -> np.ndarray:
    """Recorded frontiers as a [rounds, ceil(count/32)] uint32 array (count = M, or n for RS)."""
    rounds = ctypes.c_int32()
    words = (count + 31) // 32
    # A NULL buffer reports the recorded round count (and fails as too small
    # when there is something to copy).
    rc = lib().bp_get_trace(handle, None, 0, ctypes.byref(rounds))
    if rc not in (BP_OK, BP_ERR_INVALID_ARG):
        raise BPError(rc, "bp_get_trace")
    if rounds.value == 0:
        return np.zeros((0, words), dtype=np.uint32)
    cap = rounds.value * words
    out = np.zeros(cap, dtype=np.uint32)
    _check(lib().bp_get_trace(handle, _ptr(out), cap, ctypes.byref(rounds)), "bp_get_trace")
    return out.reshape(rounds.value, words)


def bp_get_residuals(handle) -> np.ndarray:
    m = _info(handle)[2]
    out = np.empty(m, dtype=np.float64)
    _check(lib().bp_get_residuals(handle, _ptr(out)), "bp_get_residuals")
    return out


def bp_get_profile(handle) -> dict:
    p = bp_profile()
    _check(lib().bp_get_profile(handle, ctypes.byref(p)), "bp_get_profile")
    return p.as_dict()


def bp_autotune(handle, schedule, parallelism, eps, options: bp_options | None = None,
                trial_rounds: int = 16) -> dict:
    sched = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
    r = bp_tune_result()
    _check(lib().bp_autotune(handle, sched, float(parallelism), float(eps),
                             ctypes.byref(options) if options is not None else None, int(trial_rounds),
                             ctypes.byref(r)), "bp_autotune")
    return r.as_dict()


def bp_time_update(handle, schedule, parallelism, options: bp_options | None = None, launches: int = 20) -> float:
    """Mean device ms of the update kernel over back-to-back launches."""
    sched = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
    ms = ctypes.c_double()
    _check(lib().bp_time_update(handle, sched, float(parallelism),
                                ctypes.byref(options) if options is not None else None, int(launches),
                                ctypes.byref(ms)), "bp_time_update")
    return ms.value


def bp_set_graph_parallelism(handle, p) -> None:
    arr = None if p is None else np.ascontiguousarray(p, dtype=np.float64)
    _check(lib().bp_set_graph_parallelism(handle, _ptr(arr)), "bp_set_graph_parallelism")


def bp_autotune_parallelism(handle, schedule, candidates, eps, max_rounds, options: bp_options | None = None):
    """Returns the chosen parallelism of every graph (float64 [n_graphs])."""
    sched = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
    cand = np.ascontiguousarray(candidates, dtype=np.float64)
    G = _info(handle)[3]
    out = np.empty(G, dtype=np.float64)
    _check(lib().bp_autotune_parallelism(handle, sched, _ptr(cand), int(len(cand)), float(eps), int(max_rounds),
                                         ctypes.byref(options) if options is not None else None, _ptr(out)),
           "bp_autotune_parallelism")
    return out


def bp_lbp_run_noalloc(n_vars, n_dir_edges, row_ptr, col, rev, unary_log, beta, eps, max_rounds,
                       beliefs, cuda_stream=None):
    """LBP on one binary Ising graph without any allocation by the library.
    Every array is a CUDA tensor (or a device address) the caller owns: row_ptr
    int32 [n+1], col / rev int32 [M], unary_log float32 [n*2], beta float32 [M],
    beliefs float64 [n*2] (written). Returns (rounds, converged)."""
    def dp(t):
        return t if isinstance(t, int) or t is None else t.data_ptr()
    rounds, conv = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().bp_lbp_run_noalloc(int(n_vars), int(n_dir_edges), dp(row_ptr), dp(col), dp(rev),
                                    dp(unary_log), dp(beta), float(eps), int(max_rounds), dp(beliefs),
                                    ctypes.byref(rounds), ctypes.byref(conv), cuda_stream),
           "bp_lbp_run_noalloc")
    return rounds.value, bool(conv.value)


def bp_storage_scale(handle, msg_dtype) -> float:
    """The scale of a 16-bit format ("q16" or "bf16") on the handle's binary
    Ising potentials."""
    dt = DTYPES[msg_dtype] if isinstance(msg_dtype, str) else int(msg_dtype)
    out = ctypes.c_float()
    _check(lib().bp_storage_scale(handle, dt, ctypes.byref(out)), "bp_storage_scale")
    return float(out.value)


def bp_destroy_graph(handle) -> None:
    if handle:
        lib().bp_destroy_graph(handle)


# ---------------------------------------------------------------- convenience
class Graph:
    """Owns one handle; methods forward to the C functions above."""

    def __init__(self, problem):
        self.problem = problem
        if problem.n_graphs == 1:
            self.handle = bp_create_graph(problem.n, problem.k, problem.row_ptr, problem.col,
                                          problem.rev)
        else:
            self.handle = bp_create_batch(problem.graph_var_offsets, problem.k, problem.row_ptr,
                                          problem.col, problem.rev)
        bp_set_potentials(self.handle, problem.unary_log, problem.pair_kind, problem.pair_log)

    def run(self, schedule="lbp", parallelism=1.0, eps=1e-4, max_rounds=1000, **opts):
        return bp_run(self.handle, schedule, parallelism, eps, max_rounds, bp_default_options(**opts))

    def beliefs(self):
        return bp_get_beliefs(self.handle)

    def messages(self):
        return bp_get_messages(self.handle)

    def graph_stats(self):
        return bp_get_graph_stats(self.handle)

    def storage_scale(self, msg_dtype):
        return bp_storage_scale(self.handle, msg_dtype)

    def profile(self):
        return bp_get_profile(self.handle)

    def residuals(self):
        return bp_get_residuals(self.handle)

    def autotune(self, schedule="lbp", parallelism=1.0, eps=1e-4, trial_rounds=16, **opts):
        return bp_autotune(self.handle, schedule, parallelism, eps, bp_default_options(**opts), trial_rounds)

    def set_graph_parallelism(self, p):
        bp_set_graph_parallelism(self.handle, p)

    def autotune_parallelism(self, schedule, candidates, eps=1e-4, max_rounds=1000, **opts):
        return bp_autotune_parallelism(self.handle, schedule, candidates, eps, max_rounds,
                                       bp_default_options(**opts))

    def trace(self, schedule):
        sched = SCHEDULES[schedule] if isinstance(schedule, str) else schedule
        return bp_get_trace(self.handle, self.problem.n if sched == BP_RS else self.problem.m)

    def close(self):
        bp_destroy_graph(self.handle)
        self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            if getattr(self, "handle", None):
                self.close()
        except Exception:
            pass
