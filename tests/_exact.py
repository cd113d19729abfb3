"""Independent reference computations used to pin the oracle (no oracle code).

Everything here is written directly from textbook definitions:
  * brute-force enumeration of the joint of Eq. 1 (exact marginals, tiny graphs);
  * forward-backward on a chain (exact marginals of a chain MRF);
  * a direct NumPy transcription of Eq. 2 for one message;
  * the closed form of the binary Ising message in half-log-odds;
  * serial residual BP with a binary heap (Section III-B describes the serial
    comparator as RBP driven by a priority queue).
"""
from __future__ import annotations

import heapq
import itertools

import numpy as np

from paper_1909_11469_gb300.synth import PAIR_ISING_BETA, PAIR_SHARED, PAIR_TABLE


def pair_table(prob, e: int) -> np.ndarray:
    """theta_ij(x_src, x_dst) as a [k, k] float64 array for directed edge e."""
    k = prob.k
    if prob.pair_kind == PAIR_ISING_BETA:
        s = np.array([-1.0, 1.0])
        return float(prob.pair_log[e]) * np.outer(s, s)
    if prob.pair_kind == PAIR_TABLE:
        return prob.pair_log[e * k * k:(e + 1) * k * k].astype(np.float64).reshape(k, k)
    return prob.pair_log.astype(np.float64).reshape(k, k)


def src_of(prob) -> np.ndarray:
    return np.repeat(np.arange(prob.n), np.diff(prob.row_ptr))


def brute_force_marginals(prob) -> np.ndarray:
    """Exact marginals by enumerating all k^n assignments (tiny graphs only)."""
    n, k = prob.n, prob.k
    assert k ** n <= 2 ** 21
    X = np.array(list(itertools.product(range(k), repeat=n)), dtype=np.int64)
    unary = prob.unary_log.astype(np.float64).reshape(n, k)
    logp = unary[np.arange(n)[None, :], X].sum(axis=1)
    src = src_of(prob)
    for e in range(prob.m):
        i, j = int(src[e]), int(prob.col[e])
        if i < j:
            logp += pair_table(prob, e)[X[:, i], X[:, j]]
    p = np.exp(logp - logp.max())
    p /= p.sum()
    out = np.zeros((n, k))
    for i in range(n):
        for a in range(k):
            out[i, a] = p[X[:, i] == a].sum()
    return out


def chain_marginals(prob) -> np.ndarray:
    """Forward-backward (log domain) on a chain 0 - 1 - ... - (n-1)."""
    n, k = prob.n, prob.k
    unary = prob.unary_log.astype(np.float64).reshape(n, k)
    # pairwise table between i and i+1, oriented (x_i, x_{i+1})
    src = src_of(prob)
    pairs = []
    for i in range(n - 1):
        e = [e for e in range(prob.row_ptr[i], prob.row_ptr[i + 1]) if prob.col[e] == i + 1][0]
        assert src[e] == i
        pairs.append(pair_table(prob, e))

    def lse(a, axis):
        m = a.max(axis=axis, keepdims=True)
        return (m + np.log(np.exp(a - m).sum(axis=axis, keepdims=True))).squeeze(axis)

    fwd = np.zeros((n, k))
    bwd = np.zeros((n, k))
    for i in range(1, n):
        fwd[i] = lse((fwd[i - 1] + unary[i - 1])[:, None] + pairs[i - 1], axis=0)
    for i in range(n - 2, -1, -1):
        bwd[i] = lse(pairs[i] + (bwd[i + 1] + unary[i + 1])[None, :], axis=1)
    lm = fwd + bwd + unary
    lm -= lm.max(axis=1, keepdims=True)
    pm = np.exp(lm)
    return pm / pm.sum(axis=1, keepdims=True)


def message_eq2(prob, msg: np.ndarray, e: int) -> np.ndarray:
    """Eq. 2 for directed edge e from messages msg [M, k] (probability domain)."""
    k = prob.k
    i = int(src_of(prob)[e])
    w = np.exp(prob.unary_log.astype(np.float64).reshape(prob.n, k)[i])
    for f in range(prob.row_ptr[i], prob.row_ptr[i + 1]):
        if f != e:
            w = w * msg[prob.rev[f]]
    c = np.exp(pair_table(prob, e)).T @ w
    return c / c.sum()


def ising_closed_form(prob, msg: np.ndarray, e: int) -> float:
    """Half-log-odds of the new binary message: atanh(tanh(beta) tanh(lambda_i + sum u))
    where lambda_i and u are half-log-odds of the unary and of the incoming messages."""
    i = int(src_of(prob)[e])
    un = prob.unary_log.astype(np.float64).reshape(prob.n, 2)[i]
    field = 0.5 * (un[1] - un[0])
    for f in range(prob.row_ptr[i], prob.row_ptr[i + 1]):
        if f != e:
            mm = msg[prob.rev[f]]
            field += 0.5 * np.log(mm[1] / mm[0])
    return float(np.arctanh(np.tanh(float(prob.pair_log[e])) * np.tanh(field)))


def beliefs_eq3(prob, msg: np.ndarray) -> np.ndarray:
    k = prob.k
    out = np.exp(prob.unary_log.astype(np.float64).reshape(prob.n, k))
    for i in range(prob.n):
        for f in range(prob.row_ptr[i], prob.row_ptr[i + 1]):
            out[i] *= msg[prob.rev[f]]
    return out / out.sum(axis=1, keepdims=True)


def serial_rbp(prob, eps: float, max_updates: int):
    """Serial residual BP: one message per step, always the largest residual
    (ties to the smaller id), residuals of the messages it feeds re-evaluated
    after each update. Returns (updates, converged, messages)."""
    m, k = prob.m, prob.k
    src = src_of(prob)
    msg = np.full((m, k), 1.0 / k)
    cand = np.array([message_eq2(prob, msg, e) for e in range(m)])
    res = np.abs(cand - msg).max(axis=1)
    version = np.zeros(m, dtype=np.int64)
    heap = [(-res[e], e, 0) for e in range(m)]
    heapq.heapify(heap)
    updates = 0
    while True:
        while heap and heap[0][2] != version[heap[0][1]]:
            heapq.heappop(heap)
        if not heap or -heap[0][0] < eps:
            return updates, True, msg
        if updates == max_updates:
            return updates, False, msg
        _, e, _ = heapq.heappop(heap)
        msg[e] = cand[e]
        updates += 1
        j = int(prob.col[e])
        dirty = [e] + [f for f in range(prob.row_ptr[j], prob.row_ptr[j + 1])
                       if f != prob.rev[e]]
        for f in dirty:
            cand[f] = message_eq2(prob, msg, f)
            res[f] = np.abs(cand[f] - msg[f]).max()
            version[f] += 1
            heapq.heappush(heap, (-res[f], f, int(version[f])))
        assert int(src[e]) >= 0


def grid_marginals(prob, rows: int, cols: int) -> np.ndarray:
    """Exact marginals of a binary rows x cols grid MRF (vertex r * cols + c)
    by row transfer matrices: a row's 2^cols joint states carry the row's
    unary and horizontal factors; the vertical factors between rows r and r+1
    form a 2^cols x 2^cols matrix; a forward and a backward pass over the rows
    (each step renormalised) give every row's joint distribution, summed to
    vertex marginals. Exact for any coupling; cols <= 12."""
    assert prob.k == 2 and prob.n == rows * cols and cols <= 12
    S = 1 << cols
    bits = ((np.arange(S)[:, None] >> np.arange(cols)[None, :]) & 1).astype(np.int64)   # [S, cols]
    unary = prob.unary_log.astype(np.float64).reshape(prob.n, 2)
    src = src_of(prob)
    horiz = {}
    vert = {}
    for e in range(prob.m):
        i, j = int(src[e]), int(prob.col[e])
        if i >= j:
            continue
        th = pair_table(prob, e)
        if j == i + 1 and i // cols == j // cols:
            horiz[i] = th
        elif j == i + cols:
            vert[i] = th
        else:
            raise ValueError("not a 4-neighbour grid")
    row_log = np.zeros((rows, S))
    for r in range(rows):
        for c in range(cols):
            v = r * cols + c
            row_log[r] += unary[v][bits[:, c]]
            if c + 1 < cols:
                row_log[r] += horiz[v][bits[:, c], bits[:, c + 1]]
    trans = []
    for r in range(rows - 1):
        lt = np.zeros((S, S))
        for c in range(cols):
            v = r * cols + c
            lt += vert[v][bits[:, c][:, None], bits[:, c][None, :]]
        trans.append(np.exp(lt - lt.max()))
    row_pot = np.exp(row_log - row_log.max(axis=1, keepdims=True))
    fwd = np.zeros((rows, S))
    bwd = np.ones((rows, S))
    a = row_pot[0]
    fwd[0] = a / a.sum()
    for r in range(1, rows):
        a = (fwd[r - 1] @ trans[r - 1]) * row_pot[r]
        fwd[r] = a / a.sum()
    for r in range(rows - 2, -1, -1):
        b = trans[r] @ (row_pot[r + 1] * bwd[r + 1])
        bwd[r] = b / b.sum()
    out = np.zeros((prob.n, 2))
    for r in range(rows):
        joint = fwd[r] * bwd[r]
        joint /= joint.sum()
        for c in range(cols):
            p1 = joint[bits[:, c] == 1].sum()
            out[r * cols + c] = (1.0 - p1, p1)
    return out


def kl_divergence(p: np.ndarray, q: np.ndarray) -> np.ndarray:
    """KL(p || q) of each row of two [n, k] distribution arrays."""
    p = np.asarray(p, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(p > 0, p * (np.log(p) - np.log(q)), 0.0)
    return t.sum(axis=1)
