"""Seeded synthetic inputs for loopy belief propagation on pairwise MRFs.

This module builds graph structure (CSR of directed edges with a reverse-edge
index) and draws random log-potentials. It holds none of the BP arithmetic
(no message update, no normalisation, no residual, no selection): both the CUDA
library and the FP64 CPU oracle consume the arrays it returns.

Graph conventions (Section III-B, "adjacency list ... edge and vertex IDs"):
  * directed edge e = (i -> j) lives in CSR row i: row_ptr[i] <= e < row_ptr[i+1],
    col[e] = j; neighbour lists are sorted by vertex id;
  * rev[e] is the id of the opposite directed edge (j -> i);
  * undirected-edge order is CSR order restricted to i < j.

Potential conventions (Eq. 1, stored as natural logs theta = log psi):
  * unary_log  [n, k]  theta_i(x_i)
  * pair kind 0 (Ising): beta per directed edge [M]; theta_ij(x_i, x_j) = beta * s(x_i) s(x_j)
    with spin s(0) = -1, s(1) = +1 (only k = 2);
  * pair kind 1 (table): [M, k, k], entry [e, a, b] = theta_ij(x_i = a, x_j = b) for e = (i -> j);
  * pair kind 2 (shared): one symmetric [k, k] table used on every edge.

Draw order for every generator: unary values in vertex order, then pairwise
values in undirected-edge order, from numpy.random.Generator(PCG64(seed)).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PAIR_ISING_BETA = 0
PAIR_TABLE = 1
PAIR_SHARED = 2


@dataclasses.dataclass
class Problem:
    """One pairwise MRF, or a batch of independent MRFs as one disjoint union."""

    n: int
    k: int
    row_ptr: np.ndarray          # int64 [n+1]
    col: np.ndarray              # int32 [M]
    rev: np.ndarray              # int32 [M]
    unary_log: np.ndarray        # float32 [n*k]
    pair_kind: int
    pair_log: np.ndarray         # float32, layout per pair_kind
    graph_var_offsets: np.ndarray  # int64 [G+1]; one graph -> [0, n]
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.col.shape[0])

    @property
    def n_graphs(self) -> int:
        return int(self.graph_var_offsets.shape[0] - 1)

    def graphs(self, g0: int, g1: int) -> "Problem":
        """Graphs [g0, g1) of a batch as a batch of their own, renumbered from
        vertex 0 and edge 0."""
        v0, v1 = int(self.graph_var_offsets[g0]), int(self.graph_var_offsets[g1])
        e0, e1 = int(self.row_ptr[v0]), int(self.row_ptr[v1])
        k = self.k
        if self.pair_kind == PAIR_ISING_BETA:
            pl = self.pair_log[e0:e1].copy()
        elif self.pair_kind == PAIR_TABLE:
            pl = self.pair_log[e0 * k * k:e1 * k * k].copy()
        else:
            pl = self.pair_log.copy()
        return Problem(
            n=v1 - v0, k=k,
            row_ptr=(self.row_ptr[v0:v1 + 1] - e0).astype(np.int64),
            col=(self.col[e0:e1] - v0).astype(np.int32),
            rev=(self.rev[e0:e1] - e0).astype(np.int32),
            unary_log=self.unary_log[v0 * k:v1 * k].copy(),
            pair_kind=self.pair_kind, pair_log=pl,
            graph_var_offsets=(self.graph_var_offsets[g0:g1 + 1] - v0).astype(np.int64),
            name=f"{self.name}[{g0}:{g1}]")

    def graph(self, g: int) -> "Problem":
        """Graph g of a batch, renumbered from vertex 0 and edge 0."""
        v0, v1 = int(self.graph_var_offsets[g]), int(self.graph_var_offsets[g + 1])
        e0, e1 = int(self.row_ptr[v0]), int(self.row_ptr[v1])
        k = self.k
        if self.pair_kind == PAIR_ISING_BETA:
            pl = self.pair_log[e0:e1].copy()
        elif self.pair_kind == PAIR_TABLE:
            pl = self.pair_log[e0 * k * k:e1 * k * k].copy()
        else:
            pl = self.pair_log.copy()
        return Problem(
            n=v1 - v0, k=k,
            row_ptr=(self.row_ptr[v0:v1 + 1] - e0).astype(np.int64),
            col=(self.col[e0:e1] - v0).astype(np.int32),
            rev=(self.rev[e0:e1] - e0).astype(np.int32),
            unary_log=self.unary_log[v0 * k:v1 * k].copy(),
            pair_kind=self.pair_kind, pair_log=pl,
            graph_var_offsets=np.array([0, v1 - v0], dtype=np.int64),
            name=f"{self.name}[{g}]")


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def csr_from_undirected(n: int, ei: np.ndarray, ej: np.ndarray):
    """CSR (row_ptr, col, rev) of the 2|E| directed edges of an undirected edge list.

    Rows are sorted by destination id. Self-loops and duplicate edges are rejected.
    """
    ei = np.asarray(ei, dtype=np.int64)
    ej = np.asarray(ej, dtype=np.int64)
    if np.any(ei == ej):
        raise ValueError("self-loop in edge list")
    src = np.concatenate([ei, ej])
    dst = np.concatenate([ej, ei])
    key = src * n + dst
    order = np.argsort(key, kind="stable")
    key = key[order]
    if key.size and np.any(key[1:] == key[:-1]):
        raise ValueError("duplicate edge in edge list")
    src = src[order]
    dst = dst[order]
    counts = np.bincount(src, minlength=n) if src.size else np.zeros(n, dtype=np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    rev = np.searchsorted(key, dst * n + src)
    return row_ptr, dst.astype(np.int32), rev.astype(np.int32)


def _undirected_positions(row_ptr: np.ndarray, col: np.ndarray) -> np.ndarray:
    """Directed-edge ids e = (i -> j) with i < j, in CSR order."""
    n = row_ptr.shape[0] - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    return np.nonzero(src < col)[0]


def grid_edges(rows: int, cols: int):
    """4-neighbour grid; vertex id = r * cols + c."""
    idx = np.arange(rows * cols, dtype=np.int64).reshape(rows, cols)
    h_i, h_j = idx[:, :-1].ravel(), idx[:, 1:].ravel()
    v_i, v_j = idx[:-1, :].ravel(), idx[1:, :].ravel()
    return np.concatenate([h_i, v_i]), np.concatenate([h_j, v_j])


def chain_edges(n: int):
    a = np.arange(n - 1, dtype=np.int64)
    return a, a + 1


def _ising_from_structure(n, row_ptr, col, rev, rng, lam_max, beta_max, name):
    lam = rng.uniform(-lam_max, lam_max, size=n)
    und = _undirected_positions(row_ptr, col)
    beta_u = rng.uniform(-beta_max, beta_max, size=und.shape[0])
    beta = np.zeros(col.shape[0], dtype=np.float64)
    beta[und] = beta_u
    beta[rev[und]] = beta_u
    unary = np.stack([-lam, lam], axis=1).astype(np.float32).ravel()
    return Problem(n=n, k=2, row_ptr=row_ptr, col=col, rev=rev, unary_log=unary,
                   pair_kind=PAIR_ISING_BETA, pair_log=beta.astype(np.float32),
                   graph_var_offsets=np.array([0, n], dtype=np.int64), name=name)


def ising_grid(side: int, beta_max: float, seed: int, lam_max: float = 1.0,
               cols: int | None = None) -> Problem:
    """Binary Ising grid: theta_i(x) = lambda_i s(x), lambda ~ U[-lam_max, lam_max];
    theta_ij = beta_ij s(x_i) s(x_j), beta ~ U[-beta_max, beta_max]."""
    cols = side if cols is None else cols
    n = side * cols
    row_ptr, col, rev = csr_from_undirected(n, *grid_edges(side, cols))
    return _ising_from_structure(n, row_ptr, col, rev, _rng(seed), lam_max, beta_max,
                                 f"ising{side}x{cols}_b{beta_max}_s{seed}")


def ising_chain(n: int, beta_max: float, seed: int, lam_max: float = 1.0) -> Problem:
    row_ptr, col, rev = csr_from_undirected(n, *chain_edges(n))
    return _ising_from_structure(n, row_ptr, col, rev, _rng(seed), lam_max, beta_max,
                                 f"chain{n}_b{beta_max}_s{seed}")


def ising_tree(n: int, beta_max: float, seed: int, lam_max: float = 1.0) -> Problem:
    """Random recursive tree (vertex v > 0 attaches to a uniform earlier vertex)."""
    rng = _rng(seed)
    parent = np.array([rng.integers(0, v) for v in range(1, n)], dtype=np.int64)
    row_ptr, col, rev = csr_from_undirected(n, parent, np.arange(1, n, dtype=np.int64))
    return _ising_from_structure(n, row_ptr, col, rev, rng, lam_max, beta_max,
                                 f"tree{n}_b{beta_max}_s{seed}")


def paper_ising(rows: int, cols: int, C: float, seed: int) -> Problem:
    """The paper's own Ising parametrisation (Section III-C): psi_i(x) ~ U(0,1] drawn
    independently per state; psi_ij = exp(+lambda C) when x_i = x_j, else exp(-lambda C),
    lambda ~ U[-0.5, 0.5]. A chain is rows = 1."""
    n = rows * cols
    row_ptr, col, rev = csr_from_undirected(n, *grid_edges(rows, cols))
    rng = _rng(seed)
    psi = 1.0 - rng.random(size=(n, 2))          # U(0, 1]
    und = _undirected_positions(row_ptr, col)
    lam = rng.uniform(-0.5, 0.5, size=und.shape[0])
    beta = np.zeros(col.shape[0], dtype=np.float64)
    beta[und] = lam * C
    beta[rev[und]] = lam * C
    return Problem(n=n, k=2, row_ptr=row_ptr, col=col, rev=rev,
                   unary_log=np.log(psi).astype(np.float32).ravel(),
                   pair_kind=PAIR_ISING_BETA, pair_log=beta.astype(np.float32),
                   graph_var_offsets=np.array([0, n], dtype=np.int64),
                   name=f"paper_ising{rows}x{cols}_C{C}_s{seed}")


def potts_grid(side: int, k: int, seed: int, noise_std: float = 0.3,
               diag: float = 1.0, cols: int | None = None) -> Problem:
    """Potts grid with one shared pairwise table: theta_i ~ N(0, 1) per state;
    Theta = diag * I + eta, eta symmetric with N(0, noise_std^2) upper triangle
    (diagonal included) mirrored below."""
    cols = side if cols is None else cols
    n = side * cols
    row_ptr, col, rev = csr_from_undirected(n, *grid_edges(side, cols))
    rng = _rng(seed)
    unary = rng.standard_normal(size=(n, k))
    eta = np.zeros((k, k))
    iu = np.triu_indices(k)
    eta[iu] = rng.normal(0.0, noise_std, size=iu[0].shape[0])
    eta = np.triu(eta) + np.triu(eta, 1).T
    theta = diag * np.eye(k) + eta
    return Problem(n=n, k=k, row_ptr=row_ptr, col=col, rev=rev,
                   unary_log=unary.astype(np.float32).ravel(),
                   pair_kind=PAIR_SHARED, pair_log=theta.astype(np.float32).ravel(),
                   graph_var_offsets=np.array([0, n], dtype=np.int64),
                   name=f"potts{side}x{cols}_k{k}_s{seed}")


def protein_like(n: int, seed: int, k_min: int = 2, k_max: int = 32, attach: int = 2,
                 pair_std: float = 1.0, tree: bool = False) -> Problem:
    """Synthetic stand-in with the shape of the paper's protein-folding graphs
    (Section IV-E: 2 to 81 settings per vertex, highly irregular structure; the
    dataset itself is not available): vertices join by preferential attachment,
    each new vertex linking to `attach` earlier ones (1 when tree=True) with
    probability proportional to degree + 1; vertex v has k_v states, k_v drawn
    log-uniform in [k_min, k_max] (an integer); the layout has k_max states and
    the absent ones carry unary log-potential -inf; present unaries ~ N(0, 1);
    one pairwise log-table ~ N(0, pair_std^2) per undirected edge, stored per
    directed edge with table[rev e] = table[e] transposed.
    Draw order: k_v, edges, unaries, tables."""
    rng = _rng(seed)
    kv = np.floor(np.exp(rng.uniform(np.log(k_min), np.log(k_max + 1), size=n))).astype(np.int64)
    kv = np.clip(kv, k_min, k_max)
    deg = np.zeros(n, dtype=np.float64)
    ei, ej = [], []
    links = 1 if tree else attach
    for v in range(1, n):
        cnt = min(links, v)
        w = deg[:v] + 1.0
        targets = rng.choice(v, size=cnt, replace=False, p=w / w.sum())
        for t in targets:
            ei.append(int(t))
            ej.append(v)
            deg[t] += 1
            deg[v] += 1
    row_ptr, col, rev = csr_from_undirected(n, np.array(ei, np.int64), np.array(ej, np.int64))
    unary = rng.standard_normal(size=(n, k_max))
    unary[np.arange(k_max)[None, :] >= kv[:, None]] = -np.inf
    und = _undirected_positions(row_ptr, col)
    tables = np.zeros((col.shape[0], k_max, k_max))
    for e in und:
        t = rng.normal(0.0, pair_std, size=(k_max, k_max))
        tables[e] = t
        tables[rev[e]] = t.T
    return Problem(n=n, k=k_max, row_ptr=row_ptr, col=col, rev=rev,
                   unary_log=unary.astype(np.float32).ravel(), pair_kind=PAIR_TABLE,
                   pair_log=tables.astype(np.float32).ravel(),
                   graph_var_offsets=np.array([0, n], dtype=np.int64),
                   name=f"protein_like{n}_k{k_min}-{k_max}_s{seed}")


def random_table_graph(n: int, k: int, extra_edges: int, seed: int,
                       unary_std: float = 1.0, pair_std: float = 1.0) -> Problem:
    """Random connected graph (a random tree plus extra random edges) with a
    general k-state table per edge, stored per directed edge as [M, k, k] with
    table[rev e] = table[e] transposed."""
    rng = _rng(seed)
    parent = np.array([rng.integers(0, v) for v in range(1, n)], dtype=np.int64)
    ei = list(parent)
    ej = list(range(1, n))
    seen = {(min(a, b), max(a, b)) for a, b in zip(ei, ej)}
    while len(seen) < n - 1 + extra_edges:
        a, b = (int(x) for x in rng.integers(0, n, size=2))
        if a == b or (min(a, b), max(a, b)) in seen:
            continue
        seen.add((min(a, b), max(a, b)))
        ei.append(a)
        ej.append(b)
    row_ptr, col, rev = csr_from_undirected(n, np.array(ei), np.array(ej))
    unary = rng.normal(0.0, unary_std, size=(n, k))
    und = _undirected_positions(row_ptr, col)
    tabs = rng.normal(0.0, pair_std, size=(und.shape[0], k, k))
    pair = np.zeros((col.shape[0], k, k))
    pair[und] = tabs
    pair[rev[und]] = np.transpose(tabs, (0, 2, 1))
    return Problem(n=n, k=k, row_ptr=row_ptr, col=col, rev=rev,
                   unary_log=unary.astype(np.float32).ravel(),
                   pair_kind=PAIR_TABLE, pair_log=pair.astype(np.float32).ravel(),
                   graph_var_offsets=np.array([0, n], dtype=np.int64),
                   name=f"table{n}_k{k}_s{seed}")


def _er_graph_edges(rng: np.random.Generator, n: int, mean_degree: float):
    """G(n, p) with p = mean_degree / (n - 1): the edge count is Binomial, then the
    edges are a uniform sample of distinct unordered pairs."""
    if n < 2:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    n_pairs = n * (n - 1) // 2
    p = min(1.0, mean_degree / (n - 1))
    m = int(rng.binomial(n_pairs, p))
    chosen_i = np.zeros(0, np.int64)
    chosen_j = np.zeros(0, np.int64)
    keys = np.zeros(0, np.int64)
    while keys.shape[0] < m:
        want = m - keys.shape[0]
        a = rng.integers(0, n, size=2 * want + 8)
        b = rng.integers(0, n, size=2 * want + 8)
        ok = a != b
        lo, hi = np.minimum(a[ok], b[ok]), np.maximum(a[ok], b[ok])
        cand = lo * n + hi
        allk = np.concatenate([keys, cand])
        _, first = np.unique(allk, return_index=True)
        first.sort()
        keys = allk[first][:m]
    chosen_i, chosen_j = keys // n, keys % n
    return chosen_i, chosen_j


def concat_batch(problems: list[Problem], name: str = "batch") -> Problem:
    """Disjoint union of independent graphs with the same k and pair kind."""
    if not problems:
        raise ValueError("empty batch")
    k = problems[0].k
    kind = problems[0].pair_kind
    if any(p.k != k or p.pair_kind != kind for p in problems):
        raise ValueError("batch members must share k and pair kind")
    if kind == PAIR_SHARED and any(not np.array_equal(p.pair_log, problems[0].pair_log)
                                   for p in problems):
        raise ValueError("shared-table batch members must share the table")
    v_off = np.zeros(len(problems) + 1, dtype=np.int64)
    v_off[1:] = np.cumsum([p.n for p in problems])
    e_off = np.zeros(len(problems) + 1, dtype=np.int64)
    e_off[1:] = np.cumsum([p.m for p in problems])
    row_ptr = np.concatenate([problems[0].row_ptr[:1]] +
                             [p.row_ptr[1:] + e_off[g] for g, p in enumerate(problems)])
    col = np.concatenate([p.col.astype(np.int64) + v_off[g] for g, p in enumerate(problems)])
    rev = np.concatenate([p.rev.astype(np.int64) + e_off[g] for g, p in enumerate(problems)])
    unary = np.concatenate([p.unary_log for p in problems])
    pair = problems[0].pair_log if kind == PAIR_SHARED else \
        np.concatenate([p.pair_log for p in problems])
    return Problem(n=int(v_off[-1]), k=k, row_ptr=row_ptr.astype(np.int64),
                   col=col.astype(np.int32), rev=rev.astype(np.int32),
                   unary_log=unary.astype(np.float32), pair_kind=kind,
                   pair_log=pair.astype(np.float32), graph_var_offsets=v_off, name=name)


def er_batch(n_graphs: int, seed: int, n_min: int = 50, n_max: int = 5000,
             mean_degree: float = 4.0, lam_max: float = 1.0, beta_max: float = 3.0) -> Problem:
    """Batch of Erdos-Renyi binary Ising MRFs: n = round(exp(U[ln n_min, ln n_max])),
    G(n, mean_degree / (n - 1)), lambda ~ U[-lam_max, lam_max], beta ~ U[-beta_max, beta_max].
    Per graph: size, then edges, then lambda (vertex order), then beta (undirected-edge order)."""
    rng = _rng(seed)
    members = []
    for g in range(n_graphs):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        ei, ej = _er_graph_edges(rng, n, mean_degree)
        row_ptr, col, rev = csr_from_undirected(n, ei, ej)
        members.append(_ising_from_structure(n, row_ptr, col, rev, rng, lam_max, beta_max,
                                             f"er{g}"))
    return concat_batch(members, name=f"er_batch{n_graphs}_s{seed}")


def ising_grid_batch(side: int, beta_max: float, seeds, lam_max: float = 1.0) -> Problem:
    """Several seeds of the same Ising grid as one batch (graph g = seeds[g])."""
    seeds = list(seeds)
    return concat_batch([ising_grid(side, beta_max, s, lam_max) for s in seeds],
                        name=f"ising{side}_b{beta_max}_x{len(seeds)}")
