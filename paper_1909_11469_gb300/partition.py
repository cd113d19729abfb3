"""Partition of one large graph across ranks (one process per GPU).

A single graph too large for one GPU, or whose round time one GPU bounds,
splits into vertex blocks: rank r owns a set of vertices and every directed
message that leaves them (CSR rows of its vertices). A message update of an
owned vertex's out-edge needs the messages INTO that vertex (Eq. 2), so each
rank also keeps a slot for every incoming message from a vertex it does not
own (a halo). One round of any schedule then needs exactly one exchange: each
rank sends the messages it committed on cut edges to the rank that owns their
destination, which stores them in its halo slots. The convergence test and
RnBP's EdgeRatio (Section IV-A) need the global max residual and the global
count of messages with residual >= eps: one 16-byte all-reduce (a max and a
sum) per round. RnBP's random filter is keyed by the global edge id, so the
partitioned run draws the same frontier as one process. RBP and RS need a
global top-k (a histogram all-reduce per radix pass), so they do not partition
as cheaply.

Partitions: `grid_blocks` cuts a rows x cols grid (vertex r * cols + c) into
pr x pc rectangles (cut ~ perimeter, the natural choice for the Ising grids);
`contiguous_ranges` cuts any CSR into contiguous vertex ranges balanced by
directed edges (the edge cut of a general graph, no reordering).

`build_plans` turns an owner array into per-rank plans: local numbering
(owned vertices first, in global order, then halo vertices), the local CSR of
the owned rows with local column ids, and for every neighbouring rank the
global ids of the messages sent to it and received from it, in one agreed
order (sorted by global edge id), with the local slots they come from and go
to. Host logic only (NumPy); the exchange itself is NCCL send/recv or a copy
into the peer's memory on the data path.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def grid_blocks(rows: int, cols: int, pr: int, pc: int) -> np.ndarray:
    """Owner rank of every vertex of a rows x cols grid cut into pr x pc
    rectangles (rank = block row * pc + block column); block boundaries split
    the rows and the columns as evenly as integers allow."""
    if pr < 1 or pc < 1 or pr > rows or pc > cols:
        raise ValueError("block counts out of range")
    rb = (np.arange(rows) * pr) // rows
    cb = (np.arange(cols) * pc) // cols
    return (rb[:, None] * pc + cb[None, :]).reshape(-1).astype(np.int32)


def contiguous_ranges(row_ptr: np.ndarray, world: int) -> np.ndarray:
    """Owner rank of every vertex: contiguous vertex ranges, rank r ending
    where the running count of directed edges first reaches (r + 1) / world of
    the total (a rank's share exceeds the ideal by less than one vertex's
    degree)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    n = row_ptr.shape[0] - 1
    if world < 1:
        raise ValueError("world must be >= 1")
    total = int(row_ptr[-1])
    owner = np.empty(n, dtype=np.int32)
    start = 0
    for r in range(world):
        if r == world - 1:
            end = n
        else:
            target = (r + 1) * total / world
            end = int(np.searchsorted(row_ptr[1:], target, side="left")) + 1 if total > 0 else start
            end = max(start, min(end, n))
        owner[start:end] = r
        start = end
    return owner


@dataclasses.dataclass
class RankPlan:
    """What rank `rank` holds and exchanges each round.

    vertices[:n_owned] are the owned global vertex ids (ascending), the rest
    the halo vertices (sources of incoming cut messages). Local directed edge
    ids [0, n_local_edges) are the out-edges of the owned vertices in CSR
    order (global ids `edges`); local ids [n_local_edges, n_local_edges +
    n_halo_slots) are the halo slots, one per incoming cut message (global ids
    `halo_edges`). row_ptr / col describe the owned rows with local vertex ids;
    rev[e] is the local slot of the reverse message of local edge e (an owned
    edge or a halo slot). send[q] / recv[q]: (global message ids, local slots)
    exchanged with rank q, sorted by global id, so that rank p's send[q] equals
    rank q's recv[p] element for element."""
    rank: int
    vertices: np.ndarray
    n_owned: int
    edges: np.ndarray
    halo_edges: np.ndarray
    row_ptr: np.ndarray
    col: np.ndarray
    rev: np.ndarray
    send: dict
    recv: dict

    @property
    def n_local_edges(self) -> int:
        return int(self.edges.shape[0])

    @property
    def n_halo_slots(self) -> int:
        return int(self.halo_edges.shape[0])

    def exchange_bytes(self, bytes_per_message: int) -> int:
        """Bytes this rank sends per round (one value per cut message)."""
        return bytes_per_message * sum(int(ids.shape[0]) for ids, _ in self.send.values())


def build_plans(row_ptr, col, rev, owner) -> list[RankPlan]:
    """Per-rank plans of the partition `owner` (owner[v] = rank of vertex v)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    rev = np.asarray(rev, dtype=np.int64)
    owner = np.asarray(owner, dtype=np.int64)
    n = row_ptr.shape[0] - 1
    m = col.shape[0]
    if owner.shape[0] != n:
        raise ValueError("owner must have one entry per vertex")
    world = int(owner.max()) + 1 if n else 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    edge_owner = owner[src]                       # a message lives with its source vertex
    dst_owner = owner[col] if m else np.zeros(0, np.int64)
    plans = []
    for r in range(world):
        owned = np.nonzero(owner == r)[0]
        my_edges = np.nonzero(edge_owner == r)[0]           # CSR order = ascending global id
        # incoming cut messages: reverses of my out-edges whose destination is remote
        cut_out = my_edges[dst_owner[my_edges] != r]
        halo_edges = np.sort(rev[cut_out])
        halo_vertices = np.unique(src[halo_edges]) if halo_edges.size else np.zeros(0, np.int64)
        vertices = np.concatenate([owned, halo_vertices])
        vloc = np.full(n, -1, dtype=np.int64)
        vloc[vertices] = np.arange(vertices.shape[0])
        eloc = np.full(m, -1, dtype=np.int64)
        eloc[my_edges] = np.arange(my_edges.shape[0])
        eloc[halo_edges] = my_edges.shape[0] + np.arange(halo_edges.shape[0])
        deg = np.diff(row_ptr)[owned]
        lrow = np.zeros(owned.shape[0] + 1, dtype=np.int64)
        np.cumsum(deg, out=lrow[1:])
        lcol = vloc[col[my_edges]]
        lrev = eloc[rev[my_edges]]
        send, recv = {}, {}
        for q in range(world):
            if q == r:
                continue
            out_q = my_edges[dst_owner[my_edges] == q]          # I compute these, q needs them
            if out_q.size:
                send[q] = (out_q, eloc[out_q])
            in_q = halo_edges[edge_owner[halo_edges] == q]       # q computes these, I need them
            if in_q.size:
                recv[q] = (in_q, eloc[in_q])
        plans.append(RankPlan(rank=r, vertices=vertices, n_owned=int(owned.shape[0]), edges=my_edges,
                              halo_edges=halo_edges, row_ptr=lrow, col=lcol, rev=lrev, send=send, recv=recv))
    return plans


def cut_messages(plans: list[RankPlan]) -> int:
    """Directed messages that cross ranks per round (each sent once)."""
    return sum(int(ids.shape[0]) for p in plans for ids, _ in p.send.values())
