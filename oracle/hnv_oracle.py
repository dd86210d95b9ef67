"""HyperNetVec multilevel V-cycle: the plain CPU FP64 oracle.

TEST INFRASTRUCTURE ONLY. This module is the slow, obviously-correct
statement of what the GPU library computes; only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm
may import it. The library never calls it and shares no code with it.

It follows the paper (Maleki, Saless, Wall, Pingali: "HyperNetVec: Fast and
Scalable Hierarchical Embedding for Hypergraphs", arXiv 2103.09660):

* the hypergraph ``H = (V, E)`` with hyperedge weights and its star
  expansion ``H*`` (Section 1.1);
* coarsening, Algorithm 1 and the text of Section 3.1 (assign every node to
  one of its hyperedges, merge the nodes assigned to the same hyperedge,
  drop a hyperedge once all its nodes are merged, connect rep(v) to rep(e));
* projection, last paragraph of the smoothing description in Section 3.3
  (a merged node's embedding is given to every node it merged);
* refinement, Algorithm 2 and the smoothing/relaxation formulas of
  Section 3.3 (weighted neighbour mean, then ``(1-w) z + w z~``);
* the V-cycle: refine at every level from the coarsest to the original
  (Section 2.1.1 "Multi-level Embedding", Section 3 overview, Fig. 1).

Arithmetic is float64 throughout; integer work is exact. Library primitives
used as single steps: ``numpy.lexsort``/``numpy.unique`` (sorting) and the
scipy CSR-times-dense product (a sparse matmul; each row sums its entries in
ascending column order).

Readings of points the paper leaves open are marked READING below; the
same list is kept in the design notes of the repository.

Parity status: every function here is pinned by the CPU tests (brute force on
tiny hypergraphs, dense-matrix refinement, closed forms, invariants,
SplitMix64 test vectors, a hand-worked coarsening example).
"""

from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence, Tuple

import numpy as np
import scipy.sparse as sp

# ---------------------------------------------------------------------------
# Constants
# ---------------------------------------------------------------------------

ASSIGN_HASH = 0
ASSIGN_LOW_DEGREE = 1
ASSIGN_HIGH_WEIGHT = 2
ASSIGN_EXPLICIT = 3
ASSIGN_COSINE = 4

# Feature values are checked against this bound so that no sum of squares
# can overflow float32 (|x| <= 1e15: x^2 <= 1e30, and up to 2^24 of them).
FEATURE_ABS_MAX = 1e15

SWEEP_TWO_PHASE = 0
SWEEP_JACOBI = 1

_M64 = (1 << 64) - 1
# SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
# generators", OOPSLA 2014): golden-ratio increment and finaliser constants.
GOLDEN_GAMMA = 0x9E3779B97F4A7C15
_MIX_C1 = 0xBF58476D1CE4E5B9
_MIX_C2 = 0x94D049BB133111EB


# ---------------------------------------------------------------------------
# Hashing: the deterministic stand-in for the paper's random tie-break
# ---------------------------------------------------------------------------

def mix64_int(z: int) -> int:
    """SplitMix64 finaliser on a Python int (wrapping uint64 arithmetic)."""
    z &= _M64
    z = ((z ^ (z >> 30)) * _MIX_C1) & _M64
    z = ((z ^ (z >> 27)) * _MIX_C2) & _M64
    return z ^ (z >> 31)


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on a uint64 array (numpy wraps modulo 2**64)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_MIX_C1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_MIX_C2)
    return z ^ (z >> np.uint64(31))


def level_salt(seed: int, level: int) -> int:
    """Per-level salt ``mix64(seed + level * gamma)``."""
    return mix64_int((seed + level * GOLDEN_GAMMA) & _M64)


def hash_priority(edge_ids: np.ndarray, seed: int, level: int) -> np.ndarray:
    """``prio_l(e) = mix64(e XOR salt_l)`` for hyperedge IDs at level ``l``.

    READING (Section 3.1): with no node features every incident hyperedge of
    a node ties, and the paper breaks ties by a random choice among the
    node's hyperedges. The oracle and the library make that choice with one
    hash per hyperedge per level, identical for all nodes, so nodes that share
    a hyperedge agree and merge, and the hierarchy is reproducible.
    """
    salt = np.uint64(level_salt(seed, level))
    return mix64(np.asarray(edge_ids, dtype=np.uint64) ^ salt)


# ---------------------------------------------------------------------------
# Incidence structure of one level
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Level:
    """One level's hypergraph as incidence CSR (hyperedge -> nodes) and CSC
    (node -> hyperedges), both with ascending, duplicate-free rows.

    ``orig_e[e]`` is the level-0 ID of hyperedge ``e`` (a coarse hyperedge is
    the representative of exactly one fine hyperedge, Section 3.1)."""

    n: int
    m: int
    e_ptr: np.ndarray       # int64 [m+1]
    e_nodes: np.ndarray     # int64 [nnz]
    v_ptr: np.ndarray       # int64 [n+1]
    v_edges: np.ndarray     # int64 [nnz]
    w: np.ndarray           # float64 [m], weights as given (float32 values)
    w32: np.ndarray         # float32 [m], the same weights at input precision
    orig_e: np.ndarray      # int64 [m]

    @property
    def nnz(self) -> int:
        return int(self.e_ptr[-1])

    def size_e(self) -> np.ndarray:
        return np.diff(self.e_ptr)

    def deg_v(self) -> np.ndarray:
        """Weighted node degree ``sum_{e ∋ v} w_e`` (Section 3.3: the
        denominator of the smoothing formula; the plain degree when all
        weights are 1)."""
        out = np.zeros(self.n, dtype=np.float64)
        np.add.at(out, np.repeat(np.arange(self.n), np.diff(self.v_ptr)),
                  self.w[self.v_edges])
        return out


def _csr_from_pairs(rows: np.ndarray, cols: np.ndarray, n_rows: int
                    ) -> Tuple[np.ndarray, np.ndarray]:
    """Sorted, duplicate-free CSR from (row, col) pairs."""
    if rows.size:
        order = np.lexsort((cols, rows))
        r = rows[order]
        c = cols[order]
        keep = np.ones(r.size, dtype=bool)
        keep[1:] = (r[1:] != r[:-1]) | (c[1:] != c[:-1])
        r, c = r[keep], c[keep]
    else:
        r = rows.astype(np.int64)
        c = cols.astype(np.int64)
    ptr = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=n_rows), out=ptr[1:])
    return ptr, c.astype(np.int64)


def build_level(n: int, m: int, edge_ptr: Sequence[int], edge_nodes: Sequence[int],
                weights: Optional[Sequence[float]] = None,
                orig_e: Optional[np.ndarray] = None) -> Level:
    """Incidence structure of ``H = (V, E, w)`` (Section 1.1, star expansion):
    members are deduplicated and sorted; the CSC is the transpose.

    Raises ValueError for an out-of-range node, an empty hyperedge (the
    paper's hyperedges are non-empty subsets of V) or a non-positive or
    non-finite weight."""
    edge_ptr = np.asarray(edge_ptr, dtype=np.int64)
    edge_nodes = np.asarray(edge_nodes, dtype=np.int64)
    if edge_ptr.shape != (m + 1,) or edge_ptr[0] != 0 or np.any(np.diff(edge_ptr) < 0):
        raise ValueError("edge_ptr must be non-decreasing, start at 0, length m+1")
    if edge_nodes.size != edge_ptr[-1]:
        raise ValueError("edge_nodes length must equal edge_ptr[m]")
    if edge_nodes.size and (edge_nodes.min() < 0 or edge_nodes.max() >= n):
        raise ValueError("node id out of range")
    if np.any(np.diff(edge_ptr) == 0):
        raise ValueError("empty hyperedge")
    if weights is None:
        w32 = np.ones(m, dtype=np.float32)
    else:
        w32 = np.asarray(weights, dtype=np.float32)
    if w32.shape != (m,) or not np.all(np.isfinite(w32)) or np.any(w32 <= 0):
        raise ValueError("weights must be finite and > 0")
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(edge_ptr))
    e_ptr, e_nodes = _csr_from_pairs(rows, edge_nodes, m)
    v_ptr, v_edges = _csr_from_pairs(e_nodes, np.repeat(np.arange(m, dtype=np.int64),
                                                         np.diff(e_ptr)), n)
    if orig_e is None:
        orig_e = np.arange(m, dtype=np.int64)
    return Level(n=n, m=m, e_ptr=e_ptr, e_nodes=e_nodes, v_ptr=v_ptr,
                 v_edges=v_edges, w=w32.astype(np.float64), w32=w32,
                 orig_e=np.asarray(orig_e, dtype=np.int64))


# ---------------------------------------------------------------------------
# Coarsening (Algorithm 1, Section 3.1)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class CoarsenParams:
    policy: int = ASSIGN_HASH
    seed: int = 0
    min_nodes: int = 200
    max_levels: int = 32
    # ASSIGN_EXPLICIT: uint64 table [max_levels, m0]; entry [l, orig_e(e)]
    # is the priority of hyperedge e at level l (test-only policy).
    explicit_prio: Optional[np.ndarray] = None
    # ASSIGN_COSINE: level-0 node features, float32 [n0, k].
    features: Optional[np.ndarray] = None


def priorities(lv: Level, params: CoarsenParams, level: int) -> np.ndarray:
    """The uint64 key each node minimises over its hyperedges, ties going to
    the smaller hyperedge ID.

    HASH (default): the per-level hash (see ``hash_priority``).
    LOW_DEGREE: ``(min(|e|, 2^24-1) << 40) | (hash >> 24)`` -- smallest
      hyperedge first, hash among equal sizes (Section 3.1: "weights or
      degrees of a hyperedge").
    HIGH_WEIGHT: ``((2^32-1 - bits32(w_e)) << 32) | (hash >> 32)`` -- heaviest
      hyperedge first (positive float32 weights order like their bits).
    EXPLICIT: caller table indexed by (level, level-0 hyperedge ID).
    """
    e_ids = np.arange(lv.m, dtype=np.uint64)
    h = hash_priority(e_ids, params.seed, level)
    if params.policy == ASSIGN_HASH:
        return h
    if params.policy == ASSIGN_LOW_DEGREE:
        size = np.minimum(lv.size_e(), (1 << 24) - 1).astype(np.uint64)
        return (size << np.uint64(40)) | (h >> np.uint64(24))
    if params.policy == ASSIGN_HIGH_WEIGHT:
        bits = lv.w32.view(np.uint32).astype(np.uint64)
        return ((np.uint64(0xFFFFFFFF) - bits) << np.uint64(32)) | (h >> np.uint64(32))
    if params.policy == ASSIGN_EXPLICIT:
        tab = np.asarray(params.explicit_prio, dtype=np.uint64)
        return tab[level, lv.orig_e]
    raise ValueError("unknown assignment policy")


def assign_hyperedges(lv: Level, prio: np.ndarray) -> np.ndarray:
    """AssignHyperedge(v) for every node (Algorithm 1, Section 3.1):
    ``c(v) = argmin_{e in N(v)} (prio(e), e)``; ``-1`` if ``N(v)`` is empty."""
    c = np.full(lv.n, -1, dtype=np.int64)
    if lv.nnz == 0:
        return c
    node_of = np.repeat(np.arange(lv.n, dtype=np.int64), np.diff(lv.v_ptr))
    edge = lv.v_edges
    # sort incidences by (node, prio(edge), edge); the first of each node wins
    order = np.lexsort((edge, prio[edge], node_of))
    first = np.ones(order.size, dtype=bool)
    first[1:] = node_of[order][1:] != node_of[order][:-1]
    c[node_of[order][first]] = edge[order][first]
    return c


# ---------------------------------------------------------------------------
# Feature-based assignment (Section 3.1, nodes with features)
#
# The choice of c(v) is an argmax over floating-point scores, so it is taken
# in float32 with every rounding step written out, in the order the GPU
# kernels use: sums run one term at a time in a fixed order, products and
# quotients are rounded separately (no fused multiply-add), square roots
# are IEEE-rounded. numpy float32 arithmetic rounds each operation, so the
# float32 steps below are that definition.
# ---------------------------------------------------------------------------

def check_features(X: np.ndarray, n: int) -> np.ndarray:
    """Level-0 node features as float32 [n, k], k >= 1, finite, |x| <= 1e15."""
    X = np.asarray(X)
    if X.ndim != 2 or X.shape[0] != n or X.shape[1] < 1:
        raise ValueError("features must be [n, k] with k >= 1")
    X = X.astype(np.float32)
    if not np.all(np.isfinite(X)) or np.any(np.abs(X) > FEATURE_ABS_MAX):
        raise ValueError("features must be finite with |x| <= 1e15")
    return X


def segment_means_f32(ptr: np.ndarray, idx: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Row r of the result: the float32 mean of X[idx[ptr[r]:ptr[r+1]]],
    summed one row at a time in list order, then divided by the count (a
    row with an empty list is 0)."""
    rows = ptr.size - 1
    k = X.shape[1]
    cnt = np.diff(ptr)
    acc = np.zeros((rows, k), dtype=np.float32)
    for j in range(int(cnt.max()) if rows else 0):
        sel = np.nonzero(cnt > j)[0]
        acc[sel] = acc[sel] + X[idx[ptr[sel] + j]]
    den = np.maximum(cnt, 1).astype(np.float32)
    return (acc / den[:, None]).astype(np.float32)


def row_norms_f32(F: np.ndarray) -> np.ndarray:
    """sqrt(sum_i F[:, i] * F[:, i]), squares added in dimension order."""
    acc = np.zeros(F.shape[0], dtype=np.float32)
    for i in range(F.shape[1]):
        acc = acc + F[:, i] * F[:, i]
    return np.sqrt(acc).astype(np.float32)


def edge_features(lv: Level, X: np.ndarray) -> np.ndarray:
    """ComputeEdgeFeature (Algorithm 1, Section 3.1): the feature vector of a
    hyperedge is the mean of its members' features (members in ascending
    node order)."""
    return segment_means_f32(lv.e_ptr, lv.e_nodes, X)


def cosine_scores(lv: Level, X: np.ndarray, FE: np.ndarray) -> np.ndarray:
    """cos(f(e), f(v)) = f(e).f(v) / (|f(e)| |f(v)|) for every incidence, in
    CSC order (node-major, ascending hyperedge). READING: where either norm
    is 0 the cosine is undefined; its score is taken as 0."""
    node_of = row_of(lv.v_ptr)
    edge = lv.v_edges
    dot = np.zeros(edge.size, dtype=np.float32)
    for i in range(X.shape[1]):
        dot = dot + FE[edge, i] * X[node_of, i]
    den = row_norms_f32(FE)[edge] * row_norms_f32(X)[node_of]
    score = np.zeros(edge.size, dtype=np.float32)
    ok = den > 0
    score[ok] = dot[ok] / den[ok]
    return score


def assign_cosine(lv: Level, X: np.ndarray, prio: np.ndarray) -> np.ndarray:
    """AssignHyperedge with features: ``c(v) = argmax_{e in N(v)} cos(f(e),
    f(v))``. READING of the tie rule (the paper picks at random): among
    equal scores the smallest ``(prio(e), e)`` wins, the same per-level hash
    order as the featureless rule. ``-1`` if ``N(v)`` is empty."""
    c = np.full(lv.n, -1, dtype=np.int64)
    if lv.nnz == 0:
        return c
    score = cosine_scores(lv, X, edge_features(lv, X))
    node_of = row_of(lv.v_ptr)
    edge = lv.v_edges
    order = np.lexsort((edge, prio[edge], -score, node_of))
    first = np.ones(order.size, dtype=bool)
    first[1:] = node_of[order][1:] != node_of[order][:-1]
    c[node_of[order][first]] = edge[order][first]
    return c


def merge_features(rep_v: np.ndarray, n2: int, X: np.ndarray) -> np.ndarray:
    """Coarse node features X' (Algorithm 1's output). READING (the merge rule
    is not stated): the mean of the merged nodes' features, in ascending
    fine-node order."""
    order = np.argsort(rep_v, kind="stable")
    ptr = np.zeros(n2 + 1, dtype=np.int64)
    np.cumsum(np.bincount(rep_v, minlength=n2), out=ptr[1:])
    return segment_means_f32(ptr, order, X)


def coarsen_level(lv: Level, params: CoarsenParams, level: int,
                  X: Optional[np.ndarray] = None) -> Tuple[np.ndarray, np.ndarray, Level]:
    """One coarsening step of Algorithm 1.

    Returns ``rep_v[n]`` (coarse node of each node), ``rep_e[m]`` (coarse
    hyperedge ID if kept, else ``-1 - c`` where ``c`` is the coarse node the
    hyperedge collapsed into) and the coarse level.

    Steps (Section 3.1, Algorithm 1):
    1. AssignHyperedge: ``c(v)`` as in ``assign_hyperedges``.
    2. FindAssignedNodes/Merge/addNode: nodes with equal ``c(v)`` form one
       coarse node. READING: a node in no hyperedge stays a coarse node of its
       own (the paper is silent; this keeps rep a partition map). Coarse IDs
       are the ranks of the keys ``c(v)`` (assigned) or ``m + v`` (alone):
       hyperedge-formed nodes first in hyperedge order, then lone nodes in
       node order (a canonical numbering; the paper does not fix one).
    3. addHedge: READING of "if all nodes of a hyperedge are merged, we remove
       that hyperedge": ``e`` is kept iff its members map to at least two
       distinct coarse nodes. Algorithm 1's test ``|M| != |e|`` (every member
       assigned to ``e`` itself) is the case that always collapses to one
       node; the rule here also removes hyperedges whose members all merged
       through other hyperedges, which also matches the dataset cleaning that
       removes one-node hyperedges. Kept hyperedges keep their order and
       weight; hyperedges with equal member sets stay distinct.
    4. addEdge(rep(e), rep(v)) for v in e: coarse members are the distinct
       ``rep_v`` of the members, ascending.
    """
    if params.policy == ASSIGN_COSINE:
        prio = hash_priority(np.arange(lv.m, dtype=np.uint64), params.seed, level)
        c = assign_cosine(lv, X, prio)
    else:
        prio = priorities(lv, params, level)
        c = assign_hyperedges(lv, prio)
    key = np.where(c >= 0, c, lv.m + np.arange(lv.n, dtype=np.int64))
    uniq = np.unique(key)
    rep_v = np.searchsorted(uniq, key).astype(np.int64)
    n2 = int(uniq.size)

    # image of every hyperedge under rep_v, as a sorted set
    row = np.repeat(np.arange(lv.m, dtype=np.int64), lv.size_e())
    img_ptr, img_nodes = _csr_from_pairs(row, rep_v[lv.e_nodes], lv.m)
    img_size = np.diff(img_ptr)
    keep = img_size >= 2
    new_id = np.cumsum(keep) - 1
    m2 = int(keep.sum())
    # every hyperedge is non-empty, so a removed one has exactly one image
    rep_e = np.empty(lv.m, dtype=np.int64)
    rep_e[keep] = new_id[keep]
    rep_e[~keep] = -1 - img_nodes[img_ptr[:-1][~keep]]

    kept_entries = np.repeat(keep, img_size)
    coarse_row = new_id[row_of(img_ptr)[kept_entries]]
    coarse_col = img_nodes[kept_entries]
    e_ptr2 = np.zeros(m2 + 1, dtype=np.int64)
    np.cumsum(img_size[keep], out=e_ptr2[1:])
    v_ptr2, v_edges2 = _csr_from_pairs(coarse_col, coarse_row, n2)
    nxt = Level(n=n2, m=m2, e_ptr=e_ptr2, e_nodes=coarse_col.astype(np.int64),
                v_ptr=v_ptr2, v_edges=v_edges2, w=lv.w[keep], w32=lv.w32[keep],
                orig_e=lv.orig_e[keep])
    return rep_v, rep_e, nxt


def row_of(ptr: np.ndarray) -> np.ndarray:
    """Row index of every entry of a CSR with row pointer ``ptr``."""
    return np.repeat(np.arange(ptr.size - 1, dtype=np.int64), np.diff(ptr))


@dataclasses.dataclass
class Hierarchy:
    levels: List[Level]
    rep_v: List[np.ndarray]     # rep_v[l]: level l -> level l+1
    rep_e: List[np.ndarray]
    # ASSIGN_COSINE: node features of every level (float32 [n_l, k])
    features: Optional[List[np.ndarray]] = None


def coarsen(lv0: Level, params: CoarsenParams) -> Hierarchy:
    """Repeat Algorithm 1's loop body level by level.

    READING of the depth: Algorithm 1 takes a depth K; the experiments stop
    by level count or once the coarsest graph is small enough (Section 3.2).
    Coarsen while ``n_l > min_nodes``, ``l < max_levels`` and ``m_l > 0``;
    a step that merges nothing (``n_{l+1} == n_l``) is discarded and ends
    the loop."""
    levels = [lv0]
    rv: List[np.ndarray] = []
    re: List[np.ndarray] = []
    feats = None
    if params.policy == ASSIGN_COSINE:
        if params.features is None:
            raise ValueError("the cosine policy needs node features")
        feats = [check_features(params.features, lv0.n)]
    while True:
        cur = levels[-1]
        ell = len(levels) - 1
        if not (cur.n > params.min_nodes and ell < params.max_levels and cur.m > 0):
            break
        rep_v, rep_e, nxt = coarsen_level(cur, params, ell, feats[-1] if feats else None)
        if nxt.n == cur.n:
            break
        levels.append(nxt)
        rv.append(rep_v)
        re.append(rep_e)
        if feats is not None:
            feats.append(merge_features(rep_v, nxt.n, feats[-1]))
    return Hierarchy(levels=levels, rep_v=rv, rep_e=re, features=feats)


# ---------------------------------------------------------------------------
# Projection (Section 3.3, initial embeddings of the finer levels)
# ---------------------------------------------------------------------------

def project(rep_v: np.ndarray, rep_e: np.ndarray, zc_v: np.ndarray,
            zc_e: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """A fine node takes its coarse node's embedding (Section 3.3). READING
    for hyperedges (the paper is silent): a kept hyperedge takes its coarse
    hyperedge's embedding; a removed one takes the embedding of the coarse
    node it collapsed into, which is also the mean of its projected
    members."""
    zc_v = np.asarray(zc_v, dtype=np.float64)
    zc_e = np.asarray(zc_e, dtype=np.float64)
    zf_v = zc_v[rep_v]
    zf_e = np.empty((rep_e.size, zc_v.shape[1]), dtype=np.float64)
    kept = rep_e >= 0
    zf_e[kept] = zc_e[rep_e[kept]]
    zf_e[~kept] = zc_v[-1 - rep_e[~kept]]
    return zf_v, zf_e


# ---------------------------------------------------------------------------
# Refinement (Algorithm 2, Section 3.3)
# ---------------------------------------------------------------------------

def incidence_matrices(lv: Level) -> Tuple[sp.csr_matrix, sp.csr_matrix]:
    """``H_e`` (m x n, ones: hyperedge rows) and ``H_v`` (n x m, entry
    ``w_e``: node rows) of the star expansion, both CSR with ascending
    columns."""
    He = sp.csr_matrix((np.ones(lv.nnz), lv.e_nodes, lv.e_ptr), shape=(lv.m, lv.n))
    Hv = sp.csr_matrix((lv.w[lv.v_edges], lv.v_edges, lv.v_ptr), shape=(lv.n, lv.m))
    He.has_sorted_indices = True
    Hv.has_sorted_indices = True
    return He, Hv


def smooth_edges(lv: Level, He: sp.csr_matrix, z_v: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """``z~_e = sum_{v in e} w_e z_v / sum_{v in e} w_e``: every incidence of
    ``e`` carries ``w_e``, so this is the plain mean over the members
    (Section 3.3 smoothing formula). Returns (z~, has_neighbours)."""
    size = lv.size_e().astype(np.float64)
    has = size > 0
    zt = He @ z_v
    zt[has] /= size[has, None]
    return zt, has


def smooth_nodes(lv: Level, Hv: sp.csr_matrix, deg_v: np.ndarray, z_e: np.ndarray
                 ) -> Tuple[np.ndarray, np.ndarray]:
    """``z~_v = sum_{e ∋ v} w_e z_e / sum_{e ∋ v} w_e`` (Section 3.3)."""
    has = np.diff(lv.v_ptr) > 0
    zt = Hv @ z_e
    zt[has] /= deg_v[has, None]
    return zt, has


def relax(z: np.ndarray, zt: np.ndarray, has: np.ndarray, omega: float) -> np.ndarray:
    """``z <- (1 - omega) z + omega z~`` on rows that have neighbours; rows
    with an empty neighbourhood are left as they are (READING: the paper's
    formula is undefined there)."""
    out = z.copy()
    out[has] = (1.0 - omega) * z[has] + omega * zt[has]
    return out


# bfloat16: the IEEE binary32 layout cut to 16 bits (1 sign, 8 exponent and
# 7 fraction bits), so 8 significant bits and binary32's exponent range.
BF16_SIGNIFICANT_BITS = 8
BF16_MIN_NORMAL_EXP = -126


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Rounds float64 values to the nearest bfloat16 value, ties to the one
    with an even last significand bit (IEEE round-to-nearest-even), and
    returns them as float64 (exactly). A value with binary exponent E (that
    is, in [2^E, 2^(E+1))) is a multiple of 2^(E-7) in bfloat16; below the
    smallest normal 2^-126 the spacing stays 2^-133. numpy's ``rint`` rounds
    halves to even, and scaling by powers of two is exact, so every step
    here is exact but the one rounding. Values beyond bfloat16's range are
    not expected (the embeddings are convex combinations of the input)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    nz = x != 0
    _, e = np.frexp(x[nz])                      # |x| = f * 2^e, 0.5 <= f < 1
    exp = np.maximum(e - 1, BF16_MIN_NORMAL_EXP)
    q = np.ldexp(1.0, exp - (BF16_SIGNIFICANT_BITS - 1))
    out[nz] = np.rint(x[nz] / q) * q
    return out


STORAGE_F64 = None
STORAGE_BF16 = "bf16"


def _store(z: np.ndarray, storage) -> np.ndarray:
    """The rows as they are stored between half-sweeps: unchanged, or
    rounded to bfloat16 (the library's BF16 storage keeps rows in bfloat16
    and does its arithmetic in float32; the oracle does its arithmetic in
    float64 and rounds each stored value once)."""
    if storage is None:
        return z
    if storage == STORAGE_BF16:
        return round_bf16(z)
    raise ValueError("unknown storage %r" % (storage,))


def refine(lv: Level, z_v: np.ndarray, z_e: np.ndarray, omega: float,
           sweeps: int, mode: int = SWEEP_TWO_PHASE, storage=None
           ) -> Tuple[np.ndarray, np.ndarray]:
    """Algorithm 2: ``sweeps`` iterations of smoothing plus relaxation over
    the star expansion of one level.

    READING of the update order: Algorithm 2 writes every update from the
    previous iterate (``SWEEP_JACOBI``), while the text says hyperedge
    embeddings are updated from the nodes and node embeddings from the
    hyperedges, and frames the scheme as SOR. The default
    ``SWEEP_TWO_PHASE`` updates all hyperedges from the current nodes, then
    all nodes from the new hyperedges; both are provided.

    ``storage=STORAGE_BF16`` rounds every relaxed row to bfloat16 as it is
    stored (see ``_store``); the input rows must then be bfloat16 values."""
    z_v = np.array(z_v, dtype=np.float64)
    z_e = np.array(z_e, dtype=np.float64)
    He, Hv = incidence_matrices(lv)
    deg = lv.deg_v()
    for _ in range(sweeps):
        if mode == SWEEP_TWO_PHASE:
            zt_e, has_e = smooth_edges(lv, He, z_v)
            z_e = _store(relax(z_e, zt_e, has_e, omega), storage)
            zt_v, has_v = smooth_nodes(lv, Hv, deg, z_e)
            z_v = _store(relax(z_v, zt_v, has_v, omega), storage)
        elif mode == SWEEP_JACOBI:
            zt_e, has_e = smooth_edges(lv, He, z_v)
            zt_v, has_v = smooth_nodes(lv, Hv, deg, z_e)
            z_e = _store(relax(z_e, zt_e, has_e, omega), storage)
            z_v = _store(relax(z_v, zt_v, has_v, omega), storage)
        else:
            raise ValueError("unknown sweep mode")
    return z_v, z_e


def refine_until(lv: Level, z_v: np.ndarray, z_e: np.ndarray, omega: float,
                 max_sweeps: int, eps: float, mode: int = SWEEP_TWO_PHASE):
    """Refinement with the stopping rule the experiments name as an
    alternative to a fixed sweep count (Section 4, experimental setup): stop
    once the difference between two consecutive iterates is at most eps.
    READING of "difference": the largest absolute change of any coordinate
    of any node or hyperedge row during one sweep. At most max_sweeps
    sweeps. Returns (z_v, z_e, sweeps_done, per-sweep differences)."""
    z_v = np.array(z_v, dtype=np.float64)
    z_e = np.array(z_e, dtype=np.float64)
    deltas = []
    for _ in range(max_sweeps):
        nv, ne = refine(lv, z_v, z_e, omega, 1, mode)
        dv = float(np.abs(nv - z_v).max()) if nv.size else 0.0
        de = float(np.abs(ne - z_e).max()) if ne.size else 0.0
        z_v, z_e = nv, ne
        deltas.append(max(dv, de))
        if deltas[-1] <= eps:
            break
    return z_v, z_e, len(deltas), deltas


# ---------------------------------------------------------------------------
# The V-cycle
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class VCycleResult:
    z_v: np.ndarray
    z_e: np.ndarray
    per_level: List[Tuple[np.ndarray, np.ndarray]]   # refined (z_v, z_e) per level


def vcycle(h: Hierarchy, z_coarsest: np.ndarray, omega: float, sweeps: int,
           mode: int = SWEEP_TWO_PHASE, keep_levels: bool = False,
           storage=None) -> VCycleResult:
    """Refine the coarsest level from its initial embedding, then for every
    finer level project and refine, down to the original hypergraph
    (Section 3 overview, Fig. 1). ``z_coarsest`` holds the coarsest nodes'
    rows first, then its hyperedges'. ``storage`` is passed to ``refine``
    (projection copies stored rows, so it needs no rounding of its own)."""
    L = len(h.levels) - 1
    top = h.levels[L]
    z = np.asarray(z_coarsest, dtype=np.float64)
    if z.shape[0] != top.n + top.m:
        raise ValueError("z_coarsest must have n_L + m_L rows")
    z_v, z_e = refine(top, z[:top.n], z[top.n:], omega, sweeps, mode, storage)
    per = [None] * (L + 1)
    if keep_levels:
        per[L] = (z_v, z_e)
    for ell in range(L - 1, -1, -1):
        z_v, z_e = project(h.rep_v[ell], h.rep_e[ell], z_v, z_e)
        z_v, z_e = refine(h.levels[ell], z_v, z_e, omega, sweeps, mode, storage)
        if keep_levels:
            per[ell] = (z_v, z_e)
    return VCycleResult(z_v=z_v, z_e=z_e, per_level=per)


# ---------------------------------------------------------------------------
# Reverse mode (adjoint) of the two-phase V-cycle
# ---------------------------------------------------------------------------
#
# The forward map is (w0, Z^L) -> (Z_V^0, Z_E^0): the level-l weights are the
# level-0 weights of the hyperedges they came from, w_l = w0[orig_e_l], and
# enter the node half-sweeps through the weighted mean
#   z~_v = s_v / D_v,   s_v = sum_{e ∋ v} w_e z_e,   D_v = sum_{e ∋ v} w_e,
# so d z~_v / d w_e = (z_e - z~_v) / D_v. Reverse mode follows the sweeps
# backwards; every step is the transpose of the forward step.

def with_weights(h: Hierarchy, w0: np.ndarray) -> Hierarchy:
    """The same hierarchy with level-0 weights `w0` (float64) propagated to
    every level through orig_e (coarse hyperedges keep their weight)."""
    w0 = np.asarray(w0, dtype=np.float64)
    levels = []
    for lv in h.levels:
        w = w0[lv.orig_e]
        levels.append(dataclasses.replace(lv, w=w, w32=w.astype(np.float32)))
    return Hierarchy(levels=levels, rep_v=h.rep_v, rep_e=h.rep_e)


def refine_states(lv: Level, z_v: np.ndarray, z_e: np.ndarray, omega: float, sweeps: int):
    """Two-phase refinement keeping every iterate: [(z_v^0, z_e^0), ...,
    (z_v^k, z_e^k)]."""
    states = [(np.array(z_v, dtype=np.float64), np.array(z_e, dtype=np.float64))]
    for _ in range(sweeps):
        states.append(refine(lv, states[-1][0], states[-1][1], omega, 1, SWEEP_TWO_PHASE))
    return states


def refine_backward(lv: Level, states, omega: float, g_v: np.ndarray, g_e: np.ndarray):
    """Adjoint of two-phase `refine`: from dL/d(z_v^k, z_e^k) to
    dL/d(z_v^0, z_e^0) and dL/dw (this level's weights)."""
    He, Hv = incidence_matrices(lv)
    size = lv.size_e().astype(np.float64)
    deg = lv.deg_v()
    has_v = np.diff(lv.v_ptr) > 0
    has_e = size > 0
    g_v = np.array(g_v, dtype=np.float64)
    g_e = np.array(g_e, dtype=np.float64)
    dw = np.zeros(lv.m)
    for i in range(len(states) - 1, 0, -1):
        _, ze_i = states[i]
        zv_prev, _ = states[i - 1]
        # node half-sweep of sweep i: z_v^i = (1-w) z_v^{i-1} + w s_v / D_v
        zt_v, _ = smooth_nodes(lv, Hv, deg, ze_i)
        a = np.zeros_like(g_v)
        a[has_v] = g_v[has_v] / deg[has_v, None]
        A = He @ a                                         # sum_{v in e} a_v
        c = np.einsum("ij,ij->i", a, zt_v)                 # <a_v, z~_v>
        dw += omega * (np.einsum("ij,ij->i", A, ze_i) - He @ c)
        g_e = g_e + omega * lv.w[:, None] * A
        g_v[has_v] *= (1.0 - omega)
        # hyperedge half-sweep of sweep i: z_e^i = (1-w) z_e^{i-1} + w mean_{v in e} z_v^{i-1}
        b = np.zeros_like(g_e)
        b[has_e] = g_e[has_e] / size[has_e, None]
        g_v = g_v + omega * (He.T @ b)
        g_e[has_e] *= (1.0 - omega)
    return g_v, g_e, dw


def project_backward(rep_v: np.ndarray, rep_e: np.ndarray, n_c: int, m_c: int,
                     gf_v: np.ndarray, gf_e: np.ndarray):
    """Adjoint of `project`: a coarse row collects the gradients of every fine
    row copied from it."""
    d = gf_v.shape[1]
    gc_v = np.zeros((n_c, d))
    gc_e = np.zeros((m_c, d))
    np.add.at(gc_v, rep_v, gf_v)
    kept = rep_e >= 0
    np.add.at(gc_e, rep_e[kept], gf_e[kept])
    np.add.at(gc_v, -1 - rep_e[~kept], gf_e[~kept])
    return gc_v, gc_e


def vcycle_grad(h: Hierarchy, z_coarsest: np.ndarray, omega: float, sweeps: int,
                g_v0: np.ndarray, g_e0: np.ndarray):
    """dL/dw0 and dL/dZ^L of the two-phase V-cycle, given dL/dZ_V^0 and
    dL/dZ_E^0. Forward states are recomputed level by level from the
    levels' starting rows (checkpoints)."""
    L = len(h.levels) - 1
    top = h.levels[L]
    z = np.asarray(z_coarsest, dtype=np.float64)
    starts = [None] * (L + 1)
    starts[L] = (z[:top.n], z[top.n:])
    zv, ze = refine(top, starts[L][0], starts[L][1], omega, sweeps)
    for ell in range(L - 1, -1, -1):
        zv, ze = project(h.rep_v[ell], h.rep_e[ell], zv, ze)
        starts[ell] = (zv, ze)
        zv, ze = refine(h.levels[ell], zv, ze, omega, sweeps)
    m0 = h.levels[0].m
    dw0 = np.zeros(m0)
    g_v, g_e = np.asarray(g_v0, dtype=np.float64), np.asarray(g_e0, dtype=np.float64)
    for ell in range(0, L + 1):
        lv = h.levels[ell]
        states = refine_states(lv, starts[ell][0], starts[ell][1], omega, sweeps)
        g_v, g_e, dw = refine_backward(lv, states, omega, g_v, g_e)
        np.add.at(dw0, lv.orig_e, dw)
        if ell < L:
            nxt = h.levels[ell + 1]
            g_v, g_e = project_backward(h.rep_v[ell], h.rep_e[ell], nxt.n, nxt.m, g_v, g_e)
    return dw0, np.vstack([g_v, g_e])
