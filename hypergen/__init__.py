"""Seeded synthetic hypergraphs with planted communities.

This module is the only code shared by the CUDA path's tests/bench and the
oracle: it draws inputs and holds none of the embedding method's arithmetic.

The paper evaluates on citation, co-authorship and social hypergraphs whose
hyperedges are mostly drawn from one class/community and whose sizes are
heavy-tailed (Section 4, Tables 1 and 3; Friendster groups are capped at 500).
None of those datasets is available here, so a planted-community generator
stands in for them:

* ``comm = rng.permutation(n) % C``: equal-size communities, uncorrelated
  with node ID;
* per hyperedge ``e``: size ``min(cap, 2 + Zipf(alpha))`` (also ``<= n``),
  a uniform home community, and members drawn one by one -- with
  probability ``p_in`` uniformly from the home community, otherwise
  uniformly from all nodes; a member already in ``e`` is redrawn;
* weights all 1, or ``Uniform[0.5, 2.0)`` per hyperedge;
* then the paper's dataset cleaning (Section 4, "Datasets" of the node
  classification study): hyperedges with fewer than two distinct members
  and nodes in no hyperedge are removed, and both are relabelled compactly
  in ascending original ID.

Draw order (fixed; changing it changes every dataset):
  1. ``rng.permutation(n)``                       -> communities
  2. ``rng.zipf(alpha, m)``                        -> sizes
  3. ``rng.integers(0, C, m)``                     -> home communities
  4. ``rng.uniform(0.5, 2.0, m)`` (weighted only)  -> weights
  5. rounds of member draws: for every missing member, in hyperedge order,
     one ``rng.random`` (inside/outside) and one ``rng.random`` (position),
     drawn as two arrays of the round's length; duplicates are rejected
     (first occurrence wins) and the next round redraws what is missing.

Members are returned in acceptance order (not sorted, not deduplicated
against nothing else), so the library's own incidence build does the sort.
"""

from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional

import numpy as np

__all__ = [
    "Hypergraph",
    "GenSpec",
    "CONFIGS",
    "planted_hypergraph",
    "coarsest_embedding",
    "random_small_hypergraph",
    "induced_subhypergraph",
]


@dataclasses.dataclass
class Hypergraph:
    """A hypergraph as hyperedge member lists (CSR over hyperedges).

    ``edge_ptr[m+1]`` (int64) and ``edge_nodes[nnz]`` (int32) list the
    members of hyperedge ``e`` in ``edge_nodes[edge_ptr[e]:edge_ptr[e+1]]``;
    ``weights[m]`` is float32; ``labels[n]`` is the planted community of each
    node (int32), or None.
    """

    n: int
    m: int
    edge_ptr: np.ndarray
    edge_nodes: np.ndarray
    weights: np.ndarray
    labels: Optional[np.ndarray] = None

    @property
    def nnz(self) -> int:
        return int(self.edge_ptr[-1])

    def members(self, e: int) -> np.ndarray:
        return self.edge_nodes[self.edge_ptr[e]:self.edge_ptr[e + 1]]


@dataclasses.dataclass(frozen=True)
class GenSpec:
    """Generator and method parameters of one named workload."""

    name: str
    n: int
    m: int
    C: int
    alpha: float
    cap: int
    p_in: float
    weighted: bool
    d: int
    sweeps: int
    min_nodes: int
    max_levels: int
    seed: int = 0


# The workloads: a small case the oracle finishes in seconds, the 1M-node
# plain-FP32 case, the 4M-node precision case, the 200K-node differentiation
# case (three coarsenings = four refined levels).
CONFIGS: Dict[str, GenSpec] = {
    "small_2k": GenSpec("small_2k", n=2_000, m=1_000, C=8, alpha=2.0, cap=50,
                        p_in=0.8, weighted=False, d=32, sweeps=10,
                        min_nodes=200, max_levels=32),
    "planted_1m": GenSpec("planted_1m", n=1_000_000, m=1_000_000, C=64,
                          alpha=1.8, cap=5_000, p_in=0.7, weighted=True,
                          d=128, sweeps=20, min_nodes=10_000, max_levels=32),
    "planted_4m": GenSpec("planted_4m", n=4_000_000, m=8_000_000, C=64,
                          alpha=1.8, cap=5_000, p_in=0.7, weighted=True,
                          d=128, sweeps=20, min_nodes=10_000, max_levels=32),
    "diff_200k": GenSpec("diff_200k", n=200_000, m=150_000, C=16, alpha=1.8,
                         cap=5_000, p_in=0.7, weighted=True, d=64, sweeps=10,
                         min_nodes=0, max_levels=3),
}


def batch_specs(count: int = 256, n_min: int = 1_000, n_max: int = 100_000,
                seed: int = 0) -> List[GenSpec]:
    """The batching workload: ``count`` independent planted-community
    hypergraphs, node counts log-uniform in [n_min, n_max] (seeded), 0.8 n
    hyperedges of size 2+Zipf(2.0) capped at 500, 8 communities, p_in 0.8,
    unit weights, d = 64, 10 sweeps per level, each coarsened down to
    max(200, n / 100) nodes."""
    rng = np.random.default_rng([seed, 0xBA7C4])
    ns = np.exp(rng.uniform(np.log(n_min), np.log(n_max), count)).astype(np.int64)
    return [GenSpec("batch_%d" % i, n=int(n), m=int(0.8 * n), C=8, alpha=2.0, cap=500,
                    p_in=0.8, weighted=False, d=64, sweeps=10,
                    min_nodes=max(200, int(n) // 100), max_levels=32,
                    seed=seed * 1_000_003 + i + 1)
            for i, n in enumerate(ns)]


def planted_features(hg: Hypergraph, k: int, sigma: float = 1.0, seed: int = 0) -> np.ndarray:
    """Node features for feature-based coarsening: planted-community
    Gaussians. Each community c draws a centre mu_c ~ N(0, I_k); node v gets
    mu_{label(v)} + sigma * N(0, I_k). float32 [n, k]. Seeded."""
    if hg.labels is None:
        raise ValueError("planted features need community labels")
    rng = np.random.default_rng([seed, 0xFEA7])
    C = int(hg.labels.max()) + 1 if hg.n else 0
    mu = rng.standard_normal((C, k))
    noise = rng.standard_normal((hg.n, k))
    return (mu[hg.labels] + sigma * noise).astype(np.float32)


def _first_occurrences(keys: np.ndarray) -> np.ndarray:
    """Indices of the first occurrence of each distinct value of ``keys``."""
    order = np.argsort(keys, kind="stable")
    sk = keys[order]
    first = np.ones(sk.size, dtype=bool)
    first[1:] = sk[1:] != sk[:-1]
    return order[first]


def _draw_members(rng, n, m, sizes, home, comm, C, p_in):
    """Member draws (step 5 of the draw order). Returns (eid, node) in
    acceptance order."""
    comm_nodes = np.argsort(comm, kind="stable").astype(np.int64)
    comm_count = np.bincount(comm, minlength=C).astype(np.int64)
    comm_start = np.concatenate([[0], np.cumsum(comm_count)[:-1]])

    need = sizes.astype(np.int64).copy()
    acc_keys = np.empty(0, dtype=np.int64)      # eid * n + node, accepted
    acc_eid = []
    acc_node = []
    while True:
        live = np.nonzero(need > 0)[0]
        if live.size == 0:
            break
        eid = np.repeat(live, need[live])
        u = rng.random(eid.size)
        r = rng.random(eid.size)
        h = home[eid]
        csize = comm_count[h]
        inside = (u < p_in) & (csize > 0)
        pos_in = np.minimum((r * csize).astype(np.int64), np.maximum(csize - 1, 0))
        pos_all = np.minimum((r * n).astype(np.int64), n - 1)
        node = np.where(inside, comm_nodes[np.minimum(comm_start[h] + pos_in, n - 1)], pos_all)
        keys = eid * n + node
        # first occurrence within this round ...
        keep = np.zeros(keys.size, dtype=bool)
        keep[_first_occurrences(keys)] = True
        # ... and not already accepted in an earlier round
        if acc_keys.size:
            pos = np.minimum(np.searchsorted(acc_keys, keys), acc_keys.size - 1)
            keep &= acc_keys[pos] != keys
        acc_eid.append(eid[keep])
        acc_node.append(node[keep])
        acc_keys = np.sort(np.concatenate([acc_keys, keys[keep]]))
        need -= np.bincount(eid[keep], minlength=m)
    eids = np.concatenate(acc_eid) if acc_eid else np.empty(0, np.int64)
    nodes = np.concatenate(acc_node) if acc_node else np.empty(0, np.int64)
    order = np.argsort(eids, kind="stable")          # acceptance order within e
    return eids[order], nodes[order]


def planted_hypergraph(n: int, m: int, C: int, alpha: float, cap: int,
                       p_in: float, weighted: bool, seed: int = 0,
                       clean: bool = True) -> Hypergraph:
    """Draw a planted-community hypergraph (see the module docstring)."""
    if n < 1 or m < 0 or C < 1:
        raise ValueError("need n >= 1, m >= 0, C >= 1")
    rng = np.random.default_rng(seed)
    comm = (rng.permutation(n) % C).astype(np.int64)
    sizes = np.minimum(np.minimum(cap, 2 + rng.zipf(alpha, m)), n).astype(np.int64)
    home = rng.integers(0, C, m).astype(np.int64)
    if weighted:
        weights = rng.uniform(0.5, 2.0, m).astype(np.float32)
    else:
        weights = np.ones(m, dtype=np.float32)
    eid, node = _draw_members(rng, n, m, sizes, home, comm, C, p_in)
    counts = np.bincount(eid, minlength=m)
    ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    hg = Hypergraph(n=n, m=m, edge_ptr=ptr, edge_nodes=node.astype(np.int32),
                    weights=weights, labels=comm.astype(np.int32))
    return clean_hypergraph(hg) if clean else hg


def clean_hypergraph(hg: Hypergraph) -> Hypergraph:
    """Dataset cleaning of the paper's evaluation: drop hyperedges with fewer
    than two distinct members, then nodes in no hyperedge; relabel both in
    ascending original ID. Member order within a hyperedge is preserved."""
    m = hg.m
    counts = np.diff(hg.edge_ptr)
    eid = np.repeat(np.arange(m, dtype=np.int64), counts)
    keys = eid * max(hg.n, 1) + hg.edge_nodes.astype(np.int64)
    distinct = np.bincount(eid[_first_occurrences(keys)], minlength=m)
    keep_e = distinct >= 2
    keep_inc = keep_e[eid]
    eid_k = eid[keep_inc]
    node_k = hg.edge_nodes[keep_inc].astype(np.int64)
    used = np.zeros(hg.n, dtype=bool)
    used[node_k] = True
    new_node = np.cumsum(used) - 1
    new_e = np.cumsum(keep_e) - 1
    m2 = int(keep_e.sum())
    n2 = int(used.sum())
    counts2 = np.bincount(new_e[eid_k], minlength=m2)
    ptr2 = np.concatenate([[0], np.cumsum(counts2)]).astype(np.int64)
    labels = hg.labels[used] if hg.labels is not None else None
    return Hypergraph(n=n2, m=m2, edge_ptr=ptr2,
                      edge_nodes=new_node[node_k].astype(np.int32),
                      weights=hg.weights[keep_e].astype(np.float32),
                      labels=labels)


def generate(spec: GenSpec) -> Hypergraph:
    """The hypergraph of a named workload."""
    return planted_hypergraph(spec.n, spec.m, spec.C, spec.alpha, spec.cap,
                              spec.p_in, spec.weighted, seed=spec.seed)


def coarsest_embedding(rows: int, d: int, seed: int = 0) -> np.ndarray:
    """Seeded N(0,1) embedding of the coarsest level, rounded to float32.

    Stands in for the initial embedding method run on the coarsest star
    expansion (Section 3.2). Rows are the coarsest nodes first, then its
    hyperedges. Stream: ``default_rng([seed, 0x5eed])``.
    """
    rng = np.random.default_rng([seed, 0x5EED])
    return rng.standard_normal((rows, d)).astype(np.float32)


def random_small_hypergraph(rng: np.random.Generator, n: int, m: int,
                            max_size: int, weighted: bool = False,
                            allow_dups: bool = False) -> Hypergraph:
    """A tiny random hypergraph (no cleaning): every hyperedge is a
    non-empty set of members in random order; with ``allow_dups`` a member
    may be repeated (the library must deduplicate)."""
    ptr = [0]
    nodes = []
    for _ in range(m):
        s = int(rng.integers(1, min(max_size, n) + 1))
        mem = list(rng.choice(n, size=s, replace=False))
        if allow_dups and s > 0 and rng.random() < 0.3:
            mem.append(mem[int(rng.integers(0, len(mem)))])
        rng.shuffle(mem)
        nodes.extend(int(x) for x in mem)
        ptr.append(len(nodes))
    w = (rng.uniform(0.5, 2.0, m) if weighted else np.ones(m)).astype(np.float32)
    return Hypergraph(n=n, m=m, edge_ptr=np.array(ptr, dtype=np.int64),
                      edge_nodes=np.array(nodes, dtype=np.int32), weights=w)


def induced_subhypergraph(hg: Hypergraph, keep_nodes: int, seed: int = 0) -> Hypergraph:
    """Restriction to ``keep_nodes`` nodes chosen by a seeded permutation:
    hyperedges keep only their chosen members, then the dataset cleaning
    runs again. Used to run the oracle on a subsample of a large workload."""
    rng = np.random.default_rng([seed, 0x5AB])
    chosen = np.zeros(hg.n, dtype=bool)
    chosen[rng.permutation(hg.n)[:keep_nodes]] = True
    counts = np.diff(hg.edge_ptr)
    eid = np.repeat(np.arange(hg.m, dtype=np.int64), counts)
    inc = chosen[hg.edge_nodes]
    counts2 = np.bincount(eid[inc], minlength=hg.m)
    sub = Hypergraph(n=hg.n, m=hg.m,
                     edge_ptr=np.concatenate([[0], np.cumsum(counts2)]).astype(np.int64),
                     edge_nodes=hg.edge_nodes[inc], weights=hg.weights, labels=hg.labels)
    return clean_hypergraph(sub)
