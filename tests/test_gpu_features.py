"""Feature-based coarsening (HNV_ASSIGN_COSINE, Section 3.1) against the
oracle: the hierarchy (every integer array) and every level's node
features must be equal bit for bit. The cosines decide an argmax, so both
sides take every float32 step with the same rounding (see hnv.h)."""

import numpy as np
import pytest

import hypergen
from oracle import hnv_oracle as O

from _helpers import assert_hierarchy_equal, oracle_level0, small_cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2103_09660_gb300 import build
    build.build()
    import paper_2103_09660_gb300 as mod
    import torch
    assert torch.cuda.is_available()
    return mod


def _check(H, hg, X, **kw):
    h = O.coarsen(oracle_level0(hg), O.CoarsenParams(policy=O.ASSIGN_COSINE, features=X, **kw))
    with H.Graph.from_hypergraph(hg) as G:
        G.set_node_features(X)
        G.coarsen(policy=H.ASSIGN_COSINE, **kw)
        assert_hierarchy_equal(G, h)
        for ell, F in enumerate(h.features):
            np.testing.assert_array_equal(G.level_features(ell), F)
    return h


def test_hand_worked_example(H):
    X = np.array([[1, 0], [1, 0], [1, 0], [0, 1], [0, 1], [0, 1]], dtype=np.float32)
    edges = [[0, 1, 2], [2, 3], [3, 4, 5], [1, 4]]
    hg = hypergen.Hypergraph(n=6, m=4, edge_ptr=np.array([0, 3, 5, 8, 10], dtype=np.int64),
                             edge_nodes=np.concatenate(edges).astype(np.int32),
                             weights=np.ones(4, dtype=np.float32))
    h = _check(H, hg, X, min_nodes=1, max_levels=1)
    assert h.rep_v[0].tolist() == [0, 0, 0, 1, 1, 1]


@pytest.mark.parametrize("k", [1, 3, 8, 32])
def test_random_small_graphs(H, k):
    for case, hg in enumerate(small_cases(20 + k, 30, n_max=60, m_max=50, size_max=9)):
        rng = np.random.default_rng(case)
        X = rng.standard_normal((hg.n, k)).astype(np.float32)
        if case % 5 == 0:
            X[rng.integers(0, hg.n)] = 0.0          # a zero-norm node
        if case % 7 == 0:
            X = np.round(X)                         # many exact ties
        _check(H, hg, X, min_nodes=2, seed=case)


def test_small_workload_planted_features(H):
    spec = hypergen.CONFIGS["small_2k"]
    hg = hypergen.generate(spec)
    for k, sigma in ((16, 0.5), (64, 2.0)):
        _check(H, hg, hypergen.planted_features(hg, k, sigma=sigma, seed=k),
               min_nodes=spec.min_nodes)


def test_mid_size(H):
    hg = hypergen.planted_hypergraph(50_000, 40_000, C=16, alpha=1.8, cap=5000, p_in=0.7,
                                     weighted=True, seed=7)
    X = hypergen.planted_features(hg, 24, sigma=1.0, seed=7)
    _check(H, hg, X, min_nodes=500, max_levels=4)


def test_hub_node_takes_the_long_row_path(H):
    """A node in 6,000 hyperedges: its assignment runs in the block-per-row
    kernel (rows longer than 4,096 incidences)."""
    rng = np.random.default_rng(3)
    n = 8000
    edges = [[0, i, i + 1] for i in range(1, 6001)]
    edges += [sorted(rng.choice(np.arange(1, n), 4, replace=False).tolist()) for _ in range(3000)]
    ptr = np.concatenate([[0], np.cumsum([len(e) for e in edges])]).astype(np.int64)
    hg = hypergen.Hypergraph(n=n, m=len(edges), edge_ptr=ptr,
                             edge_nodes=np.concatenate(edges).astype(np.int32),
                             weights=np.ones(len(edges), dtype=np.float32))
    X = rng.standard_normal((n, 12)).astype(np.float32)
    h = _check(H, hg, X, min_nodes=100, max_levels=3)
    assert int(np.diff(h.levels[0].v_ptr).max()) > 4096


def test_feature_errors(H):
    hg = hypergen.random_small_hypergraph(np.random.default_rng(0), 10, 5, 4)
    with H.Graph.from_hypergraph(hg) as G:
        with pytest.raises(H.HNVError) as ei:
            G.coarsen(policy=H.ASSIGN_COSINE, min_nodes=1)
        assert ei.value.code == -8                   # no features yet
        for bad in (np.full((10, 3), np.nan, dtype=np.float32),
                    np.full((10, 3), 3e15, dtype=np.float32)):
            with pytest.raises(H.HNVError) as ei:
                G.set_node_features(bad)
            assert ei.value.code == -1
        with pytest.raises(H.HNVError) as ei:
            G.level_features(0)
        assert ei.value.code == -8
        G.set_node_features(np.ones((10, 3), dtype=np.float32))
        np.testing.assert_array_equal(G.level_features(0), np.ones((10, 3), dtype=np.float32))
