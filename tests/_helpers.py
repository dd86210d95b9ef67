"""Shared helpers of the test-suite (comparisons, builders). Not a test file."""

import numpy as np

import hypergen
from oracle import hnv_oracle as O

# Parity bar for float32 embeddings against the float64 oracle: per level,
# max over rows u of ||z_gpu,u - z_ref,u||_inf / max(||z_ref,u||_inf,
# 1e-3 * rms(z_ref)). The floor keeps the ratio meaningful on rows that are
# nearly zero.
FP32_TOL = 1e-5


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.size == 0:
        return 0.0
    rms = float(np.sqrt(np.mean(ref * ref)))
    den = np.maximum(np.abs(ref).max(axis=1), 1e-3 * rms)
    den = np.maximum(den, 1e-30)
    return float((np.abs(got - ref).max(axis=1) / den).max())


def oracle_level0(hg):
    return O.build_level(hg.n, hg.m, hg.edge_ptr, hg.edge_nodes, hg.weights)


def csr_lists(ptr, idx):
    return [idx[ptr[i]:ptr[i + 1]].tolist() for i in range(len(ptr) - 1)]


def gpu_level_arrays(G, level):
    import paper_2103_09660_gb300 as H
    return {
        "e_ptr": G.level_array(level, H.ARR_E_PTR),
        "e_nodes": G.level_array(level, H.ARR_E_NODES),
        "v_ptr": G.level_array(level, H.ARR_V_PTR),
        "v_edges": G.level_array(level, H.ARR_V_EDGES),
        "w": G.level_array(level, H.ARR_W),
        "deg_v": G.level_array(level, H.ARR_DEG_V),
    }


def assert_level_equal(G, level, lv):
    """Bit-exact comparison of one level's integer arrays and weights."""
    a = gpu_level_arrays(G, level)
    n, m, nnz = G.level_info(level)
    assert (n, m, nnz) == (lv.n, lv.m, lv.nnz), (level, (n, m, nnz), (lv.n, lv.m, lv.nnz))
    np.testing.assert_array_equal(a["e_ptr"], lv.e_ptr)
    np.testing.assert_array_equal(a["e_nodes"], lv.e_nodes)
    np.testing.assert_array_equal(a["v_ptr"], lv.v_ptr)
    np.testing.assert_array_equal(a["v_edges"], lv.v_edges)
    np.testing.assert_array_equal(a["w"], lv.w32)
    np.testing.assert_allclose(a["deg_v"], lv.deg_v(), rtol=2e-6, atol=0)


def assert_hierarchy_equal(G, h):
    import paper_2103_09660_gb300 as H
    assert G.num_levels == len(h.levels)
    for ell, lv in enumerate(h.levels):
        assert_level_equal(G, ell, lv)
        if ell + 1 < len(h.levels):
            np.testing.assert_array_equal(G.level_array(ell, H.ARR_REP_V), h.rep_v[ell])
            np.testing.assert_array_equal(G.level_array(ell, H.ARR_REP_E), h.rep_e[ell])


def small_cases(seed, count, n_max=40, m_max=30, size_max=8):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        n = int(rng.integers(1, n_max + 1))
        m = int(rng.integers(1, m_max + 1))
        yield hypergen.random_small_hypergraph(rng, n, m, max_size=size_max,
                                               weighted=bool(rng.integers(0, 2)),
                                               allow_dups=True)
