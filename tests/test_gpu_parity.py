"""GPU path vs the CPU FP64 oracle, through the C ABI (libhnv.so).

Bars: integer work (incidence build, coarsening, rep maps) bit-exact;
projection bitwise; float32 refinement within FP32_TOL of the float64 oracle
(metric in tests/_helpers.py).
"""

import numpy as np
import pytest

import hypergen
from oracle import hnv_oracle as O

from _helpers import (FP32_TOL, assert_hierarchy_equal, assert_level_equal, oracle_level0,
                      rel_err, small_cases)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2103_09660_gb300 import build
    build.build()
    import paper_2103_09660_gb300 as mod
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return mod


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _np(t):
    import torch
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def _ok(G):
    """No device-side wait of the graph's kernels gave up."""
    G.sync_status()


# ---------------------------------------------------------------------------
# Incidence build and coarsening: bit-exact
# ---------------------------------------------------------------------------

def test_build_incidence_small_random(H):
    for hg in small_cases(1, 40):
        lv = oracle_level0(hg)
        for on_dev in (False, True):
            with H.Graph.from_hypergraph(hg, on_device=on_dev) as G:
                assert_level_equal(G, 0, lv)


def test_build_without_weights_means_unit(H):
    hg = next(small_cases(2, 1))
    with H.Graph(hg.n, hg.m, hg.edge_ptr, hg.edge_nodes, None) as G:
        np.testing.assert_array_equal(G.level_array(0, H.ARR_W), np.ones(hg.m, np.float32))


@pytest.mark.parametrize("policy", [0, 1, 2])
def test_coarsen_random_small_all_policies(H, policy):
    for i, hg in enumerate(small_cases(10 + policy, 30)):
        lv = oracle_level0(hg)
        h = O.coarsen(lv, O.CoarsenParams(policy=policy, seed=i, min_nodes=1, max_levels=8))
        with H.Graph.from_hypergraph(hg) as G:
            G.coarsen(policy=policy, seed=i, min_nodes=1, max_levels=8)
            assert_hierarchy_equal(G, h)


def test_coarsen_hand_worked_example(H):
    import os
    from test_oracle_pins import _parse_golden
    g = _parse_golden(os.path.join(os.path.dirname(__file__), "golden",
                                   "coarsen_worked_example.txt"))
    ptr = [0]
    nodes = []
    for e in range(g["m"]):
        nodes += g["edges"][e]
        ptr.append(len(nodes))
    tab = np.zeros((8, g["m"]), dtype=np.uint64)
    for (ell, e), p in g["prio"].items():
        tab[ell, e] = p
    lv0 = O.build_level(g["n"], g["m"], ptr, nodes)
    h = O.coarsen(lv0, O.CoarsenParams(policy=O.ASSIGN_EXPLICIT, min_nodes=0, max_levels=8,
                                       explicit_prio=tab))
    with H.Graph(g["n"], g["m"], np.array(ptr, np.int64), np.array(nodes, np.int32)) as G:
        L = G.coarsen(policy=H.ASSIGN_EXPLICIT, min_nodes=0, max_levels=8, explicit_prio=tab)
        assert L == 4
        assert_hierarchy_equal(G, h)
        assert G.level_array(0, H.ARR_REP_V).tolist() == g["rep_v"][0]
        assert G.level_array(1, H.ARR_REP_E).tolist() == g["rep_e"][1]


def test_coarsen_small_workload_bit_exact(H):
    spec = hypergen.CONFIGS["small_2k"]
    hg = hypergen.generate(spec)
    h = O.coarsen(oracle_level0(hg), O.CoarsenParams(min_nodes=spec.min_nodes,
                                                     max_levels=spec.max_levels))
    with H.Graph.from_hypergraph(hg, on_device=True) as G:
        G.coarsen(min_nodes=spec.min_nodes, max_levels=spec.max_levels)
        assert_hierarchy_equal(G, h)
        # coarsening again replaces the hierarchy
        G.coarsen(min_nodes=spec.min_nodes, max_levels=2)
        assert G.num_levels == 3


def test_long_rows_and_skew(H):
    """One 5000-member hyperedge, one node in 3000 hyperedges, lone nodes."""
    rng = np.random.default_rng(7)
    n, edges = 6000, []
    edges.append(rng.choice(5800, 5000, replace=False))
    for _ in range(3000):
        edges.append(np.concatenate([[5999], rng.choice(5800, 2, replace=False)]))
    ptr = np.concatenate([[0], np.cumsum([len(e) for e in edges])]).astype(np.int64)
    nodes = np.concatenate(edges).astype(np.int32)
    w = rng.uniform(0.5, 2.0, len(edges)).astype(np.float32)
    hg = hypergen.Hypergraph(n=n, m=len(edges), edge_ptr=ptr, edge_nodes=nodes, weights=w)
    lv = oracle_level0(hg)
    h = O.coarsen(lv, O.CoarsenParams(min_nodes=10, seed=3))
    import torch
    with H.Graph.from_hypergraph(hg) as G:
        G.coarsen(min_nodes=10, seed=3)
        assert_hierarchy_equal(G, h)
        for ell, lvl in enumerate(h.levels):
            for d in (8, 128):
                z = np.random.default_rng(ell).standard_normal((lvl.n + lvl.m, d)).astype(np.float32)
                zv, ze = _t(z[:lvl.n]), _t(z[lvl.n:])
                for mode in (H.SWEEP_TWO_PHASE, H.SWEEP_JACOBI):
                    a, b = zv.clone(), ze.clone()
                    G.refine(ell, a, b, 0.5, 3, mode)
                    _ok(G)
                    rv, re = O.refine(lvl, z[:lvl.n], z[lvl.n:], 0.5, 3, mode)
                    assert rel_err(_np(a), rv) < FP32_TOL
                    assert rel_err(_np(b), re) < FP32_TOL


@pytest.mark.parametrize("n", [5000, 300000])
def test_long_member_lists_with_repeats(H, n):
    """Hyperedges of 300, 1000 and 6000 members drawn with replacement (many
    repeats) among 4000 short ones, also with repeats. n = 5000 keeps the
    distinct-value bitmaps of the member and image sorts flat; n = 300000
    (most nodes alone) takes the two-level bitmap at the build and on the
    coarse levels. The hierarchy must equal the oracle's bit for bit."""
    rng = np.random.default_rng(11)
    edges = [rng.integers(0, n, size) for size in (300, 1000, 6000)]
    for _ in range(4000):
        edges.append(rng.integers(0, min(n, 20000), int(rng.integers(2, 12))))
    ptr = np.concatenate([[0], np.cumsum([len(e) for e in edges])]).astype(np.int64)
    hg = hypergen.Hypergraph(n=n, m=len(edges), edge_ptr=ptr,
                             edge_nodes=np.concatenate(edges).astype(np.int32),
                             weights=rng.uniform(0.5, 2.0, len(edges)).astype(np.float32))
    lv = oracle_level0(hg)
    h = O.coarsen(lv, O.CoarsenParams(min_nodes=100, max_levels=3, seed=5))
    for on_dev in (False, True):
        with H.Graph.from_hypergraph(hg, on_device=on_dev) as G:
            G.coarsen(min_nodes=100, max_levels=3, seed=5)
            assert_hierarchy_equal(G, h)


# ---------------------------------------------------------------------------
# Refinement and projection
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d", [4, 12, 32, 64, 128, 160, 256, 1024])
def test_refine_one_level_widths(H, d):
    spec = hypergen.CONFIGS["small_2k"]
    hg = hypergen.generate(spec)
    lv = oracle_level0(hg)
    z = np.random.default_rng(d).standard_normal((lv.n + lv.m, d)).astype(np.float32)
    with H.Graph.from_hypergraph(hg) as G:
        for mode in (H.SWEEP_TWO_PHASE, H.SWEEP_JACOBI):
            zv, ze = _t(z[:lv.n]), _t(z[lv.n:])
            G.refine(0, zv, ze, 0.5, 4, mode)
            _ok(G)
            rv, re = O.refine(lv, z[:lv.n], z[lv.n:], 0.5, 4, mode)
            assert rel_err(_np(zv), rv) < FP32_TOL
            assert rel_err(_np(ze), re) < FP32_TOL


def test_refine_random_small_graphs(H):
    for i, hg in enumerate(small_cases(20, 25)):
        lv = oracle_level0(hg)
        d = 4 * int(np.random.default_rng(i).integers(1, 20))
        z = np.random.default_rng(100 + i).standard_normal((lv.n + lv.m, d)).astype(np.float32)
        om = float(np.random.default_rng(i).uniform(0, 1))
        with H.Graph.from_hypergraph(hg) as G:
            for mode in (H.SWEEP_TWO_PHASE, H.SWEEP_JACOBI):
                zv, ze = _t(z[:lv.n]), _t(z[lv.n:])
                G.refine(0, zv, ze, om, 3, mode)
                rv, re = O.refine(lv, z[:lv.n], z[lv.n:], om, 3, mode)
                assert rel_err(_np(zv), rv) < FP32_TOL
                assert rel_err(_np(ze), re) < FP32_TOL


def test_refine_special_cases(H):
    spec = hypergen.CONFIGS["small_2k"]
    hg = hypergen.generate(spec)
    lv = oracle_level0(hg)
    d = 32
    z = np.random.default_rng(0).standard_normal((lv.n + lv.m, d)).astype(np.float32)
    with H.Graph.from_hypergraph(hg) as G:
        # omega = 0 and zero sweeps: identity, bitwise
        for om, k in ((0.0, 5), (0.5, 0)):
            zv, ze = _t(z[:lv.n]), _t(z[lv.n:])
            G.refine(0, zv, ze, om, k)
            assert np.array_equal(_np(zv), z[:lv.n]) and np.array_equal(_np(ze), z[lv.n:])
        # constant embeddings are a fixed point (unit weights: up to rounding
        # of the reciprocal degree)
        zv = _t(np.full((lv.n, d), 0.75))
        ze = _t(np.full((lv.m, d), 0.75))
        G.refine(0, zv, ze, 0.5, 10)
        assert np.abs(_np(zv) - 0.75).max() <= 4e-7 and np.abs(_np(ze) - 0.75).max() <= 4e-7
        # determinism: identical inputs give bitwise identical outputs
        outs = []
        for _ in range(2):
            zv, ze = _t(z[:lv.n]), _t(z[lv.n:])
            G.refine(0, zv, ze, 0.5, 5)
            outs.append((_np(zv), _np(ze)))
        assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_project_bitwise(H):
    spec = hypergen.CONFIGS["small_2k"]
    hg = hypergen.generate(spec)
    h = O.coarsen(oracle_level0(hg), O.CoarsenParams(min_nodes=spec.min_nodes))
    import torch
    with H.Graph.from_hypergraph(hg) as G:
        G.coarsen(min_nodes=spec.min_nodes)
        for ell in range(len(h.levels) - 1):
            f, c = h.levels[ell], h.levels[ell + 1]
            for d in (4, 36, 128):
                zc = np.random.default_rng(ell * 7 + d).standard_normal((c.n + c.m, d)).astype(np.float32)
                zf_v = torch.full((f.n, d), float("nan"), device="cuda")
                zf_e = torch.full((f.m, d), float("nan"), device="cuda")
                G.project(ell, _t(zc[:c.n]), _t(zc[c.n:]), zf_v, zf_e)
                rv, re = O.project(h.rep_v[ell], h.rep_e[ell], zc[:c.n], zc[c.n:])
                assert np.array_equal(_np(zf_v), rv) and np.array_equal(_np(zf_e), re)


@pytest.mark.parametrize("mode", [0, 1])
def test_vcycle_small_workload(H, mode):
    spec = hypergen.CONFIGS["small_2k"]
    hg = hypergen.generate(spec)
    h = O.coarsen(oracle_level0(hg), O.CoarsenParams(min_nodes=spec.min_nodes))
    top = h.levels[-1]
    zc = hypergen.coarsest_embedding(top.n + top.m, spec.d, seed=0)
    ref = O.vcycle(h, zc, 0.5, spec.sweeps, mode)
    import torch
    with H.Graph.from_hypergraph(hg, on_device=True) as G:
        G.coarsen(min_nodes=spec.min_nodes)
        zv = torch.empty((hg.n, spec.d), device="cuda")
        ze = torch.empty((hg.m, spec.d), device="cuda")
        G.vcycle(_t(zc), zv, ze, 0.5, spec.sweeps, mode)
        _ok(G)
        assert rel_err(_np(zv), ref.z_v) < FP32_TOL
        assert rel_err(_np(ze), ref.z_e) < FP32_TOL
        # host buffers: same result, copies inside the call
        hv = np.empty((hg.n, spec.d), np.float32)
        he = np.empty((hg.m, spec.d), np.float32)
        G.vcycle(np.ascontiguousarray(zc), hv, he, 0.5, spec.sweeps, mode)
        assert np.array_equal(hv, _np(zv).astype(np.float32))
        assert np.array_equal(he, _np(ze).astype(np.float32))


def test_vcycle_mid_size(H):
    hg = hypergen.planted_hypergraph(30_000, 25_000, C=16, alpha=1.8, cap=2_000, p_in=0.7,
                                     weighted=True, seed=5)
    h = O.coarsen(oracle_level0(hg), O.CoarsenParams(min_nodes=1_000))
    top = h.levels[-1]
    d = 64
    zc = hypergen.coarsest_embedding(top.n + top.m, d, seed=1)
    ref = O.vcycle(h, zc, 0.5, 8, O.SWEEP_TWO_PHASE, keep_levels=True)
    import torch
    with H.Graph.from_hypergraph(hg) as G:
        G.coarsen(min_nodes=1_000)
        assert_hierarchy_equal(G, h)
        zv = torch.empty((hg.n, d), device="cuda")
        ze = torch.empty((hg.m, d), device="cuda")
        G.vcycle(_t(zc), zv, ze, 0.5, 8)
        assert rel_err(_np(zv), ref.z_v) < FP32_TOL
        assert rel_err(_np(ze), ref.z_e) < FP32_TOL


def test_single_level_vcycle(H):
    """A graph that cannot coarsen (min_nodes above n): the V-cycle is one
    refinement of level 0 from the given embedding."""
    hg = next(small_cases(33, 1, n_max=30))
    lv = oracle_level0(hg)
    import torch
    with H.Graph.from_hypergraph(hg) as G:
        assert G.coarsen(min_nodes=10_000) == 1
        z = np.random.default_rng(1).standard_normal((lv.n + lv.m, 8)).astype(np.float32)
        zv = torch.empty((lv.n, 8), device="cuda")
        ze = torch.empty((lv.m, 8), device="cuda")
        G.vcycle(_t(z), zv, ze, 0.5, 4)
        rv, re = O.refine(lv, z[:lv.n], z[lv.n:], 0.5, 4)
        assert rel_err(_np(zv), rv) < FP32_TOL and rel_err(_np(ze), re) < FP32_TOL


# ---------------------------------------------------------------------------
# Errors: invalid input is reported, never faults
# ---------------------------------------------------------------------------

def test_error_codes(H):
    import torch
    ptr = np.array([0, 2, 4], np.int64)
    with pytest.raises(H.HNVError) as ei:
        H.Graph(3, 2, ptr, np.array([0, 1, 2, 3], np.int32))
    assert ei.value.code == -2                              # node out of range
    for on_dev in (False, True):
        args = (np.array([0, 2, 2], np.int64), np.array([0, 1], np.int32))
        if on_dev:
            args = tuple(torch.from_numpy(a).cuda() for a in args)
        with pytest.raises(H.HNVError) as ei:
            H.Graph(3, 2, *args)
        assert ei.value.code == -1                          # empty hyperedge
    with pytest.raises(H.HNVError) as ei:
        H.Graph(3, 1, np.array([0, 2], np.int64), np.array([0, 1], np.int32),
                np.array([-1.0], np.float32))
    assert ei.value.code == -1                              # bad weight
    with H.Graph(3, 2, ptr, np.array([0, 1, 1, 2], np.int32)) as G:
        zv = torch.zeros((3, 6), device="cuda")
        ze = torch.zeros((2, 6), device="cuda")
        with pytest.raises(H.HNVError) as ei:
            G.refine(0, zv, ze)
        assert ei.value.code == -7                          # d % 4 != 0
        zv = torch.zeros((3, 8), device="cuda")
        ze = torch.zeros((2, 8), device="cuda")
        with pytest.raises(H.HNVError) as ei:
            G.refine(3, zv, ze)
        assert ei.value.code == -2                          # level out of range
        with pytest.raises(H.HNVError) as ei:
            G.refine(0, zv, ze, omega=1.5)
        assert ei.value.code == -1
        with pytest.raises(H.HNVError) as ei:
            G.project(0, zv, ze, zv, ze)                    # no coarse level yet
        assert ei.value.code == -2
        L = H.lib()
        assert L.hnv_refine(G.handle, 0, zv.data_ptr(), ze.data_ptr(), H.BF16, 12, 0.5, 1, 0,
                            None) == -7                     # BF16 needs d % 8 == 0
        assert L.hnv_refine(G.handle, 0, zv.data_ptr() + 4, ze.data_ptr(), H.F32, 8, 0.5, 1, 0,
                            None) == -1                     # misaligned
    # the context is still usable after the reported errors
    hg = next(small_cases(3, 1))
    with H.Graph.from_hypergraph(hg) as G:
        assert_level_equal(G, 0, oracle_level0(hg))


def test_allocator_hook_failure_is_reported(H):
    """An allocator that fails: the call returns HNV_ERR_OOM and frees what
    it had; restoring the default allocator works again."""
    import ctypes
    L = H.lib()
    AF = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    FF = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
    fail = AF(lambda nbytes, s, ctx: None)
    nofree = FF(lambda p, s, ctx: None)
    hg = next(small_cases(4, 1))
    assert L.hnv_set_allocator(ctypes.cast(fail, ctypes.c_void_p),
                               ctypes.cast(nofree, ctypes.c_void_p), None) == 0
    try:
        with pytest.raises(H.HNVError) as ei:
            H.Graph.from_hypergraph(hg)
        assert ei.value.code == -4
    finally:
        assert L.hnv_set_allocator(None, None, None) == 0
    with H.Graph.from_hypergraph(hg) as G:
        assert_level_equal(G, 0, oracle_level0(hg))
