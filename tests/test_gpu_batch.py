"""Batched V-cycle (hnv_batch_*) against the per-graph V-cycle and the
oracle. Per row, the batched kernels sum the same incidences in the same
order as the single-graph kernels (the order does not depend on lanes per
row, row-class boundaries or the graph's position in the batch), so the
batched results equal the per-graph ones bit for bit."""

import numpy as np
import pytest

import hypergen
from oracle import hnv_oracle as O

from _helpers import FP32_TOL, oracle_level0, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2103_09660_gb300 import build
    build.build()
    import paper_2103_09660_gb300 as mod
    import torch
    assert torch.cuda.is_available()
    return mod


def _graphs(H, count, seed, weighted=True):
    rng = np.random.default_rng(seed)
    hgs, Gs = [], []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(200), np.log(6000))))
        hg = hypergen.planted_hypergraph(n, int(0.8 * n), C=8, alpha=2.0, cap=300, p_in=0.8,
                                         weighted=weighted, seed=seed * 1000 + i)
        G = H.Graph.from_hypergraph(hg)
        G.coarsen(min_nodes=max(50, hg.n // 50), seed=i)
        hgs.append(hg)
        Gs.append(G)
    return hgs, Gs


def _run_single(H, G, zc_i, d, dt, sweeps):
    import torch
    n0, m0, _ = G.level_info(0)
    zv = torch.empty((n0, d), dtype=dt, device="cuda")
    ze = torch.empty((m0, d), dtype=dt, device="cuda")
    G.vcycle(zc_i, zv, ze, 0.5, sweeps)
    return zv, ze


@pytest.mark.parametrize("dtname,d", [("f32", 32), ("f32", 64), ("bf16", 64), ("f32", 128)])
def test_batch_equals_per_graph(H, dtname, d):
    import torch
    dt = torch.float32 if dtname == "f32" else torch.bfloat16
    hgs, Gs = _graphs(H, 12, seed=3 + d)
    depths = {G.num_levels for G in Gs}
    assert len(depths) > 1            # graphs of different depth in one batch
    with H.Batch(Gs) as B:
        assert B.kernel == H.BATCH_KERNEL_PER_CLASS           # the default
        co, vo, eo = B.offsets()
        zc = torch.randn((int(co[-1]), d), device="cuda").to(dt)
        zv = torch.empty((int(vo[-1]), d), dtype=dt, device="cuda")
        ze = torch.empty((int(eo[-1]), d), dtype=dt, device="cuda")
        # both half-sweep kernels; direct launches, capture, replay, and a
        # switch back to the first kernel (re-capture)
        for kernel, use_graph in ((H.BATCH_KERNEL_PERSISTENT, False),
                                  (H.BATCH_KERNEL_PERSISTENT, True),
                                  (H.BATCH_KERNEL_PERSISTENT, True),
                                  (H.BATCH_KERNEL_PER_CLASS, False),
                                  (H.BATCH_KERNEL_PER_CLASS, True),
                                  (H.BATCH_KERNEL_PERSISTENT, True)):
            B.kernel = kernel
            zv.fill_(float("nan"))
            ze.fill_(float("nan"))
            B.vcycle(zc, zv, ze, 0.5, 4, use_cuda_graph=use_graph)
            torch.cuda.synchronize()
            for G in Gs:
                G.sync_status()          # no work item was out of bounds
            for i, G in enumerate(Gs):
                sv, se = _run_single(H, G, zc[co[i]:co[i + 1]].contiguous(), d, dt, 4)
                assert torch.equal(sv, zv[vo[i]:vo[i + 1]]) and torch.equal(se, ze[eo[i]:eo[i + 1]])
        with pytest.raises(H.HNVError):
            B.kernel = 7
    for G in Gs:
        G.close()


def test_batch_autotune_keeps_results_and_matches_oracle(H):
    import torch
    d = 64
    hgs, Gs = _graphs(H, 10, seed=11)
    with H.Batch(Gs) as B:
        co, vo, eo = B.offsets()
        zc = torch.randn((int(co[-1]), d), device="cuda")
        zv = torch.empty((int(vo[-1]), d), device="cuda")
        ze = torch.empty((int(eo[-1]), d), device="cuda")
        B.vcycle(zc, zv, ze, 0.5, 3)
        before = (zv.clone(), ze.clone())
        t = B.autotune(H.F32, d)
        assert t["a_max"] < t["b_max"] < t["c_max"] and t["lanes_a"] >= 1
        assert t["kernel"] == B.kernel and t["persistent_ms"] > 0 and t["best_ms"] > 0
        assert t["best_ms"] <= t["persistent_ms"]
        B.vcycle(zc, zv, ze, 0.5, 3)
        torch.cuda.synchronize()
        assert torch.equal(before[0], zv) and torch.equal(before[1], ze)
        t2 = B.autotune(H.F32, d)
        assert t2["from_cache"] == 1 and t2["a_max"] == t["a_max"]
        assert t2["kernel"] == t["kernel"] == B.kernel
        # two graphs against the FP64 oracle
        for i in (0, len(Gs) - 1):
            lv0 = oracle_level0(hgs[i])
            h = O.coarsen(lv0, O.CoarsenParams(min_nodes=max(50, hgs[i].n // 50), seed=i))
            ref = O.vcycle(h, zc[co[i]:co[i + 1]].double().cpu().numpy(), 0.5, 3)
            assert rel_err(zv[vo[i]:vo[i + 1]].double().cpu().numpy(), ref.z_v) < FP32_TOL
            assert rel_err(ze[eo[i]:eo[i + 1]].double().cpu().numpy(), ref.z_e) < FP32_TOL
    for G in Gs:
        G.close()


def test_batch_rejects_bad_arguments(H):
    import torch
    hgs, Gs = _graphs(H, 2, seed=5)
    with H.Batch(Gs) as B:
        co, vo, eo = B.offsets()
        zc = torch.zeros((int(co[-1]), 12), device="cuda")
        zv = torch.zeros((int(vo[-1]), 12), device="cuda")
        ze = torch.zeros((int(eo[-1]), 12), device="cuda")
        with pytest.raises(H.HNVError) as ei:
            B.vcycle(zc, zv, ze)
        assert ei.value.code == -7
    for G in Gs:
        G.close()


def _hub_graph(n, hub_edges, seed):
    """A hypergraph whose node 0 is in `hub_edges` hyperedges (a split row of
    many chunks on the node side), plus random small hyperedges."""
    rng = np.random.default_rng(seed)
    edges = [[0, 1 + (i % (n - 2)), 2 + (i % (n - 2))] for i in range(hub_edges)]
    edges += [sorted(rng.choice(np.arange(1, n), 3, replace=False).tolist()) for _ in range(n)]
    ptr = np.concatenate([[0], np.cumsum([len(e) for e in edges])]).astype(np.int64)
    return hypergen.Hypergraph(n=n, m=len(edges), edge_ptr=ptr,
                               edge_nodes=np.concatenate(edges).astype(np.int32),
                               weights=rng.uniform(0.5, 2.0, len(edges)).astype(np.float32))


@pytest.mark.parametrize("dtname,d", [("bf16", 8), ("f32", 1024)])
def test_batch_edge_shapes(H, dtname, d):
    """Width extremes (one 16-byte vector per row; 256 per row), a graph that
    is not coarsened at all next to deeper ones, a node in 9,000 hyperedges
    (split rows with many chunks), zero sweeps and omega = 0 (identity)."""
    import torch
    dt = torch.float32 if dtname == "f32" else torch.bfloat16
    hgs = [_hub_graph(3000, 9000, 1),
           hypergen.generate(hypergen.CONFIGS["small_2k"]),
           hypergen.random_small_hypergraph(np.random.default_rng(2), 30, 20, 5)]
    Gs = []
    for i, hg in enumerate(hgs):
        G = H.Graph.from_hypergraph(hg)
        G.coarsen(min_nodes=10 ** 9 if i == 2 else 100, seed=i)   # graph 2: one level
        Gs.append(G)
    assert Gs[2].num_levels == 1 and Gs[0].num_levels > 1
    with H.Batch(Gs) as B:
        co, vo, eo = B.offsets()
        zc = torch.randn((int(co[-1]), d), device="cuda").to(dt)
        zv = torch.empty((int(vo[-1]), d), dtype=dt, device="cuda")
        ze = torch.empty((int(eo[-1]), d), dtype=dt, device="cuda")
        for kernel, omega, sweeps in ((H.BATCH_KERNEL_PERSISTENT, 0.5, 3),
                                      (H.BATCH_KERNEL_PER_CLASS, 0.5, 3),
                                      (H.BATCH_KERNEL_PERSISTENT, 0.5, 0),
                                      (H.BATCH_KERNEL_PERSISTENT, 0.0, 2)):
            B.kernel = kernel
            B.vcycle(zc, zv, ze, omega, sweeps)
            torch.cuda.synchronize()
            for i, G in enumerate(Gs):
                G.sync_status()
                n0, m0, _ = G.level_info(0)
                sv = torch.empty((n0, d), dtype=dt, device="cuda")
                se = torch.empty((m0, d), dtype=dt, device="cuda")
                G.vcycle(zc[co[i]:co[i + 1]].contiguous(), sv, se, omega, sweeps)
                assert torch.equal(sv, zv[vo[i]:vo[i + 1]]) and torch.equal(se, ze[eo[i]:eo[i + 1]])
    for G in Gs:
        G.close()


def test_batch_goes_stale_when_a_graph_is_coarsened_again(H):
    import torch
    hgs, Gs = _graphs(H, 3, seed=9)
    with H.Batch(Gs) as B:
        co, vo, eo = B.offsets()
        zc = torch.zeros((int(co[-1]), 16), device="cuda")
        zv = torch.zeros((int(vo[-1]), 16), device="cuda")
        ze = torch.zeros((int(eo[-1]), 16), device="cuda")
        B.vcycle(zc, zv, ze)
        Gs[1].coarsen(min_nodes=5, seed=1)
        with pytest.raises(H.HNVError) as ei:
            B.vcycle(zc, zv, ze)
        assert ei.value.code == -8
    for G in Gs:
        G.close()
