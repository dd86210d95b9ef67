"""Full-size parity on the 1M-node workload that bench.py times.

* The whole hierarchy (5 levels: CSR, CSC, weights, rep maps) bit-exact
  against the oracle's.
* One two-phase sweep of every level from the same seeded float32 rows,
  compared with the oracle's float64 sweep on every row.
* The whole V-cycle (20 sweeps on each of the 5 levels, d = 128) element by
  element against the oracle's float64 V-cycle on every level, the oracle
  run over column blocks in worker processes; hnv_vcycle's output equals
  the level-by-level result bit for bit.
* Properties of the full V-cycle at this size: a constant embedding is a
  fixed point of projection and refinement, and two runs are bitwise equal.
"""

import numpy as np
import pytest

import hypergen
from oracle import hnv_oracle as O

from _helpers import (FP32_TOL, assert_bf16_close, assert_hierarchy_equal, bf16_errors,
                      oracle_level0, oracle_vcycle_columns, rel_err)

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def H():
    from paper_2103_09660_gb300 import build
    build.build()
    import paper_2103_09660_gb300 as mod
    import torch
    assert torch.cuda.is_available()
    return mod


@pytest.fixture(scope="module")
def workload():
    spec = hypergen.CONFIGS["planted_1m"]
    hg = hypergen.generate(spec)
    h = O.coarsen(oracle_level0(hg), O.CoarsenParams(min_nodes=spec.min_nodes,
                                                     max_levels=spec.max_levels, seed=spec.seed))
    return spec, hg, h


def test_fullsize_hierarchy_and_one_sweep_per_level(H, workload):
    import torch
    spec, hg, h = workload
    with H.Graph.from_hypergraph(hg, on_device=True) as G:
        G.coarsen(min_nodes=spec.min_nodes, max_levels=spec.max_levels, seed=spec.seed)
        assert_hierarchy_equal(G, h)
        for ell, lv in enumerate(h.levels):
            z = hypergen.coarsest_embedding(lv.n + lv.m, spec.d, seed=100 + ell)
            zv = torch.from_numpy(z[:lv.n]).cuda()
            ze = torch.from_numpy(z[lv.n:]).cuda()
            G.refine(ell, zv, ze, 0.5, 1)
            rv, re = O.refine(lv, z[:lv.n], z[lv.n:], 0.5, 1)
            torch.cuda.synchronize()
            ev = rel_err(zv.double().cpu().numpy(), rv)
            ee = rel_err(ze.double().cpu().numpy(), re)
            assert ev < FP32_TOL and ee < FP32_TOL, (ell, ev, ee)


def test_fullsize_vcycle_against_fp64_oracle(H, workload, tmp_path):
    """The V-cycle bench.py times, compared on every element of every level."""
    import torch
    spec, hg, h = workload
    top = h.levels[-1]
    zc = hypergen.coarsest_embedding(top.n + top.m, spec.d, seed=spec.seed)
    with H.Graph.from_hypergraph(hg, on_device=True) as G:
        G.coarsen(min_nodes=spec.min_nodes, max_levels=spec.max_levels, seed=spec.seed)
        zcd = torch.from_numpy(zc).cuda()
        per = _levels_on_gpu(H, G, zcd, spec.sweeps)
        zv = torch.empty((hg.n, spec.d), device="cuda")
        ze = torch.empty((hg.m, spec.d), device="cuda")
        G.vcycle(zcd, zv, ze, 0.5, spec.sweeps)
        G.sync_status()
        assert torch.equal(torch.cat([zv, ze]), per[0])
        got = [p.cpu() for p in per]
        del per, zv, ze
    ref = oracle_vcycle_columns(h, zc, 0.5, spec.sweeps, str(tmp_path))
    for l in range(len(h.levels)):
        r = ref(l)
        err = rel_err(got[l].double().numpy(), r)
        print("level %d: rows %d, max row-relative error %.2e" % (l, r.shape[0], err))
        assert err < FP32_TOL, (l, err)


def test_fullsize_vcycle_properties(H, workload):
    import torch
    spec, hg, h = workload
    top = h.levels[-1]
    with H.Graph.from_hypergraph(hg, on_device=True) as G:
        G.coarsen(min_nodes=spec.min_nodes, max_levels=spec.max_levels, seed=spec.seed)
        zv = torch.empty((hg.n, spec.d), device="cuda")
        ze = torch.empty((hg.m, spec.d), device="cuda")
        # fixed point: constant rows stay constant through every level
        zc = torch.full((top.n + top.m, spec.d), 0.625, device="cuda")
        G.vcycle(zc, zv, ze, 0.5, spec.sweeps)
        torch.cuda.synchronize()
        assert float((zv - 0.625).abs().max()) < 1e-5
        assert float((ze - 0.625).abs().max()) < 1e-5
        # determinism: the seeded V-cycle twice, bitwise equal
        zc = torch.from_numpy(hypergen.coarsest_embedding(top.n + top.m, spec.d, seed=0)).cuda()
        G.vcycle(zc, zv, ze, 0.5, spec.sweeps)
        a_v, a_e = zv.clone(), ze.clone()
        G.vcycle(zc, zv, ze, 0.5, spec.sweeps)
        torch.cuda.synchronize()
        assert torch.equal(a_v, zv) and torch.equal(a_e, ze)
        # every output row is finite and inside the range of the seed rows
        # (each update is a convex combination: maximum principle)
        lo, hi = float(zc.min()), float(zc.max())
        assert float(zv.min()) >= lo and float(zv.max()) <= hi
        assert float(ze.min()) >= lo and float(ze.max()) <= hi


# ---------------------------------------------------------------------------
# BF16 storage at the 4M-node / 8M-hyperedge size: the FP64 oracle runs on a
# 250,000-node induced sub-hypergraph drawn from the same seed
# ---------------------------------------------------------------------------

def _oracle_vcycle_cols(args):
    """Oracle V-cycle of a block of embedding columns (refinement treats every
    column independently, so column blocks are independent computations),
    exact and with bfloat16 storage."""
    arrays, params, zc_block, sweeps = args
    n, m, ptr, nodes, w = arrays
    h = O.coarsen(O.build_level(n, m, ptr, nodes, w), O.CoarsenParams(**params))
    res = O.vcycle(h, zc_block, 0.5, sweeps, keep_levels=True)
    r16 = O.vcycle(h, zc_block, 0.5, sweeps, keep_levels=True, storage=O.STORAGE_BF16)
    return [np.vstack(p) for p in res.per_level], [np.vstack(p) for p in r16.per_level]


def _levels_on_gpu(H, G, zc, sweeps):
    import torch
    L = G.num_levels - 1
    sizes = [G.level_info(l) for l in range(L + 1)]
    out = [None] * (L + 1)
    n = sizes[L][0]
    z = zc.clone()
    G.refine(L, z[:n], z[n:], 0.5, sweeps)
    out[L] = z
    for l in range(L - 1, -1, -1):
        n, m, _ = sizes[l]
        zf = torch.empty((n + m, zc.shape[1]), dtype=zc.dtype, device=zc.device)
        nc = sizes[l + 1][0]
        G.project(l, out[l + 1][:nc], out[l + 1][nc:], zf[:n], zf[n:])
        G.refine(l, zf[:n], zf[n:], 0.5, sweeps)
        out[l] = zf
    G.sync_status()
    return out


def test_fullsize_bf16_subsample_against_fp64(H):
    import multiprocessing as mp
    import os
    import torch
    spec = hypergen.CONFIGS["planted_4m"]
    hg = hypergen.generate(spec)
    sub = hypergen.induced_subhypergraph(hg, 250_000, seed=spec.seed)
    del hg
    params = dict(min_nodes=spec.min_nodes, max_levels=spec.max_levels, seed=spec.seed)
    with H.Graph.from_hypergraph(sub, on_device=True) as G:
        L = G.coarsen(**params)
        nL, mL, _ = G.level_info(L - 1)
        zc = torch.from_numpy(hypergen.coarsest_embedding(nL + mL, spec.d, seed=spec.seed))
        zc = zc.to(torch.bfloat16).float()          # both precisions start here
        z32 = _levels_on_gpu(H, G, zc.cuda(), spec.sweeps)
        z16 = _levels_on_gpu(H, G, zc.cuda().to(torch.bfloat16), spec.sweeps)
        blocks = max(1, min(16, os.cpu_count() or 1))
        cols = np.array_split(np.arange(spec.d), blocks)
        arrays = (sub.n, sub.m, sub.edge_ptr, sub.edge_nodes, sub.weights)
        with mp.get_context("spawn").Pool(blocks) as pool:
            parts = pool.map(_oracle_vcycle_cols, [(arrays, params, zc.numpy()[:, c].astype(np.float64),
                                                    spec.sweeps) for c in cols])
        M = float(zc.abs().max())
        for l in range(L):
            ref = torch.from_numpy(np.hstack([p[0][l] for p in parts])).cuda()
            ref16 = np.hstack([p[1][l] for p in parts])
            e32 = float((z32[l].double() - ref).abs().max()) / M
            e16 = float((z16[l].double() - ref).abs().max()) / M
            got16 = z16[l].double().cpu().numpy()
            p_max, p_rms = bf16_errors(got16, ref16)
            half_sweeps = 2 * spec.sweeps * (L - l)           # along the path to level l
            print("level %d: fp32 %.2e  bf16 vs fp64 %.4f (bar %.3f)  bf16 vs bf16-storage "
                  "oracle: max %.2e rms %.2e" % (l, e32, e16, half_sweeps * 2.0 ** -8, p_max, p_rms))
            assert e32 < 1e-5
            assert_bf16_close(got16, ref16, ("level", l))
            assert e16 <= half_sweeps * 2.0 ** -8


# ---------------------------------------------------------------------------
# Gradients at the 200K-node differentiation size: the FP64 oracle's adjoint
# and central differences (h = 1e-3) of the FP64 oracle's forward map
# ---------------------------------------------------------------------------

def _oracle_fwd_cols(args):
    arrays, params, w0, zc_block, omega, sweeps = args
    n, m, ptr, nodes, w = arrays
    h = O.coarsen(O.build_level(n, m, ptr, nodes, w), O.CoarsenParams(**params))
    return O.vcycle(O.with_weights(h, w0), zc_block, omega, sweeps).z_v


def _oracle_grad_cols(args):
    arrays, params, w0, zc_block, gv_block, omega, sweeps = args
    n, m, ptr, nodes, w = arrays
    h = O.coarsen(O.build_level(n, m, ptr, nodes, w), O.CoarsenParams(**params))
    return O.vcycle_grad(O.with_weights(h, w0), zc_block, omega, sweeps, gv_block,
                         np.zeros((m, gv_block.shape[1])))


def _ce(z_sub, head, labels):
    logits = z_sub @ head
    logits = logits - logits.max(axis=1, keepdims=True)
    p = np.exp(logits)
    p /= p.sum(axis=1, keepdims=True)
    loss = -np.log(p[np.arange(len(labels)), labels]).mean()
    p[np.arange(len(labels)), labels] -= 1.0
    return loss, (p / len(labels)) @ head.T


def test_fullsize_gradient_against_fp64(H):
    import multiprocessing as mp
    import os
    import torch
    spec = hypergen.CONFIGS["diff_200k"]
    hg = hypergen.generate(spec)
    params = dict(min_nodes=spec.min_nodes, max_levels=spec.max_levels, seed=spec.seed)
    om, k, d = 0.5, spec.sweeps, spec.d
    classes = int(hg.labels.max()) + 1
    gen = torch.Generator().manual_seed(spec.seed)
    head = torch.randn(d, classes, generator=gen, dtype=torch.float64) / d ** 0.5
    sub = torch.randperm(hg.n, generator=gen)[: hg.n // 10]
    labels = torch.from_numpy(hg.labels.astype(np.int64))[sub]
    with H.Graph.from_hypergraph(hg, on_device=True) as G:
        L = G.coarsen(**params)
        assert L == 4
        nL, mL, _ = G.level_info(L - 1)
        zc = torch.from_numpy(hypergen.coarsest_embedding(nL + mL, d, seed=spec.seed)).cuda()
        w = torch.from_numpy(hg.weights.copy()).cuda().requires_grad_(True)
        z = zc.clone().requires_grad_(True)
        zv, _ = H.vcycle_autograd(G, w, z, om, k)
        torch.nn.functional.cross_entropy(zv[sub.cuda()] @ head.float().cuda(),
                                          labels.cuda()).backward()
        G.sync_status()
        gw, gz = w.grad.double().cpu().numpy(), z.grad.double().cpu().numpy()
    blocks = max(1, min(16, os.cpu_count() or 1))
    cols = np.array_split(np.arange(d), blocks)
    arrays = (hg.n, hg.m, hg.edge_ptr, hg.edge_nodes, hg.weights)
    w64 = hg.weights.astype(np.float64)
    zc64 = zc.double().cpu().numpy()
    sub_np, head_np, lab_np = sub.numpy(), head.numpy(), labels.numpy()
    with mp.get_context("spawn").Pool(blocks) as pool:
        zv64 = np.hstack(pool.map(_oracle_fwd_cols, [(arrays, params, w64, zc64[:, c], om, k)
                                                     for c in cols]))
        _, gsub = _ce(zv64[sub_np], head_np, lab_np)
        gv64 = np.zeros_like(zv64)
        gv64[sub_np] = gsub
        grads = pool.map(_oracle_grad_cols, [(arrays, params, w64, zc64[:, c], gv64[:, c], om, k)
                                             for c in cols])
        dw64 = sum(g[0] for g in grads)
        dz64 = np.hstack([g[1] for g in grads])
        ew = np.abs(gw - dw64).max() / np.abs(dw64).max()
        ez = np.abs(gz - dz64).max() / np.abs(dz64).max()
        print("gradient vs FP64 oracle adjoint: weights %.2e, coarsest rows %.2e" % (ew, ez))
        assert ew < 1e-4 and ez < 1e-4

        # central differences of the oracle's forward map, h = 1e-3
        def loss64(wv, zz, col=None):
            if col is None:
                zvv = np.hstack(pool.map(_oracle_fwd_cols, [(arrays, params, wv, zz[:, c], om, k)
                                                            for c in cols]))
            else:
                zvv = zv64.copy()
                zvv[:, col] = _oracle_fwd_cols((arrays, params, wv, zz[:, [col]], om, k))[:, 0]
            return _ce(zvv[sub_np], head_np, lab_np)[0]

        hfd = 1e-3
        for j in np.argsort(-np.abs(gw))[:2]:
            e = np.zeros_like(w64)
            e[j] = hfd
            fd = (loss64(w64 + e, zc64) - loss64(w64 - e, zc64)) / (2 * hfd)
            print("w[%d]: gpu %.6e  oracle fd %.6e" % (j, gw[j], fd))
            assert abs(gw[j] - fd) <= 1e-3 * abs(fd)
        for flat in np.argsort(-np.abs(gz).ravel())[:2]:
            i, c = divmod(int(flat), d)
            e = np.zeros_like(zc64)
            e[i, c] = hfd
            fd = (loss64(w64, zc64 + e, c) - loss64(w64, zc64 - e, c)) / (2 * hfd)
            print("zc[%d,%d]: gpu %.6e  oracle fd %.6e" % (i, c, gz[i, c], fd))
            assert abs(gz[i, c] - fd) <= 1e-3 * abs(fd)
