"""BF16 embedding storage with FP32 accumulation.

Two comparisons per case:

* the pin: the oracle run with the same storage (every stored row rounded
  to bfloat16 after each relaxation, arithmetic in float64). The GPU and the
  oracle then hold values on the same bfloat16 grid and differ only where a
  float32 and a float64 sum round to neighbouring grid values; the bars
  (tests/_helpers.py: every value within 4u of the largest, RMS within u/8,
  u = 2^-8) fail for any systematic error of 1% or more;
* a sanity bound against the exact FP64 oracle: every half-sweep stores
  with an error of at most u * |value|, every update is a convex
  combination (the error present is not amplified in the max-norm), so
  after K half-sweeps the difference is at most K * u * M, M = max |start|.

Both sides start from the same bfloat16-rounded rows.
"""

import numpy as np
import pytest

import hypergen
from oracle import hnv_oracle as O

from _helpers import U_BF16, assert_bf16_close, oracle_level0

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2103_09660_gb300 import build
    build.build()
    import paper_2103_09660_gb300 as mod
    import torch
    assert torch.cuda.is_available()
    return mod


def _bf16(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).cuda()


def _f64(t):
    import torch
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def _global_err(got, ref, M):
    return float(np.abs(got - ref).max() / M)


@pytest.mark.parametrize("d", [8, 32, 128, 256])
def test_bf16_refine_one_level(H, d):
    spec = hypergen.CONFIGS["small_2k"]
    hg = hypergen.generate(spec)
    lv = oracle_level0(hg)
    k = 3
    with H.Graph.from_hypergraph(hg) as G:
        for mode in (H.SWEEP_TWO_PHASE, H.SWEEP_JACOBI):
            z = np.random.default_rng(d + mode).standard_normal((lv.n + lv.m, d)).astype(np.float32)
            zb = _bf16(z)
            z0 = _f64(zb)                              # the rounded start, exactly
            zv, ze = zb[:lv.n].clone(), zb[lv.n:].clone()
            G.refine(0, zv, ze, 0.5, k, mode)
            G.sync_status()
            got = np.vstack([_f64(zv), _f64(ze)])
            bv, be = O.refine(lv, z0[:lv.n], z0[lv.n:], 0.5, k, mode, storage=O.STORAGE_BF16)
            assert_bf16_close(got, np.vstack([bv, be]), ("one level", d, mode))
            rv, re = O.refine(lv, z0[:lv.n], z0[lv.n:], 0.5, k, mode)
            M = np.abs(z0).max()
            err = max(_global_err(_f64(zv), rv, M), _global_err(_f64(ze), re, M))
            assert err <= 2 * k * U_BF16, err


def test_bf16_split_rows_and_projection(H):
    import torch
    rng = np.random.default_rng(3)
    edges = [rng.choice(5800, 5000, replace=False)]
    for _ in range(3000):
        edges.append(np.concatenate([[5999], rng.choice(5800, 2, replace=False)]))
    ptr = np.concatenate([[0], np.cumsum([len(e) for e in edges])]).astype(np.int64)
    hg = hypergen.Hypergraph(n=6000, m=len(edges), edge_ptr=ptr,
                             edge_nodes=np.concatenate(edges).astype(np.int32),
                             weights=rng.uniform(0.5, 2.0, len(edges)).astype(np.float32))
    lv = oracle_level0(hg)
    h = O.coarsen(lv, O.CoarsenParams(min_nodes=10, seed=3))
    d = 128
    with H.Graph.from_hypergraph(hg) as G:
        G.coarsen(min_nodes=10, seed=3)
        for ell, lvl in enumerate(h.levels):
            z0 = _f64(_bf16(np.random.default_rng(ell).standard_normal((lvl.n + lvl.m, d))))
            zv, ze = _bf16(z0[:lvl.n]), _bf16(z0[lvl.n:])
            G.refine(ell, zv, ze, 0.5, 2)
            G.sync_status()
            bv, be = O.refine(lvl, z0[:lvl.n], z0[lvl.n:], 0.5, 2, storage=O.STORAGE_BF16)
            assert_bf16_close(np.vstack([_f64(zv), _f64(ze)]), np.vstack([bv, be]),
                              ("split rows", ell))
            rv, re = O.refine(lvl, z0[:lvl.n], z0[lvl.n:], 0.5, 2)
            M = np.abs(z0).max()
            assert max(_global_err(_f64(zv), rv, M), _global_err(_f64(ze), re, M)) <= 4 * U_BF16
        # projection copies bfloat16 bits
        f, c = h.levels[0], h.levels[1]
        zc = _bf16(np.random.default_rng(9).standard_normal((c.n + c.m, d)))
        zf_v = torch.zeros((f.n, d), dtype=torch.bfloat16, device="cuda")
        zf_e = torch.zeros((f.m, d), dtype=torch.bfloat16, device="cuda")
        G.project(0, zc[:c.n], zc[c.n:], zf_v, zf_e)
        rv, re = O.project(h.rep_v[0], h.rep_e[0], _f64(zc[:c.n]), _f64(zc[c.n:]))
        assert np.array_equal(_f64(zf_v), rv) and np.array_equal(_f64(zf_e), re)


def _levels_on_gpu(G, zc, sweeps):
    """The V-cycle level by level (refine the coarsest, then project and
    refine each finer level); every level's refined rows, nodes first."""
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


def test_bf16_vcycle_error_per_level_and_vs_fp32(H):
    import torch
    spec = hypergen.CONFIGS["small_2k"]
    hg = hypergen.generate(spec)
    h = O.coarsen(oracle_level0(hg), O.CoarsenParams(min_nodes=spec.min_nodes))
    top = h.levels[-1]
    zc = hypergen.coarsest_embedding(top.n + top.m, spec.d, seed=0)
    zcb = _bf16(zc)
    zc0 = _f64(zcb)
    ref = O.vcycle(h, zc0, 0.5, spec.sweeps, keep_levels=True)
    ref16 = O.vcycle(h, zc0, 0.5, spec.sweeps, keep_levels=True, storage=O.STORAGE_BF16)
    with H.Graph.from_hypergraph(hg) as G:
        G.coarsen(min_nodes=spec.min_nodes)
        # every level against the bfloat16-storage oracle
        per = _levels_on_gpu(G, zcb, spec.sweeps)
        L = len(h.levels) - 1
        M = np.abs(zc0).max()
        for l in range(L + 1):
            got = _f64(per[l])
            assert_bf16_close(got, np.vstack(ref16.per_level[l]), ("level", l))
            # sanity: within the worst-case bound of the exact oracle, which
            # grows linearly with the half-sweeps along the path to level l
            K = 2 * spec.sweeps * (L + 1 - l)
            assert _global_err(got, np.vstack(ref.per_level[l]), M) <= K * U_BF16
        zv = torch.empty((hg.n, spec.d), dtype=torch.bfloat16, device="cuda")
        ze = torch.empty((hg.m, spec.d), dtype=torch.bfloat16, device="cuda")
        G.vcycle(zcb, zv, ze, 0.5, spec.sweeps)
        G.sync_status()
        # the V-cycle entry point gives the level-by-level result bit for bit
        assert torch.equal(torch.cat([zv, ze]), per[0])
        assert_bf16_close(np.vstack([_f64(zv), _f64(ze)]), np.vstack([ref16.z_v, ref16.z_e]),
                          "vcycle")
        err = max(_global_err(_f64(zv), ref.z_v, M), _global_err(_f64(ze), ref.z_e, M))
        # the float32 path from the same start is much closer to the exact oracle
        zv32 = torch.empty((hg.n, spec.d), device="cuda")
        ze32 = torch.empty((hg.m, spec.d), device="cuda")
        G.vcycle(zcb.float(), zv32, ze32, 0.5, spec.sweeps)
        e32 = max(_global_err(_f64(zv32), ref.z_v, M), _global_err(_f64(ze32), ref.z_e, M))
        assert e32 < 1e-5 and e32 < err
        # host buffers (CPU bfloat16 tensors): same bits as the device run
        hv = torch.empty((hg.n, spec.d), dtype=torch.bfloat16)
        he = torch.empty((hg.m, spec.d), dtype=torch.bfloat16)
        G.vcycle(zcb.cpu(), hv, he, 0.5, spec.sweeps)
        assert torch.equal(hv, zv.cpu()) and torch.equal(he, ze.cpu())


def test_bf16_rejects_bad_width(H):
    import torch
    hg = hypergen.random_small_hypergraph(np.random.default_rng(0), 10, 5, 4)
    with H.Graph.from_hypergraph(hg) as G:
        zv = torch.zeros((10, 12), dtype=torch.bfloat16, device="cuda")
        ze = torch.zeros((5, 12), dtype=torch.bfloat16, device="cuda")
        with pytest.raises(H.HNVError) as ei:
            G.refine(0, zv, ze)
        assert ei.value.code == -7
