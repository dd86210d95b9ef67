"""BF16 embedding storage with FP32 accumulation, against the FP64 oracle.

Error bar (derived from the arithmetic, not fitted): every half-sweep
stores its rows rounded to bfloat16, an error of at most u * |value| with
u = 2^-8 (8 significant bits, round to nearest). Every update is a convex
combination of the previous values, so (maximum principle) no value leaves
[min, max] of the starting rows and the error already present is not
amplified in the max-norm. After K half-sweeps the GPU result therefore
differs from the exact result by at most K * u * M, M = max |starting
value|. Projection copies bits and adds nothing. The oracle starts from the
same bfloat16-rounded rows (promoted exactly to float64).
"""

import numpy as np
import pytest

import hypergen
from oracle import hnv_oracle as O

from _helpers import oracle_level0

pytestmark = pytest.mark.gpu
U_BF16 = 2.0 ** -8


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
            rv, re = O.refine(lv, z0[:lv.n], z0[lv.n:], 0.5, k, mode)
            M = np.abs(z0).max()
            err = max(_global_err(_f64(zv), rv, M), _global_err(_f64(ze), re, M))
            assert err <= 2 * k * U_BF16, err
            # rounding, not a systematic error: the mean error is far smaller
            mean = np.abs(np.vstack([_f64(zv), _f64(ze)]) - np.vstack([rv, re])).mean() / M
            assert mean <= U_BF16, mean


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
    with H.Graph.from_hypergraph(hg) as G:
        G.coarsen(min_nodes=spec.min_nodes)
        zv = torch.empty((hg.n, spec.d), dtype=torch.bfloat16, device="cuda")
        ze = torch.empty((hg.m, spec.d), dtype=torch.bfloat16, device="cuda")
        G.vcycle(zcb, zv, ze, 0.5, spec.sweeps)
        G.sync_status()
        K = 2 * spec.sweeps * len(h.levels)          # half-sweeps along the V-cycle
        M = np.abs(zc0).max()
        err = max(_global_err(_f64(zv), ref.z_v, M), _global_err(_f64(ze), ref.z_e, M))
        assert err <= K * U_BF16, err
        # the float32 path from the same start is within the same bar of the
        # bfloat16 one, and much closer to the oracle
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
