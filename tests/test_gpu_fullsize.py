"""Full-size parity on the 1M-node workload that bench.py times.

* The whole hierarchy (5 levels: CSR, CSC, weights, rep maps) bit-exact
  against the oracle's.
* One two-phase sweep of every level from the same seeded float32 rows,
  compared with the oracle's float64 sweep on every row.
* Properties of the full V-cycle at this size: a constant embedding is a
  fixed point of projection and refinement, and two runs are bitwise equal.
"""

import numpy as np
import pytest

import hypergen
from oracle import hnv_oracle as O

from _helpers import FP32_TOL, assert_hierarchy_equal, oracle_level0, rel_err

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
