"""The epsilon stopping rule (hnv_refine_until; Section 4 names it as the
alternative to a fixed iteration count) against the oracle's
refine_until."""

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


def _rows(z):
    import torch
    return torch.from_numpy(np.ascontiguousarray(z, dtype=np.float32)).cuda()


def test_stops_where_the_oracle_stops(H):
    hg = hypergen.generate(hypergen.CONFIGS["small_2k"])
    lv = oracle_level0(hg)
    z = np.random.default_rng(1).standard_normal((lv.n + lv.m, 32)).astype(np.float32)
    z64 = z.astype(np.float64)
    _, _, _, deltas = O.refine_until(lv, z64[:lv.n], z64[lv.n:], 0.5, 40, -1.0)
    # an eps whose first crossing is at a sweep with a clear margin on both sides
    for j in range(10, 39):
        lo, hi = deltas[j], min(deltas[:j])
        if hi > lo * 1.05:
            eps = lo * 1.02
            break
    else:
        pytest.skip("no clear crossing")
    rv, re, done, dl = O.refine_until(lv, z64[:lv.n], z64[lv.n:], 0.5, 40, eps)
    assert done == j + 1
    with H.Graph.from_hypergraph(hg) as G:
        zv, ze = _rows(z[:lv.n]), _rows(z[lv.n:])
        got_done, got_delta = G.refine_until(0, zv, ze, 0.5, 40, eps)
        assert got_done == done
        assert abs(got_delta - dl[-1]) <= 1e-3 * dl[-1] + 1e-6
        assert rel_err(zv.double().cpu().numpy(), rv) < FP32_TOL
        assert rel_err(ze.double().cpu().numpy(), re) < FP32_TOL


def test_negative_eps_is_a_fixed_count_and_constants_stop_at_once(H):
    import torch
    hg = hypergen.generate(hypergen.CONFIGS["small_2k"])
    lv = oracle_level0(hg)
    z = np.random.default_rng(2).standard_normal((lv.n + lv.m, 16)).astype(np.float32)
    with H.Graph.from_hypergraph(hg) as G:
        a_v, a_e = _rows(z[:lv.n]), _rows(z[lv.n:])
        b_v, b_e = a_v.clone(), a_e.clone()
        done, _ = G.refine_until(0, a_v, a_e, 0.5, 6, -1.0)
        G.refine(0, b_v, b_e, 0.5, 6)
        torch.cuda.synchronize()
        assert done == 6 and torch.equal(a_v, b_v) and torch.equal(a_e, b_e)
        # unit weights and rows of 1.0: every relaxation returns 1.0 exactly
        c_v = torch.ones((lv.n, 16), device="cuda")
        c_e = torch.ones((lv.m, 16), device="cuda")
        done, delta = G.refine_until(0, c_v, c_e, 0.5, 9, 0.0)
        assert (done, delta) == (1, 0.0)
        # BF16 rows run too (the difference is taken on the stored values)
        h_v, h_e = _rows(z[:lv.n]).bfloat16(), _rows(z[lv.n:]).bfloat16()
        done, delta = G.refine_until(0, h_v, h_e, 0.5, 50, 1e-2)
        assert 1 <= done <= 50 and (delta <= 1e-2 or done == 50)
        with pytest.raises(H.HNVError):
            G.refine_until(0, a_v, a_e, 0.5, -1, 1e-3)


def test_jacobi_mode_stops_where_the_oracle_stops(H):
    hg = hypergen.generate(hypergen.CONFIGS["small_2k"])
    lv = oracle_level0(hg)
    z = np.random.default_rng(3).standard_normal((lv.n + lv.m, 16)).astype(np.float32)
    z64 = z.astype(np.float64)
    _, _, _, deltas = O.refine_until(lv, z64[:lv.n], z64[lv.n:], 0.5, 30, -1.0, O.SWEEP_JACOBI)
    for j in range(5, 29):
        if min(deltas[:j]) > deltas[j] * 1.05:
            eps = deltas[j] * 1.02
            break
    else:
        pytest.skip("no clear crossing")
    rv, re, done, _ = O.refine_until(lv, z64[:lv.n], z64[lv.n:], 0.5, 30, eps, O.SWEEP_JACOBI)
    with H.Graph.from_hypergraph(hg) as G:
        zv, ze = _rows(z[:lv.n]), _rows(z[lv.n:])
        got, _ = G.refine_until(0, zv, ze, 0.5, 30, eps, H.SWEEP_JACOBI)
        assert got == done
        assert rel_err(zv.double().cpu().numpy(), rv) < FP32_TOL
        assert rel_err(ze.double().cpu().numpy(), re) < FP32_TOL
