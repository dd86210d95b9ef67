"""Pins of the oracle's adjoint (reverse mode of the V-cycle) against
float64 central differences of the oracle's forward map, and the
dot-product identity <J x, y> = <x, J^T y> for the linear part."""

import numpy as np

import hypergen
from oracle import hnv_oracle as O


def _tiny_case(seed, n=14, m=10):
    rng = np.random.default_rng(seed)
    hg = hypergen.random_small_hypergraph(rng, n, m, max_size=5, weighted=True)
    lv = O.build_level(hg.n, hg.m, hg.edge_ptr, hg.edge_nodes, hg.weights)
    h = O.coarsen(lv, O.CoarsenParams(min_nodes=2, seed=seed))
    return rng, h


def _mid_case(seed, n=30, m=24):
    """Coarsened only to 8 nodes, so the coarsest level keeps hyperedges. (On
    the tiny cases most components end as one coarsest node with no
    hyperedges: every row of a component is then equal on every level, the
    sweeps act as the identity and the weight gradients vanish.)"""
    rng = np.random.default_rng(seed)
    hg = hypergen.random_small_hypergraph(rng, n, m, max_size=5, weighted=True)
    lv = O.build_level(hg.n, hg.m, hg.edge_ptr, hg.edge_nodes, hg.weights)
    h = O.coarsen(lv, O.CoarsenParams(min_nodes=8, seed=seed))
    return rng, h


def _loss(h, w0, zc, om, k, Gv, Ge):
    r = O.vcycle(O.with_weights(h, w0), zc, om, k)
    return float((Gv * r.z_v).sum() + (Ge * r.z_e).sum())


def test_adjoint_matches_central_differences():
    for seed in range(9):
        rng, h = _tiny_case(seed) if seed < 6 else _mid_case(seed)
        lv0, top = h.levels[0], h.levels[-1]
        d, om, k = 3, float(rng.uniform(0.2, 0.8)), 3
        w0 = rng.uniform(0.5, 2.0, lv0.m)
        zc = rng.standard_normal((top.n + top.m, d))
        Gv = rng.standard_normal((lv0.n, d))
        Ge = rng.standard_normal((lv0.m, d))
        dw, dz = O.vcycle_grad(O.with_weights(h, w0), zc, om, k, Gv, Ge)
        eps = 1e-6
        fd_w = np.array([(_loss(h, w0 + eps * e, zc, om, k, Gv, Ge) -
                          _loss(h, w0 - eps * e, zc, om, k, Gv, Ge)) / (2 * eps)
                         for e in np.eye(lv0.m)])
        np.testing.assert_allclose(dw, fd_w, rtol=1e-6, atol=1e-7)
        if seed >= 6:
            assert np.abs(fd_w).max() > 1e-3  # the mid cases have weight gradients
        fd_z = np.zeros_like(zc)
        for i in range(zc.shape[0]):
            for j in range(d):
                e = np.zeros_like(zc)
                e[i, j] = eps
                fd_z[i, j] = (_loss(h, w0, zc + e, om, k, Gv, Ge) -
                              _loss(h, w0, zc - e, om, k, Gv, Ge)) / (2 * eps)
        np.testing.assert_allclose(dz, fd_z, rtol=1e-6, atol=1e-7)


def test_adjoint_dot_product_identity():
    """For fixed weights the V-cycle is linear in Z^L: <J x, y> = <x, J^T y>."""
    rng, h = _tiny_case(11, n=20, m=14)
    lv0, top = h.levels[0], h.levels[-1]
    d, om, k = 4, 0.5, 4
    x = rng.standard_normal((top.n + top.m, d))
    yv = rng.standard_normal((lv0.n, d))
    ye = rng.standard_normal((lv0.m, d))
    r = O.vcycle(h, x, om, k)
    _, jt_y = O.vcycle_grad(h, x, om, k, yv, ye)
    lhs = (r.z_v * yv).sum() + (r.z_e * ye).sum()
    rhs = (x * jt_y).sum()
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_weight_gradient_vanishes_on_constant_rows():
    """With every row equal to one constant, z_e = z~_v everywhere, so every
    weight derivative is zero (the weighted mean of equal rows does not
    depend on the weights)."""
    rng, h = _tiny_case(3)
    lv0, top = h.levels[0], h.levels[-1]
    zc = np.full((top.n + top.m, 2), 0.7)
    dw, _ = O.vcycle_grad(h, zc, 0.5, 3, rng.standard_normal((lv0.n, 2)),
                          rng.standard_normal((lv0.m, 2)))
    assert np.abs(dw).max() < 1e-12


def test_adjoint_at_small_and_unit_omega():
    """omega = 0.02 (weight gradients of size omega, the GPU backward's
    hardest case), omega = 1 (z_v^i = z~_v) and omega = 0 (every sweep the
    identity: zero weight gradients, coarsest-row gradients the summed
    projections) against float64 central differences."""
    tested = 0
    for seed in range(3):
        rng, h = _mid_case(seed)
        lv0, top = h.levels[0], h.levels[-1]
        d, k = 3, 3
        w0 = rng.uniform(0.5, 2.0, lv0.m)
        zc = rng.standard_normal((top.n + top.m, d))
        Gv = rng.standard_normal((lv0.n, d))
        Ge = rng.standard_normal((lv0.m, d))
        for om in (0.02, 1.0, 0.0):
            dw, dz = O.vcycle_grad(O.with_weights(h, w0), zc, om, k, Gv, Ge)
            eps = 1e-6
            fd_w = np.array([(_loss(h, w0 + eps * e, zc, om, k, Gv, Ge) -
                              _loss(h, w0 - eps * e, zc, om, k, Gv, Ge)) / (2 * eps)
                             for e in np.eye(lv0.m)])
            if om == 0.0:
                assert not np.any(dw)
                assert np.abs(fd_w).max() < 1e-8
            else:
                # float64 differences of a loss of size ~10 carry ~1e-9 of noise
                scale = np.abs(fd_w).max()
                tested += scale > 1e-4
                np.testing.assert_allclose(dw, fd_w, rtol=0, atol=max(1e-6 * scale, 1e-8))
            i, j = int(rng.integers(zc.shape[0])), int(rng.integers(d))
            e = np.zeros_like(zc)
            e[i, j] = eps
            fd = (_loss(h, w0, zc + e, om, k, Gv, Ge) - _loss(h, w0, zc - e, om, k, Gv, Ge)) / (2 * eps)
            assert abs(dz[i, j] - fd) <= 1e-6 * max(1.0, abs(fd))
    assert tested == 6
