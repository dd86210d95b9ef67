"""Reverse mode of the GPU V-cycle against the FP64 oracle's adjoint (which
is itself pinned by float64 central differences), float32 central
differences on the GPU (h = 1e-3), and the dot-product identity.

Bar for GPU vs oracle gradients: 1e-4 of the largest gradient entry (both
passes are float32 sequences of convex combinations and their transposes;
observed errors are ~1e-6 of the largest entry)."""

import numpy as np
import pytest

import hypergen
from oracle import hnv_oracle as O

from _helpers import oracle_level0, small_cases

pytestmark = pytest.mark.gpu
GRAD_TOL = 1e-4


@pytest.fixture(scope="module")
def H():
    from paper_2103_09660_gb300 import build
    build.build()
    import paper_2103_09660_gb300 as mod
    import torch
    assert torch.cuda.is_available()
    return mod


def _gpu_grads(H, G, w0, zc, gv, ge, om, k):
    import torch
    dev = "cuda"
    d = zc.shape[1]
    G.set_weights(w0.astype(np.float32))
    n0, m0, _ = G.level_info(0)
    ck = torch.empty(H.hnv_checkpoint_floats(G.handle, d), device=dev)
    zv = torch.empty((n0, d), device=dev)
    ze = torch.empty((m0, d), device=dev)
    zct = torch.from_numpy(zc.astype(np.float32)).to(dev)
    H.hnv_vcycle_save(G.handle, zct, zv, ze, ck, om, k, G.stream)
    gw = torch.empty(m0, device=dev)
    gz = torch.empty_like(zct)
    H.hnv_vcycle_backward(G.handle, ck, torch.from_numpy(gv.astype(np.float32)).to(dev),
                          torch.from_numpy(ge.astype(np.float32)).to(dev), gw, gz, om, k,
                          G.stream)
    G.sync_status()
    return gw.double().cpu().numpy(), gz.double().cpu().numpy(), zv, ze


def _check_case(H, hg, seed, d=8, om=0.5, k=3, min_nodes=2, need_dw=False, max_levels=32):
    rng = np.random.default_rng(seed)
    lv0 = oracle_level0(hg)
    h = O.coarsen(lv0, O.CoarsenParams(min_nodes=min_nodes, max_levels=max_levels, seed=seed))
    top = h.levels[-1]
    w0 = rng.uniform(0.5, 2.0, lv0.m).astype(np.float32).astype(np.float64)
    zc = rng.standard_normal((top.n + top.m, d)).astype(np.float32).astype(np.float64)
    gv = rng.standard_normal((lv0.n, d)).astype(np.float32).astype(np.float64)
    ge = rng.standard_normal((lv0.m, d)).astype(np.float32).astype(np.float64)
    hw = O.with_weights(h, w0)
    dw_ref, dz_ref = O.vcycle_grad(hw, zc, om, k, gv, ge)
    if need_dw:  # the case must exercise the weight gradients
        assert np.abs(dw_ref).max() > 1e-3 * np.abs(gv).max() * np.abs(zc).max()
    with H.Graph.from_hypergraph(hg) as G:
        G.coarsen(min_nodes=min_nodes, max_levels=max_levels, seed=seed)
        dw, dz, zv, ze = _gpu_grads(H, G, w0, zc, gv, ge, om, k)
        # the checkpointed forward is the plain V-cycle with these weights
        ref = O.vcycle(hw, zc, om, k)
        assert np.abs(zv.double().cpu().numpy() - ref.z_v).max() <= 1e-5 * max(1.0, np.abs(ref.z_v).max())
    # normalise by the largest entry, floored at 1e-2 of the size of the two
    # sums a weight-gradient entry is the difference of (about |G| |z|): an
    # exactly-zero gradient (every member of a hyperedge in one coarse row)
    # is a difference of equal float32 sums and leaves ~eps |G| |z| of noise
    # (a weight gradient is omega times such a difference, so its floor
    # scales with omega; at omega = 0 it must be exactly zero)
    floor = 1e-2 * np.abs(gv).max() * np.abs(zc).max()
    if om == 0.0:
        assert not np.any(dw)
        ew = 0.0
    else:
        ew = np.abs(dw - dw_ref).max() / max(np.abs(dw_ref).max(), om * floor)
    ez = np.abs(dz - dz_ref).max() / max(np.abs(dz_ref).max(), floor)
    assert ew < GRAD_TOL and ez < GRAD_TOL, (ew, ez, np.abs(dw_ref).max(), np.abs(dw).max())
    return ew, ez


def test_adjoint_small_random_graphs(H):
    """Random small graphs, coarsened to 2 nodes (the deepest hierarchies;
    their weight gradients are often zero, see test_adjoint_omega_extremes)
    and to 8 nodes or 4 levels (coarsest levels with hyperedges)."""
    for i, hg in enumerate(small_cases(40, 15, n_max=30, m_max=20)):
        for om in (0.5, 0.3):
            _check_case(H, hg, seed=i, d=4 * (1 + i % 3), om=om, k=2 + i % 3)
            _check_case(H, hg, seed=i, d=4 * (1 + i % 3), om=om, k=2 + i % 3, min_nodes=8,
                        max_levels=4)


def test_adjoint_omega_extremes(H):
    """omega near 0, where z~_v = s_v / D_v carries a weight gradient of
    size omega and must not be recovered from consecutive iterates (which
    would leave eps |z| / omega of error in it); omega = 1 (z_v^i = z~_v);
    omega = 0 (every sweep the identity, weight gradients exactly zero).
    The graphs are coarsened only to 8 nodes or 4 levels so that the coarsest
    level keeps hyperedges and the weight gradients do not vanish."""
    for i in range(6):
        rng = np.random.default_rng(100 + i)
        hg = hypergen.random_small_hypergraph(rng, 30 + 2 * i, 24 + i, max_size=5,
                                              weighted=True)
        for om in (0.02, 0.001, 1.0, 0.0):
            _check_case(H, hg, seed=100 + i, d=8, om=om, k=3, min_nodes=8, max_levels=4,
                        need_dw=om > 0)


def test_adjoint_skewed_split_rows(H):
    rng = np.random.default_rng(5)
    edges = [rng.choice(3000, 2000, replace=False)]
    for _ in range(1500):
        edges.append(np.concatenate([[2999], rng.choice(2900, 2, replace=False)]))
    for _ in range(500):
        edges.append(rng.choice(2900, int(rng.integers(2, 9)), replace=False))
    ptr = np.concatenate([[0], np.cumsum([len(e) for e in edges])]).astype(np.int64)
    hg = hypergen.Hypergraph(n=3000, m=len(edges), edge_ptr=ptr,
                             edge_nodes=np.concatenate(edges).astype(np.int32),
                             weights=np.ones(len(edges), np.float32))
    _check_case(H, hg, seed=1, d=32, k=3, min_nodes=20)


def test_adjoint_small_workload(H):
    spec = hypergen.CONFIGS["small_2k"]
    hg = hypergen.generate(spec)
    _check_case(H, hg, seed=0, d=32, k=5, min_nodes=spec.min_nodes)


def test_autograd_function_and_finite_differences(H):
    """CE loss of a fixed linear head on a node subset, through
    torch.autograd; spot-check against float32 central differences on the GPU
    (h = 1e-3) for a few weights and embedding entries."""
    import torch
    hg = hypergen.planted_hypergraph(3000, 2000, C=4, alpha=1.8, cap=200, p_in=0.8,
                                     weighted=True, seed=2)
    d, om, k = 16, 0.5, 4
    gen = torch.Generator().manual_seed(0)
    with H.Graph.from_hypergraph(hg) as G:
        G.coarsen(min_nodes=200, seed=0)
        nL, mL, _ = G.level_info(G.num_levels - 1)
        head = (torch.randn(d, 4, generator=gen) / d ** 0.5).cuda()
        sub = torch.randperm(hg.n, generator=gen)[: hg.n // 10].cuda()
        labels = torch.from_numpy(hg.labels.astype(np.int64)).cuda()[sub]
        w0 = torch.from_numpy(hg.weights.copy()).cuda().requires_grad_(True)
        zc = torch.randn((nL + mL, d), generator=gen).cuda().requires_grad_(True)

        def loss_of(w, z):
            zv, _ = H.vcycle_autograd(G, w, z, om, k)
            return torch.nn.functional.cross_entropy(zv[sub] @ head, labels)

        loss = loss_of(w0, zc)
        loss.backward()
        gw, gz = w0.grad.clone(), zc.grad.clone()
        assert torch.isfinite(gw).all() and torch.isfinite(gz).all()
        h = 1e-3
        with torch.no_grad():
            for j in torch.argsort(gw.abs(), descending=True)[:4].tolist():
                e = torch.zeros_like(w0)
                e[j] = h
                fd = (loss_of(w0 + e, zc) - loss_of(w0 - e, zc)) / (2 * h)
                assert abs(float(fd) - float(gw[j])) <= 0.05 * abs(float(gw[j])) + 3e-4, (j, float(fd), float(gw[j]))
            flat = gz.flatten()
            for j in torch.argsort(flat.abs(), descending=True)[:4].tolist():
                e = torch.zeros_like(flat)
                e[j] = h
                e = e.view_as(zc)
                fd = (loss_of(w0, zc + e) - loss_of(w0, zc - e)) / (2 * h)
                assert abs(float(fd) - float(flat[j])) <= 0.05 * abs(float(flat[j])) + 3e-4, (j, float(fd), float(flat[j]))
        # and against the FP64 oracle through the same loss gradient
        zv, _ = H.vcycle_autograd(G, w0.detach(), zc.detach(), om, k)
        zv = zv.detach().requires_grad_(True)
        torch.nn.functional.cross_entropy(zv[sub] @ head, labels).backward()
        gv = zv.grad.double().cpu().numpy()
    lv0 = oracle_level0(hg)
    h_ = O.coarsen(lv0, O.CoarsenParams(min_nodes=200, seed=0))
    dw_ref, dz_ref = O.vcycle_grad(O.with_weights(h_, hg.weights.astype(np.float64)),
                                   zc.detach().double().cpu().numpy(), om, k, gv,
                                   np.zeros((lv0.m, d)))
    assert np.abs(gw.double().cpu().numpy() - dw_ref).max() <= GRAD_TOL * np.abs(dw_ref).max()
    assert np.abs(gz.double().cpu().numpy() - dz_ref).max() <= GRAD_TOL * np.abs(dz_ref).max()


def test_dot_product_identity_gpu(H):
    import torch
    spec = hypergen.CONFIGS["small_2k"]
    hg = hypergen.generate(spec)
    rng = np.random.default_rng(4)
    d, om, k = 16, 0.5, 4
    with H.Graph.from_hypergraph(hg) as G:
        G.coarsen(min_nodes=spec.min_nodes)
        nL, mL, _ = G.level_info(G.num_levels - 1)
        x = rng.standard_normal((nL + mL, d))
        yv = rng.standard_normal((hg.n, d))
        ye = rng.standard_normal((hg.m, d))
        _, jt_y, zv, ze = _gpu_grads(H, G, hg.weights.astype(np.float64), x, yv, ye, om, k)
        lhs = float((zv.double().cpu().numpy() * yv).sum() + (ze.double().cpu().numpy() * ye).sum())
        rhs = float((x.astype(np.float32).astype(np.float64) * jt_y).sum())
    assert abs(lhs - rhs) <= 1e-4 * max(1.0, abs(lhs))


def test_set_weights_rejects_bad_weights(H):
    hg = next(small_cases(7, 1))
    with H.Graph.from_hypergraph(hg) as G:
        w = np.ones(hg.m, np.float32)
        w[0] = -1.0
        with pytest.raises(H.HNVError) as ei:
            G.set_weights(w)
        assert ei.value.code == -1


def test_backward_phase_timing(H):
    """The backward records its three phases (replay, reverse, projection)
    with events and algorithmic bytes when timing is on."""
    import torch
    spec = hypergen.CONFIGS["small_2k"]
    hg = hypergen.generate(spec)
    rng = np.random.default_rng(3)
    d, om, k = 16, 0.5, 3
    with H.Graph.from_hypergraph(hg) as G:
        L = G.coarsen(min_nodes=spec.min_nodes, seed=0)
        nL, mL, _ = G.level_info(L - 1)
        zc = rng.standard_normal((nL + mL, d))
        gv = rng.standard_normal((hg.n, d))
        ge = rng.standard_normal((hg.m, d))
        w0 = rng.uniform(0.5, 2.0, hg.m)
        H.timing_reset()
        H.timing_enable(True)
        try:
            _gpu_grads(H, G, w0, zc, gv, ge, om, k)
            torch.cuda.synchronize()
        finally:
            H.timing_enable(False)
        for ph in (H.PHASE_ADJOINT_REPLAY, H.PHASE_ADJOINT_REVERSE, H.PHASE_ADJOINT_PROJECT):
            ms, launches, by = H.timing_read(ph)
            assert launches == L and ms > 0 and by > 0, (ph, ms, launches, by)
        H.timing_reset()
