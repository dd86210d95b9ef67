"""hnv_refine_noalloc: refinement for callers that may not allocate device
memory during the call (programs that reserve their whole device budget up
front and treat any later cudaMalloc as an error).

The entry point keeps its split-row scratch in a fixed array inside the
library. These tests call it through the C ABI and compare it with
hnv_refine, the entry point that allocates its scratch, on a hypergraph
whose long rows (more than 128 incidences) make the scratch matter. They
check two calls in a row (the array keeps the previous call's contents),
that no allocation is requested (a failing allocator hook is installed for
the call), and that a level too large for the array is refused with
HNV_ERR_TOO_LARGE before any kernel runs.

This file is named to be collected last.
"""

import ctypes

import numpy as np
import pytest

import hypergen

from _helpers import FP32_TOL, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2103_09660_gb300 import build
    build.build()
    import paper_2103_09660_gb300 as mod
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return mod


def _skewed_hypergraph(seed):
    """A 6,000-node hypergraph with one 5,000-member hyperedge and one node
    in 3,000 three-member hyperedges: both half-sweeps have split rows."""
    rng = np.random.default_rng(seed)
    edges = [rng.choice(5800, 5000, replace=False)]
    for _ in range(3000):
        edges.append(np.concatenate([[5999], rng.choice(5800, 2, replace=False)]))
    ptr = np.concatenate([[0], np.cumsum([len(e) for e in edges])]).astype(np.int64)
    return hypergen.Hypergraph(n=6000, m=len(edges), edge_ptr=ptr,
                               edge_nodes=np.concatenate(edges).astype(np.int32),
                               weights=rng.uniform(0.5, 2.0, len(edges)).astype(np.float32))


def _call_noalloc(H, G, level, zv, ze, omega, sweeps):
    return H.lib().hnv_refine_noalloc(G.handle, level, zv.data_ptr(), ze.data_ptr(), H.F32,
                                      zv.shape[1], omega, sweeps,
                                      H._stream_handle(G.stream))


@pytest.mark.parametrize("d", [32, 128])
def test_noalloc_matches_allocating_refine_twice(H, d):
    import torch
    hg = _skewed_hypergraph(1)
    with H.Graph.from_hypergraph(hg) as G:
        G.coarsen(min_nodes=10, seed=3)
        for level in range(G.num_levels):
            n, m, _ = G.level_info(level)
            z = torch.from_numpy(np.random.default_rng(level + d).standard_normal(
                (n + m, d)).astype(np.float32)).cuda()
            ref_v, ref_e = z[:n].clone(), z[n:].clone()
            G.refine(level, ref_v, ref_e, 0.5, 3)          # allocating entry point
            for call in range(2):                          # two calls in a row
                zv, ze = z[:n].clone(), z[n:].clone()
                assert _call_noalloc(H, G, level, zv, ze, 0.5, 3) == 0, \
                    H.lib().hnv_last_error_detail()
                torch.cuda.synchronize()
                assert rel_err(zv.double().cpu().numpy(), ref_v.double().cpu().numpy()) < FP32_TOL
                assert rel_err(ze.double().cpu().numpy(), ref_e.double().cpu().numpy()) < FP32_TOL


def _install_counting_allocator(H, calls):
    """A device allocator hook that records every request and grants none
    (it returns NULL, so an allocating call fails with HNV_ERR_OOM)."""
    AF = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    FF = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
    fail_alloc = AF(lambda nbytes, s, ctx: calls.append(nbytes))
    no_free = FF(lambda p, s, ctx: calls.append(-1))
    assert H.lib().hnv_set_allocator(ctypes.cast(fail_alloc, ctypes.c_void_p),
                                     ctypes.cast(no_free, ctypes.c_void_p), None) == 0
    return fail_alloc, no_free          # keep the callbacks alive while installed


def test_noalloc_requests_no_allocation(H):
    """On a graph that has never refined (so it holds no split-row scratch),
    the no-allocation entry point runs with an allocator hook that refuses
    everything; as a positive control, hnv_refine on a second such graph does
    ask that hook for memory. The reference rows come from the second graph
    after the hook is removed."""
    import torch
    hg = _skewed_hypergraph(2)
    L = H.lib()
    with H.Graph.from_hypergraph(hg) as G, H.Graph.from_hypergraph(hg) as G2:
        n, m, _ = G.level_info(0)
        z = torch.from_numpy(np.random.default_rng(0).standard_normal(
            (n + m, 64)).astype(np.float32)).cuda()
        zv, ze = z[:n].clone(), z[n:].clone()
        rv, re_ = z[:n].clone(), z[n:].clone()
        torch.cuda.synchronize()

        calls = []
        keep = _install_counting_allocator(H, calls)
        try:
            rc = _call_noalloc(H, G, 0, zv, ze, 0.5, 2)
            torch.cuda.synchronize()
        finally:
            assert L.hnv_set_allocator(None, None, None) == 0
        assert rc == 0, L.hnv_last_error_detail()
        assert calls == []

        control = []
        keep = _install_counting_allocator(H, control)
        try:
            rc2 = L.hnv_refine(G2.handle, 0, rv.data_ptr(), re_.data_ptr(), H.F32, 64, 0.5, 2,
                               H.SWEEP_TWO_PHASE, H._stream_handle(G2.stream))
            torch.cuda.synchronize()
        finally:
            assert L.hnv_set_allocator(None, None, None) == 0
        del keep
        assert rc2 == -4, rc2                    # HNV_ERR_OOM: the hook refused
        assert any(c > 0 for c in control)       # hnv_refine did ask for memory

        G2.refine(0, rv, re_, 0.5, 2)            # reference, allocator restored
        torch.cuda.synchronize()
        assert rel_err(zv.double().cpu().numpy(), rv.double().cpu().numpy()) < FP32_TOL
        assert rel_err(ze.double().cpu().numpy(), re_.double().cpu().numpy()) < FP32_TOL


def test_noalloc_refuses_levels_beyond_the_scratch(H):
    import torch
    # one hyperedge of 600,000 members: 4,688 chunks * 1,024 floats * 4 bytes
    # is more than the 16 MiB array
    n = 600_000
    ptr = np.array([0, n, n + 2], np.int64)
    nodes = np.concatenate([np.arange(n), [0, 1]]).astype(np.int32)
    L = H.lib()
    with H.Graph(n, 2, ptr, nodes) as G:
        # the size check comes before any use of the embeddings, so small
        # stand-in buffers suffice
        zv = torch.zeros(64, device="cuda")
        ze = torch.zeros(64, device="cuda")
        assert L.hnv_refine_noalloc(G.handle, 0, zv.data_ptr(), ze.data_ptr(), H.F32, 1024,
                                    0.5, 1, None) == -3          # HNV_ERR_TOO_LARGE
        assert b"static scratch" in L.hnv_last_error_detail()
        assert L.hnv_refine_noalloc(G.handle, 0, zv.data_ptr(), ze.data_ptr(), H.BF16, 1024,
                                    0.5, 1, None) == -7          # F32 only
