"""Device-side failure reporting, tested without faulting the GPU.

A refinement kernel that waits on an mbarrier (the TMA gather) gives every
wait a time limit; when a wait gives up it records a timeout in the graph's
error word, returns, and the host reads HNV_ERR_TIMEOUT from
hnv_sync_status. hnv_selftest_wait_timeout runs one such wait on an
mbarrier that nothing completes (no copy in flight), so the limit must run
out. The tests check the status, that it is cleared once read, and that the
context keeps working (a refinement afterwards still matches the oracle).
"""

import time

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


def test_bounded_wait_gives_up_and_reports_timeout(H):
    import torch
    hg = hypergen.generate(hypergen.CONFIGS["small_2k"])
    lv = oracle_level0(hg)
    with H.Graph.from_hypergraph(hg) as G:
        G.sync_status()                                   # nothing recorded yet
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        assert H.lib().hnv_selftest_wait_timeout(G.handle, 20000,
                                                 H._stream_handle(G.stream)) == 0
        with pytest.raises(H.HNVError) as ei:
            G.sync_status()
        waited = time.perf_counter() - t0
        assert ei.value.code == -6                        # HNV_ERR_TIMEOUT
        assert waited >= 0.018                            # the 20 ms limit ran out
        G.sync_status()                                   # read once, then cleared
        # the context is still usable
        z = np.random.default_rng(0).standard_normal((lv.n + lv.m, 32)).astype(np.float32)
        zv, ze = torch.from_numpy(z[:lv.n]).cuda(), torch.from_numpy(z[lv.n:]).cuda()
        G.refine(0, zv, ze, 0.5, 3)
        G.sync_status()
        rv, re = O.refine(lv, z[:lv.n], z[lv.n:], 0.5, 3)
        assert rel_err(zv.double().cpu().numpy(), rv) < FP32_TOL
        assert rel_err(ze.double().cpu().numpy(), re) < FP32_TOL


def test_selftest_rejects_bad_arguments(H):
    hg = hypergen.random_small_hypergraph(np.random.default_rng(0), 10, 5, 4)
    with H.Graph.from_hypergraph(hg) as G:
        s = H._stream_handle(G.stream)
        assert H.lib().hnv_selftest_wait_timeout(G.handle, 0, s) == -1
        assert H.lib().hnv_selftest_wait_timeout(G.handle, 2_000_000, s) == -1
        assert H.lib().hnv_selftest_wait_timeout(None, 100, s) == -1
        G.sync_status()                                   # nothing was launched


def test_release_cached_memory_keeps_graphs_working(H):
    import torch
    hg = hypergen.generate(hypergen.CONFIGS["small_2k"])
    spec = hypergen.CONFIGS["small_2k"]
    with H.Graph.from_hypergraph(hg) as G:
        G.coarsen(min_nodes=spec.min_nodes)
        top = G.level_info(G.num_levels - 1)
        zc = torch.randn((top[0] + top[1], 32), device="cuda")
        zv = torch.empty((hg.n, 32), device="cuda")
        ze = torch.empty((hg.m, 32), device="cuda")
        G.vcycle(zc, zv, ze, 0.5, 3)
        a = (zv.clone(), ze.clone())
        torch.cuda.synchronize()
        assert H.lib().hnv_release_cached_memory() == 0
        G.vcycle(zc, zv, ze, 0.5, 3)                      # allocates afresh
        torch.cuda.synchronize()
        assert torch.equal(a[0], zv) and torch.equal(a[1], ze)
