"""The node-side panel plan (build_panel_plan): node rows cut at hyperedge-ID
panel boundaries, items listed panel by panel, pieces reduced in order.

The plan is chosen per level from the size of the hyperedge table; the
environment variable HNV_PANELS forces a panel count for every level. It
is read once per process, so the forced runs go through child processes
that rerun the parity, BF16, adjoint and batch tests with odd panel
counts (ragged boundaries, many split rows on every level)."""

import os
import subprocess
import sys

import numpy as np
import pytest

import hypergen
from oracle import hnv_oracle as O

from _helpers import FP32_TOL, oracle_level0, rel_err

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run_forced(panels, files, k=None):
    env = dict(os.environ, HNV_PANELS=str(panels))
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "gpu"]
    cmd += [os.path.join(ROOT, "tests", f) for f in files]
    if k:
        cmd += ["-k", k]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]


def test_forced_three_panels_parity():
    _run_forced(3, ["test_gpu_parity.py"],
                "widths or long_rows or random_small_graphs or special_cases or vcycle or project")


def test_forced_five_panels_bf16_adjoint_batch():
    _run_forced(5, ["test_gpu_bf16.py", "test_gpu_adjoint.py", "test_gpu_batch.py"])


@pytest.fixture(scope="module")
def H():
    from paper_2103_09660_gb300 import build
    build.build()
    import paper_2103_09660_gb300 as mod
    import torch
    assert torch.cuda.is_available()
    return mod


def test_panels_chosen_by_size_match_oracle(H):
    """A level whose hyperedge table (200,000 rows x 512 bytes) exceeds the
    panel threshold, with long node rows (about 530 incidences): the default
    rule picks panels; one and three sweeps against the oracle."""
    import torch
    rng = np.random.default_rng(7)
    n, m, k = 3000, 200_000, 8
    # k distinct members per hyperedge: a random start plus k steps of 97 (mod n)
    nodes = ((rng.integers(0, n, m)[:, None] + 97 * np.arange(k)) % n).astype(np.int32)
    hg = hypergen.Hypergraph(n=n, m=m, edge_ptr=np.arange(0, m * k + 1, k, dtype=np.int64),
                             edge_nodes=nodes.ravel(),
                             weights=rng.uniform(0.5, 2.0, m).astype(np.float32))
    lv = oracle_level0(hg)
    d = 128
    with H.Graph.from_hypergraph(hg) as G:
        for sweeps in (1, 3):
            z = rng.standard_normal((n + m, d)).astype(np.float32)
            zv = torch.from_numpy(z[:n]).cuda()
            ze = torch.from_numpy(z[n:]).cuda()
            G.refine(0, zv, ze, 0.5, sweeps)
            G.sync_status()
            rv, re = O.refine(lv, z[:n].astype(np.float64), z[n:].astype(np.float64), 0.5, sweeps)
            assert rel_err(zv.double().cpu().numpy(), rv) < FP32_TOL
            assert rel_err(ze.double().cpu().numpy(), re) < FP32_TOL
