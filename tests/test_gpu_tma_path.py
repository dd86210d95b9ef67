"""The opt-in TMA-gather refinement path (HNV_GATHER=tma) against the
oracle, run in a child process because the path is chosen once per
process."""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_tma_gather_path_parity():
    env = dict(os.environ, HNV_GATHER="tma")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "gpu", os.path.join(ROOT, "tests", "test_gpu_parity.py"),
                        "-k", "widths or long_rows or vcycle_small or random_small_graphs"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
