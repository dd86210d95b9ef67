"""Host logic of bench.py that needs no GPU: the two arms describe the same
workload, and the ncu traffic summary groups launches into half-sweeps."""

import csv
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import hypergen  # noqa: E402


class _Args:
    workload = "small_2k"
    dtype = "f32"


def test_workload_config_is_the_same_for_both_arms():
    spec = hypergen.CONFIGS["small_2k"]
    hg = hypergen.generate(spec)
    a = bench.workload_config(_Args, spec, hg, 1)
    assert a["workload"] == "small_2k" and a["n"] == hg.n and a["nnz"] == hg.nnz
    assert a["d"] == spec.d and a["sweeps_per_level"] == spec.sweeps
    assert "fit in L2" in a["l2"]                 # 1,842 x 32 floats is far below L2
    assert bench.workload_config(_Args, spec, hg, 4)["parallelism"] == "replicas"


def test_traffic_summary_groups_half_sweeps(tmp_path, capsys):
    """Two sweeps: hyperedge side = packed short rows + long rows + reduction,
    node side = weighted short + long rows; a coarsening kernel between."""
    rows = [["ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value"]]
    seq = [("pack_col_row(int)", 0), ("gather_packed_kernel<float, 16, 2>(x)", 1),
           ("gather_kernel<float, 32, 1, 0>(x)", 1), ("finalize_kernel<float>(x)", 1),
           ("gather_kernel<float, 16, 2, 1>(x)", 2), ("gather_kernel<float, 32, 1, 1>(x)", 2),
           ("gather_packed16_kernel<float, 16, 2>(x)", 3), ("gather_kernel<float, 32, 1, 0>(x)", 3),
           ("gather_kernel<float, 32, 1, 1>(x)", 4), ("rs_scatter(x)", 0)]
    for i, (name, _) in enumerate(seq):
        rows.append([str(i), name, "gpu__time_duration.sum", "ns", "1000"])
        rows.append([str(i), name, "dram__bytes_read.sum", "byte", "100"])
        rows.append([str(i), name, "dram__bytes_write.sum", "byte", "10"])
    p = tmp_path / "t.csv"
    with open(p, "w", newline="") as f:
        f.write("==PROF== a banner line\n")
        csv.writer(f).writerows(rows)
    bench.traffic_summary(str(p))
    out = json.loads(capsys.readouterr().out)
    e, v = out["refine_e_half_sweep"], out["refine_v_half_sweep"]
    assert e["half_sweeps"] == 2 and v["half_sweeps"] == 2
    assert e["dram_bytes_per_launch"] == (3 + 2) * 110 // 2
    assert v["dram_bytes_per_launch"] == (2 + 1) * 110 // 2
    assert e["source_sha256_16"] == bench.source_hash()
