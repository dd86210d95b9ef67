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


def _ncu_csv(path, seq):
    rows = [["ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value"]]
    for i, (name, byts) in enumerate(seq):
        rows.append([str(i), name, "gpu__time_duration.sum", "ns", "1000"])
        rows.append([str(i), name, "dram__bytes_read.sum", "byte", str(byts)])
        rows.append([str(i), name, "dram__bytes_write.sum", "byte", "10"])
    with open(path, "w", newline="") as f:
        f.write("==PROF== a banner line\n")
        csv.writer(f).writerows(rows)


def test_traffic_summary_groups_half_sweeps_per_level(tmp_path, capsys):
    """Two levels, one sweep each: hyperedge side = packed short rows + long
    rows + reduction, node side = weighted short + long rows + reduction;
    the result averages the levels."""
    lvl0 = [("gather_packed_kernel<float, 16, 2, 1, 4>(x)", 100),
            ("gather_packed_kernel<float, 16, 2, 2, 4>(x)", 100),
            ("gather_kernel<float, 32, 1, 0>(x)", 100), ("finalize_kernel<float>(x)", 100),
            ("gather_kernel<float, 16, 2, 1>(x)", 100), ("gather_kernel<float, 32, 1, 1>(x)", 100),
            ("finalize_kernel<float>(x)", 100), ("combine_kernel<float>(x)", 100)]
    lvl1 = [("gather_packed_kernel<float, 16, 2, 1, 4>(x)", 300),
            ("gather_kernel<float, 32, 1, 0>(x)", 300),
            ("gather_kernel<float, 32, 1, 1>(x)", 300)]
    _ncu_csv(tmp_path / "l0.csv", lvl0)
    _ncu_csv(tmp_path / "l1.csv", lvl1)
    bench.traffic_summary([str(tmp_path / "l0.csv"), str(tmp_path / "l1.csv")])
    out = json.loads(capsys.readouterr().out)
    e, v = out["refine_e_half_sweep"], out["refine_v_half_sweep"]
    assert [x["dram_bytes"] for x in e["levels"]] == [4 * 110, 2 * 310]
    assert [x["dram_bytes"] for x in v["levels"]] == [4 * 110, 310]
    assert e["dram_bytes_per_launch"] == (4 * 110 + 2 * 310) // 2
    assert v["dram_bytes_per_launch"] == (4 * 110 + 310) // 2
    assert e["source_sha256_16"] == bench.source_hash()


def test_traffic_is_read_only_for_the_current_sources(tmp_path, monkeypatch):
    f = tmp_path / "t.json"
    f.write_text(json.dumps({"refine_e_half_sweep": {"dram_bytes_per_launch": 5,
                                                     "source_sha256_16": bench.source_hash()},
                             "refine_v_half_sweep": {"dram_bytes_per_launch": 7,
                                                     "source_sha256_16": "stale"}}))
    monkeypatch.setattr(bench, "TRAFFIC_JSON", str(f))
    assert bench.load_traffic("refine_e_half_sweep") == 5
    assert bench.load_traffic("refine_v_half_sweep") is None
