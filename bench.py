"""Benchmark of the HyperNetVec V-cycle hot path on GB300.

One step = the whole hot path over the 1M-node planted-community workload
(1,000,000 nodes, 1,000,000 hyperedges, sizes 2+Zipf(1.8) capped at 5,000,
weights U[0.5,2), d=128, 20 two-phase sweeps per level, coarsened to
<= 10,000 nodes): build the incidence (level 0), coarsen level by level,
refine the coarsest level from the seeded embedding, then project and refine
every finer level.

Metric: refinement updates per second, where one update is one incidence
times one embedding element (sum over levels of 2 * nnz_l * d * sweeps per
step), divided by the whole step time (build and coarsening included).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import hypergen  # noqa: E402

METRIC = "refine incidence-nnz×d updates/s"
UNIT = "updates/s"
WORKLOAD = "planted_1m"


# ---------------------------------------------------------------------------
# distributed helpers (replicas: one independent V-cycle per GPU)
# ---------------------------------------------------------------------------

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws, backend):
    import torch.distributed as dist
    if ws > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend)


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int, device=None) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_config(args, spec, hg, ws: int) -> dict:
    """The workload a line is measured on (the same for both arms)."""
    return {"workload": args.workload, "n": hg.n, "m": hg.m, "nnz": hg.nnz, "d": spec.d,
            "sweeps_per_level": spec.sweeps, "omega": 0.5, "sweep": "two_phase",
            "min_nodes": spec.min_nodes, "max_levels": spec.max_levels,
            "storage": "bf16 rows, f32 sums" if args.dtype == "bf16" else "f32",
            "l2": ("inputs larger than L2 (node and hyperedge embedding tables)"
                   if max(hg.n, hg.m) * spec.d * 4 > 129e6 else
                   "tables fit in L2; no flush between steps (the incidence build and "
                   "coarsening of each step rewrite every array)"),
            "parallelism": "replicas" if ws > 1 else "single GPU"}


def shard_units(weights, ws: int, rank: int) -> list:
    """Indices of the units (independent graphs) rank `rank` of `ws` takes:
    longest-processing-time first, each unit to the rank with the least
    weight so far (ties to the lower rank). Every rank computes the same
    assignment; every unit goes to exactly one rank."""
    load = [0.0] * ws
    mine = []
    for i in sorted(range(len(weights)), key=lambda i: (-weights[i], i)):
        r = min(range(ws), key=lambda q: (load[q], q))
        load[r] += weights[i]
        if r == rank:
            mine.append(i)
    return sorted(mine)


def _rank_entry(rank, n, port, target, argv):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(n),
                      LOCAL_WORLD_SIZE=str(n), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    target(argv)


def spawn_ranks(n: int, target, argv) -> None:
    """Runs target(argv) in n child processes with the torch.distributed
    environment set as torchrun sets it (RANK, LOCAL_RANK, WORLD_SIZE,
    MASTER_ADDR=127.0.0.1, a free MASTER_PORT): `bench.py --gpus N` started
    without a launcher starts its own ranks. Raises if a rank fails."""
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    mp.start_processes(_rank_entry, args=(n, port, target, argv), nprocs=n, join=True,
                       start_method="spawn")


def aggregate(units_per_rank: float, seconds: list) -> float:
    """Whole-job throughput: units of all ranks over the slowest rank."""
    return units_per_rank * len(seconds) / max(seconds)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.uuid:
            cmd += ["--id=" + self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, mx, power = [], [], []
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            try:
                sm.append(float(f[2]))
                mx.append(float(f[3]))
                power.append(float(f[4]))
            except ValueError:
                continue
            for nm, v in zip(names, f[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "power_w_max": float(max(power)), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU oracle baseline (the cpu_baseline leg, the reference arm, --oracle-study)
#
# The FP64 oracle runs the same V-cycle on the host cores. Its coarsening is
# sequential integer work and is timed once, on one core. Projection and
# refinement act on every embedding column on its own, so a block of columns
# is the same computation restricted to those columns: worker processes,
# forked before this process touches CUDA, take column blocks. Throughput is
# refinement updates (2 * nnz_l * d * sweeps per level) per second.
# ---------------------------------------------------------------------------

_OH = {}   # the oracle hierarchy and coarsest rows, set before workers fork


def host_cores() -> int:
    return len(os.sched_getaffinity(0))


def oracle_prepare(hg, spec):
    """Builds the oracle's hierarchy (timed: level-0 incidence, coarsening)
    and the coarsest rows; kept in _OH for forked workers."""
    from oracle import hnv_oracle as O
    t0 = time.perf_counter()
    lv0 = O.build_level(hg.n, hg.m, hg.edge_ptr, hg.edge_nodes, hg.weights)
    t1 = time.perf_counter()
    h = O.coarsen(lv0, O.CoarsenParams(min_nodes=spec.min_nodes, max_levels=spec.max_levels,
                                       seed=spec.seed))
    t2 = time.perf_counter()
    top = h.levels[-1]
    _OH["h"] = h
    _OH["zc"] = hypergen.coarsest_embedding(top.n + top.m, spec.d, seed=spec.seed).astype(np.float64)
    _OH["sweeps"] = spec.sweeps
    return {"build_s": t1 - t0, "coarsen_s": t2 - t1}


def _oracle_vcycle_worker(cols):
    """The oracle V-cycle (refine the coarsest level, then project and refine
    every finer level) on the given columns; seconds per phase and updates."""
    from oracle import hnv_oracle as O
    h, sweeps = _OH["h"], _OH["sweeps"]
    z = _OH["zc"][:, cols]
    L = len(h.levels) - 1
    tr = tp = 0.0
    upd = 0.0
    top = h.levels[L]
    t0 = time.perf_counter()
    z_v, z_e = O.refine(top, z[:top.n], z[top.n:], 0.5, sweeps)
    tr += time.perf_counter() - t0
    upd += 2.0 * top.nnz * len(cols) * sweeps
    for ell in range(L - 1, -1, -1):
        t0 = time.perf_counter()
        z_v, z_e = O.project(h.rep_v[ell], h.rep_e[ell], z_v, z_e)
        t1 = time.perf_counter()
        z_v, z_e = O.refine(h.levels[ell], z_v, z_e, 0.5, sweeps)
        t2 = time.perf_counter()
        tp += t1 - t0
        tr += t2 - t1
        upd += 2.0 * h.levels[ell].nnz * len(cols) * sweeps
    return {"refine_s": tr, "project_s": tp, "updates": upd}


def _oracle_level_worker(args):
    """One level of the V-cycle (project from seeded coarse rows, then the
    level's sweeps) on the given columns; the reference arm's step sample."""
    from oracle import hnv_oracle as O
    ell, cols = args
    h, sweeps = _OH["h"], _OH["sweeps"]
    lv = h.levels[ell]
    rng = np.random.default_rng(1000 + ell)
    t0 = time.perf_counter()
    if ell + 1 < len(h.levels):
        c = h.levels[ell + 1]
        zc = rng.standard_normal((c.n + c.m, len(cols)))
        t0 = time.perf_counter()
        z_v, z_e = O.project(h.rep_v[ell], h.rep_e[ell], zc[:c.n], zc[c.n:])
    else:
        z = _OH["zc"][:, cols]
        z_v, z_e = z[:lv.n], z[lv.n:]
    t1 = time.perf_counter()
    O.refine(lv, z_v, z_e, 0.5, sweeps)
    t2 = time.perf_counter()
    return {"refine_s": t2 - t1, "project_s": t1 - t0,
            "updates": 2.0 * lv.nnz * len(cols) * sweeps}


def oracle_pool(procs):
    """A pool forked now (the caller has not initialised CUDA), sharing _OH."""
    import multiprocessing as mp
    return mp.get_context("fork").Pool(procs)


def oracle_vcycle_timed(pool, procs, cols_per_proc, d):
    """The oracle V-cycle on procs * cols_per_proc columns, one block per
    process (all at once); wall time and summed per-phase worker seconds."""
    blocks = [list(range(i * cols_per_proc, (i + 1) * cols_per_proc)) for i in range(procs)]
    blocks = [[c % d for c in b] for b in blocks]
    t0 = time.perf_counter()
    parts = pool.map(_oracle_vcycle_worker, blocks) if procs > 1 else [_oracle_vcycle_worker(blocks[0])]
    wall = time.perf_counter() - t0
    return {"wall_s": wall, "columns": procs * cols_per_proc,
            "updates": sum(p["updates"] for p in parts),
            "refine_s_max": max(p["refine_s"] for p in parts),
            "project_s_max": max(p["project_s"] for p in parts)}


def cpu_baseline_line(hg, spec, prep, pool, procs):
    """cpu_baseline of the bench line: the oracle V-cycle on all host cores
    (one column per process) and on one core (one column), scaled to the
    workload's d columns; coarsening (one core) added once."""
    d = spec.d
    allc = oracle_vcycle_timed(pool, procs, 1, d)
    one = oracle_vcycle_timed(None, 1, 1, d)
    full_updates = allc["updates"] / allc["columns"] * d
    # all cores: d columns take ceil(d / procs) waves of the measured wall time
    waves = -(-d // procs)
    t_all = prep["build_s"] + prep["coarsen_s"] + waves * allc["wall_s"]
    t_one = prep["build_s"] + prep["coarsen_s"] + d * one["wall_s"]
    return {
        "value": full_updates / t_all, "unit": UNIT, "cores": procs, "kind": "oracle",
        "sample": ("FP64 oracle V-cycle of the workload (5 levels, %d sweeps per level): "
                   "incidence build and coarsening timed whole on one core; projection and "
                   "refinement on %d of the %d columns, one per process on %d cores, scaled "
                   "to %d columns (%d waves)" % (spec.sweeps, allc["columns"], d, procs, d,
                                                   waves)),
        "seconds_per_vcycle": t_all,
        "phases_s": {"build": prep["build_s"], "coarsen": prep["coarsen_s"],
                     "refine_project_all_cores_per_wave": allc["wall_s"],
                     "refine_per_wave": allc["refine_s_max"],
                     "project_per_wave": allc["project_s_max"]},
        "one_core": {"value": full_updates / t_one, "cores": 1, "seconds_per_vcycle": t_one,
                     "sample": "the same V-cycle on one column in one process, scaled to %d "
                               "columns" % d},
        "host_cores_available": host_cores(),
    }


def run_oracle_study(args):
    """The FP64 oracle's whole V-cycle per phase on all host cores (column
    blocks across processes) and on one core, every column, median of 3."""
    spec = hypergen.CONFIGS[args.workload]
    hg = hypergen.generate(spec)
    prep = oracle_prepare(hg, spec)
    procs = host_cores()
    d = spec.d
    pool = oracle_pool(procs)
    runs_all, runs_one = [], []
    for _ in range(3):
        runs_all.append(oracle_vcycle_timed(pool, procs, -(-d // procs), d))
    pool.close()
    one_cols = -(-d // procs)
    for _ in range(3):
        runs_one.append(oracle_vcycle_timed(None, 1, one_cols, d))
    med = lambda xs, k: float(np.median([x[k] for x in xs]))
    updates = runs_all[0]["updates"] / runs_all[0]["columns"] * d
    t_all = prep["build_s"] + prep["coarsen_s"] + med(runs_all, "wall_s")
    t_one = prep["build_s"] + prep["coarsen_s"] + med(runs_one, "wall_s") * d / one_cols
    print(json.dumps({
        "study": "FP64 oracle V-cycle on the host cores", "workload": args.workload,
        "n": hg.n, "m": hg.m, "nnz": hg.nnz, "d": d, "sweeps_per_level": spec.sweeps,
        "levels": len(_OH["h"].levels), "updates_per_vcycle": updates,
        "build_s": prep["build_s"], "coarsen_s": prep["coarsen_s"],
        "all_cores": {"cores": procs, "columns_per_process": -(-d // procs),
                      "refine_project_wall_s_median": med(runs_all, "wall_s"),
                      "refine_s_median": med(runs_all, "refine_s_max"),
                      "project_s_median": med(runs_all, "project_s_max"),
                      "vcycle_s": t_all, "updates_per_s": updates / t_all},
        "one_core": {"cores": 1, "columns_measured": one_cols,
                     "refine_project_s_median": med(runs_one, "wall_s"),
                     "vcycle_s_scaled": t_one, "updates_per_s": updates / t_one},
        "runs": 3}))


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

TRAFFIC_SOURCES = ("paper_2103_09660_gb300/csrc/refine.cu",
                   "paper_2103_09660_gb300/csrc/refine_device.cuh",
                   "paper_2103_09660_gb300/csrc/incidence.cu")
TRAFFIC_JSON = os.path.join(ROOT, "profiles", "traffic_refine_planted_1m.json")


def source_hash():
    """Hash of the sources that decide the refinement kernels' DRAM traffic
    (the gather and reduction kernels and the work plans)."""
    h = hashlib.sha256()
    for rel in TRAFFIC_SOURCES:
        h.update(open(os.path.join(ROOT, rel), "rb").read())
    return h.hexdigest()[:16]


def load_traffic(kernel_tag):
    """DRAM bytes per half-sweep from the committed ncu data file, if it was
    taken on the current kernel sources; else None."""
    try:
        rec = json.load(open(TRAFFIC_JSON)).get(kernel_tag)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_sha256_16") != source_hash():
        return None
    return rec.get("dram_bytes_per_launch")


def _half_sweeps(csv_path):
    """Per side, the DRAM bytes and ncu time of each half-sweep in an ncu CSV
    of gpu__time_duration.sum, dram__bytes_read.sum and dram__bytes_write.sum
    over refinement launches (a half-sweep: one side's gather launches, then
    its split-row reduction)."""
    import csv
    rows = list(csv.reader(open(csv_path)))
    hdr = next(i for i, r in enumerate(rows) if "Kernel Name" in r and "Metric Name" in r)
    h = rows[hdr]
    ii, ki, mi, vi = (h.index("ID"), h.index("Kernel Name"), h.index("Metric Name"),
                      h.index("Metric Value"))
    launches = {}
    for r in rows[hdr + 1:]:
        if len(r) <= vi:
            continue
        rec = launches.setdefault(int(r[ii]), {"name": r[ki]})
        rec[r[mi]] = float(r[vi].replace(",", ""))
    out = {"E": [], "V": []}
    phase = None
    for lid in sorted(launches):
        rec = launches[lid]
        name = rec["name"]
        if "gather_packed" in name:             # the packed short rows: hyperedge side
            side = "E"
        elif "gather_kernel<" in name and "batched" not in name:
            side = "V" if name.split("<", 1)[1].split(">", 1)[0].rstrip().endswith("1") else "E"
        elif (("finalize_kernel<" in name or "combine_kernel<" in name) and phase is not None
              and "batched" not in name):
            side = phase
        else:
            phase = None
            continue
        if side != phase and "finalize" not in name and "combine" not in name:
            out[side].append([0.0, 0.0])
        phase = side
        out[side][-1][0] += rec.get("dram__bytes_read.sum", 0.0) + rec.get("dram__bytes_write.sum", 0.0)
        out[side][-1][1] += rec.get("gpu__time_duration.sum", 0.0)
    return out


def traffic_summary(csv_paths):
    """DRAM bytes per refinement half-sweep, averaged over the levels, from
    one ncu CSV per level (each capturing one sweep of that level: the
    launches of `bench.py --refine-level L --sweeps 1` whose names match
    gather, finalize or combine). Prints the JSON that bench.py reads."""
    if isinstance(csv_paths, str):
        csv_paths = [csv_paths]
    per = {"E": [], "V": []}
    for p in csv_paths:
        hs = _half_sweeps(p)
        for side in ("E", "V"):
            if hs[side]:
                b = sum(x[0] for x in hs[side]) / len(hs[side])
                t = sum(x[1] for x in hs[side]) / len(hs[side])
                per[side].append({"csv": os.path.basename(p), "dram_bytes": round(b),
                                  "ncu_us": round(t / 1e3, 1)})
    out = {}
    for side, tag in (("E", "refine_e_half_sweep"), ("V", "refine_v_half_sweep")):
        if per[side]:
            out[tag] = {"dram_bytes_per_launch":
                        round(sum(x["dram_bytes"] for x in per[side]) / len(per[side])),
                        "levels": per[side], "source_sha256_16": source_hash()}
    print(json.dumps(out, indent=1))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except ValueError:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def run_ours(args, ws, rank, local):
    spec = hypergen.CONFIGS[args.workload]
    hg = hypergen.generate(spec)
    # the CPU oracle's workers fork before this process initialises CUDA
    pool = prep = None
    procs = host_cores()
    if not args.no_cpu_baseline and ws == 1:
        prep = oracle_prepare(hg, spec)
        pool = oracle_pool(procs)

    import torch
    import paper_2103_09660_gb300 as H
    from paper_2103_09660_gb300 import build as B

    if torch.cuda.device_count() <= local:
        raise SystemExit("rank %d needs GPU %d but %d are visible" %
                         (rank, local, torch.cuda.device_count()))
    if ws > 1:
        init_dist(ws, "nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    H.lib()
    stream = torch.cuda.current_stream()

    d_ptr = torch.from_numpy(hg.edge_ptr).to(dev)
    d_nodes = torch.from_numpy(hg.edge_nodes).to(dev)
    d_w = torch.from_numpy(hg.weights).to(dev)

    # learn the hierarchy once (deterministic), then seed the coarsest level
    with H.Graph(hg.n, hg.m, d_ptr, d_nodes, d_w) as G:
        L = G.coarsen(min_nodes=spec.min_nodes, max_levels=spec.max_levels, seed=spec.seed)
        sizes = [G.level_info(l) for l in range(L)]
    n_L, m_L, _ = sizes[-1]
    tdt = torch.bfloat16 if args.dtype == "bf16" else torch.float32
    zc_t = torch.from_numpy(hypergen.coarsest_embedding(n_L + m_L, spec.d, seed=spec.seed)).to(tdt)
    d_zc = zc_t.to(dev)
    z_v = torch.empty((hg.n, spec.d), dtype=tdt, device=dev)
    z_e = torch.empty((hg.m, spec.d), dtype=tdt, device=dev)
    updates = float(sum(2.0 * nnz * spec.d * spec.sweeps for (_, _, nnz) in sizes))

    def step():
        g = H.hnv_build_incidence(hg.n, hg.m, d_ptr, d_nodes, d_w, stream)
        try:
            H.hnv_coarsen(g, seed=spec.seed, min_nodes=spec.min_nodes, max_levels=spec.max_levels)
            H.hnv_vcycle(g, d_zc, z_v, z_e, 0.5, spec.sweeps, H.SWEEP_TWO_PHASE, stream)
        finally:
            H.lib().hnv_graph_free(g)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region: inputs resident in HBM ----
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    H.timing_reset()
    H.timing_enable(True)
    launches0 = H.kernel_launch_count()
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clock_rec = clocks.stop()
    launches = H.kernel_launch_count() - launches0
    H.timing_enable(False)
    sec = ev0.elapsed_time(ev1) / 1e3
    sec_max = max_over_ranks(sec, ws, dev)
    phases = {}
    for name, ph in (("build", H.PHASE_BUILD), ("coarsen", H.PHASE_COARSEN),
                     ("project", H.PHASE_PROJECT), ("refine_e", H.PHASE_REFINE_E),
                     ("refine_v", H.PHASE_REFINE_V)):
        ms, cnt, by = H.timing_read(ph)
        phases[name] = {"ms_per_step": ms / args.steps, "launches": cnt, "alg_bytes": by}

    # ---- end to end through the public API: host buffers, copies inside ----
    pin_ptr = torch.from_numpy(hg.edge_ptr).pin_memory().numpy()
    pin_nodes = torch.from_numpy(hg.edge_nodes).pin_memory().numpy()
    pin_w = torch.from_numpy(hg.weights).pin_memory().numpy()
    pin_zc = zc_t.pin_memory()
    out_v = torch.empty((hg.n, spec.d), dtype=tdt).pin_memory()
    out_e = torch.empty((hg.m, spec.d), dtype=tdt).pin_memory()

    def step_host():
        g = H.hnv_build_incidence(hg.n, hg.m, pin_ptr, pin_nodes, pin_w, stream)
        try:
            H.hnv_coarsen(g, seed=spec.seed, min_nodes=spec.min_nodes, max_levels=spec.max_levels)
            H.hnv_vcycle(g, pin_zc, out_v, out_e, 0.5, spec.sweeps, H.SWEEP_TWO_PHASE, stream)
        finally:
            H.lib().hnv_graph_free(g)

    e2e_steps = max(1, min(args.steps, 5))
    step_host()
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        step_host()
    torch.cuda.synchronize()
    e2e_sec = (time.perf_counter() - t0) / e2e_steps
    e2e_max = max_over_ranks(e2e_sec, ws, dev)
    h2d = (hg.edge_ptr.nbytes + hg.edge_nodes.nbytes + hg.weights.nbytes +
           pin_zc.numel() * pin_zc.element_size())
    d2h = (out_v.numel() + out_e.numel()) * out_v.element_size()

    # the same host<->device copies alone (pinned buffers, one stream): the
    # part of the end-to-end time that is transfer
    ptr_t, nodes_t, w_t = (torch.from_numpy(pin_ptr), torch.from_numpy(pin_nodes),
                           torch.from_numpy(pin_w))
    dst = [torch.empty_like(x, device=dev) for x in (ptr_t, nodes_t, w_t, pin_zc)]
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for rep in range(2):
        c0.record(stream)
        for src_t, dst_t in zip((ptr_t, nodes_t, w_t, pin_zc), dst):
            dst_t.copy_(src_t, non_blocking=True)
        out_v.copy_(z_v, non_blocking=True)
        out_e.copy_(z_e, non_blocking=True)
        c1.record(stream)
        torch.cuda.synchronize()
    copy_ms = c0.elapsed_time(c1)
    del dst

    if rank != 0:
        return None

    # ---- roofline of the dominant kernel (the heavier refinement half-sweep) ----
    peaks, peak_src = measured_peaks()
    dom = max(("refine_e", "refine_v"), key=lambda k: phases[k]["ms_per_step"])
    ms_tot = phases[dom]["ms_per_step"] * args.steps
    achieved = phases[dom]["alg_bytes"] / (ms_tot / 1e3) / 1e9 if ms_tot > 0 else 0.0
    peak = float(peaks.get("hbm_gbs", 6800.0))
    tag = "refine_v_half_sweep" if dom == "refine_v" else "refine_e_half_sweep"
    traffic = load_traffic(tag)
    n_half = phases[dom]["launches"]          # half-sweeps over the timed steps
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "alg_bytes_per_launch": round(phases[dom]["alg_bytes"] / max(n_half, 1)),
                "launch": "one half-sweep of one level (its gather launches and split-row "
                          "reduction), averaged over the levels of the V-cycle",
                "kernel": tag + " (gather_kernel + finalize_kernel)",
                "peak_source": peak_src + " hbm_gbs (copy bandwidth)",
                "bytes": "compulsory: neighbour table once, own rows read+written, indices, "
                         "pointers, weights, normalisers"}

    # ---- CPU oracle on the host cores ----
    cpu = None
    if pool is not None:
        cpu = cpu_baseline_line(hg, spec, prep, pool, procs)
        pool.close()

    value = aggregate(updates, [sec_max / args.steps] * ws)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sec_max / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.dtype,
        "data": "synthetic",
        "config": workload_config(args, spec, hg, ws),
        "hierarchy": {"levels": len(sizes), "level_sizes": [list(s) for s in sizes],
                      "updates_per_step": updates},
        "vcycle_ms": sec_max / args.steps * 1e3,
        "phase_ms_per_step": {k: round(v["ms_per_step"], 3) for k, v in phases.items()},
        "refine_only_updates_per_s": updates / ((phases["refine_e"]["ms_per_step"] +
                                                 phases["refine_v"]["ms_per_step"]) / 1e3),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": aggregate(updates, [e2e_max] * ws), "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": e2e_max * 1e3, "steps": e2e_steps,
                "copies_alone_ms": round(copy_ms, 3),
                "copies_alone_GBps": round((h2d + d2h) / (copy_ms / 1e3) / 1e9, 1)},
        "gpu_launches": int(launches),
        "clocks": clock_rec,
    }
    return line


def run_reference(args, ws, rank, local):
    """The reference arm: the CPU FP64 oracle on the host cores, rank 0 only.
    Step k is one level of the V-cycle (projection from seeded coarse rows,
    then the level's sweeps), the levels taken in turn from the coarsest, on
    one column per process over all host cores; the hierarchy is built once
    before the steps."""
    if rank != 0:
        return None
    spec = hypergen.CONFIGS[args.workload]
    hg = hypergen.generate(spec)
    prep = oracle_prepare(hg, spec)
    procs = host_cores()
    pool = oracle_pool(procs)
    L = len(_OH["h"].levels)
    order = list(range(L - 1, -1, -1))

    def step(k):
        ell = order[k % L]
        t0 = time.perf_counter()
        parts = pool.map(_oracle_level_worker, [(ell, [c % spec.d]) for c in range(procs)])
        return sum(p["updates"] for p in parts), time.perf_counter() - t0

    for k in range(args.warmup):
        step(k)
    tot_u, tot_t = 0.0, 0.0
    for k in range(args.steps):
        u, t = step(args.warmup + k)
        tot_u += u
        tot_t += t
    pool.close()
    value = tot_u / tot_t
    sample = ("FP64 oracle, one V-cycle level per step (levels in turn from the coarsest: "
              "projection and %d sweeps) on %d columns, one per process on %d cores; "
              "hierarchy built once before the steps (build %.1f s, coarsening %.1f s)"
              % (spec.sweeps, procs, procs, prep["build_s"], prep["coarsen_s"]))
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_t / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(args, spec, hg, ws),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_gather_ceiling(args):
    """Gather ceilings of this GPU (random 512-byte rows by table size and
    route, and a copy): builds and runs paper_2103_09660_gb300/probes/
    gather_ceiling.cu. The refinement kernels are held against these."""
    from paper_2103_09660_gb300 import build as B
    src = os.path.join(ROOT, "paper_2103_09660_gb300", "probes", "gather_ceiling.cu")
    exe = os.path.join(B.BUILD, "gather_ceiling")
    os.makedirs(B.BUILD, exist_ok=True)
    subprocess.run([B.nvcc()] + B.ARCH + ["-O3", "-std=c++17", "-o", exe, src], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    if r.returncode != 0:
        raise SystemExit("gather ceiling probe failed (%d): %s" % (r.returncode, r.stderr.strip()))
    print(r.stdout.strip())


def run_refine_level(args):
    """Profiling aid: build and coarsen the workload up to `level`, then run
    `sweeps` two-phase sweeps of that level on random rows, and print the
    per-half-sweep device times. Few launches precede the refinement, which
    keeps ncu captures of it short."""
    import torch
    import paper_2103_09660_gb300 as H
    from paper_2103_09660_gb300 import build as B
    B.build()
    spec = hypergen.CONFIGS[args.workload]
    hg = hypergen.generate(spec)
    with H.Graph.from_hypergraph(hg, on_device=True) as G:
        if args.refine_level > 0:
            G.coarsen(min_nodes=spec.min_nodes, max_levels=args.refine_level, seed=spec.seed)
        lvl = min(args.refine_level, G.num_levels - 1)
        n, m, nnz = G.level_info(lvl)
        gen = torch.Generator(device="cuda").manual_seed(0)
        z_v = torch.randn((n, spec.d), device="cuda", generator=gen)
        z_e = torch.randn((m, spec.d), device="cuda", generator=gen)
        torch.cuda.synchronize()
        H.timing_reset()
        H.timing_enable(True)
        G.refine(lvl, z_v, z_e, 0.5, args.sweeps)
        torch.cuda.synchronize()
        H.timing_enable(False)
        out = {"level": lvl, "n": n, "m": m, "nnz": nnz, "d": spec.d, "sweeps": args.sweeps}
        for nm, ph in (("refine_e", H.PHASE_REFINE_E), ("refine_v", H.PHASE_REFINE_V)):
            ms, c, by = H.timing_read(ph)
            out[nm] = {"ms_per_launch": ms / max(c, 1),
                       "alg_GBps": by / (ms / 1e3) / 1e9 if ms > 0 else 0.0}
        print(json.dumps(out))


# ---------------------------------------------------------------------------
# Precision study: BF16 storage vs FP32 on the same GPU
# ---------------------------------------------------------------------------

def gpu_levels(H, G, zc, sweeps):
    """The V-cycle run level by level through the ABI; returns each level's
    refined rows (nodes then hyperedges) as device tensors."""
    import torch
    L = G.num_levels - 1
    sizes = [G.level_info(l) for l in range(L + 1)]
    out = [None] * (L + 1)
    n, m, _ = sizes[L]
    z = zc.clone()
    G.refine(L, z[:n], z[n:], 0.5, sweeps)
    out[L] = z
    for l in range(L - 1, -1, -1):
        n, m, _ = sizes[l]
        zf = torch.empty((n + m, zc.shape[1]), dtype=zc.dtype, device=zc.device)
        nc = sizes[l + 1][0]
        G.project(l, out[l + 1][:nc], out[l + 1][nc:], zf[:n], zf[n:])
        G.refine(l, zf[:n], zf[n:], 0.5, sweeps)
        out[l] = zf
    G.sync_status()
    return out


def level_errors(got, ref):
    """(max |diff| / max |ref|, max row-relative error with the 1e-3 rms floor)."""
    import torch
    g = got.double()
    r = ref.double() if hasattr(ref, "double") else torch.from_numpy(ref).to(g.device)
    diff = (g - r).abs()
    glob = float(diff.max() / r.abs().max())
    rms = float(torch.sqrt((r * r).mean()))
    den = torch.clamp(r.abs().max(dim=1).values, min=1e-3 * rms)
    row = float((diff.max(dim=1).values / den).max())
    return glob, row


def run_precision_study(args):
    """BF16 storage vs FP32 on the same GPU: V-cycle time and per-level
    difference, both precisions starting from the same bfloat16-rounded
    coarsest rows. (The comparison with the FP64 oracle on an induced
    subsample is a GPU test: tests/test_gpu_fullsize.py.)"""
    import torch
    import paper_2103_09660_gb300 as H
    from paper_2103_09660_gb300 import build as B
    B.build()
    spec = hypergen.CONFIGS[args.workload]
    hg = hypergen.generate(spec)
    params = dict(min_nodes=spec.min_nodes, max_levels=spec.max_levels, seed=spec.seed)
    dev = torch.device("cuda", 0)
    rows = []
    timing = {}
    with H.Graph.from_hypergraph(hg, on_device=True) as G:
        L = G.coarsen(**params)
        sizes = [G.level_info(l) for l in range(L)]
        nL, mL, _ = sizes[-1]
        zc = torch.from_numpy(hypergen.coarsest_embedding(nL + mL, spec.d, seed=spec.seed))
        zc = zc.to(torch.bfloat16).to(dev)
        for name, dt in (("fp32", torch.float32), ("bf16", torch.bfloat16)):
            zv = torch.empty((hg.n, spec.d), dtype=dt, device=dev)
            ze = torch.empty((hg.m, spec.d), dtype=dt, device=dev)
            zci = zc.to(dt)
            G.vcycle(zci, zv, ze, 0.5, spec.sweeps)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                G.vcycle(zci, zv, ze, 0.5, spec.sweeps)
            e1.record()
            torch.cuda.synchronize()
            G.sync_status()
            timing[name] = e0.elapsed_time(e1) / args.steps
            del zv, ze
        z32 = gpu_levels(H, G, zc.float(), spec.sweeps)
        z16 = gpu_levels(H, G, zc, spec.sweeps)
        for l in range(L):
            rows.append({"level": l, "n": sizes[l][0], "m": sizes[l][1], "nnz": sizes[l][2],
                         "bf16_vs_fp32": level_errors(z16[l], z32[l])})
    updates = float(sum(2.0 * nnz * spec.d * spec.sweeps for (_, _, nnz) in sizes))
    print(json.dumps({
        "study": "bf16 storage vs fp32", "workload": args.workload,
        "n": hg.n, "m": hg.m, "nnz": hg.nnz, "d": spec.d, "sweeps_per_level": spec.sweeps,
        "vcycle_ms": timing, "speedup_bf16_over_fp32": timing["fp32"] / timing["bf16"],
        "refine_updates_per_s": {k: updates / (v / 1e3) for k, v in timing.items()},
        "error_metrics": "(max|diff|/max|ref|, max row-relative with 1e-3 rms floor)",
        "levels": rows}))


# ---------------------------------------------------------------------------
# Differentiation study: forward + backward of a node-classification loss
# through the V-cycle, against the forward alone
# ---------------------------------------------------------------------------

def run_autograd_study(args):
    """Forward + backward of a node-classification loss through the V-cycle
    against the forward alone (float32). (Gradient parity with the FP64
    oracle at this size is a GPU test: tests/test_gpu_fullsize.py.)"""
    import torch
    import paper_2103_09660_gb300 as H
    from paper_2103_09660_gb300 import build as B
    B.build()
    spec = hypergen.CONFIGS[args.workload]
    hg = hypergen.generate(spec)
    params = dict(min_nodes=spec.min_nodes, max_levels=spec.max_levels, seed=spec.seed)
    om, k, d = 0.5, spec.sweeps, spec.d
    classes = int(hg.labels.max()) + 1
    gen = torch.Generator().manual_seed(spec.seed)
    head = torch.randn(d, classes, generator=gen) / d ** 0.5
    sub = torch.randperm(hg.n, generator=gen)[: hg.n // 10]
    labels = torch.from_numpy(hg.labels.astype(np.int64))[sub]
    dev = torch.device("cuda", 0)
    with H.Graph.from_hypergraph(hg, on_device=True) as G:
        L = G.coarsen(**params)
        nL, mL, _ = G.level_info(L - 1)
        zc = torch.from_numpy(hypergen.coarsest_embedding(nL + mL, d, seed=spec.seed)).to(dev)
        w0 = torch.from_numpy(hg.weights.copy()).to(dev)
        head_d, sub_d, lab_d = head.to(dev), sub.to(dev), labels.to(dev)
        zv = torch.empty((hg.n, d), device=dev)
        ze = torch.empty((hg.m, d), device=dev)
        G.set_weights(w0)

        def fwd():
            H.hnv_vcycle(G.handle, zc, zv, ze, om, k, H.SWEEP_TWO_PHASE, G.stream)

        def fwd_bwd():
            w = w0.clone().requires_grad_(True)
            z = zc.clone().requires_grad_(True)
            zvo, _ = H.vcycle_autograd(G, w, z, om, k)
            torch.nn.functional.cross_entropy(zvo[sub_d] @ head_d, lab_d).backward()

        def timed(fn, reps):
            for _ in range(2):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        t_fwd = timed(fwd, args.steps)
        t_fb = timed(fwd_bwd, args.steps)
        # the backward alone, and its phases (CUDA events the library records
        # on the launching stream, with each phase's algorithmic bytes)
        n0, m0 = hg.n, hg.m
        ck = torch.empty(H.hnv_checkpoint_floats(G.handle, d), device=dev)
        gen2 = torch.Generator().manual_seed(spec.seed + 1)
        g_v = torch.randn(n0, d, generator=gen2).to(dev)
        g_e = torch.randn(m0, d, generator=gen2).to(dev)
        g_w, g_z = torch.empty(m0, device=dev), torch.empty_like(zc)
        H.hnv_vcycle_save(G.handle, zc, zv, ze, ck, om, k, G.stream)

        def bwd():
            H.hnv_vcycle_backward(G.handle, ck, g_v, g_e, g_w, g_z, om, k, G.stream)

        t_bwd = timed(bwd, args.steps)
        H.timing_reset()
        H.timing_enable(True)
        for _ in range(args.steps):
            bwd()
        torch.cuda.synchronize()
        H.timing_enable(False)
        peak, peak_src = measured_peaks()
        hbm = float(peak.get("hbm_gbs", 6800.0))
        phases = {}
        for nm, ph in (("replay", H.PHASE_ADJOINT_REPLAY), ("reverse", H.PHASE_ADJOINT_REVERSE),
                       ("project", H.PHASE_ADJOINT_PROJECT)):
            ms, c, by = H.timing_read(ph)
            ms, by = ms / args.steps, by / args.steps
            gbs = by / (ms / 1e3) / 1e9 if ms > 0 else 0.0
            phases[nm] = {"ms": ms, "alg_GB": by / 1e9, "alg_GBps": gbs,
                          "frac_of_hbm": gbs / hbm}
        H.timing_reset()
        if args.profile_backward:
            # one backward call bracketed for `ncu --profile-from-start off`
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
            bwd()
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
        G.sync_status()
    print(json.dumps({
        "study": "forward+backward vs forward (float32)", "workload": args.workload,
        "n": hg.n, "m": hg.m, "nnz": hg.nnz, "d": d, "levels": L, "sweeps_per_level": k,
        "loss": "softmax cross-entropy of a seeded %dx%d linear head on a seeded %d-node subset"
                % (d, classes, len(sub)),
        "forward_ms": t_fwd, "forward_backward_ms": t_fb, "ratio": t_fb / t_fwd,
        "backward_ms": t_bwd, "backward_phases": phases,
        "hbm_peak_GBps": hbm, "peak_source": peak_src + " hbm_gbs (copy bandwidth)"}))


def run_feature_study(args):
    """Feature rule (cosine, Section 3.1) against the hash rule on the same
    hypergraph: coarsening time (CUDA events), levels, sizes, and how well
    the first level's coarse nodes keep the planted communities together
    (purity: the share of nodes whose coarse node's majority community is
    their own). GPU only; the bit-exact comparison with the oracle is
    tests/test_gpu_features.py."""
    import torch
    import paper_2103_09660_gb300 as H
    from paper_2103_09660_gb300 import build as B
    B.build()
    spec = hypergen.CONFIGS[args.workload]
    hg = hypergen.generate(spec)
    X = hypergen.planted_features(hg, args.feature_dim, sigma=args.feature_sigma, seed=spec.seed)
    dev = torch.device("cuda", 0)
    Xd = torch.from_numpy(X).to(dev)
    labels = hg.labels.astype(np.int64)

    def purity(rep):
        n2 = int(rep.max()) + 1
        C = int(labels.max()) + 1
        tab = np.zeros((n2, C), dtype=np.int64)
        np.add.at(tab, (rep, labels), 1)
        return float(tab.max(axis=1).sum() / labels.size)

    out = {"study": "feature rule vs hash rule (coarsening)", "workload": args.workload,
           "n": hg.n, "m": hg.m, "nnz": hg.nnz, "feature_dim": args.feature_dim,
           "feature_sigma": args.feature_sigma, "min_nodes": spec.min_nodes,
           "max_levels": spec.max_levels}
    with H.Graph.from_hypergraph(hg, on_device=True) as G:
        G.set_node_features(Xd)
        for name, policy in (("hash", H.ASSIGN_HASH), ("cosine", H.ASSIGN_COSINE)):
            ts = []
            for _ in range(max(args.steps, 1) + 1):
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                L = G.coarsen(policy=policy, seed=spec.seed, min_nodes=spec.min_nodes,
                              max_levels=spec.max_levels)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            sizes = [G.level_info(l)[:2] for l in range(L)]
            rep0 = G.level_array(0, H.ARR_REP_V).astype(np.int64) if L > 1 else None
            out[name] = {"coarsen_ms": float(np.median(ts[1:])), "levels": L,
                         "level_sizes": sizes,
                         "level1_purity": purity(rep0) if rep0 is not None else None}
        G.sync_status()
    print(json.dumps(out))


def run_batch_study(args):
    """The batching workload (256 planted hypergraphs, 1K..100K nodes, d=64):
    the V-cycle of every graph looped through the single-graph path (FP32 and
    BF16) against the batched path (BF16 and FP32; direct launches, one
    captured CUDA graph, autotuned row classes). Device-resident buffers,
    CUDA-event timing on one stream; all variants give the same rows per
    dtype (tests/test_gpu_batch.py checks that).

    Under torchrun the graphs are independent units: each rank takes its
    share (shard_units, balanced by node count), no data moves between
    ranks, and every time is the slowest rank's; throughput counts the
    updates of all ranks."""
    import torch
    import paper_2103_09660_gb300 as H
    from paper_2103_09660_gb300 import build as B
    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        init_dist(ws, "nccl")
    B.build()
    all_specs = hypergen.batch_specs(args.batch_count)
    specs = [all_specs[i] for i in shard_units([sp.n for sp in all_specs], ws, rank)]
    t0 = time.time()
    hgs = [hypergen.generate(sp) for sp in specs]
    t_gen = time.time() - t0
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    Gs = []
    t0 = time.time()
    for sp, hg in zip(specs, hgs):
        G = H.Graph.from_hypergraph(hg, stream=stream)
        G.coarsen(min_nodes=sp.min_nodes, max_levels=sp.max_levels, seed=sp.seed)
        Gs.append(G)
    torch.cuda.synchronize()
    t_build = time.time() - t0
    d, om, k = specs[0].d, 0.5, specs[0].sweeps
    updates = 0
    for G in Gs:
        for lv in range(G.num_levels):
            n, m, _ = G.level_info(lv)
            updates += (n + m) * k
    bat = H.Batch(Gs)
    co, vo, eo = bat.offsets()
    zc32 = torch.cat([torch.from_numpy(hypergen.coarsest_embedding(
        int(co[i + 1] - co[i]), d, seed=specs[i].seed)) for i in range(len(Gs))]).to(dev)
    bufs = {}
    for name, dt in (("f32", torch.float32), ("bf16", torch.bfloat16)):
        bufs[name] = (zc32.to(dt), torch.empty((int(vo[-1]), d), dtype=dt, device=dev),
                      torch.empty((int(eo[-1]), d), dtype=dt, device=dev))

    def loop(name):
        zc, zv, ze = bufs[name]
        for i, G in enumerate(Gs):
            H.hnv_vcycle(G.handle, zc[co[i]:co[i + 1]], zv[vo[i]:vo[i + 1]], ze[eo[i]:eo[i + 1]],
                         om, k, H.SWEEP_TWO_PHASE, stream)

    def batched(name, graph):
        zc, zv, ze = bufs[name]
        return lambda: bat.vcycle(zc, zv, ze, om, k, use_cuda_graph=graph)

    total_updates = updates
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([float(updates)], dtype=torch.float64, device=dev)
        dist.all_reduce(t)
        total_updates = float(t.item())

    def timed(fn):
        for _ in range(max(args.warmup, 1)):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            barrier(ws)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            l0 = H.kernel_launch_count()
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = max_over_ranks(float(np.median(ts)), ws, dev)
        return {"ms": ms, "updates_per_s": total_updates / (ms / 1e3),
                "launches_rank0": int(H.kernel_launch_count() - l0)}

    # compulsory bytes of the batched sweeps per V-cycle (the refinement
    # half-sweeps' formula of the single-graph roofline, summed over graphs
    # and levels; projection not included)
    def sweep_bytes(es):
        tot = 0.0
        for G in Gs:
            for lv in range(G.num_levels):
                n, m, nnz = G.level_info(lv)
                be = es * (n * d + 2.0 * m * d) + 4.0 * (nnz + 2.0 * m + 1.0)
                bv = es * (m * d + 2.0 * n * d) + 4.0 * (2.0 * nnz + 2.0 * n + 1.0)
                tot += k * (be + bv)
        return tot
    peak = float(measured_peaks()[0].get("hbm_gbs", 6800.0))

    res = {}
    res["loop_f32"] = timed(lambda: loop("f32"))
    res["loop_bf16"] = timed(lambda: loop("bf16"))
    for kname, kern in (("per_class", H.BATCH_KERNEL_PER_CLASS),
                        ("persistent", H.BATCH_KERNEL_PERSISTENT)):
        bat.kernel = kern
        res["batched_f32_%s_direct" % kname] = timed(batched("f32", False))
        res["batched_f32_%s_graph" % kname] = timed(batched("f32", True))
        res["batched_bf16_%s_direct" % kname] = timed(batched("bf16", False))
        res["batched_bf16_%s_graph" % kname] = timed(batched("bf16", True))
    t0 = time.time()
    tune = bat.autotune(H.BF16, d, om)
    t_tune = time.time() - t0
    res["batched_bf16_graph_tuned"] = timed(batched("bf16", True))
    tune32 = bat.autotune(H.F32, d, om)
    res["batched_f32_graph_tuned"] = timed(batched("f32", True))
    for key, r in res.items():
        if key.startswith("batched"):
            by = sweep_bytes(2 if "bf16" in key else 4)
            r["sweep_compulsory_GB"] = by / 1e9
            r["roofline_frac_of_measured_hbm"] = by / (r["ms"] / 1e3) / 1e9 / peak
    levels = [G.num_levels for G in Gs]
    for G in Gs:
        G.sync_status()
    bat.close()
    for G in Gs:
        G.close()
    if rank != 0:
        return
    print(json.dumps({
        "study": "batched V-cycle vs looping the single-graph path", "n_gpus": ws,
        "scaling": "weak" if ws > 1 else None,
        "graphs_rank0": len(Gs), "graphs": len(all_specs), "nodes_rank0": int(vo[-1]),
        "hyperedges_rank0": int(eo[-1]), "updates_per_vcycle_all_ranks": total_updates,
        "incidences_rank0": int(sum(h.nnz for h in hgs)), "d": d, "sweeps_per_level": k,
        "levels_min": min(levels), "levels_max": max(levels),
        "updates_per_vcycle_rank0": updates, "results": res,
        "speedup_batched_bf16_tuned_vs_loop_f32":
            res["loop_f32"]["ms"] / res["batched_bf16_graph_tuned"]["ms"],
        "speedup_batched_f32_tuned_vs_loop_f32":
            res["loop_f32"]["ms"] / res["batched_f32_graph_tuned"]["ms"],
        "roofline_note": "sweep_compulsory_GB over the whole V-cycle time (projection and "
                         "launch gaps included) against the measured copy bandwidth",
        "tuning_bf16": tune, "tuning_f32": tune32, "autotune_s": t_tune,
        "generate_s": t_gen, "build_coarsen_s": t_build}))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(hypergen.CONFIGS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--refine-level", type=int, default=None,
                    help="profiling aid: only refine this level (see run_refine_level)")
    ap.add_argument("--sweeps", type=int, default=2)
    ap.add_argument("--dtype", choices=["f32", "bf16"], default="f32",
                    help="embedding storage of the timed V-cycle (sums are float32 either way)")
    ap.add_argument("--precision-study", action="store_true",
                    help="BF16 vs FP32 per level and V-cycle time (use with --workload planted_4m)")
    ap.add_argument("--traffic-summary", default=None, nargs="+", metavar="NCU_CSV",
                    help="print DRAM bytes per refinement half-sweep from ncu CSVs (one per level)")
    ap.add_argument("--feature-study", action="store_true",
                    help="feature (cosine) vs hash coarsening on the workload")
    ap.add_argument("--feature-dim", type=int, default=32)
    ap.add_argument("--feature-sigma", type=float, default=1.0)
    ap.add_argument("--batch-study", action="store_true",
                    help="batched V-cycle over many hypergraphs vs looping the single-graph path")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--gather-ceiling", action="store_true",
                    help="measure the GPU's random-row gather ceilings (a probe, no method)")
    ap.add_argument("--oracle-study", action="store_true",
                    help="FP64 oracle V-cycle per phase on all host cores and on one core")
    ap.add_argument("--autograd-study", action="store_true",
                    help="forward+backward vs forward time (use with --workload diff_200k)")
    ap.add_argument("--profile-backward", action="store_true",
                    help="with --autograd-study: one more backward call between "
                         "cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    args = ap.parse_args(argv)
    if args.gpus < 1:
        raise SystemExit("--gpus must be >= 1")
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # no launcher: start one rank per GPU here (each rank re-enters main)
        spawn_ranks(args.gpus, main, list(argv) if argv is not None else sys.argv[1:])
        return
    ws, rank, local = dist_env()
    if ws != args.gpus:
        raise SystemExit("--gpus %d but WORLD_SIZE=%d: launch one rank per GPU" % (args.gpus, ws))
    if args.refine_level is not None:
        run_refine_level(args)
        return
    if args.precision_study:
        run_precision_study(args)
        return
    if args.autograd_study:
        run_autograd_study(args)
        return
    if args.oracle_study:
        run_oracle_study(args)
        return
    if args.gather_ceiling:
        run_gather_ceiling(args)
        return
    if args.batch_study:
        run_batch_study(args)
        return
    if args.feature_study:
        run_feature_study(args)
        return
    if args.traffic_summary:
        traffic_summary(args.traffic_summary)
        return
    if args.impl == "reference":
        line = run_reference(args, ws, rank, local)
    else:
        line = run_ours(args, ws, rank, local)
    if line is not None and rank == 0:
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
