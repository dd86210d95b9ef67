"""Shared helpers of the test-suite (comparisons, builders). Not a test file."""

import numpy as np

import hypergen
from oracle import hnv_oracle as O

# Parity bar for float32 embeddings against the float64 oracle: per level,
# max over rows u of ||z_gpu,u - z_ref,u||_inf / max(||z_ref,u||_inf,
# 1e-3 * rms(z_ref)). The floor keeps the ratio meaningful on rows that are
# nearly zero.
FP32_TOL = 1e-5


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.size == 0:
        return 0.0
    rms = float(np.sqrt(np.mean(ref * ref)))
    den = np.maximum(np.abs(ref).max(axis=1), 1e-3 * rms)
    den = np.maximum(den, 1e-30)
    return float((np.abs(got - ref).max(axis=1) / den).max())


def oracle_level0(hg):
    return O.build_level(hg.n, hg.m, hg.edge_ptr, hg.edge_nodes, hg.weights)


def csr_lists(ptr, idx):
    return [idx[ptr[i]:ptr[i + 1]].tolist() for i in range(len(ptr) - 1)]


def gpu_level_arrays(G, level):
    import paper_2103_09660_gb300 as H
    return {
        "e_ptr": G.level_array(level, H.ARR_E_PTR),
        "e_nodes": G.level_array(level, H.ARR_E_NODES),
        "v_ptr": G.level_array(level, H.ARR_V_PTR),
        "v_edges": G.level_array(level, H.ARR_V_EDGES),
        "w": G.level_array(level, H.ARR_W),
        "deg_v": G.level_array(level, H.ARR_DEG_V),
    }


def assert_level_equal(G, level, lv):
    """Bit-exact comparison of one level's integer arrays and weights."""
    a = gpu_level_arrays(G, level)
    n, m, nnz = G.level_info(level)
    assert (n, m, nnz) == (lv.n, lv.m, lv.nnz), (level, (n, m, nnz), (lv.n, lv.m, lv.nnz))
    np.testing.assert_array_equal(a["e_ptr"], lv.e_ptr)
    np.testing.assert_array_equal(a["e_nodes"], lv.e_nodes)
    np.testing.assert_array_equal(a["v_ptr"], lv.v_ptr)
    np.testing.assert_array_equal(a["v_edges"], lv.v_edges)
    np.testing.assert_array_equal(a["w"], lv.w32)
    np.testing.assert_allclose(a["deg_v"], lv.deg_v(), rtol=2e-6, atol=0)


def assert_hierarchy_equal(G, h):
    import paper_2103_09660_gb300 as H
    assert G.num_levels == len(h.levels)
    for ell, lv in enumerate(h.levels):
        assert_level_equal(G, ell, lv)
        if ell + 1 < len(h.levels):
            np.testing.assert_array_equal(G.level_array(ell, H.ARR_REP_V), h.rep_v[ell])
            np.testing.assert_array_equal(G.level_array(ell, H.ARR_REP_E), h.rep_e[ell])


def small_cases(seed, count, n_max=40, m_max=30, size_max=8):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        n = int(rng.integers(1, n_max + 1))
        m = int(rng.integers(1, m_max + 1))
        yield hypergen.random_small_hypergraph(rng, n, m, max_size=size_max,
                                               weighted=bool(rng.integers(0, 2)),
                                               allow_dups=True)


# Parity bar for bfloat16 row storage against the oracle run with the same
# storage (oracle.refine(..., storage=STORAGE_BF16)): both store every row
# on the bfloat16 grid, and a stored value can differ only where the float32
# sum before rounding (GPU) and the float64 one (oracle) fall on opposite
# sides of a rounding boundary. Such a flip moves one value by one bfloat16
# ulp (at most 2^-7 of its magnitude); later updates are convex combinations,
# so its effect does not grow, and a flip shifts a neighbour's sum by a
# fraction of an ulp, so flips stay rare. Bars: every value within 4 * u of
# the level's largest magnitude, and the RMS difference within u / 8 of the
# level's RMS (u = 2^-8, bfloat16's unit roundoff). A systematic error of
# 1% of every value is 20 times the RMS bar.
U_BF16 = 2.0 ** -8
BF16_MAX_BAR = 4 * U_BF16
BF16_RMS_BAR = U_BF16 / 8


def bf16_errors(got, ref):
    """(max |got - ref| / max |ref|, rms(got - ref) / rms(ref))."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.size == 0:
        return 0.0, 0.0
    diff = got - ref
    M = max(float(np.abs(ref).max()), 1e-30)
    rms = max(float(np.sqrt(np.mean(ref * ref))), 1e-30)
    return float(np.abs(diff).max()) / M, float(np.sqrt(np.mean(diff * diff))) / rms


def assert_bf16_close(got, ref, what=""):
    emax, erms = bf16_errors(got, ref)
    assert emax <= BF16_MAX_BAR and erms <= BF16_RMS_BAR, (what, emax, erms)
    return emax, erms


# ---------------------------------------------------------------------------
# The oracle over column blocks in worker processes. Refinement and
# projection act on every embedding column on its own, so a V-cycle over a
# block of columns is the same computation as the full one restricted to
# those columns. Workers are started with "spawn" (the test process has a
# CUDA context) and read the oracle's hierarchy from .npy files (memory
# mapped) instead of coarsening again.
# ---------------------------------------------------------------------------

_LEVEL_ARRAYS = ("e_ptr", "e_nodes", "v_ptr", "v_edges", "w", "w32", "orig_e")


def save_hierarchy(h, path):
    import json
    import os
    os.makedirs(path, exist_ok=True)
    meta = {"levels": [[lv.n, lv.m] for lv in h.levels]}
    for l, lv in enumerate(h.levels):
        for a in _LEVEL_ARRAYS:
            np.save(os.path.join(path, "l%d_%s.npy" % (l, a)), getattr(lv, a))
    for l in range(len(h.rep_v)):
        np.save(os.path.join(path, "rep_v%d.npy" % l), h.rep_v[l])
        np.save(os.path.join(path, "rep_e%d.npy" % l), h.rep_e[l])
    with open(os.path.join(path, "meta.json"), "w") as f:
        json.dump(meta, f)


def load_hierarchy(path):
    import json
    import os
    meta = json.load(open(os.path.join(path, "meta.json")))
    levels = []
    for l, (n, m) in enumerate(meta["levels"]):
        arr = {a: np.load(os.path.join(path, "l%d_%s.npy" % (l, a)), mmap_mode="r")
               for a in _LEVEL_ARRAYS}
        levels.append(O.Level(n=n, m=m, **arr))
    L = len(levels) - 1
    rv = [np.load(os.path.join(path, "rep_v%d.npy" % l), mmap_mode="r") for l in range(L)]
    re = [np.load(os.path.join(path, "rep_e%d.npy" % l), mmap_mode="r") for l in range(L)]
    return O.Hierarchy(levels=levels, rep_v=rv, rep_e=re)


def oracle_vcycle_block(args):
    """Worker: the oracle V-cycle of one block of columns, every level kept;
    writes level l's rows (nodes, then hyperedges) to <out>/b<block>_l<l>.npy
    and returns the number of levels."""
    import os
    hpath, out, block, zc_block, omega, sweeps, storage = args
    h = load_hierarchy(hpath)
    res = O.vcycle(h, zc_block, omega, sweeps, keep_levels=True, storage=storage)
    for l, (zv, ze) in enumerate(res.per_level):
        np.save(os.path.join(out, "b%d_l%d.npy" % (block, l)), np.vstack([zv, ze]))
    return len(res.per_level)


def oracle_vcycle_columns(h, zc, omega, sweeps, workdir, storage=None, processes=None):
    """The oracle V-cycle of every column of zc, computed over column blocks
    in spawned worker processes. Returns a function level -> rows (float64,
    nodes first), read back from workdir."""
    import multiprocessing as mp
    import os
    procs = processes or max(1, min(16, os.cpu_count() or 1))
    hpath = os.path.join(workdir, "hierarchy")
    if not os.path.exists(os.path.join(hpath, "meta.json")):
        save_hierarchy(h, hpath)
    out = os.path.join(workdir, "vcycle_%s" % (storage or "f64"))
    os.makedirs(out, exist_ok=True)
    cols = [c for c in np.array_split(np.arange(zc.shape[1]), procs) if c.size]
    zc = np.asarray(zc, dtype=np.float64)
    with mp.get_context("spawn").Pool(len(cols)) as pool:
        pool.map(oracle_vcycle_block, [(hpath, out, b, np.ascontiguousarray(zc[:, c]), omega,
                                        sweeps, storage) for b, c in enumerate(cols)])

    def level(l):
        return np.hstack([np.load(os.path.join(out, "b%d_l%d.npy" % (b, l)))
                          for b in range(len(cols))])
    return level
