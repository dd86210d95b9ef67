"""Pins of the CPU FP64 oracle against things other than itself.

* SplitMix64: published test vectors of the generator whose finaliser the
  per-level hash uses (Steele, Lea & Flood 2014; Vigna's reference code).
* Coarsening (Algorithm 1, Section 3.1): a hand-worked example
  (tests/golden/coarsen_worked_example.txt), and a brute-force restatement
  with Python sets and dicts run exhaustively on tiny hypergraphs and on
  random ones up to 12 nodes; level invariants; the Table 5 trend.
* Refinement (Algorithm 2, Section 3.3): dense-matrix form of the smoothing
  operator built from the star-expansion Laplacian ``L = D - A``; closed
  form on one two-node hyperedge; fixed point; conservation of ``d^T z``
  (Jacobi); maximum principle; ``omega = 0`` identity; many-sweep limit.
* Projection and the V-cycle: brute force with dicts, dense operators.
"""

import itertools
import os

import numpy as np
import pytest

import hypergen
from oracle import hnv_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# SplitMix64
# ---------------------------------------------------------------------------

def _splitmix_stream(seed, k):
    s = seed
    out = []
    for _ in range(k):
        s = (s + O.GOLDEN_GAMMA) & ((1 << 64) - 1)
        out.append(O.mix64_int(s))
    return out


def test_splitmix64_published_vectors():
    # first outputs of SplitMix64 seeded with 0 and with 1234567
    assert _splitmix_stream(0, 2) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4]
    assert _splitmix_stream(1234567, 5) == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_mix64_vector_matches_scalar():
    rng = np.random.default_rng(3)
    xs = rng.integers(0, 2**63, 200, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    vec = O.mix64(xs)
    assert [int(v) for v in vec] == [O.mix64_int(int(x)) for x in xs]
    assert O.level_salt(7, 3) == O.mix64_int(7 + 3 * O.GOLDEN_GAMMA)


# ---------------------------------------------------------------------------
# Hand-worked coarsening example
# ---------------------------------------------------------------------------

def _parse_golden(path):
    spec = {"edges": {}, "prio": {}, "levels": {}, "rep_v": {}, "rep_e": {}}
    cur = None
    for raw in open(path):
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        head, _, tail = line.partition(":")
        toks = head.split()
        vals = [int(x) for x in tail.split()] if ":" in line else []
        if toks[0] == "input":
            spec["n"], spec["m"] = int(toks[2]), int(toks[4])
        elif toks[0] == "edge":
            spec["edges"][int(toks[1])] = vals
        elif toks[0] == "prio":
            spec["prio"][(int(toks[1]), int(toks[2]))] = int(toks[3])
        elif toks[0] == "level":
            cur = int(toks[1])
            spec["levels"][cur] = {"n": int(toks[3]), "m": int(toks[5]), "csr": {}, "csc": {}}
        elif toks[0] in ("csr", "csc"):
            spec["levels"][cur][toks[0]][int(toks[1])] = vals
        elif toks[0] in ("rep_v", "rep_e"):
            spec[toks[0]][int(toks[1])] = vals
    return spec


def test_coarsen_hand_worked_example():
    g = _parse_golden(os.path.join(GOLDEN, "coarsen_worked_example.txt"))
    n, m = g["n"], g["m"]
    ptr = [0]
    nodes = []
    for e in range(m):
        nodes += g["edges"][e]
        ptr.append(len(nodes))
    lv0 = O.build_level(n, m, ptr, nodes)
    tab = np.zeros((8, m), dtype=np.uint64)
    for (ell, e), p in g["prio"].items():
        tab[ell, e] = p
    h = O.coarsen(lv0, O.CoarsenParams(policy=O.ASSIGN_EXPLICIT, min_nodes=0,
                                       max_levels=8, explicit_prio=tab))
    assert len(h.levels) == len(g["levels"])
    for ell, want in g["levels"].items():
        lv = h.levels[ell]
        assert (lv.n, lv.m) == (want["n"], want["m"])
        for e, mem in want["csr"].items():
            assert list(lv.e_nodes[lv.e_ptr[e]:lv.e_ptr[e + 1]]) == mem
        for v, eds in want["csc"].items():
            assert list(lv.v_edges[lv.v_ptr[v]:lv.v_ptr[v + 1]]) == eds
    for ell, want in g["rep_v"].items():
        assert list(h.rep_v[ell]) == want
    for ell, want in g["rep_e"].items():
        assert list(h.rep_e[ell]) == want


# ---------------------------------------------------------------------------
# Brute-force restatement of one coarsening step with sets and dicts
# ---------------------------------------------------------------------------

def brute_coarsen_step(n, edges, prio):
    """edges: list of sets; prio: list of ints. Returns rep_v (list), rep_e
    (list), coarse edges (list of sorted lists), kept fine ids."""
    nbrs = {v: [e for e, s in enumerate(edges) if v in s] for v in range(n)}
    choice = {}
    for v in range(n):
        if nbrs[v]:
            best = nbrs[v][0]
            for e in nbrs[v][1:]:
                if (prio[e], e) < (prio[best], best):
                    best = e
            choice[v] = ("edge", best)
        else:
            choice[v] = ("alone", v)
    # hyperedge-formed coarse nodes first (by hyperedge id), then lone nodes
    groups = sorted(set(choice.values()), key=lambda t: (0 if t[0] == "edge" else 1, t[1]))
    gid = {g: i for i, g in enumerate(groups)}
    rep_v = [gid[choice[v]] for v in range(n)]
    rep_e, coarse, kept = [], [], []
    for e, s in enumerate(edges):
        img = sorted({rep_v[v] for v in s})
        if len(img) >= 2:
            rep_e.append(len(coarse))
            coarse.append(img)
            kept.append(e)
        else:
            rep_e.append(-1 - img[0])
    return rep_v, rep_e, coarse, kept


def _level_from_sets(n, edges, w=None):
    ptr = [0]
    nodes = []
    for s in edges:
        nodes += sorted(s)
        ptr.append(len(nodes))
    return O.build_level(n, len(edges), ptr, nodes, w)


def _check_step_against_brute(lv, params, ell):
    edges = [set(lv.e_nodes[lv.e_ptr[e]:lv.e_ptr[e + 1]].tolist()) for e in range(lv.m)]
    prio = [int(p) for p in O.priorities(lv, params, ell)]
    rv, re, coarse, kept = brute_coarsen_step(lv.n, edges, prio)
    rep_v, rep_e, nxt = O.coarsen_level(lv, params, ell)
    assert rep_v.tolist() == rv
    assert rep_e.tolist() == re
    assert nxt.n == (max(rv) + 1 if rv else 0) and nxt.m == len(coarse)
    for e, mem in enumerate(coarse):
        assert nxt.e_nodes[nxt.e_ptr[e]:nxt.e_ptr[e + 1]].tolist() == mem
    assert np.array_equal(nxt.w32, lv.w32[kept])
    assert np.array_equal(nxt.orig_e, lv.orig_e[kept])
    # the CSC is the transpose, rows ascending
    for v in range(nxt.n):
        want = [e for e, mem in enumerate(coarse) if v in mem]
        assert nxt.v_edges[nxt.v_ptr[v]:nxt.v_ptr[v + 1]].tolist() == want
    return nxt


def test_coarsen_exhaustive_tiny():
    """Every hypergraph on 4 nodes with 1..3 hyperedges (each a non-empty
    subset), under several explicit priority orders."""
    n = 4
    subsets = [set(c) for r in range(1, n + 1) for c in itertools.combinations(range(n), r)]
    rng = np.random.default_rng(0)
    count = 0
    for k in (1, 2, 3):
        for combo in itertools.product(range(len(subsets)), repeat=k):
            if k == 3 and rng.random() > 0.25:   # a quarter of the 3375 triples
                continue
            edges = [subsets[i] for i in combo]
            lv = _level_from_sets(n, edges)
            tab = rng.integers(0, 4, size=(1, k)).astype(np.uint64)  # many ties
            params = O.CoarsenParams(policy=O.ASSIGN_EXPLICIT, explicit_prio=tab)
            _check_step_against_brute(lv, params, 0)
            count += 1
    assert count > 900


@pytest.mark.parametrize("policy", [O.ASSIGN_HASH, O.ASSIGN_LOW_DEGREE, O.ASSIGN_HIGH_WEIGHT])
def test_coarsen_random_small_against_brute(policy):
    rng = np.random.default_rng(10 + policy)
    for trial in range(60):
        n = int(rng.integers(1, 13))
        m = int(rng.integers(1, 9))
        hg = hypergen.random_small_hypergraph(rng, n, m, max_size=5, weighted=True)
        lv = O.build_level(hg.n, hg.m, hg.edge_ptr, hg.edge_nodes, hg.weights)
        params = O.CoarsenParams(policy=policy, seed=int(rng.integers(0, 2**32)))
        ell = 0
        while lv.m > 0 and ell < 6:
            nxt = _check_step_against_brute(lv, params, ell)
            if nxt.n == lv.n:
                break
            lv = nxt
            ell += 1


def test_priority_policies_definitions():
    # LOW_DEGREE orders by size first; HIGH_WEIGHT by weight, heaviest first
    lv = _level_from_sets(6, [{0, 1, 2}, {0, 1}, {3, 4, 5, 0}], w=[1.0, 2.0, 0.5])
    p = O.CoarsenParams(policy=O.ASSIGN_LOW_DEGREE, seed=1)
    pr = O.priorities(lv, p, 0)
    assert pr[1] < pr[0] < pr[2]
    p = O.CoarsenParams(policy=O.ASSIGN_HIGH_WEIGHT, seed=1)
    pr = O.priorities(lv, p, 0)
    assert pr[1] < pr[0] < pr[2]
    c = O.assign_hyperedges(lv, pr)
    assert c[0] == 1 and c[2] == 0 and c[3] == 2


def test_build_level_dedupes_and_validates():
    lv = O.build_level(4, 2, [0, 4, 6], [3, 1, 3, 0, 2, 2])
    assert lv.e_nodes.tolist() == [0, 1, 3, 2]
    assert lv.e_ptr.tolist() == [0, 3, 4]
    assert lv.v_ptr.tolist() == [0, 1, 2, 3, 4]
    assert lv.v_edges.tolist() == [0, 0, 1, 0]
    with pytest.raises(ValueError):
        O.build_level(3, 1, [0, 2], [0, 3])
    with pytest.raises(ValueError):
        O.build_level(3, 2, [0, 2, 2], [0, 1])
    with pytest.raises(ValueError):
        O.build_level(3, 1, [0, 2], [0, 1], [0.0])
    with pytest.raises(ValueError):
        O.build_level(3, 1, [0, 2], [0, 1], [float("nan")])


def _check_hierarchy_invariants(h):
    for ell, (lv, nxt) in enumerate(zip(h.levels[:-1], h.levels[1:])):
        rv, re = h.rep_v[ell], h.rep_e[ell]
        # rep_v maps onto [0, n_{l+1}): the coarse nodes partition the nodes
        assert rv.min() == 0 and rv.max() == nxt.n - 1
        assert np.unique(rv).size == nxt.n
        # kept hyperedges are numbered 0..m'-1 in order; removed ones point at
        # a coarse node that is the image of all their members
        kept = re >= 0
        assert np.array_equal(re[kept], np.arange(nxt.m))
        for e in np.nonzero(~kept)[0][:200]:
            mem = lv.e_nodes[lv.e_ptr[e]:lv.e_ptr[e + 1]]
            assert np.all(rv[mem] == -1 - re[e])
        # every kept hyperedge has >= 2 members, rows ascending and unique
        sz = np.diff(nxt.e_ptr)
        assert np.all(sz >= 2)
        for ptr, idx in ((nxt.e_ptr, nxt.e_nodes), (nxt.v_ptr, nxt.v_edges)):
            row = O.row_of(ptr)
            same = row[1:] == row[:-1]
            assert np.all(idx[1:][same] > idx[:-1][same])
        # CSR and CSC describe the same incidences
        a = set(zip(O.row_of(nxt.e_ptr).tolist(), nxt.e_nodes.tolist()))
        b = set(zip(nxt.v_edges.tolist(), O.row_of(nxt.v_ptr).tolist()))
        assert a == b


def test_hierarchy_invariants_and_trend_small_workload():
    spec = hypergen.CONFIGS["small_2k"]
    g = hypergen.generate(spec)
    lv0 = O.build_level(g.n, g.m, g.edge_ptr, g.edge_nodes, g.weights)
    h = O.coarsen(lv0, O.CoarsenParams(min_nodes=spec.min_nodes, max_levels=spec.max_levels))
    assert len(h.levels) >= 4
    assert h.levels[-1].n <= spec.min_nodes < h.levels[-2].n
    _check_hierarchy_invariants(h)
    # Table 5 trend: the node contraction ratio n_{l+1}/n_l grows toward 1
    # over the levels, and hyperedges shrink more slowly than nodes.
    nr = [b.n / a.n for a, b in zip(h.levels[:-1], h.levels[1:])]
    mr = [b.m / a.m for a, b in zip(h.levels[:-1], h.levels[1:])]
    assert nr[0] < nr[-1] < 1.0
    assert all(x < y for x, y in zip(nr, mr))


def test_coarsen_stop_rules():
    lv = _level_from_sets(5, [{0, 1}, {1, 2}, {2, 3}, {3, 4}])
    assert len(O.coarsen(lv, O.CoarsenParams(min_nodes=5)).levels) == 1
    assert len(O.coarsen(lv, O.CoarsenParams(min_nodes=0, max_levels=0)).levels) == 1
    h = O.coarsen(lv, O.CoarsenParams(min_nodes=0, max_levels=1))
    assert len(h.levels) == 2
    # a level without hyperedges stops; a step that merges nothing is discarded
    lv2 = _level_from_sets(3, [{0}, {1}, {2}])
    h2 = O.coarsen(lv2, O.CoarsenParams(min_nodes=0))
    assert len(h2.levels) == 1   # every node keeps its own one-node hyperedge: nothing merges


# ---------------------------------------------------------------------------
# Refinement pins
# ---------------------------------------------------------------------------

def dense_star_operator(lv, omega):
    """(n+m)x(n+m) matrices of one Jacobi sweep and of the two half-sweeps,
    built from the star expansion: A has w_e on (v, e) and (e, v); D is its
    row sum (weighted degree, Section 3.3); a row with D = 0 is the identity.
    Node rows come first."""
    n, m = lv.n, lv.m
    N = n + m
    A = np.zeros((N, N))
    for e in range(m):
        for v in lv.e_nodes[lv.e_ptr[e]:lv.e_ptr[e + 1]]:
            A[v, n + e] = lv.w[e]
            A[n + e, v] = lv.w[e]
    D = A.sum(axis=1)
    P = np.eye(N)
    nz = D > 0
    P[nz] = (1 - omega) * np.eye(N)[nz] + omega * A[nz] / D[nz, None]
    PV = np.eye(N)
    PE = np.eye(N)
    PV[:n] = P[:n]
    PE[n:] = P[n:]
    return P, PV, PE, A, D


@pytest.mark.parametrize("mode", [O.SWEEP_TWO_PHASE, O.SWEEP_JACOBI])
def test_refine_matches_dense_operator(mode):
    rng = np.random.default_rng(5 + mode)
    for trial in range(25):
        n = int(rng.integers(2, 20))
        m = int(rng.integers(1, 15))
        hg = hypergen.random_small_hypergraph(rng, n, m, max_size=6, weighted=bool(trial % 2))
        lv = O.build_level(hg.n, hg.m, hg.edge_ptr, hg.edge_nodes, hg.weights)
        omega = float(rng.uniform(0.1, 0.9))
        k = int(rng.integers(1, 6))
        d = 3
        z = rng.standard_normal((n + m, d))
        P, PV, PE, _, _ = dense_star_operator(lv, omega)
        step = P if mode == O.SWEEP_JACOBI else PV @ PE
        want = np.linalg.matrix_power(step, k) @ z
        zv, ze = O.refine(lv, z[:n], z[n:], omega, k, mode)
        np.testing.assert_allclose(np.vstack([zv, ze]), want, rtol=1e-12, atol=1e-12)


def test_refine_two_node_closed_form():
    lv = _level_from_sets(2, [{0, 1}], w=[1.7])
    a, b, ze = np.array([[1.0, -2.0]]), np.array([[3.0, 5.0]]), np.array([[0.5, 0.25]])
    om = 0.3
    zv, ze2 = O.refine(lv, np.vstack([a, b]), ze, om, 1, O.SWEEP_TWO_PHASE)
    e_new = (1 - om) * ze + om * (a + b) / 2
    np.testing.assert_allclose(ze2, e_new, rtol=0, atol=1e-15)
    np.testing.assert_allclose(zv[0:1], (1 - om) * a + om * e_new, rtol=0, atol=1e-15)
    np.testing.assert_allclose(zv[1:2], (1 - om) * b + om * e_new, rtol=0, atol=1e-15)


def _random_level(rng, n, m, weighted=True):
    hg = hypergen.random_small_hypergraph(rng, n, m, max_size=8, weighted=weighted)
    return O.build_level(hg.n, hg.m, hg.edge_ptr, hg.edge_nodes, hg.weights)


def test_refine_fixed_point_and_identity():
    rng = np.random.default_rng(9)
    lv = _random_level(rng, 40, 30)
    zc = np.full((lv.n + lv.m, 4), 0.37)
    for mode in (O.SWEEP_TWO_PHASE, O.SWEEP_JACOBI):
        zv, ze = O.refine(lv, zc[:lv.n], zc[lv.n:], 0.5, 7, mode)
        assert np.max(np.abs(np.vstack([zv, ze]) - 0.37)) < 1e-15
    z = rng.standard_normal((lv.n + lv.m, 4))
    zv, ze = O.refine(lv, z[:lv.n], z[lv.n:], 0.0, 5)
    assert np.array_equal(np.vstack([zv, ze]), z)


def test_refine_jacobi_conserves_degree_weighted_sum():
    rng = np.random.default_rng(11)
    lv = _random_level(rng, 60, 40)
    d_v = lv.deg_v()
    d_e = lv.size_e() * lv.w
    dvec = np.concatenate([d_v, d_e])
    z = rng.standard_normal((lv.n + lv.m, 5))
    before = dvec @ z
    zv, ze = O.refine(lv, z[:lv.n], z[lv.n:], 0.5, 9, O.SWEEP_JACOBI)
    after = dvec @ np.vstack([zv, ze])
    np.testing.assert_allclose(after, before, rtol=1e-12, atol=1e-12)


def _components(lv):
    parent = list(range(lv.n + lv.m))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x
    for e in range(lv.m):
        for v in lv.e_nodes[lv.e_ptr[e]:lv.e_ptr[e + 1]]:
            parent[find(int(v))] = find(lv.n + e)
    return np.array([find(i) for i in range(lv.n + lv.m)])


@pytest.mark.parametrize("mode", [O.SWEEP_TWO_PHASE, O.SWEEP_JACOBI])
def test_refine_maximum_principle_and_limit(mode):
    rng = np.random.default_rng(13 + mode)
    lv = _random_level(rng, 50, 35)
    comp = _components(lv)
    z = rng.standard_normal((lv.n + lv.m, 3))
    zv, ze = O.refine(lv, z[:lv.n], z[lv.n:], 0.5, 4, mode)
    out = np.vstack([zv, ze])
    for c in np.unique(comp):
        sel = comp == c
        assert np.all(out[sel].max(axis=0) <= z[sel].max(axis=0) + 1e-14)
        assert np.all(out[sel].min(axis=0) >= z[sel].min(axis=0) - 1e-14)
    # many sweeps: constant per connected component; Jacobi's limit is the
    # degree-weighted mean of the start
    zv, ze = O.refine(lv, z[:lv.n], z[lv.n:], 0.5, 3000, mode)
    out = np.vstack([zv, ze])
    dvec = np.concatenate([lv.deg_v(), lv.size_e() * lv.w])
    for c in np.unique(comp):
        sel = comp == c
        if sel.sum() == 1:
            continue
        assert np.ptp(out[sel], axis=0).max() < 1e-8
        if mode == O.SWEEP_JACOBI:
            want = dvec[sel] @ z[sel] / dvec[sel].sum()
            np.testing.assert_allclose(out[sel][0], want, atol=1e-8)


# ---------------------------------------------------------------------------
# Projection and V-cycle
# ---------------------------------------------------------------------------

def test_project_brute_force_and_collapse_mean():
    rng = np.random.default_rng(17)
    lv = _random_level(rng, 12, 9, weighted=False)
    rep_v, rep_e, nxt = O.coarsen_level(lv, O.CoarsenParams(seed=3), 0)
    zc = rng.standard_normal((nxt.n + nxt.m, 4))
    zf_v, zf_e = O.project(rep_v, rep_e, zc[:nxt.n], zc[nxt.n:])
    for v in range(lv.n):
        assert np.array_equal(zf_v[v], zc[rep_v[v]])
    for e in range(lv.m):
        mem = lv.e_nodes[lv.e_ptr[e]:lv.e_ptr[e + 1]]
        if rep_e[e] >= 0:
            assert np.array_equal(zf_e[e], zc[nxt.n + rep_e[e]])
        else:
            # a removed hyperedge takes the mean of its projected members
            np.testing.assert_allclose(zf_e[e], zf_v[mem].mean(axis=0), rtol=0, atol=1e-15)


def test_vcycle_matches_dense_composition():
    rng = np.random.default_rng(21)
    for trial in range(6):
        lv = _random_level(rng, 14, 10, weighted=bool(trial % 2))
        h = O.coarsen(lv, O.CoarsenParams(min_nodes=2, seed=trial))
        L = len(h.levels) - 1
        d, om, k = 3, 0.5, 3
        top = h.levels[L]
        z = rng.standard_normal((top.n + top.m, d))
        # dense: R_L, then (projection matrix, R_l) for l = L-1..0
        _, PV, PE, _, _ = dense_star_operator(top, om)
        cur = np.linalg.matrix_power(PV @ PE, k) @ z
        for ell in range(L - 1, -1, -1):
            fine, coarse = h.levels[ell], h.levels[ell + 1]
            Pi = np.zeros((fine.n + fine.m, coarse.n + coarse.m))
            for v in range(fine.n):
                Pi[v, h.rep_v[ell][v]] = 1
            for e in range(fine.m):
                r = h.rep_e[ell][e]
                Pi[fine.n + e, coarse.n + r if r >= 0 else -1 - r] = 1
            _, PV, PE, _, _ = dense_star_operator(fine, om)
            cur = np.linalg.matrix_power(PV @ PE, k) @ (Pi @ cur)
        res = O.vcycle(h, z, om, k)
        np.testing.assert_allclose(np.vstack([res.z_v, res.z_e]), cur, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------
# Generator sanity (the shared seeded inputs)
# ---------------------------------------------------------------------------

def test_generator_is_seeded_and_clean():
    spec = hypergen.CONFIGS["small_2k"]
    a = hypergen.generate(spec)
    b = hypergen.generate(spec)
    assert np.array_equal(a.edge_ptr, b.edge_ptr) and np.array_equal(a.edge_nodes, b.edge_nodes)
    sizes = np.diff(a.edge_ptr)
    assert sizes.min() >= 2 and sizes.max() <= spec.cap
    assert np.bincount(a.edge_nodes, minlength=a.n).min() >= 1
    for e in range(a.m):
        mem = a.members(e)
        assert np.unique(mem).size == mem.size
    z = hypergen.coarsest_embedding(10, 4, seed=0)
    assert z.dtype == np.float32 and np.array_equal(z, hypergen.coarsest_embedding(10, 4, seed=0))
