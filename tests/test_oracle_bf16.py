"""Pins of the oracle's bfloat16 storage mode (CPU).

``round_bf16`` is checked against hand-worked values, against every
bfloat16 grid point and midpoint of several binades (brute force), and
against torch's own float32 -> bfloat16 conversion, an implementation the
oracle does not use. The storage mode of ``refine`` is checked by the
properties it must have: results on the bfloat16 grid, no change without
storage, bit-exact fixed points on representable constants, and the
worst-case distance to the exact oracle.
"""

import numpy as np
import pytest

import hypergen
from oracle import hnv_oracle as O

from _helpers import oracle_level0

U = 2.0 ** -8


def test_round_bf16_hand_values():
    # the bfloat16 neighbours of 1 are 1 - 2^-8 (below) and 1 + 2^-7 (above)
    cases = {
        1.0: 1.0,
        1.0 + 2.0 ** -8: 1.0,                        # a tie: the even neighbour (1)
        1.0 + 3 * 2.0 ** -8: 1.0 + 2.0 ** -6,        # a tie: 1 + 2^-6 is even
        1.0 + 2.0 ** -8 + 2.0 ** -30: 1.0 + 2.0 ** -7,
        -(1.0 + 2.0 ** -8 + 2.0 ** -30): -(1.0 + 2.0 ** -7),
        1.0 - 2.0 ** -9: 1.0,                        # a tie: 1 - 2^-8 has fraction 127 (odd)
        1.0 - 2.0 ** -9 - 2.0 ** -30: 1.0 - 2.0 ** -8,
        3.0: 3.0,
        255.5: 256.0,                                # 255.5 lies halfway: 256 is even
        0.1: 0.10009765625,                          # 0x3DCD
        0.0: 0.0,
        2.0 ** -133: 2.0 ** -133,                    # the smallest subnormal
        1.5 * 2.0 ** -133: 2.0 ** -132,              # a subnormal tie to even
    }
    got = O.round_bf16(np.array(list(cases.keys())))
    np.testing.assert_array_equal(got, np.array(list(cases.values())))


def _grid(lo_exp, hi_exp):
    """Every positive bfloat16 value with exponent in [lo_exp, hi_exp]."""
    vals = []
    for e in range(lo_exp, hi_exp + 1):
        for f in range(128):
            vals.append((1.0 + f / 128.0) * 2.0 ** e)
    return np.array(vals)


def test_round_bf16_brute_force_grid_and_midpoints():
    g = _grid(-10, 10)
    np.testing.assert_array_equal(O.round_bf16(g), g)            # grid points stay
    np.testing.assert_array_equal(O.round_bf16(-g), -g)
    mid = (g[:-1] + g[1:]) / 2                                   # exact in float64
    r = O.round_bf16(mid)
    lower, upper = g[:-1], g[1:]
    # a midpoint goes to the neighbour whose 7-bit fraction is even
    frac_lower = np.rint((lower / 2.0 ** np.floor(np.log2(lower)) - 1.0) * 128).astype(int)
    want = np.where(frac_lower % 2 == 0, lower, upper)
    np.testing.assert_array_equal(r, want)
    # just off the midpoint: to the nearer neighbour
    np.testing.assert_array_equal(O.round_bf16(mid * (1 + 1e-12)), upper)
    np.testing.assert_array_equal(O.round_bf16(mid * (1 - 1e-12)), lower)


def test_round_bf16_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(200_000) * np.exp(rng.uniform(-40, 40, 200_000))).astype(np.float32)
    x = np.concatenate([x, np.float32([1e-39, -3e-40, 1e-45, 6e-39])])   # subnormals
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(O.round_bf16(x.astype(np.float64)), want)


def test_round_bf16_error_bound():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(100_000) * 10.0
    r = O.round_bf16(x)
    assert np.all(np.abs(r - x) <= U * np.abs(x))


def _small():
    spec = hypergen.CONFIGS["small_2k"]
    hg = hypergen.generate(spec)
    return spec, hg, oracle_level0(hg)


def test_bf16_storage_refine_properties():
    spec, hg, lv = _small()
    rng = np.random.default_rng(2)
    z = O.round_bf16(rng.standard_normal((lv.n + lv.m, 16)))
    for mode in (O.SWEEP_TWO_PHASE, O.SWEEP_JACOBI):
        bv, be = O.refine(lv, z[:lv.n], z[lv.n:], 0.5, 4, mode, storage=O.STORAGE_BF16)
        # every stored value is on the bfloat16 grid
        np.testing.assert_array_equal(O.round_bf16(bv), bv)
        np.testing.assert_array_equal(O.round_bf16(be), be)
        # worst case: 8 half-sweeps, u * max|z| each, not amplified
        rv, re = O.refine(lv, z[:lv.n], z[lv.n:], 0.5, 4, mode)
        M = np.abs(z).max()
        assert np.abs(np.vstack([bv, be]) - np.vstack([rv, re])).max() <= 8 * U * M
        # and not identical: the rounding does happen
        assert not np.array_equal(bv, rv)
        # without storage rounding the mode is the plain oracle, bit for bit
        pv, pe = O.refine(lv, z[:lv.n], z[lv.n:], 0.5, 4, mode, storage=None)
        np.testing.assert_array_equal(pv, rv)
        np.testing.assert_array_equal(pe, re)
    # a representable constant is a fixed point, bit for bit
    c = np.full((lv.n + lv.m, 4), 0.625)
    bv, be = O.refine(lv, c[:lv.n], c[lv.n:], 0.5, 3, storage=O.STORAGE_BF16)
    assert np.all(bv == 0.625) and np.all(be == 0.625)


def test_bf16_storage_vcycle_stays_near_exact():
    spec, hg, lv = _small()
    h = O.coarsen(lv, O.CoarsenParams(min_nodes=spec.min_nodes))
    top = h.levels[-1]
    zc = O.round_bf16(hypergen.coarsest_embedding(top.n + top.m, 8, seed=0).astype(np.float64))
    r16 = O.vcycle(h, zc, 0.5, spec.sweeps, storage=O.STORAGE_BF16)
    r64 = O.vcycle(h, zc, 0.5, spec.sweeps)
    K = 2 * spec.sweeps * len(h.levels)
    M = np.abs(zc).max()
    diff = np.vstack([r16.z_v, r16.z_e]) - np.vstack([r64.z_v, r64.z_e])
    assert np.abs(diff).max() <= K * U * M
    np.testing.assert_array_equal(O.round_bf16(r16.z_v), r16.z_v)
