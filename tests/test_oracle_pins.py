"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or weight, a wrong pass or dimension, an off-by-one at a block edge,
a wrong rounding of the error-bound constants) fails at least one of them.
None of them re-types the oracle's formulas: traversal and stencil choice come
from the level definition of Eq. 3 (tests/bruteforce.py), weights from the
Lagrange formula in exact rationals, remainders from their closed forms.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

from paper_2507_11165_gb300 import fields
from tests import bruteforce as bf

SHAPES = [((9, 9, 9), 8), ((10, 7, 13), 8), ((17, 17, 17), 16), ((33, 20, 5), 16), ((12, 30), 4),
          ((21,), 4), ((5, 1, 19), 8), ((2, 3, 4), 2), ((1, 1, 1), 8), ((40,), 32)]


def _random_levels(rng, L, shape):
    n3 = bf.dims3(shape)
    act = bf.active_dims(n3)
    interp = rng.integers(0, 2, size=L).astype(np.uint8)
    order = np.zeros((L, 3), dtype=np.uint8)
    for l in range(L):
        perm = list(rng.permutation(act)) + [d for d in range(3) if d not in act]
        order[l] = perm
    return interp, order


# --------------------------------------------------------------------------
# Error-bound constants (Eq. 1; value-range-relative bound, Sec. 6.1.4)
# --------------------------------------------------------------------------
def test_eps_constants_rel(oracle_mod):
    x = np.array([0.5, -1.0, 3.0, np.nan, np.inf, 2.0], dtype=np.float32)
    c = oracle_mod.eps_constants(x, oracle_mod.REL, 1e-3)
    # range over finite values = 3 - (-1) = 4; eps = 1e-3 * 4 in double
    eps = 1e-3 * 4.0
    assert c["eps"] == eps
    assert c["vmin"] == -1.0 and c["vmax"] == 3.0
    # eb_f: largest float32 not above eps
    f = np.float32(eps)
    if float(f) > eps:
        f = np.nextafter(f, np.float32(0))
    assert c["eb_f"] == f and float(c["eb_f"]) <= eps
    assert float(np.nextafter(c["eb_f"], np.float32(1))) > eps
    assert c["ebx2_f"] == np.float32(2 * eps)
    assert c["r_f"] == np.float32(1.0 / (2 * eps))


def test_eps_constants_abs_and_constant(oracle_mod):
    x = np.full(100, 7.25, dtype=np.float32)
    c = oracle_mod.eps_constants(x, oracle_mod.REL, 1e-2)
    assert c["eps"] == 1e-2  # constant field: range 0 -> eps = eb
    c = oracle_mod.eps_constants(x, oracle_mod.ABS, 0.5)
    assert c["eb_f"] == 0.5 and c["ebx2_f"] == 1.0 and c["r_f"] == 1.0
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.eps_constants(x, oracle_mod.ABS, 0.0)
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.eps_constants(x, oracle_mod.ABS, float("nan"))


def test_eps_signed_zero(oracle_mod):
    x = np.array([-0.0, 1.0], dtype=np.float32)
    c = oracle_mod.eps_constants(x, oracle_mod.REL, 1e-3)
    assert np.signbit(c["vmin"]) == False  # noqa: E712


# --------------------------------------------------------------------------
# Traversal: level, pass dimension and stencil case of every point
# --------------------------------------------------------------------------
@pytest.mark.parametrize("shape,A", SHAPES)
def test_trace_matches_bruteforce(oracle_mod, shape, A):
    rng = np.random.default_rng(sum(shape) * 31 + A)
    L = oracle_mod.n_levels(A)
    for trial in range(3):
        interp, order = _random_levels(rng, L, shape)
        lvl, d, k = oracle_mod.trace(shape, A, interp, order)
        blvl, bd, bk = bf.trace(shape, A, interp, order)
        assert np.array_equal(lvl, blvl)
        assert np.array_equal(d, bd)
        assert np.array_equal(k, bk)
        assert bf.check_causality(shape, A, interp, order) == 0


def test_trace_exhaustive_9cubed(oracle_mod):
    """All 12^3 per-level configurations on one 9^3 block (A = 8)."""
    shape, A = (9, 9, 9), 8
    perms = list(itertools.permutations(range(3)))
    cfgs = [(i, p) for i in (1, 0) for p in perms]
    n3 = bf.dims3(shape)
    # brute-force per-level tables are independent across levels: check each
    # level's configs once, then every combination through the oracle.
    ref = {}
    for l in range(3):
        for (i, p) in cfgs:
            interp = np.array([i] * 3, dtype=np.uint8)
            order = np.array([p] * 3, dtype=np.uint8)
            lv, dd, kk = bf.trace(shape, A, interp, order)
            m = lv == l
            ref[(l, i, p)] = (m, dd[m], kk[m])
    for c2, c1, c0 in itertools.product(cfgs, repeat=3):
        interp = np.array([c0[0], c1[0], c2[0]], dtype=np.uint8)
        order = np.array([c0[1], c1[1], c2[1]], dtype=np.uint8)
        lvl, d, k = oracle_mod.trace(shape, A, interp, order)
        for l, c in enumerate((c0, c1, c2)):
            m, dd, kk = ref[(l, c[0], c[1])]
            assert np.array_equal(lvl == l, m)
            assert np.array_equal(d[m], dd) and np.array_equal(k[m], kk)
    assert n3 == (9, 9, 9)


# --------------------------------------------------------------------------
# Stencil weights: polynomial exactness and Lagrange remainders
# --------------------------------------------------------------------------
def _linear_field(shape, coef=(3, 2, -1, 4)):
    n3 = bf.dims3(shape)
    g = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in n3], indexing="ij")
    f = coef[0] + coef[1] * g[0] + coef[2] * g[1] + coef[3] * g[2]
    return f.reshape(shape).astype(np.float32)


@pytest.mark.parametrize("shape,A", [((17, 17, 17), 16), ((17, 33, 9), 8), ((33, 65), 16), ((65,), 32),
                                     ((9, 9, 9), 4)])
def test_linear_field_all_zero_codes(oracle_mod, shape, A):
    """On (kA+1)-sized fields every stencil is exact for a linear field: code 128 everywhere."""
    x = _linear_field(shape)
    L = oracle_mod.n_levels(A)
    rng = np.random.default_rng(7)
    c = oracle_mod.eps_constants(x, oracle_mod.ABS, 0.25)
    for _ in range(4):
        interp, order = _random_levels(rng, L, shape)
        out = oracle_mod.compress(x, A, interp, order, c)
        assert np.all(out["codes"] == 128)
        assert np.array_equal(out["recon"].view(np.uint32), x.view(np.uint32))


@pytest.mark.parametrize("shape,A", [((10, 7, 13), 8), ((30,), 16), ((20, 19), 4)])
def test_linear_field_ragged(oracle_mod, shape, A):
    """Ragged edges: only the copy case (no right neighbour, no f(c-3s)) may miss."""
    x = _linear_field(shape, coef=(1, 1, 2, -3))
    L = oracle_mod.n_levels(A)
    interp, order = oracle_mod.levels(L, oracle_mod.CUBIC)
    c = oracle_mod.eps_constants(x, oracle_mod.ABS, 0.25)
    out = oracle_mod.compress(x, A, interp, order, c)
    lvl, d, k = bf.trace(shape, A, interp, order)
    copy = k == 5
    assert np.all(out["codes"][~copy] == 128)
    assert copy.any()


def _int_poly(shape, rng, deg=3, scale=16):
    """Integer polynomial field (times 16, so every Lagrange residual is an integer)."""
    n3 = bf.dims3(shape)
    g = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in n3], indexing="ij")
    f = np.zeros(n3)
    for d in range(3):
        cs = rng.integers(-2, 3, size=deg + 1)
        for p, cc in enumerate(cs):
            f += cc * g[d] ** p
    f *= scale
    assert np.abs(f).max() < 2 ** 23
    return f.reshape(shape).astype(np.float32)


@pytest.mark.parametrize("shape,A", [((17, 9, 10), 8), ((33,), 16), ((13, 21), 4), ((9, 9, 9), 8),
                                     ((6, 11, 7), 4)])
def test_codes_equal_lagrange_residual(oracle_mod, shape, A):
    """With 2*eps = 1 and integer residuals the closed loop is lossless, so each
    code is 128 + (x - exact Lagrange prediction from x), or 0 when out of range."""
    rng = np.random.default_rng(11)
    L = oracle_mod.n_levels(A)
    x = _int_poly(shape, rng)
    c = oracle_mod.eps_constants(x, oracle_mod.ABS, 0.5)
    for _ in range(3):
        interp, order = _random_levels(rng, L, shape)
        out = oracle_mod.compress(x, A, interp, order, c)
        assert np.array_equal(out["recon"].view(np.uint32), x.view(np.uint32))
        res = bf.open_loop_residuals(x, A, interp, order)
        codes = out["codes"].reshape(bf.dims3(shape))
        for g, r in res.items():
            assert r.denominator == 1
            want = 128 + int(r) if abs(r) <= 127 else 0
            assert codes[g] == want, (g, r, codes[g])


def test_remainder_closed_forms(oracle_mod):
    """Lagrange remainders at the midpoint, in closed form (1D, A = 8, s = 1..4).

    f = c2 t^2 + c3 t^3 around the predicted point:
      cubic 4-point:      0                    (exact to degree 3)
      quadratic (-1,1,3): +3 s^3 c3
      quadratic (-3,-1,1): -3 s^3 c3
      linear midpoint:    -s^2 c2
    """
    A = 8
    n = 17
    xs = np.arange(n, dtype=np.float64)
    for (c2, c3) in [(0, 1), (1, 0), (2, -1), (-1, 2)]:
        # f(t) = 16 (c2 t^2 + c3 t^3) with t in grid units
        f = (16 * (c2 * xs ** 2 + c3 * xs ** 3)).astype(np.float32)
        cst = oracle_mod.eps_constants(f, oracle_mod.ABS, 0.5)
        for interp in (oracle_mod.CUBIC, oracle_mod.LINEAR):
            it, od = oracle_mod.levels(3, interp, (0, 1, 2))
            out = oracle_mod.compress(f, A, it, od, cst)
            codes = out["codes"].astype(int) - 128
            for g in range(n):
                if g % 8 == 0:
                    continue
                l = bf.trailing_zeros(g, 3)
                s = 1 << l
                cc = g % 8
                # expected residual of 16 * (c2 t^2 + c3 t^3) around t0 = g:
                # shift to the local polynomial: c2' = c2 + 3 c3 g, c3' = c3
                c2l = c2 + 3 * c3 * g
                if interp == oracle_mod.LINEAR or (cc - 3 * s < 0 and cc + 3 * s > 8):
                    want = -16 * s * s * c2l
                elif cc - 3 * s >= 0 and cc + 3 * s <= 8:
                    want = 0
                elif cc + 3 * s <= 8:
                    want = 16 * 3 * s ** 3 * c3
                else:
                    want = -16 * 3 * s ** 3 * c3
                got = codes[g] if out["codes"][g] != 0 else None
                if abs(want) <= 127:
                    assert got == want, (c2, c3, interp, g, got, want)
                else:
                    assert out["codes"][g] == 0


# --------------------------------------------------------------------------
# Quantizer special cases (Sec. 5.2.1)
# --------------------------------------------------------------------------
def test_huge_eps_all_zero_codes(oracle_mod):
    x = fields.bumps_field((20, 17, 9), seed=3)
    A, L = 8, 3
    # each pass's stencil has absolute weight sum <= 2 and there are <= 3L passes
    eps = 2.0 ** (3 * L + 2) * float(np.abs(x).max())
    c = oracle_mod.eps_constants(x, oracle_mod.ABS, eps)
    it, od = oracle_mod.levels(L)
    out = oracle_mod.compress(x, A, it, od, c)
    col = oracle_mod.collect(x, out["codes"], A)
    assert np.all(out["codes"] == 128) and col["n_out"] == 0


def test_tiny_eps_all_outliers(oracle_mod):
    x = fields.bumps_field((20, 17, 9), seed=4)
    A, L = 8, 3
    c = oracle_mod.eps_constants(x, oracle_mod.REL, 1e-30)
    it, od = oracle_mod.levels(L)
    out = oracle_mod.compress(x, A, it, od, c)
    col = oracle_mod.collect(x, out["codes"], A)
    n_anchor = int(np.prod(oracle_mod.anchor_dims(x.shape, A)))
    assert col["n_out"] == x.size - n_anchor
    assert np.array_equal(out["recon"].view(np.uint32), x.view(np.uint32))
    assert np.array_equal(np.sort(col["out_idx"]), col["out_idx"])


def test_constant_field(oracle_mod):
    x = np.full((19, 23, 5), -2.5, dtype=np.float32)
    c = oracle_mod.eps_constants(x, oracle_mod.REL, 1e-4)
    it, od = oracle_mod.levels(3)
    out = oracle_mod.compress(x, 8, it, od, c)
    assert np.all(out["codes"] == 128)
    assert np.array_equal(out["recon"], x)


def test_nonfinite_values_are_outliers(oracle_mod):
    x = fields.bumps_field((17, 17, 17), seed=5)
    x[3, 5, 7] = np.nan
    x[10, 1, 2] = np.inf
    x[16, 16, 15] = -np.inf
    A = 16
    it, od = oracle_mod.levels(4)
    out = oracle_mod.full_compress(x, A, it, od, oracle_mod.REL, 1e-3)
    for g in [(3, 5, 7), (10, 1, 2), (16, 16, 15)]:
        assert out["codes"][g] == 0
        assert out["recon"][g].view(np.uint32) == x[g].view(np.uint32)
    r = oracle_mod.decompress(x.shape, A, it, od, out["consts"]["ebx2_f"], out["codes"], out["anchors"],
                              out["out_idx"], out["out_val"])
    assert np.array_equal(r.view(np.uint32), out["recon"].view(np.uint32))


def test_code_range(oracle_mod):
    x = fields.bumps_field((33, 33, 17), seed=9)
    it, od = oracle_mod.levels(4)
    out = oracle_mod.full_compress(x, 16, it, od, oracle_mod.REL, 1e-4)
    codes = out["codes"]
    assert codes.min() >= 0 and codes.max() <= 255
    assert out["hist"].sum() == x.size - np.prod(oracle_mod.anchor_dims(x.shape, 16))
    assert out["hist"][0] == out["n_out"]


# --------------------------------------------------------------------------
# Eq. 1 and the round trip
# --------------------------------------------------------------------------
CASES = [
    (lambda: fields.bumps_field((64, 64, 64), seed=0), 8, 1e-3),
    (lambda: fields.lognormal_grf((48, 40, 56), seed=1), 16, 1e-2),
    (lambda: fields.lognormal_grf((48, 40, 56), seed=1), 16, 1e-4),
    (lambda: fields.fronts_2d((90, 180), seed=2), 16, 1e-3),
    (lambda: fields.stratified_3d((20, 50, 50), seed=3), 16, 1e-4),
    (lambda: fields.bumps_field((100,), seed=6), 8, 1e-3),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_error_bound_and_roundtrip(oracle_mod, case):
    make, A, eb = CASES[case]
    x = make()
    L = oracle_mod.n_levels(A)
    rng = np.random.default_rng(case)
    for trial in range(2):
        interp, order = _random_levels(rng, L, x.shape)
        out = oracle_mod.full_compress(x, A, interp, order, oracle_mod.REL, eb)
        eps = out["consts"]["eps"]
        err = np.abs(out["recon"].astype(np.float64) - x.astype(np.float64))
        assert err.max() < eps  # Eq. 1 (strict, see the eb_f reading)
        r = oracle_mod.decompress(x.shape, A, interp, order, out["consts"]["ebx2_f"], out["codes"],
                                  out["anchors"], out["out_idx"], out["out_val"])
        assert np.array_equal(r.view(np.uint32), out["recon"].view(np.uint32))
        # anchors verbatim
        sl = tuple(slice(0, None, A) for _ in x.shape)
        assert np.array_equal(out["anchors"], x[sl].reshape(-1))


def test_block_order_and_slab_independence(oracle_mod):
    """Blocks are independent (Sec. 3.2): processing order and slab splits at a
    multiple of A do not change any output."""
    x = fields.lognormal_grf((41, 30, 27), seed=8)
    A = 8
    L = 3
    it, od = _random_levels(np.random.default_rng(1), L, x.shape)
    c = oracle_mod.eps_constants(x, oracle_mod.REL, 1e-3)
    full = oracle_mod.compress(x, A, it, od, c)
    nb = int(np.prod(oracle_mod.block_grid(x.shape, A)))
    rev = oracle_mod.compress(x, A, it, od, c, tiles=np.arange(nb)[::-1])
    assert np.array_equal(full["codes"], rev["codes"])
    assert np.array_equal(full["recon"].view(np.uint32), rev["recon"].view(np.uint32))
    cut = 2 * A
    lo = oracle_mod.compress(np.ascontiguousarray(x[:cut + 1]), A, it, od, c)
    hi = oracle_mod.compress(np.ascontiguousarray(x[cut:]), A, it, od, c)
    assert np.array_equal(lo["codes"], full["codes"][:cut + 1])
    assert np.array_equal(hi["codes"], full["codes"][cut:])
    assert np.array_equal(hi["recon"].view(np.uint32), full["recon"][cut:].view(np.uint32))


def test_collect_definition(oracle_mod):
    x = fields.bumps_field((30, 20, 10), seed=12)
    it, od = oracle_mod.levels(3)
    c = oracle_mod.eps_constants(x, oracle_mod.REL, 1e-5)
    out = oracle_mod.compress(x, 8, it, od, c)
    col = oracle_mod.collect(x, out["codes"], 8)
    mask = out["codes"] == 0
    sl = tuple(slice(0, None, 8) for _ in x.shape)
    anchor = np.zeros(x.shape, dtype=bool)
    anchor[sl] = True
    mask &= ~anchor
    want = np.flatnonzero(mask.reshape(-1))
    assert np.array_equal(col["out_idx"], want.astype(np.uint32))
    assert np.array_equal(col["out_val"], x.reshape(-1)[want])
    h = np.bincount(out["codes"][~anchor], minlength=256)
    assert np.array_equal(col["hist"], h)
    # capacity smaller than the count: the count still reports everything
    small = oracle_mod.collect(x, out["codes"], 8, out_cap=3)
    assert small["n_out"] == col["n_out"] and np.array_equal(small["out_idx"], want[:3])


# --------------------------------------------------------------------------
# Auto-tuning (Sec. 5.1.3)
# --------------------------------------------------------------------------
def test_tune_samples(oracle_mod):
    # 0.2 % of the points in whole blocks: 0.002 * 512^3 / 16^3 = 65.5 -> 66
    assert oracle_mod.tune_samples((512, 512, 512), 16) == 66
    assert oracle_mod.tune_samples((64, 64, 64), 8) == 1  # 1.02 -> 1
    assert oracle_mod.tune_samples((1800, 3600), 16) == 51  # 0.002*6.48e6/256 = 50.6
    assert oracle_mod.tune_samples((100, 500, 500), 16) == 12  # 12.2
    assert oracle_mod.tune_samples((17, 17, 17), 16) == 1


def test_tune_configs(oracle_mod):
    """1D sequences (cubic, then linear, permutations in lexicographic order);
    with md, then the multi-dimensional scheme (cubic, then linear) when two
    or more dims are active."""
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    one_d = [(1, p) for p in perms] + [(0, p) for p in perms]
    assert oracle_mod.tune_configs((4, 5, 6)) == one_d
    assert oracle_mod.tune_configs((4, 5, 6), md=True) == one_d + [(3, (0, 1, 2)), (2, (0, 1, 2))]
    two_d = [(1, (1, 2, 0)), (1, (2, 1, 0)), (0, (1, 2, 0)), (0, (2, 1, 0))]
    assert oracle_mod.tune_configs((7, 9)) == two_d
    assert oracle_mod.tune_configs((7, 9), md=True) == two_d + [(3, (1, 2, 0)), (2, (1, 2, 0))]
    assert oracle_mod.tune_configs((9,)) == oracle_mod.tune_configs((9,), md=True) == [(1, (2, 0, 1)), (0, (2, 0, 1))]


@pytest.mark.parametrize("shape,A,md", [((40, 33, 35), 16, False), ((64, 64, 64), 8, True), ((100, 120), 16, True),
                                        ((300,), 8, False), ((40, 33, 35), 16, True)])
def test_tune_errors_bruteforce(oracle_mod, shape, A, md):
    x = fields.bumps_field(shape, seed=13)
    err = oracle_mod.tune_errors(x, A, md=md)
    L = oracle_mod.n_levels(A)
    cfgs = oracle_mod.tune_configs(shape, md=md)
    m = oracle_mod.tune_samples(shape, A)
    nb = oracle_mod.block_grid(shape, A)
    nblocks = int(np.prod(nb))
    stride = nblocks // m
    n3 = bf.dims3(shape)
    x3 = x.reshape(n3).astype(np.float64)
    want = np.zeros((L, len(cfgs)))
    npts = np.zeros((L, len(cfgs)))
    for k in range(m):
        t = k * stride
        tb = (t // (nb[1] * nb[2]), (t // nb[2]) % nb[1], t % nb[2])
        lo = [tb[d] * A for d in range(3)]
        hi = [min(lo[d] + A, n3[d] - 1) if n3[d] > 1 else 0 for d in range(3)]
        sub = x3[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1]
        for ci, (ip, od) in enumerate(cfgs):
            interp = [ip] * L
            order = [od] * L
            res = bf.open_loop_residuals(sub.astype(np.float32), A, interp, order)
            for g, r in res.items():
                l = bf.point_level(g, sub.shape, L)
                want[l, ci] += abs(float(r))
                npts[l, ci] += 1
    # the oracle evaluates each |x - p| in float32: a few ulps of max|x| per point
    tol = npts * 8 * float(np.finfo(np.float32).eps) * float(np.abs(x).max()) + 1e-7 * want
    assert np.all(np.abs(err - want) <= tol), (err, want)


def test_tune_select_argmin(oracle_mod):
    # 2D: 4 one-dimensional candidates, then multi-dimensional cubic and linear
    err = np.array([[3.0, 1.0, 1.0, 2.0], [0.0] * 4])
    interp, order = oracle_mod.tune_select((7, 9), 4, err)
    assert list(interp) == [1, 1]
    assert [tuple(o) for o in order] == [(2, 1, 0), (1, 2, 0)]
    err = np.array([[3.0, 1.0, 1.0, 2.0, 0.5, 4.0], [2.0, 2.0, 2.0, 2.0, 2.0, 1.0]])
    interp, order = oracle_mod.tune_select((7, 9), 4, err, md=True)
    assert list(interp) == [3, 2]


# --------------------------------------------------------------------------
# Entropy-based size estimate
# --------------------------------------------------------------------------
def test_entropy_estimate(oracle_mod):
    h = np.full(256, 10, dtype=np.uint32)
    e = oracle_mod.entropy_cr(h, 0, 0, 2560)
    assert abs(e["entropy_bits"] - 8.0) < 1e-12 and e["est_bytes"] == 2560
    h = np.zeros(256, dtype=np.uint32)
    h[128] = 1000
    e = oracle_mod.entropy_cr(h, 5, 7, 1012)
    assert e["entropy_bits"] == 0.0 and e["est_bytes"] == 8 * 5 + 4 * 7
    h = np.zeros(256, dtype=np.uint32)
    h[[127, 129]] = 4
    e = oracle_mod.entropy_cr(h, 0, 0, 8)
    assert e["entropy_bits"] == 1.0 and e["est_bytes"] == 1


def test_quantizer_boundaries(oracle_mod):
    """1D, A = 2, eps = 0.5 (2 eps = 1): the middle point is predicted as the
    mean of its two zero neighbours, so its code is fixed by x alone.

    |x - x'| must be strictly below eb_f (an error equal to the bound is an
    outlier), and |t| must be below 127.5 (codes 1..255)."""
    c = oracle_mod.eps_constants(np.zeros(3, np.float32), oracle_mod.ABS, 0.5)
    it, od = oracle_mod.levels(1, oracle_mod.LINEAR)
    cases = [(0.25, 128), (0.5, 0), (0.75, 129), (-0.75, 127), (1.5, 0), (127.25, 255), (-127.25, 1),
             (127.5, 0), (-127.5, 0), (126.75, 255), (3.0, 131)]
    for v, want in cases:
        x = np.array([0.0, v, 0.0], dtype=np.float32)
        out = oracle_mod.compress(x, 2, it, od, c)
        assert out["codes"][1] == want, (v, out["codes"][1], want)
        if want:
            assert abs(out["recon"][1] - v) < 0.5
        else:
            assert out["recon"][1] == v


# --------------------------------------------------------------------------
# Multi-dimensional interpolation scheme (Sec. 5.1.2)
# --------------------------------------------------------------------------
MD_SHAPES = [((9, 9, 9), 8), ((10, 7, 13), 8), ((17, 17, 17), 16), ((33, 20, 5), 16), ((12, 30), 4),
             ((5, 6, 7), 2), ((20, 19), 8)]


def _md_levels(rng, L, shape, p_md=0.6):
    """Random per-level configurations, each level multi-dimensional with probability p_md."""
    interp, order = _random_levels(rng, L, shape)
    for l in range(L):
        if rng.uniform() < p_md:
            interp[l] = bf.MD_LINEAR + int(rng.integers(0, 2))
    return interp, order


@pytest.mark.parametrize("shape,A", MD_SHAPES)
def test_md_trace_matches_bruteforce(oracle_mod, shape, A):
    """Level, averaged dims and their stencil order of every point, against the
    brute force built from the phase definition (points with 1, 2, 3 odd
    coordinates; the highest-order stencils averaged)."""
    rng = np.random.default_rng(31)
    L = oracle_mod.n_levels(A)
    for _ in range(4):
        interp, order = _md_levels(rng, L, shape)
        lvl, d, k = oracle_mod.trace(shape, A, interp, order)
        bl, bd, bk = bf.trace(shape, A, interp, order)
        assert np.array_equal(lvl, bl) and np.array_equal(d, bd) and np.array_equal(k, bk)
    for spline in (0, 1):
        assert bf.md_check_causality(shape, A, [spline] * L) == 0


@pytest.mark.parametrize("shape,A", [((17, 17, 17), 16), ((17, 33, 9), 8), ((33, 65), 16), ((9, 9, 9), 4)])
def test_md_linear_field_all_zero_codes(oracle_mod, shape, A):
    """Every stencil is exact for a linear field, so is every mean of them."""
    x = _linear_field(shape)
    L = oracle_mod.n_levels(A)
    c = oracle_mod.eps_constants(x, oracle_mod.ABS, 0.25)
    for spline in (bf.MD_LINEAR, bf.MD_CUBIC):
        interp = np.full(L, spline, dtype=np.uint8)
        order = np.tile(np.array([0, 1, 2], dtype=np.uint8), (L, 1))
        out = oracle_mod.compress(x, A, interp, order, c)
        assert np.all(out["codes"] == 128)
        assert np.array_equal(out["recon"].view(np.uint32), x.view(np.uint32))


@pytest.mark.parametrize("shape,A", [((17, 9, 10), 8), ((9, 9, 9), 8), ((13, 21), 4), ((6, 11, 7), 4)])
def test_md_codes_equal_exact_mean_residual(oracle_mod, shape, A):
    """Integer polynomial fields times 96: every 1D prediction is a multiple of
    6, so means of two and of three are exact integers, the closed loop is
    lossless at 2*eps = 1 and each code is 128 + (x - the exact mean of the
    highest-order predictions), or 0 out of range.  A wrong phase, a wrong
    choice of averaged dims or a wrong mean moves codes."""
    rng = np.random.default_rng(17)
    L = oracle_mod.n_levels(A)
    x = (_int_poly(shape, rng, deg=2, scale=1).astype(np.float64) * 96).astype(np.float32)
    c = oracle_mod.eps_constants(x, oracle_mod.ABS, 0.5)
    for _ in range(3):
        interp, order = _md_levels(rng, L, shape, p_md=1.0)
        out = oracle_mod.compress(x, A, interp, order, c)
        assert np.array_equal(out["recon"].view(np.uint32), x.view(np.uint32))
        res = bf.open_loop_residuals(x, A, interp, order)
        codes = out["codes"].reshape(bf.dims3(shape))
        for g, r in res.items():
            assert r.denominator == 1
            want = 128 + int(r) if abs(r) <= 127 else 0
            assert codes[g] == want, (g, r, codes[g])


def test_md_mean_of_two_and_three(oracle_mod):
    """Hand values on one 3x3x3 block (A = 2, one level, linear splines) of
    f = x*y*z + x*y: the point (1,1,1) averages three midpoint predictions,
    (1,1,0) two; with 2*eps = 1 the codes are 128 + x - mean."""
    n = 3
    g = np.meshgrid(*[np.arange(n, dtype=np.float64)] * 3, indexing="ij")
    f = (g[0] * g[1] * g[2] + g[0] * g[1]) * 6.0
    x = f.astype(np.float32)
    c = oracle_mod.eps_constants(x, oracle_mod.ABS, 0.5)
    interp = np.array([bf.MD_LINEAR], dtype=np.uint8)
    order = np.array([[0, 1, 2]], dtype=np.uint8)
    out = oracle_mod.compress(x, 2, interp, order, c)
    codes = out["codes"].astype(int) - 128
    # (1,0,0): along x only: (f(0,0,0) + f(2,0,0)) / 2 = 0 = f -> 0
    assert codes[1, 0, 0] == 0
    # (1,1,0): x and y midpoints of f = 6xy at z = 0: along x (0,1,0)=0,(2,1,0)=12 -> 6;
    # along y (1,0,0)=0,(1,2,0)=12 -> 6; mean 6 = f(1,1,0) -> 0
    assert codes[1, 1, 0] == 0
    # (1,1,1): f = 6xyz + 6xy; along x: (f(0,1,1) + f(2,1,1))/2 = (0 + 24)/2 = 12,
    # along y: (f(1,0,1) + f(1,2,1))/2 = (0 + 24)/2 = 12, along z: (f(1,1,0) + f(1,1,2))/2 = (6 + 18)/2 = 12;
    # mean 12 = f(1,1,1) -> 0
    assert codes[1, 1, 1] == 0
    # f = 6 x^2 y: at (1,1,0): along x (0 + 24)/2 = 12 vs f = 6 -> residual -6;
    # along y (0 + 12)/2 = 6 -> 0; both linear: mean 9 -> code -3
    x2 = (6.0 * g[0] ** 2 * g[1]).astype(np.float32)
    out = oracle_mod.compress(x2, 2, interp, order, oracle_mod.eps_constants(x2, oracle_mod.ABS, 0.5))
    assert int(out["codes"][1, 1, 0]) - 128 == 6 - 9


@pytest.mark.parametrize("shape,A,workers", [((70, 40, 36), 16, 3), ((33, 20, 17), 8, 4), ((1, 90, 70), 16, 2)])
def test_parallel_oracle_equals_serial(oracle_mod, shape, A, workers):
    """The multi-threaded oracle leg of the benchmark (blocks split into d0
    slabs over host threads) gives the serial oracle's codes, anchors and
    reconstruction bit for bit, and its decompression the same field."""
    x = fields.lognormal_grf(shape, seed=3)
    c = oracle_mod.eps_constants(x, oracle_mod.REL, 1e-3)
    L = oracle_mod.n_levels(A)
    interp, order = oracle_mod.levels(L, oracle_mod.CUBIC, (0, 1, 2))
    a = oracle_mod.compress(x, A, interp, order, c)
    b = oracle_mod.compress_parallel(x, A, interp, order, c, workers)
    for k in ("codes", "anchors"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["recon"].view(np.uint32), b["recon"].view(np.uint32))
    col = oracle_mod.collect(x, a["codes"], A)
    y = oracle_mod.decompress_parallel(x.shape, A, interp, order, c["ebx2_f"], a["codes"], a["anchors"],
                                       col["out_idx"], col["out_val"], workers)
    assert np.array_equal(y.view(np.uint32), a["recon"].view(np.uint32))
