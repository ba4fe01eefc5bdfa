"""Pins of the oracle's quantization-code reordering (Sec. 5.2.2, Eq. 3).

The printed mapping is checked against a different formulation of what the
paper says it does: the codes of one interpolation level lie together,
coarser levels first (the anchors at the front), and within a level they keep
the row-major order of the field -- i.e. I is the position of a point in the
stable sort of all points by descending level.  The level of a point comes
from its definition (the largest l <= log2 A with 2^l dividing every
coordinate), found here by trial division.
"""
import numpy as np
import pytest

import oracle

SHAPES = [((9, 9, 9), 8), ((10, 7, 13), 8), ((17, 17, 17), 16), ((33, 20, 5), 16), ((12, 30), 4),
          ((21,), 4), ((5, 1, 19), 8), ((2, 3, 4), 2), ((1, 1, 1), 8), ((40,), 32), ((6, 11, 14), 4),
          ((1, 18, 1), 2), ((3, 3, 3), 16)]


def _dims3(shape):
    return (1,) * (3 - len(shape)) + tuple(shape)


def _level(c, A):
    l = 0
    while 2 ** (l + 1) <= A and all(v % 2 ** (l + 1) == 0 for v in c):
        l += 1
    return l


def _sorted_positions(shape, A):
    d = _dims3(shape)
    pts = [(x, y, z) for x in range(d[0]) for y in range(d[1]) for z in range(d[2])]
    lv = [_level(c, A) for c in pts]
    order = sorted(range(len(pts)), key=lambda p: -lv[p])  # stable: row-major within a level
    pos = np.empty(len(pts), dtype=np.int64)
    pos[order] = np.arange(len(pts))
    return pos, np.array(lv)


@pytest.mark.parametrize("shape,A", SHAPES)
def test_matches_stable_sort_by_level(shape, A):
    pos, _ = _sorted_positions(shape, A)
    assert np.array_equal(oracle.reorder_index(shape, A), pos)


@pytest.mark.parametrize("shape,A", SHAPES)
def test_level_blocks_start_at_prefix(shape, A):
    """Level l < log2 A starts after the f_x(l) f_y(l) f_z(l) coarser points,
    f(0) = floor((d + 1) / 2), f(k + 1) = floor((f(k) + 1) / 2) (Eq. 3's
    prefix, which counts the points whose coordinates are all multiples of
    2^(l + 1))."""
    I = oracle.reorder_index(shape, A)
    _, lv = _sorted_positions(shape, A)
    L = A.bit_length() - 1
    d = _dims3(shape)
    f = [(n + 1) // 2 for n in d]
    for l in range(L):
        sel = lv == l
        if sel.any():
            assert I[sel].min() == f[0] * f[1] * f[2]
            assert I[sel].max() == (I.size if l == 0 else prefix_prev) - 1
        prefix_prev = f[0] * f[1] * f[2]
        f = [(n + 1) // 2 for n in f]
    n_anchor = int(np.prod([(n - 1) // A + 1 for n in d]))
    assert np.array_equal(np.sort(I[lv == L]), np.arange(n_anchor))


def test_level0_rank_is_the_printed_formula():
    """For l = 0, Eq. 3 as printed on the global grid: x dy dz + y dz + z
    minus the all-even points before (x, y, z)."""
    shape, A = (7, 10, 9), 4
    I = oracle.reorder_index(shape, A)
    dx, dy, dz = shape
    h = lambda v: (v + 1) // 2
    pre0 = h(dx) * h(dy) * h(dz)
    p = 0
    for x in range(dx):
        for y in range(dy):
            for z in range(dz):
                if x % 2 or y % 2 or z % 2:
                    r = x * dy * dz + y * dz + z - h(x) * h(dy) * h(dz)
                    r -= (x % 2 == 0) * h(y) * h(dz) + (x % 2 == 0 and y % 2 == 0) * h(z)
                    assert I[p] == pre0 + r
                p += 1


@pytest.mark.parametrize("shape,A", [((33, 47, 65), 16), ((64, 64, 64), 8), ((1000,), 16), ((129, 77), 32),
                                     ((48, 48, 48), 2)])
def test_bijection(shape, A):
    I = oracle.reorder_index(shape, A)
    assert np.array_equal(np.sort(I), np.arange(I.size))


def test_roundtrip_and_grouping():
    rng = np.random.default_rng(3)
    shape, A = (20, 33, 18), 8
    c = rng.integers(0, 256, size=shape, dtype=np.uint8)
    seq = oracle.reorder_codes(c, A)
    assert np.array_equal(oracle.unreorder_codes(seq, shape, A), c)
    # a field holding each point's level comes out non-increasing
    _, lv = _sorted_positions(shape, A)
    s = oracle.reorder_codes(lv.astype(np.uint8).reshape(shape), A)
    assert np.all(np.diff(s.astype(np.int64)) <= 0)


def test_rejects_bad_stride():
    with pytest.raises(ValueError):
        oracle.reorder_index((8, 8, 8), 12)
    with pytest.raises(ValueError):
        oracle.reorder_index((8, 8, 8), 1)
