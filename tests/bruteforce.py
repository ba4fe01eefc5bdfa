"""Independent brute-force formulations used to pin the oracle (test helpers).

Nothing here is copied from the oracle: the level of a point is derived from
the trailing zeros of its coordinates (the level definition of Eq. 3), the
pass from the last dimension of the level's sequence whose coordinate is an
odd multiple of the stride, and the prediction weights from the Lagrange
formula over the available nodes, in exact rational arithmetic.
"""
from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np

LINEAR, CUBIC = 0, 1
MD_LINEAR, MD_CUBIC = 2, 3  # multi-dimensional scheme; its spline is interp - 2

# order of each stencil case (the numbering of stencil_nodes): cubic 3,
# quadratic 2, linear midpoint / extrapolation 1, copy 0
ORDER_OF_CASE = {1: 3, 2: 2, 3: 2, 0: 1, 4: 1, 5: 0}


def trailing_zeros(v, cap):
    if v == 0:
        return cap
    n = 0
    while v % 2 == 0:
        v //= 2
        n += 1
    return min(n, cap)


def dims3(shape):
    return (1,) * (3 - len(shape)) + tuple(int(s) for s in shape)


def active_dims(n3):
    return [d for d in range(3) if n3[d] > 1]


def point_level(g, n3, L):
    """Level of the prediction of point g; L for an anchor (Eq. 3's level)."""
    act = active_dims(n3)
    if not act:
        return L
    return min(trailing_zeros(g[d], L) for d in act)


def point_direction(g, lvl, order_l):
    """The last dimension of the level's sequence along which g is an odd multiple of 2^lvl."""
    s = 1 << lvl
    last = None
    for d in order_l:
        if g[d] % s == 0 and (g[d] // s) % 2 == 1:
            last = d
    return last


def stencil_nodes(g, d, lvl, n_d, A, interp):
    """(case, node offsets in units of the stride) for point g predicted along d."""
    s = 1 << lvl
    b = g[d] // A
    c = g[d] - b * A
    e = min(A, n_d - 1 - b * A)
    have_r = c + s <= e
    have_l3 = c - 3 * s >= 0
    have_r3 = c + 3 * s <= e
    if not have_r:
        return (4, (-3, -1)) if have_l3 else (5, (-1,))
    if interp == LINEAR:
        return 0, (-1, 1)
    if have_l3 and have_r3:
        return 1, (-3, -1, 1, 3)
    if have_r3:
        return 2, (-1, 1, 3)
    if have_l3:
        return 3, (-3, -1, 1)
    return 0, (-1, 1)


def lagrange_weights(nodes):
    """Exact weights of the Lagrange interpolant through ``nodes`` evaluated at 0."""
    w = []
    for i, ni in enumerate(nodes):
        num = Fraction(1)
        for j, nj in enumerate(nodes):
            if j != i:
                num *= Fraction(0 - nj, ni - nj)
        w.append(num)
    return w


def md_odd_dims(g, lvl, n3):
    """Active dims along which g is an odd multiple of 2^lvl."""
    s = 1 << lvl
    return [d for d in active_dims(n3) if g[d] % s == 0 and (g[d] // s) % 2 == 1]


def md_choice(g, lvl, n3, A, spline):
    """Multi-dimensional scheme at point g: the dims whose 1D stencils have
    the highest order among the odd dims, that order, and their node sets."""
    odd = md_odd_dims(g, lvl, n3)
    st = {d: stencil_nodes(g, d, lvl, n3[d], A, spline) for d in odd}
    best = max(ORDER_OF_CASE[st[d][0]] for d in odd)
    use = [d for d in odd if ORDER_OF_CASE[st[d][0]] == best]
    return use, best, {d: st[d][1] for d in use}


def trace(shape, A, interp, order):
    """(lvl, dir, case) arrays like the oracle's trace, from the definitions above
    (multi-dimensional levels: dir = 3 + mask of the averaged dims, case = their order)."""
    n3 = dims3(shape)
    L = A.bit_length() - 1
    lvl = np.full(n3, -1, dtype=np.int8)
    dr = np.full(n3, -1, dtype=np.int8)
    kc = np.full(n3, -1, dtype=np.int8)
    for g in itertools.product(*[range(n) for n in n3]):
        l = point_level(g, n3, L)
        if l >= L:
            continue
        if interp[l] >= MD_LINEAR:
            use, best, _ = md_choice(g, l, n3, A, interp[l] - MD_LINEAR)
            lvl[g], dr[g], kc[g] = l, 3 + sum(1 << d for d in use), best
            continue
        d = point_direction(g, l, order[l])
        case, _ = stencil_nodes(g, d, l, n3[d], A, interp[l])
        lvl[g], dr[g], kc[g] = l, d, case
    return lvl.reshape(shape), dr.reshape(shape), kc.reshape(shape)


def md_check_causality(shape, A, splines):
    """Every level multi-dimensional (splines[l]): each stencil node of a point
    with k odd dims must be an anchor, on a coarser level, or on the same level
    with fewer odd dims.  Returns the number of violations."""
    n3 = dims3(shape)
    L = A.bit_length() - 1
    bad = 0
    for g in itertools.product(*[range(n) for n in n3]):
        l = point_level(g, n3, L)
        if l >= L:
            continue
        k = len(md_odd_dims(g, l, n3))
        for d in md_odd_dims(g, l, n3):
            _, nodes = stencil_nodes(g, d, l, n3[d], A, splines[l])
            for j in nodes:
                h = list(g)
                h[d] += j * (1 << l)
                h = tuple(h)
                if not all(0 <= h[q] < n3[q] for q in range(3)):
                    bad += 1
                    continue
                lh = point_level(h, n3, L)
                if lh > l or (lh == l and len(md_odd_dims(h, l, n3)) < k):
                    continue
                bad += 1
    return bad


def check_causality(shape, A, interp, order):
    """Every stencil node must be an anchor, on a coarser level, or on the same
    level in an earlier pass.  Returns the number of violations."""
    n3 = dims3(shape)
    L = A.bit_length() - 1
    bad = 0
    for g in itertools.product(*[range(n) for n in n3]):
        l = point_level(g, n3, L)
        if l >= L:
            continue
        d = point_direction(g, l, order[l])
        pos = list(order[l]).index(d)
        _, nodes = stencil_nodes(g, d, l, n3[d], A, interp[l])
        for k in nodes:
            h = list(g)
            h[d] += k * (1 << l)
            h = tuple(h)
            if not all(0 <= h[q] < n3[q] for q in range(3)):
                bad += 1
                continue
            lh = point_level(h, n3, L)
            if lh > l:
                continue
            if lh == l and list(order[l]).index(point_direction(h, l, order[l])) < pos:
                continue
            bad += 1
    return bad


def _line_prediction(x3, g, d, l, nodes):
    w = lagrange_weights(nodes)
    p = Fraction(0)
    for wi, k in zip(w, nodes):
        h = list(g)
        h[d] += k * (1 << l)
        p += wi * Fraction(float(x3[tuple(h)]))
    return p


def open_loop_residuals(x, A, interp, order):
    """Per point: x(g) - sum_i w_i x(g + n_i s e_d), exact rationals of the float inputs
    (None at anchors).  Multi-dimensional levels: x(g) - the exact mean of the
    predictions along the dims md_choice keeps."""
    n3 = dims3(x.shape)
    x3 = x.reshape(n3)
    L = A.bit_length() - 1
    out = {}
    for g in itertools.product(*[range(n) for n in n3]):
        l = point_level(g, n3, L)
        if l >= L:
            continue
        if interp[l] >= MD_LINEAR:
            use, _, nodes = md_choice(g, l, n3, A, interp[l] - MD_LINEAR)
            p = sum(_line_prediction(x3, g, d, l, nodes[d]) for d in use) / len(use)
            out[g] = Fraction(float(x3[g])) - p
            continue
        d = point_direction(g, l, order[l])
        _, nodes = stencil_nodes(g, d, l, n3[d], A, interp[l])
        w = lagrange_weights(nodes)
        p = Fraction(0)
        for wi, k in zip(w, nodes):
            h = list(g)
            h[d] += k * (1 << l)
            p += wi * Fraction(float(x3[tuple(h)]))
        out[g] = Fraction(float(x3[g])) - p
    return out
