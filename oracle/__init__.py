"""CPU oracle for the interpolation predictor / quantizer (cuSZ-Hi, arXiv 2507.11165).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
timed CPU baseline of ``bench.py`` may import this package.  The product path
(``paper_2507_11165_gb300``) never imports, links or calls it, and this package
imports nothing from the product path except the seeded input generators
(``paper_2507_11165_gb300.fields``), which hold none of the method's arithmetic.

The arithmetic lives in ``hi_oracle.c`` (plain C, float32, fixed evaluation
order, built with ``-ffp-contract=off``); this module only marshals numpy
arrays.  Sections followed: Sec. 3.1 Eq. 1 (error bound), Sec. 3.2 (anchors and
hierarchical interpolation), Sec. 5.1.1 (blocks), Sec. 5.1.2 (splines along a
dimension sequence), Sec. 5.1.3 (auto-tuning), Sec. 5.2.1 (uint8 codes and
separate outliers), Sec. 6.1.4 (value-range-relative bound).

Entropy-based size estimate (``entropy_cr``): Sec. 5.1.4 notes the Huffman
stage depends only on the code frequencies; the estimate is the order-0
entropy of the code histogram plus raw outlier and anchor bytes.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hi_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libhi_oracle.so")

CFLAGS = ["-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
          "-fno-tree-vectorize", "-fno-finite-math-only"]

LINEAR, CUBIC = 0, 1
MD_LINEAR, MD_CUBIC = 2, 3  # multi-dimensional interpolation scheme (Sec. 5.1.2)
RADIUS = 128
ABS, REL = 0, 1

_lock = threading.Lock()
_lib = None

ERRORS = {
    1: "invalid argument", 2: "out of memory", 10: "stencil point read before it was known",
    11: "point predicted twice", 12: "point never predicted", 13: "blocks disagree on a shared face",
    14: "code 0 without an outlier value", 15: "corrupt lossless stream",
}


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile hi_oracle.c into a shared library (gcc); returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            lib.hi_oracle_eps.argtypes = [ctypes.c_int, ctypes.c_double, P, i64, P, P]
            lib.hi_oracle_compress.argtypes = [P, ctypes.c_int, P, P, P, P, P, i64, P, P, P]
            lib.hi_oracle_collect.argtypes = [P, ctypes.c_int, P, P, P, P, i64, P, P]
            lib.hi_oracle_decompress.argtypes = [P, ctypes.c_int, P, P, ctypes.c_float, P, P, P, P, i64,
                                                 P, i64, P]
            lib.hi_oracle_tune_samples.argtypes = [P, ctypes.c_int]
            lib.hi_oracle_tune_samples.restype = i64
            lib.hi_oracle_tune_configs.argtypes = [P, ctypes.c_int, P, P]
            lib.hi_oracle_tune_errors.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, P]
            lib.hi_oracle_tune_errors_tiles.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, i64, P, P]
            lib.hi_oracle_tune_select.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, P]
            lib.hi_oracle_trace.argtypes = [P, ctypes.c_int, P, P, P, P, P]
            lib.hi_oracle_reorder_index.argtypes = [P, ctypes.c_int, P]
            lib.hi_oracle_tp_bound.argtypes = [i64]
            lib.hi_oracle_tp_bound.restype = i64
            lib.hi_oracle_tp_encode.argtypes = [P, i64, P, i64, P]
            lib.hi_oracle_tp_decode.argtypes = [P, i64, P, i64]
            lib.hi_oracle_hf_lengths.argtypes = [P, P]
            lib.hi_oracle_cr_bound.argtypes = [i64]
            lib.hi_oracle_cr_bound.restype = i64
            lib.hi_oracle_cr_encode.argtypes = [P, i64, P, i64, P]
            lib.hi_oracle_cr_decode.argtypes = [P, i64, P, i64]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc):
    if rc != 0:
        raise OracleError("oracle error %d: %s" % (rc, ERRORS.get(rc, "?")))


def _dims3(shape):
    shape = tuple(int(s) for s in shape)
    if not 1 <= len(shape) <= 3:
        raise ValueError("1-3 dims")
    return np.array((1,) * (3 - len(shape)) + shape, dtype=np.int64)


def levels(n_levels, interp=CUBIC, order=(0, 1, 2)):
    """Uniform per-level configuration arrays (interp[L], order[L,3])."""
    return (np.full(n_levels, interp, dtype=np.uint8),
            np.tile(np.array(order, dtype=np.uint8), (n_levels, 1)))


def eps_constants(x, eb_mode, eb):
    """(eb_f, ebx2_f, r_f, vmin, vmax, eps) for the field x (Eq. 1; value-range-relative bound)."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1)
    out = np.zeros(5, dtype=np.float32)
    eps = np.zeros(1, dtype=np.float64)
    _check(lib.hi_oracle_eps(int(eb_mode), float(eb), _p(x), x.size, _p(out), _p(eps)))
    return dict(eb_f=out[0], ebx2_f=out[1], r_f=out[2], vmin=out[3], vmax=out[4], eps=float(eps[0]))


def n_levels(A):
    L = int(A).bit_length() - 1
    if A < 2 or (1 << L) != A:
        raise ValueError("anchor stride must be a power of two")
    return L


def anchor_dims(shape, A):
    d = _dims3(shape)
    return tuple(int((n - 1) // A + 1) for n in d)


def block_grid(shape, A):
    d = _dims3(shape)
    return tuple(1 if n == 1 else int((n - 1 + A - 1) // A) for n in d)


def compress(x, A, interp, order, consts, tiles=None):
    """Predict + quantize.  Returns dict(codes, anchors, recon, written_mask_tiles).

    ``interp`` is uint8[L], ``order`` uint8[L,3] (order[l] = dimension
    sequence of level l, stride 2^l).  ``consts`` is the dict of
    :func:`eps_constants`.  With ``tiles`` (linear block ids) only those
    blocks are computed; other points of the outputs stay at their fill
    value (codes 0xFF... not meaningful)."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float32)
    dims = _dims3(x.shape)
    L = n_levels(A)
    interp = np.ascontiguousarray(interp, dtype=np.uint8).reshape(L)
    order = np.ascontiguousarray(order, dtype=np.uint8).reshape(L, 3)
    c = np.array([consts["eb_f"], consts["ebx2_f"], consts["r_f"]], dtype=np.float32)
    codes = np.zeros(x.shape, dtype=np.uint8)
    recon = np.zeros(x.shape, dtype=np.float32)
    anchors = np.zeros(anchor_dims(x.shape, A), dtype=np.float32)
    t = None if tiles is None else np.ascontiguousarray(tiles, dtype=np.int64)
    _check(lib.hi_oracle_compress(_p(dims), int(A), _p(interp), _p(order), _p(c), _p(x), _p(t),
                                  0 if t is None else t.size, _p(codes), _p(anchors), _p(recon)))
    return dict(codes=codes, anchors=anchors.reshape(-1), recon=recon)


def collect(x, codes, A, out_cap=None):
    """Outlier list (ascending index) and the 256-bin code histogram of non-anchor points."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float32)
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    dims = _dims3(x.shape)
    if out_cap is None:
        out_cap = int(np.count_nonzero(codes == 0))
    idx = np.zeros(max(out_cap, 1), dtype=np.uint32)
    val = np.zeros(max(out_cap, 1), dtype=np.float32)
    n = np.zeros(1, dtype=np.int64)
    hist = np.zeros(256, dtype=np.uint32)
    _check(lib.hi_oracle_collect(_p(dims), int(A), _p(x), _p(codes), _p(idx), _p(val), out_cap, _p(n),
                                 _p(hist)))
    k = min(int(n[0]), out_cap)
    return dict(out_idx=idx[:k].copy(), out_val=val[:k].copy(), n_out=int(n[0]), hist=hist)


def decompress(shape, A, interp, order, ebx2_f, codes, anchors, out_idx, out_val, tiles=None):
    """Level-by-level reconstruction from codes, anchors and outliers."""
    lib = _load()
    dims = _dims3(shape)
    L = n_levels(A)
    interp = np.ascontiguousarray(interp, dtype=np.uint8).reshape(L)
    order = np.ascontiguousarray(order, dtype=np.uint8).reshape(L, 3)
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    anchors = np.ascontiguousarray(anchors, dtype=np.float32)
    out_idx = np.ascontiguousarray(out_idx, dtype=np.uint32)
    out_val = np.ascontiguousarray(out_val, dtype=np.float32)
    recon = np.zeros(tuple(shape), dtype=np.float32)
    t = None if tiles is None else np.ascontiguousarray(tiles, dtype=np.int64)
    _check(lib.hi_oracle_decompress(_p(dims), int(A), _p(interp), _p(order), ctypes.c_float(ebx2_f),
                                    _p(codes), _p(anchors), _p(out_idx), _p(out_val), out_idx.size,
                                    _p(t), 0 if t is None else t.size, _p(recon)))
    return recon


def tune_samples(shape, A):
    return int(_load().hi_oracle_tune_samples(_p(_dims3(shape)), int(A)))


def tune_configs(shape, md=False):
    """Candidate (interp, order) per level in enumeration order (md: with the
    multi-dimensional scheme's two candidates)."""
    ci = np.zeros(14, dtype=np.uint8)
    co = np.zeros(42, dtype=np.uint8)
    n = _load().hi_oracle_tune_configs(_p(_dims3(shape)), int(bool(md)), _p(ci), _p(co))
    return [(int(ci[k]), tuple(int(v) for v in co[3 * k:3 * k + 3])) for k in range(n)]


def tune_errors(x, A, md=False):
    """err[L, ncfg]: open-loop sum |x - p| per level and candidate (Sec. 5.1.3)."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float32)
    L = n_levels(A)
    err = np.zeros(L * 14, dtype=np.float64)
    nc = np.zeros(1, dtype=np.int32)
    _check(lib.hi_oracle_tune_errors(_p(_dims3(x.shape)), int(A), int(bool(md)), _p(x), _p(err), _p(nc)))
    return err[:L * int(nc[0])].reshape(L, int(nc[0]))


def tune_errors_tiles(x, A, tiles, md=False):
    """err[k, L, ncfg]: the terms of :func:`tune_errors` of block tiles[k]
    (row-major block ids of x), one block at a time."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float32)
    L = n_levels(A)
    t = np.ascontiguousarray(tiles, dtype=np.int64)
    err = np.zeros(max(1, t.size) * L * 14, dtype=np.float64)
    nc = np.zeros(1, dtype=np.int32)
    _check(lib.hi_oracle_tune_errors_tiles(_p(_dims3(x.shape)), int(A), int(bool(md)), _p(x), _p(t), t.size,
                                           _p(err), _p(nc)))
    n = int(nc[0])
    return err[:t.size * L * n].reshape(t.size, L, n)


def tune_select(shape, A, err, md=False):
    lib = _load()
    L = n_levels(A)
    err = np.ascontiguousarray(err, dtype=np.float64)
    interp = np.zeros(L, dtype=np.uint8)
    order = np.zeros((L, 3), dtype=np.uint8)
    _check(lib.hi_oracle_tune_select(_p(_dims3(shape)), int(A), int(bool(md)), _p(err), _p(interp), _p(order)))
    return interp, order


def entropy_cr(hist, n_out, n_anchor, n_points, header_bytes=0):
    """Estimated compression ratio: 4 N / (ceil(N_pred H / 8) + 8 n_out + 4 n_anchor + header).

    H is the order-0 entropy (bits/symbol) of the code histogram."""
    hist = np.asarray(hist, dtype=np.float64)
    total = hist.sum()
    H = 0.0
    if total > 0:
        for c in hist:
            if c > 0:
                q = c / total
                H -= q * math.log2(q)
    nbytes = math.ceil(total * H / 8.0) + 8 * n_out + 4 * n_anchor + header_bytes
    return dict(entropy_bits=H, est_bytes=int(nbytes),
                cr=(4.0 * n_points / nbytes) if nbytes > 0 else float("inf"))


def trace(shape, A, interp, order):
    """Per point: level, dimension and stencil case of its prediction (-1 at anchors).

    Cases: 0 linear midpoint, 1 cubic 4-point, 2 quadratic without f(c-3s),
    3 quadratic without f(c+3s), 4 linear extrapolation, 5 copy of f(c-s)."""
    lib = _load()
    dims = _dims3(shape)
    L = n_levels(A)
    interp = np.ascontiguousarray(interp, dtype=np.uint8).reshape(L)
    order = np.ascontiguousarray(order, dtype=np.uint8).reshape(L, 3)
    lvl = np.zeros(tuple(shape), dtype=np.int8)
    d = np.zeros(tuple(shape), dtype=np.int8)
    k = np.zeros(tuple(shape), dtype=np.int8)
    _check(lib.hi_oracle_trace(_p(dims), int(A), _p(interp), _p(order), _p(lvl), _p(d), _p(k)))
    return lvl, d, k


def _slab_tiles(shape, A, workers):
    """Row-major block ids split into slabs of whole block planes along the
    slowest dim with more than one block (one slab list per phase: even
    slabs, then odd slabs), so that slabs that share a face plane never run
    at the same time."""
    nb = block_grid(shape, A)
    d = next((k for k in range(3) if nb[k] > 1), 2)
    per_plane = int(np.prod(nb[d + 1:], dtype=np.int64))
    n_slabs = max(1, min(nb[d], 2 * workers))
    cuts = [nb[d] * k // n_slabs for k in range(n_slabs + 1)]
    slabs = [np.arange(cuts[k] * per_plane, cuts[k + 1] * per_plane, dtype=np.int64) for k in range(n_slabs)]
    return [slabs[0::2], slabs[1::2]]


def compress_parallel(x, A, interp, order, consts, workers):
    """:func:`compress` with the independent blocks (Sec. 5.1.1) spread over
    ``workers`` host threads: the same C routine called on disjoint block
    lists into shared output arrays (the library call releases the GIL).
    Blocks that share a face plane are never processed at the same time."""
    import concurrent.futures as cf
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float32)
    dims = _dims3(x.shape)
    L = n_levels(A)
    interp = np.ascontiguousarray(interp, dtype=np.uint8).reshape(L)
    order = np.ascontiguousarray(order, dtype=np.uint8).reshape(L, 3)
    c = np.array([consts["eb_f"], consts["ebx2_f"], consts["r_f"]], dtype=np.float32)
    codes = np.zeros(x.shape, dtype=np.uint8)
    recon = np.zeros(x.shape, dtype=np.float32)
    anchors = np.zeros(anchor_dims(x.shape, A), dtype=np.float32)

    def run(t):
        return lib.hi_oracle_compress(_p(dims), int(A), _p(interp), _p(order), _p(c), _p(x), _p(t), t.size,
                                      _p(codes), _p(anchors), _p(recon))

    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        for phase in _slab_tiles(x.shape, A, workers):
            for rc in ex.map(run, phase):
                _check(rc)
    return dict(codes=codes, anchors=anchors.reshape(-1), recon=recon)


def decompress_parallel(shape, A, interp, order, ebx2_f, codes, anchors, out_idx, out_val, workers):
    """:func:`decompress` with the blocks spread over host threads as in
    :func:`compress_parallel`."""
    import concurrent.futures as cf
    lib = _load()
    dims = _dims3(shape)
    L = n_levels(A)
    interp = np.ascontiguousarray(interp, dtype=np.uint8).reshape(L)
    order = np.ascontiguousarray(order, dtype=np.uint8).reshape(L, 3)
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    anchors = np.ascontiguousarray(anchors, dtype=np.float32)
    out_idx = np.ascontiguousarray(out_idx, dtype=np.uint32)
    out_val = np.ascontiguousarray(out_val, dtype=np.float32)
    recon = np.zeros(tuple(shape), dtype=np.float32)

    def run(t):
        return lib.hi_oracle_decompress(_p(dims), int(A), _p(interp), _p(order), ctypes.c_float(ebx2_f),
                                        _p(codes), _p(anchors), _p(out_idx), _p(out_val), out_idx.size,
                                        _p(t), t.size, _p(recon))

    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        for phase in _slab_tiles(shape, A, workers):
            for rc in ex.map(run, phase):
                _check(rc)
    return recon


def full_compress(x, A, interp, order, eb_mode, eb):
    """Convenience: constants + compress + outlier/histogram collection."""
    consts = eps_constants(x, eb_mode, eb)
    out = compress(x, A, interp, order, consts)
    col = collect(x, out["codes"], A)
    out.update(col)
    out["consts"] = consts
    return out


# ---------------------------------------------------------------------------
# Quantization-code reordering (Sec. 5.2.2, Eq. 3)
# ---------------------------------------------------------------------------
def reorder_index(shape, A):
    """I(x, y, z) of Eq. 3 for every point of the field, in row-major order
    (int64, one entry per point): codes grouped by interpolation level,
    coarsest (the anchors) first, row-major within a level."""
    lib = _load()
    d = _dims3(shape)
    n_levels(A)
    out = np.empty(int(np.prod(d)), dtype=np.int64)
    _check(lib.hi_oracle_reorder_index(_p(d), int(A), _p(out)))
    return out


def reorder_codes(codes, A):
    """The code array (any 1-3D shape) as the 1D sequence of Eq. 3."""
    codes = np.ascontiguousarray(codes)
    idx = reorder_index(codes.shape, A)
    seq = np.empty(codes.size, dtype=codes.dtype)
    seq[idx] = codes.reshape(-1)
    return seq


def unreorder_codes(seq, shape, A):
    """Inverse of reorder_codes: the code array of ``shape`` from its sequence."""
    idx = reorder_index(shape, A)
    return np.asarray(seq).reshape(-1)[idx].reshape(tuple(int(s) for s in shape))


# ---------------------------------------------------------------------------
# Throughput-mode lossless pipeline TCMS1-BIT1-RRE1 (Sec. 5.2.3)
# ---------------------------------------------------------------------------
TP_CHUNK = 16384


def tp_bound(n):
    """Largest stream tp_encode can produce for n input bytes."""
    return int(_load().hi_oracle_tp_bound(int(n)))


def tp_encode(data):
    """The TCMS1-BIT1-RRE1 stream (uint8 array) of a byte sequence."""
    lib = _load()
    data = np.ascontiguousarray(data, dtype=np.uint8).reshape(-1)
    out = np.zeros(tp_bound(data.size), dtype=np.uint8)
    ln = np.zeros(1, dtype=np.int64)
    _check(lib.hi_oracle_tp_encode(_p(data), data.size, _p(out), out.size, _p(ln)))
    return out[: int(ln[0])].copy()


def tp_decode(stream, n):
    """The n bytes a TCMS1-BIT1-RRE1 stream encodes."""
    lib = _load()
    stream = np.ascontiguousarray(stream, dtype=np.uint8).reshape(-1)
    out = np.zeros(int(n), dtype=np.uint8)
    _check(lib.hi_oracle_tp_decode(_p(stream), stream.size, _p(out), int(n)))
    return out



# ---------------------------------------------------------------------------
# Compression-ratio-mode lossless pipeline HF-RRE4-TCMS8-RZE1 (Sec. 5.2.3)
# ---------------------------------------------------------------------------
def hf_lengths(freq):
    """Huffman code lengths (at most 16) of a 256-bin frequency table."""
    f = np.ascontiguousarray(freq, dtype=np.uint64).reshape(256)
    ln = np.zeros(256, dtype=np.uint8)
    _check(_load().hi_oracle_hf_lengths(_p(f), _p(ln)))
    return ln


def cr_bound(n):
    return int(_load().hi_oracle_cr_bound(int(n)))


def cr_encode(data):
    """The CR-mode stream of a byte array."""
    lib = _load()
    data = np.ascontiguousarray(data, dtype=np.uint8).reshape(-1)
    out = np.zeros(cr_bound(data.size), dtype=np.uint8)
    ln = np.zeros(1, dtype=np.int64)
    _check(lib.hi_oracle_cr_encode(_p(data), data.size, _p(out), out.size, _p(ln)))
    return out[:int(ln[0])].copy()


def cr_decode(stream, n):
    lib = _load()
    stream = np.ascontiguousarray(stream, dtype=np.uint8)
    out = np.zeros(max(int(n), 1), dtype=np.uint8)
    _check(lib.hi_oracle_cr_decode(_p(stream), stream.size, _p(out), int(n)))
    return out[:int(n)]
