"""Thin ctypes binding of the C ABI in ``include/hi.h`` (``_build/libhi.so``).

Argument marshalling only: every step of compression and decompression runs
in the library's CUDA kernels; PyTorch provides device memory and streams.
There is no fallback: without the built library every call raises.

High-level use::

    from paper_2507_11165_gb300 import hi
    c = hi.compress(x, eb=1e-3, mode="rel", anchor_stride=16, autotune=True)
    y = hi.decompress(c)            # |x - y| < eps everywhere (Eq. 1)
"""
from __future__ import annotations

import ctypes
import math
import os
import threading
from dataclasses import dataclass, field
from typing import Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhi.so")

HI_OK, HI_EINVAL, HI_ENOMEM, HI_ECAPACITY, HI_ECUDA, HI_ETIMEOUT, HI_ECORRUPT = range(7)
EB_ABS, EB_REL = 0, 1
LINEAR, CUBIC = 0, 1
MD_LINEAR, MD_CUBIC = 2, 3  # multi-dimensional interpolation scheme (Sec. 5.1.2)
MAX_LEVELS = 8
MAGIC = 0x48693235
RADIUS = 128


class HiLevel(ctypes.Structure):
    _fields_ = [("interp", ctypes.c_uint8), ("order", ctypes.c_uint8 * 3)]


class HiParams(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_uint64 * 3), ("eb", ctypes.c_double), ("eb_mode", ctypes.c_uint32),
                ("anchor_stride", ctypes.c_uint32), ("autotune", ctypes.c_uint32), ("tuning", ctypes.c_uint32),
                ("level", HiLevel * MAX_LEVELS)]


class HiHeader(ctypes.Structure):
    _fields_ = [("magic", ctypes.c_uint32), ("version", ctypes.c_uint32), ("dims", ctypes.c_uint64 * 3),
                ("anchor_stride", ctypes.c_uint32), ("eb_mode", ctypes.c_uint32), ("eb", ctypes.c_double),
                ("eps", ctypes.c_double), ("eb_f", ctypes.c_float), ("ebx2_f", ctypes.c_float),
                ("r_f", ctypes.c_float), ("vmin", ctypes.c_float), ("vmax", ctypes.c_float),
                ("status", ctypes.c_uint32), ("n_outliers", ctypes.c_uint64), ("out_cap", ctypes.c_uint64),
                ("n_anchors", ctypes.c_uint64), ("level", HiLevel * MAX_LEVELS), ("n_levels", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 7)]


class HiBatchField(ctypes.Structure):
    _fields_ = [("p", HiParams), ("d_x", ctypes.c_void_p), ("d_codes", ctypes.c_void_p),
                ("d_anchors", ctypes.c_void_p), ("d_out_idx", ctypes.c_void_p), ("d_out_val", ctypes.c_void_p),
                ("out_cap", ctypes.c_uint64), ("d_hist", ctypes.c_void_p), ("d_recon", ctypes.c_void_p),
                ("d_header", ctypes.c_void_p), ("d_out", ctypes.c_void_p)]


class HiBatchPlan(ctypes.Structure):
    _fields_ = [("n_fields", ctypes.c_uint32), ("anchor_stride", ctypes.c_uint32), ("tuning", ctypes.c_uint32),
                ("all_tma", ctypes.c_uint32), ("total_tiles", ctypes.c_uint64), ("total_chunks", ctypes.c_uint64),
                ("total_samples", ctypes.c_uint64), ("ws_bytes", ctypes.c_uint64), ("off_table", ctypes.c_uint64),
                ("off_prefix", ctypes.c_uint64), ("off_tickets", ctypes.c_uint64),
                ("off_partials", ctypes.c_uint64), ("off_err", ctypes.c_uint64),
                ("reserved", ctypes.c_uint64 * 4)]


class HiEps(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("eb_f", ctypes.c_float), ("ebx2_f", ctypes.c_float),
                ("r_f", ctypes.c_float), ("pad", ctypes.c_float)]


class HiCrEstimate(ctypes.Structure):
    _fields_ = [("entropy_bits", ctypes.c_double), ("est_bytes", ctypes.c_uint64), ("cr", ctypes.c_double),
                ("bit_rate", ctypes.c_double)]


HEADER_BYTES = ctypes.sizeof(HiHeader)
SYMBOLS = ("hi_query", "hi_compress", "hi_decompress", "hi_autotune", "hi_autotune_errors", "hi_header_read",
           "hi_status_str", "hi_version", "hi_set_stage_events", "hi_compress_static_ws", "hi_batch_query",
           "hi_batch_prepare", "hi_compress_batch", "hi_decompress_batch", "hi_batch_tune_launch", "hi_resolve_eps",
           "hi_estimate_cr",
           "hi_autotune_select", "hi_tp_query", "hi_tp_encode", "hi_tp_decode", "hi_cr_query", "hi_cr_encode",
           "hi_cr_decode", "hi_compress_seq", "hi_compress_seq_fused", "hi_reorder_codes", "hi_unreorder_codes")
STATIC_WS_BYTES = 1 << 20  # HI_STATIC_WS_BYTES
DECOMPRESS_WS_BYTES = 256  # HI_DECOMPRESS_WS_BYTES


class HiError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = int(status)
        super().__init__("%s: %s (%d)" % (what or "hi", status_str(status), self.status))


_lock = threading.Lock()
_lib = None


def lib():
    """The loaded C library (ctypes), with argument types set."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libhi.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            P, u64, sz = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_size_t
            L.hi_query.argtypes = [ctypes.POINTER(HiParams), ctypes.POINTER(u64), ctypes.POINTER(u64),
                                   ctypes.POINTER(u64), ctypes.POINTER(sz)]
            L.hi_compress.argtypes = [ctypes.POINTER(HiParams), P, P, P, P, P, u64, P, P, P, P, sz, P]
            L.hi_compress_static_ws.argtypes = [ctypes.POINTER(HiParams), P, P, P, P, P, u64, P, P, P, P]
            L.hi_compress_seq.argtypes = [ctypes.POINTER(HiParams), P, P, P, P, P, P, u64, P, P, P, P, sz, P]
            L.hi_compress_seq_fused.argtypes = [ctypes.POINTER(HiParams), P, P]
            L.hi_compress_seq_fused.restype = ctypes.c_int
            BF, BP = ctypes.POINTER(HiBatchField), ctypes.POINTER(HiBatchPlan)
            L.hi_batch_query.argtypes = [ctypes.c_uint32, BF, ctypes.POINTER(sz)]
            L.hi_batch_prepare.argtypes = [ctypes.c_uint32, BF, ctypes.c_uint32, P, sz, BP, P]
            L.hi_compress_batch.argtypes = [BP, P, P]
            L.hi_decompress_batch.argtypes = [BP, P, P, P]
            L.hi_batch_tune_launch.argtypes = [BP, P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_float), P]
            L.hi_decompress.argtypes = [ctypes.POINTER(HiParams), P, P, P, P, P, u64, P, P, P, sz, P]
            L.hi_autotune.argtypes = [ctypes.POINTER(HiParams), P, P, P, sz, P]
            L.hi_autotune_errors.argtypes = [ctypes.POINTER(HiParams), P, P, sz, P, P, P, P]
            L.hi_header_read.argtypes = [P, ctypes.POINTER(HiHeader), P]
            L.hi_reorder_codes.argtypes = [ctypes.POINTER(HiParams), P, P, P]
            L.hi_tp_query.argtypes = [u64, ctypes.POINTER(u64), ctypes.POINTER(sz)]
            L.hi_value_range.argtypes = [ctypes.POINTER(HiParams), P, P, P, sz, P]
            L.hi_tp_encode.argtypes = [P, u64, P, u64, P, P, sz, P]
            L.hi_tp_decode.argtypes = [P, u64, P, u64, P, P, sz, P]
            L.hi_cr_query.argtypes = [u64, ctypes.POINTER(u64), ctypes.POINTER(sz)]
            L.hi_cr_encode.argtypes = [P, u64, P, u64, P, P, sz, P]
            L.hi_cr_decode.argtypes = [P, u64, P, u64, P, P, sz, P]
            L.hi_unreorder_codes.argtypes = [ctypes.POINTER(HiParams), P, P, P]
            L.hi_set_stage_events.argtypes = [P, ctypes.c_uint32]
            L.hi_resolve_eps.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_float, ctypes.c_float,
                                         ctypes.POINTER(HiEps)]
            L.hi_estimate_cr.argtypes = [P, u64, u64, u64, u64, ctypes.POINTER(HiCrEstimate)]
            L.hi_autotune_select.argtypes = [ctypes.POINTER(HiParams), P, sz, ctypes.POINTER(HiParams)]
            L.hi_status_str.argtypes = [ctypes.c_int]
            L.hi_status_str.restype = ctypes.c_char_p
            L.hi_version.restype = ctypes.c_uint32
            for f in ("hi_query", "hi_compress", "hi_decompress", "hi_autotune", "hi_autotune_errors",
                      "hi_header_read", "hi_set_stage_events", "hi_compress_static_ws", "hi_batch_query",
                      "hi_batch_prepare", "hi_compress_batch", "hi_decompress_batch", "hi_batch_tune_launch",
                      "hi_resolve_eps",
                      "hi_estimate_cr", "hi_autotune_select"):
                getattr(L, f).restype = ctypes.c_int
            _lib = L
    return _lib


def status_str(s):
    try:
        return lib().hi_status_str(int(s)).decode()
    except Exception:  # library missing: still describe the code
        return {0: "ok", 1: "invalid argument", 2: "workspace too small", 3: "outlier capacity exceeded",
                4: "CUDA error", 5: "device wait timed out", 6: "corrupt compressed record"}.get(int(s), "?")


def _check(rc, what):
    if rc != HI_OK:
        raise HiError(rc, what)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def dims3(shape):
    shape = tuple(int(s) for s in shape)
    if not 1 <= len(shape) <= 3:
        raise ValueError("fields are 1-3 dimensional")
    return (1,) * (3 - len(shape)) + shape


def make_params(shape, eb, mode="rel", anchor_stride=16, autotune=True, levels=None, threads=0, buffers=0):
    """HiParams for a field of ``shape``.  ``levels``: list of (interp, order) per
    level (level l = stride 2^l), or one (interp, order) for every level.
    ``threads`` (64/128) and ``buffers`` (1/2) pick the launch shape; 0 =
    library default."""
    p = HiParams()
    for d, n in enumerate(dims3(shape)):
        p.dims[d] = n
    p.eb = float(eb)
    p.eb_mode = EB_REL if mode in ("rel", EB_REL) else EB_ABS
    p.anchor_stride = int(anchor_stride)
    p.autotune = 2 if autotune == 2 else (1 if autotune else 0)  # 2: with the multi-dimensional scheme
    p.tuning = {0: 0, 64: 1, 128: 2}[int(threads)] | ({0: 0, 1: 1, 2: 2}[int(buffers)] << 2)
    L = max(1, int(anchor_stride).bit_length() - 1)
    if levels is None:
        levels = (CUBIC, (0, 1, 2))
    if isinstance(levels, tuple) and len(levels) == 2 and isinstance(levels[0], int):
        levels = [levels] * L
    for l in range(MAX_LEVELS):
        ip, od = levels[min(l, len(levels) - 1)]
        p.level[l].interp = int(ip)
        for k in range(3):
            p.level[l].order[k] = int(od[k])
    return p


def query(p):
    n, na, nb = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    ws = ctypes.c_size_t()
    _check(lib().hi_query(ctypes.byref(p), ctypes.byref(n), ctypes.byref(na), ctypes.byref(nb), ctypes.byref(ws)),
           "hi_query")
    return dict(n_points=n.value, n_anchors=na.value, n_blocks=nb.value, ws_bytes=ws.value)


def set_stage_events(events):
    """Record ``events`` (8 torch.cuda.Event) between stages of later calls on this thread; None = off."""
    if events is None:
        _check(lib().hi_set_stage_events(None, 0), "hi_set_stage_events")
        return
    if any(e.cuda_event == 0 for e in events):
        raise ValueError("record each event once before handing it over (torch creates events lazily)")
    arr = (ctypes.c_void_p * 8)(*[ctypes.c_void_p(e.cuda_event) for e in events])
    _check(lib().hi_set_stage_events(ctypes.cast(arr, ctypes.c_void_p), 8), "hi_set_stage_events")


def read_header(d_header, stream=None):
    h = HiHeader()
    _check(lib().hi_header_read(_ptr(d_header), ctypes.byref(h), _stream(stream)), "hi_header_read")
    return h


def header_dict(h):
    return dict(magic=h.magic, version=h.version, dims=tuple(h.dims), anchor_stride=h.anchor_stride,
                eb_mode=h.eb_mode, eb=h.eb, eps=h.eps, eb_f=h.eb_f, ebx2_f=h.ebx2_f, r_f=h.r_f, vmin=h.vmin,
                vmax=h.vmax, status=h.status, n_outliers=h.n_outliers, out_cap=h.out_cap, n_anchors=h.n_anchors,
                n_levels=h.n_levels,
                levels=[(h.level[l].interp, tuple(h.level[l].order)) for l in range(h.n_levels)])


@dataclass
class Buffers:
    """Device buffers of one compression (all owned by PyTorch)."""
    params: HiParams
    shape: tuple
    codes: torch.Tensor
    anchors: torch.Tensor
    out_idx: torch.Tensor
    out_val: torch.Tensor
    hist: Optional[torch.Tensor]
    recon: Optional[torch.Tensor]
    header: torch.Tensor
    ws: torch.Tensor
    out_cap: int
    sizes: dict = field(default_factory=dict)


def default_out_cap(n_points):
    return max(4096, n_points // 16)


def alloc(p, shape, device, out_cap=None, hist=True, recon=False):
    """Allocate the device buffers of a compression of ``shape`` under ``p``."""
    sz = query(p)
    n = sz["n_points"]
    cap = default_out_cap(n) if out_cap is None else int(out_cap)
    dev = torch.device(device)
    return Buffers(
        params=p, shape=tuple(shape), sizes=sz, out_cap=cap,
        codes=torch.empty(n, dtype=torch.uint8, device=dev),
        anchors=torch.empty(max(1, sz["n_anchors"]), dtype=torch.float32, device=dev),
        out_idx=torch.empty(max(1, cap), dtype=torch.int32, device=dev),
        out_val=torch.empty(max(1, cap), dtype=torch.float32, device=dev),
        hist=torch.empty(256, dtype=torch.int32, device=dev) if hist else None,
        recon=torch.empty(n, dtype=torch.float32, device=dev) if recon else None,
        header=torch.zeros(HEADER_BYTES, dtype=torch.uint8, device=dev),
        ws=torch.empty(max(8, sz["ws_bytes"]), dtype=torch.uint8, device=dev))


def compress_into(x, b: Buffers, stream=None):
    """Enqueue hi_compress of device tensor ``x`` into preallocated buffers (no sync)."""
    if not x.is_cuda or x.dtype != torch.float32 or not x.is_contiguous():
        raise ValueError("x must be a contiguous float32 CUDA tensor")
    rc = lib().hi_compress(ctypes.byref(b.params), _ptr(x), _ptr(b.codes), _ptr(b.anchors), _ptr(b.out_idx),
                           _ptr(b.out_val), b.out_cap, _ptr(b.hist), _ptr(b.recon), _ptr(b.header), _ptr(b.ws),
                           b.ws.numel(), _stream(stream))
    _check(rc, "hi_compress")


def compress_seq_into(x, b: Buffers, seq, stream=None):
    """Enqueue hi_compress_seq of ``x`` into ``b`` and the reordered codes
    (Sec. 5.2.2, Eq. 3) into ``seq`` (n_points uint8 device bytes; no sync)."""
    if not x.is_cuda or x.dtype != torch.float32 or not x.is_contiguous():
        raise ValueError("x must be a contiguous float32 CUDA tensor")
    rc = lib().hi_compress_seq(ctypes.byref(b.params), _ptr(x), _ptr(b.codes), _ptr(seq), _ptr(b.anchors),
                               _ptr(b.out_idx), _ptr(b.out_val), b.out_cap, _ptr(b.hist), _ptr(b.recon),
                               _ptr(b.header), _ptr(b.ws), b.ws.numel(), _stream(stream))
    _check(rc, "hi_compress_seq")


def compress_seq_fused(p, codes_ptr, seq_ptr):
    """Whether hi_compress_seq with these parameters and buffer addresses
    writes the sequence from the predict-quantize kernel (host only)."""
    return bool(lib().hi_compress_seq_fused(ctypes.byref(p), ctypes.c_void_p(codes_ptr), ctypes.c_void_p(seq_ptr)))


def compress_static_ws_into(x, b: Buffers, stream=None):
    """Enqueue hi_compress_static_ws of ``x`` into ``b`` (no sync).

    The library's fixed per-device scratch serves as workspace, ``b.ws`` is
    not touched; calls that may overlap on one device race on that scratch."""
    if not x.is_cuda or x.dtype != torch.float32 or not x.is_contiguous():
        raise ValueError("x must be a contiguous float32 CUDA tensor")
    rc = lib().hi_compress_static_ws(ctypes.byref(b.params), _ptr(x), _ptr(b.codes), _ptr(b.anchors),
                                     _ptr(b.out_idx), _ptr(b.out_val), b.out_cap, _ptr(b.hist), _ptr(b.recon),
                                     _ptr(b.header), _stream(stream))
    if rc == HI_ENOMEM:
        raise HiError(rc, "hi_compress_static_ws: the field needs %d bytes of workspace, the fixed scratch "
                          "holds %d" % (query(b.params)["ws_bytes"], STATIC_WS_BYTES))
    _check(rc, "hi_compress_static_ws")


def decompress_into(b: Buffers, out, status=None, stream=None, ws=None):
    """Enqueue hi_decompress of the record in ``b`` into ``out`` (no sync).

    Uses ``b.ws`` as workspace unless ``ws`` (a uint8 device tensor) is given."""
    w = b.ws if ws is None else ws
    rc = lib().hi_decompress(ctypes.byref(b.params), _ptr(b.header), _ptr(b.codes), _ptr(b.anchors),
                             _ptr(b.out_idx), _ptr(b.out_val), b.out_cap, _ptr(out), _ptr(status), _ptr(w),
                             w.numel(), _stream(stream))
    _check(rc, "hi_decompress")


def reorder_codes(codes, p, out=None, stream=None):
    """hi_reorder_codes: the uint8 device code array of the field of ``p`` as
    the level-grouped sequence of Sec. 5.2.2, Eq. 3 (a new 1D tensor unless
    ``out`` is given; no sync)."""
    if out is None:
        out = torch.empty(codes.numel(), dtype=torch.uint8, device=codes.device)
    _check(lib().hi_reorder_codes(ctypes.byref(p), _ptr(codes), _ptr(out), _stream(stream)), "hi_reorder_codes")
    return out


def unreorder_codes(seq, p, out=None, stream=None):
    """hi_unreorder_codes: the row-major code array back from its sequence
    (a new 1D tensor unless ``out`` is given; no sync)."""
    if out is None:
        out = torch.empty(seq.numel(), dtype=torch.uint8, device=seq.device)
    _check(lib().hi_unreorder_codes(ctypes.byref(p), _ptr(seq), _ptr(out), _stream(stream)), "hi_unreorder_codes")
    return out


RANGE_WS_BYTES = DECOMPRESS_WS_BYTES + 8192


def value_range_into(x, p, header, ws, stream=None):
    """Enqueue hi_value_range of device tensor ``x`` (parameters ``p``, relative bound): the min and max
    of its finite values into the device ``header`` (no sync)."""
    _check(lib().hi_value_range(ctypes.byref(p), _ptr(x), _ptr(header), _ptr(ws), ws.numel(), _stream(stream)),
           "hi_value_range")


def tp_query(n):
    """(largest stream bytes, workspace bytes) of the TCMS1-BIT1-RRE1 pipeline for n input bytes."""
    mx, ws = ctypes.c_uint64(), ctypes.c_size_t()
    _check(lib().hi_tp_query(int(n), ctypes.byref(mx), ctypes.byref(ws)), "hi_tp_query")
    return mx.value, ws.value


def cr_query(n):
    """(largest stream bytes, workspace bytes) of the HF-RRE4-TCMS8-RZE1 pipeline for n input bytes."""
    mx, ws = ctypes.c_uint64(), ctypes.c_size_t()
    _check(lib().hi_cr_query(int(n), ctypes.byref(mx), ctypes.byref(ws)), "hi_cr_query")
    return mx.value, ws.value


class CrCodec:
    """Device buffers for hi_cr_encode / hi_cr_decode of n-byte sequences."""

    def __init__(self, n, device):
        self.n = int(n)
        mx, ws = cr_query(self.n)
        self.stream_buf = torch.empty(mx, dtype=torch.uint8, device=device)
        self.ws = torch.empty(max(ws, 16), dtype=torch.uint8, device=device)
        self.len = torch.zeros(1, dtype=torch.int64, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)

    def encode_into(self, data, stream=None):
        """Enqueue the encoding of ``data`` (n bytes, device) into ``stream_buf``; length in ``self.len``."""
        _check(lib().hi_cr_encode(_ptr(data), self.n, _ptr(self.stream_buf), self.stream_buf.numel(),
                                  _ptr(self.len), _ptr(self.ws), self.ws.numel(), _stream(stream)), "hi_cr_encode")

    def decode_into(self, stream_bytes, in_len, out, stream=None):
        """Enqueue the decoding of a stream of ``in_len`` bytes into ``out`` (n bytes); status in ``self.status``."""
        _check(lib().hi_cr_decode(_ptr(stream_bytes), int(in_len), _ptr(out), self.n, _ptr(self.status),
                                  _ptr(self.ws), self.ws.numel(), _stream(stream)), "hi_cr_decode")


class TpCodec:
    """Device buffers for hi_tp_encode / hi_tp_decode of n-byte sequences."""

    def __init__(self, n, device):
        self.n = int(n)
        mx, ws = tp_query(self.n)
        self.stream_buf = torch.empty(mx, dtype=torch.uint8, device=device)
        self.ws = torch.empty(max(ws, 16), dtype=torch.uint8, device=device)
        self.len = torch.zeros(1, dtype=torch.int64, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)

    def encode_into(self, data, stream=None):
        """Enqueue the encoding of ``data`` (n bytes, device) into ``stream_buf``; length in ``self.len``."""
        _check(lib().hi_tp_encode(_ptr(data), self.n, _ptr(self.stream_buf), self.stream_buf.numel(),
                                  _ptr(self.len), _ptr(self.ws), self.ws.numel(), _stream(stream)), "hi_tp_encode")

    def decode_into(self, stream_bytes, in_len, out, stream=None):
        """Enqueue the decoding of a stream of ``in_len`` bytes into ``out`` (n bytes); status in ``self.status``."""
        _check(lib().hi_tp_decode(_ptr(stream_bytes), int(in_len), _ptr(out), self.n, _ptr(self.status),
                                  _ptr(self.ws), self.ws.numel(), _stream(stream)), "hi_tp_decode")


def autotune_errors(b: Buffers, stream=None):
    """Per-(sample, level, candidate) auto-tune error sums left in the workspace."""
    import numpy as np
    m, L, nc = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib().hi_autotune_errors(ctypes.byref(b.params), None, None, 0, ctypes.byref(m), ctypes.byref(L),
                                    ctypes.byref(nc), _stream(stream)), "hi_autotune_errors")
    out = np.zeros(m.value * L.value * nc.value, dtype=np.float64)
    _check(lib().hi_autotune_errors(ctypes.byref(b.params), _ptr(b.ws), out.ctypes.data_as(ctypes.c_void_p),
                                    out.size, None, None, None, _stream(stream)), "hi_autotune_errors")
    return out.reshape(m.value, L.value, nc.value)


class Compressed:
    """A compressed field: device buffers plus the host copy of its header."""

    def __init__(self, b: Buffers, header: HiHeader):
        self.buffers = b
        self.h = header
        self.shape = b.shape

    @property
    def n_outliers(self):
        return int(self.h.n_outliers)

    @property
    def codes(self):
        return self.buffers.codes.view(self.shape)

    @property
    def anchors(self):
        return self.buffers.anchors[: int(self.h.n_anchors)]

    @property
    def outliers(self):
        k = min(self.n_outliers, self.buffers.out_cap)
        return self.buffers.out_idx[:k], self.buffers.out_val[:k]

    @property
    def hist(self):
        return self.buffers.hist

    @property
    def recon(self):
        return None if self.buffers.recon is None else self.buffers.recon.view(self.shape)

    def info(self):
        return header_dict(self.h)

    def estimate(self):
        return estimate_cr(self.hist.cpu().numpy(), self.n_outliers, int(self.h.n_anchors),
                           int(math.prod(self.shape)))


def compress(x, eb, mode="rel", anchor_stride=16, autotune=True, levels=None, out_cap=None, hist=True,
             recon=False, stream=None):
    """Compress a float32 field (device tensor, or host tensor copied to the current device).

    Synchronises once to read the header; if the outliers overflow the
    capacity, compresses again with the exact capacity."""
    if not x.is_cuda:
        x = x.to("cuda", non_blocking=True)
    x = x.contiguous()
    p = make_params(x.shape, eb, mode, anchor_stride, autotune, levels)
    b = alloc(p, x.shape, x.device, out_cap, hist, recon)
    compress_into(x, b, stream)
    h = read_header(b.header, stream)
    if h.status == HI_ECAPACITY:
        b = alloc(p, x.shape, x.device, int(h.n_outliers), hist, recon)
        compress_into(x, b, stream)
        h = read_header(b.header, stream)
    if h.status != HI_OK:
        raise HiError(h.status, "hi_compress (device)")
    return Compressed(b, h)


def decompress(c: Compressed, out=None, stream=None):
    b = c.buffers
    if out is None:
        out = torch.empty(b.shape, dtype=torch.float32, device=b.codes.device)
    status = torch.zeros(1, dtype=torch.int32, device=b.codes.device)
    decompress_into(b, out, status, stream)
    st = int(status.item())
    if st != HI_OK:
        raise HiError(st, "hi_decompress (device)")
    return out


# Launch shapes of the batched predict-quantize launch, in the order the
# launch-shape tuner tries them (hi_params.tuning encoding).
BATCH_SHAPES = ((128, 1), (64, 1), (128, 2), (64, 2))


def tuning_code(threads, buffers):
    return {64: 1, 128: 2}[threads] | ({1: 1, 2: 2}[buffers] << 2)


class Batch:
    """Many fields compressed together: one launch per stage for all of them
    (hi_batch_prepare / hi_compress_batch).

    ``xs``: contiguous float32 device tensors (shapes may differ); ``ebs``: one
    bound per field (or one for all); the other arguments apply to every
    field.  Buffers of each field are allocated here; ``compress()`` only
    enqueues kernels, so it can be captured in a CUDA graph.  With
    ``outs=True`` every field also gets an output tensor (``self.outs``)
    that ``decompress()`` (hi_decompress_batch) reconstructs it into."""

    def __init__(self, xs, ebs, mode="rel", anchor_stride=16, autotune=True, levels=None, out_caps=None,
                 hist=True, recon=False, tuning=0, outs=False):
        n = len(xs)
        if n == 0:
            raise ValueError("empty batch")
        if not isinstance(ebs, (list, tuple)):
            ebs = [ebs] * n
        modes = mode if isinstance(mode, (list, tuple)) else [mode] * n
        self.xs = list(xs)
        self.buffers = []
        self.outs = [torch.empty_like(x) for x in self.xs] if outs else None
        self.dstatus = torch.zeros(1, dtype=torch.int32, device=self.xs[0].device)
        arr = (HiBatchField * n)()
        for i, x in enumerate(self.xs):
            if not x.is_cuda or x.dtype != torch.float32 or not x.is_contiguous():
                raise ValueError("every field must be a contiguous float32 CUDA tensor")
            p = make_params(x.shape, ebs[i], modes[i], anchor_stride, autotune, levels)
            cap = None if out_caps is None else out_caps[i]
            b = alloc(p, x.shape, x.device, cap, hist, recon)
            self.buffers.append(b)
            arr[i].p = p
            arr[i].d_x = x.data_ptr()
            arr[i].d_codes = b.codes.data_ptr()
            arr[i].d_anchors = b.anchors.data_ptr()
            arr[i].d_out_idx = b.out_idx.data_ptr()
            arr[i].d_out_val = b.out_val.data_ptr()
            arr[i].out_cap = b.out_cap
            arr[i].d_hist = None if b.hist is None else b.hist.data_ptr()
            arr[i].d_recon = None if b.recon is None else b.recon.data_ptr()
            arr[i].d_header = b.header.data_ptr()
            arr[i].d_out = None if self.outs is None else self.outs[i].data_ptr()
        self.fields = arr
        wsb = ctypes.c_size_t()
        _check(lib().hi_batch_query(n, arr, ctypes.byref(wsb)), "hi_batch_query")
        self.ws = torch.empty(max(256, wsb.value), dtype=torch.uint8, device=self.xs[0].device)
        self.plan = HiBatchPlan()
        _check(lib().hi_batch_prepare(n, arr, tuning, _ptr(self.ws), self.ws.numel(), ctypes.byref(self.plan),
                                      _stream(None)), "hi_batch_prepare")

    def __len__(self):
        return len(self.xs)

    def compress(self, stream=None):
        """Enqueue the batch's compression (no sync)."""
        _check(lib().hi_compress_batch(ctypes.byref(self.plan), _ptr(self.ws), _stream(stream)),
               "hi_compress_batch")

    def decompress(self, stream=None):
        """Enqueue the reconstruction of every field into ``self.outs`` (no
        sync); the first error of any field goes to ``self.dstatus``."""
        _check(lib().hi_decompress_batch(ctypes.byref(self.plan), _ptr(self.ws), _ptr(self.dstatus),
                                         _stream(stream)), "hi_decompress_batch")

    def tune_launch(self, reps=3, stream=None):
        """Time every launch shape, keep the fastest; returns {shape: ms}."""
        ms = (ctypes.c_float * 4)()
        _check(lib().hi_batch_tune_launch(ctypes.byref(self.plan), _ptr(self.ws), reps, ms, _stream(stream)),
               "hi_batch_tune_launch")
        return {BATCH_SHAPES[i]: float(ms[i]) for i in range(4) if ms[i] > 0}

    @property
    def shape(self):
        t = self.plan.tuning
        return ({1: 64, 2: 128}.get(t & 3, 128), {1: 1, 2: 2}.get((t >> 2) & 3, 1))

    def set_shape(self, threads, buffers):
        self.plan.tuning = tuning_code(threads, buffers)

    def results(self, stream=None):
        """Compressed records of every field (reads the headers; synchronises)."""
        return [Compressed(b, read_header(b.header, stream)) for b in self.buffers]


def estimate_cr(hist, n_out, n_anchors, n_points, header_bytes=None):
    """Entropy-estimated size of the record (hi_estimate_cr): ceil(N_pred H / 8)
    + 8 n_out + 4 n_anchors + header bytes, H the order-0 entropy of the
    256-bin code histogram in bits (what an entropy coder such as the Huffman
    stage of Sec. 5.2.2 approaches).  Host only."""
    import numpy as np
    h = np.ascontiguousarray(np.asarray(hist).astype(np.uint32).reshape(256))
    out = HiCrEstimate()
    hb = HEADER_BYTES if header_bytes is None else int(header_bytes)
    _check(lib().hi_estimate_cr(ctypes.c_void_p(h.ctypes.data), int(n_out), int(n_anchors), int(n_points), hb,
                                ctypes.byref(out)), "hi_estimate_cr")
    return dict(entropy_bits=out.entropy_bits, est_bytes=int(out.est_bytes), cr=out.cr, bit_rate=out.bit_rate)


def resolve_eps(mode, eb, vmin, vmax):
    """The absolute bound and float32 constants of Eq. 1 for a value range
    (hi_resolve_eps): what the device derives in hi_compress, for fields
    compressed in parts at the combined range."""
    out = HiEps()
    m = {"abs": EB_ABS, "rel": EB_REL}[mode] if isinstance(mode, str) else int(mode)
    _check(lib().hi_resolve_eps(m, float(eb), float(vmin), float(vmax), ctypes.byref(out)), "hi_resolve_eps")
    return dict(eps=out.eps, eb_f=out.eb_f, ebx2_f=out.ebx2_f, r_f=out.r_f)


def tune_errors(x, anchor_stride=16, md=False, stream=None):
    """Per-sample, per-level, per-candidate auto-tune error sums of a device
    field (hi_autotune, then hi_autotune_errors): array [m, L, ncfg]."""
    if not x.is_cuda or x.dtype != torch.float32 or not x.is_contiguous():
        raise ValueError("x must be a contiguous float32 CUDA tensor")
    p = make_params(tuple(x.shape), 1.0, "abs", anchor_stride, autotune=2 if md else True)
    b = alloc(p, tuple(x.shape), x.device, out_cap=0, hist=False, recon=False)
    _check(lib().hi_autotune(ctypes.byref(p), _ptr(x), _ptr(b.header), _ptr(b.ws), b.ws.numel(), _stream(stream)),
           "hi_autotune")
    return autotune_errors(b, stream)


def autotune_select(shape, anchor_stride, err, md=False):
    """The auto-tuner's levels [(interp, order)] for a field of ``shape`` from
    its per-sample error rows err[m, L, ncfg] (hi_autotune_select): the
    choice the device makes from the same rows."""
    import numpy as np
    p = make_params(tuple(shape), 1.0, "abs", anchor_stride, autotune=2 if md else True)
    e = np.ascontiguousarray(err, dtype=np.float64).reshape(-1)
    out = HiParams()
    _check(lib().hi_autotune_select(ctypes.byref(p), ctypes.c_void_p(e.ctypes.data), e.size, ctypes.byref(out)),
           "hi_autotune_select")
    L = int(anchor_stride).bit_length() - 1
    return [(int(out.level[l].interp), tuple(int(v) for v in out.level[l].order)) for l in range(L)]


def autotune_dims(shape, anchor_stride=16, md=False):
    """(m, L, ncfg): auto-tune samples, levels and candidates of a field of ``shape``."""
    p = make_params(tuple(shape), 1.0, "abs", anchor_stride, autotune=2 if md else True)
    m, L, nc = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib().hi_autotune_errors(ctypes.byref(p), None, None, 0, ctypes.byref(m), ctypes.byref(L),
                                    ctypes.byref(nc), None), "hi_autotune_errors")
    return m.value, L.value, nc.value
