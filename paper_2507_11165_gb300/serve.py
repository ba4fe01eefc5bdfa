"""Continuous-batching request loop for compression / decompression.

Requests (compress a snapshot field, or decompress an earlier compressed
record) arrive over time.  The loop admits a waiting request as soon as a
slot (a CUDA stream) is free and its device bytes fit the memory budget next
to everything already in flight, so work of several requests overlaps on the
GPU; a finished request releases its slot and bytes, and the next waiting
ones are admitted.  Requests are admitted in arrival order (the head of the
queue waits for room; nothing behind it overtakes it).

Each request's latency runs from its arrival to the CUDA event recorded after
its last kernel, both on the device timeline of the run.  The executor does
the device work; ``GpuExecutor`` calls the library's C ABI, ``FakeExecutor``
(tests of the host logic) finishes requests after fixed durations.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time
from typing import Callable, Dict, List, Optional


@dataclasses.dataclass
class Request:
    id: int
    t: float            # arrival, seconds after the start of the run
    op: str             # "compress" or "decompress"
    side: int           # the snapshot is side^3 float32
    eb: float           # value-range-relative error bound
    seed: int = 0
    source: int = -1    # decompress: id of the compress request whose record it reads


@dataclasses.dataclass
class Done:
    id: int
    op: str
    t_arrival: float
    t_admit: float
    t_done: float        # device completion, seconds after the start
    bytes_in: int        # 4 B per point of the field
    status: int

    @property
    def latency(self):
        return self.t_done - self.t_arrival


def outlier_capacity(side: int, eb: float) -> int:
    """Outlier slots of a compress request: an eighth of the points, all of
    them at bounds of 1e-5 and below (where a quarter of a turbulent field
    can be outliers); a request that still overflows runs once more with the
    exact count."""
    n = side ** 3
    return n if eb <= 1e-5 else max(4096, n // 8)


def device_bytes(op: str, side: int, eb: float = 1e-3) -> int:
    """Device bytes a request holds while in flight (its own buffers)."""
    n = side ** 3
    if op == "compress":
        # snapshot, codes, outlier list, anchors, header, workspace
        return 4 * n + n + 8 * outlier_capacity(side, eb) + 4 * (n // 64 + 1) + 1024 + (1 << 16)
    # reconstructed field (the record it reads is held by its compress request)
    return 4 * n + 1024


class Server:
    """Admission and completion bookkeeping over an executor.

    executor.submit(req, slot) starts the request on stream `slot` and
    returns a handle; executor.poll(handle) returns None while it runs, else
    (t_done_seconds, status); executor.release(handle) frees its buffers
    (compress records stay until executor.drop_record(id)).
    """

    def __init__(self, executor, slots: int = 8, budget_bytes: int = 40 * 10 ** 9, keep_records: int = 32,
                 clock: Callable[[], float] = time.perf_counter):
        if slots < 1:
            raise ValueError("slots must be >= 1")
        self.ex = executor
        self.slots = slots
        self.budget = budget_bytes
        self.keep_records = keep_records
        self.clock = clock
        self.in_flight: Dict[int, tuple] = {}   # slot -> (req, handle, bytes, t_admit)
        self.records = collections.OrderedDict()  # compress id -> bytes held by its record
        self.bytes_in_flight = 0
        self.peak_bytes = 0
        self.peak_concurrency = 0
        self.done: List[Done] = []

    def _record_bytes(self):
        return sum(self.records.values())

    def _fits(self, need):
        return self.bytes_in_flight + self._record_bytes() + need <= self.budget

    def _free_slot(self):
        for s in range(self.slots):
            if s not in self.in_flight:
                return s
        return None

    def _retire(self, slot, t_done, status):
        req, h, b, t_admit = self.in_flight.pop(slot)
        self.bytes_in_flight -= b
        extra = self.ex.extra_bytes(h)  # a capacity re-run's larger outlier arrays stay with the record
        self.ex.release(h)
        if req.op == "compress" and status == 0:
            self.records[req.id] = self.ex.record_bytes(req) + extra
            while len(self.records) > self.keep_records:
                rid, _ = self.records.popitem(last=False)
                self.ex.drop_record(rid)
        self.done.append(Done(req.id, req.op, req.t, t_admit, t_done, 4 * req.side ** 3, status))

    def poll(self):
        n = 0
        for slot in list(self.in_flight):
            req, h, b, t_admit = self.in_flight[slot]
            r = self.ex.poll(h)
            if r is not None:
                self._retire(slot, r[0], r[1])
                n += 1
            else:
                # a capacity re-run holds more outlier memory: count it in flight
                grown = device_bytes(req.op, req.side, req.eb) + self.ex.extra_bytes(h)
                if grown != b:
                    self.bytes_in_flight += grown - b
                    self.in_flight[slot] = (req, h, grown, t_admit)
                    self.peak_bytes = max(self.peak_bytes, self.bytes_in_flight + self._record_bytes())
        return n

    def run(self, requests: List[Request], idle_sleep: float = 0.0) -> List[Done]:
        """Serve the requests (sorted by arrival); returns one Done per request."""
        pending = collections.deque(sorted(requests, key=lambda r: r.t))
        t0 = self.clock()
        self.ex.start()
        while pending or self.in_flight:
            now = self.clock() - t0
            self.poll()
            admitted = False
            while pending and pending[0].t <= now:
                req = pending[0]
                if req.op == "decompress" and req.source not in self.records:
                    if any(v[0].id == req.source for v in self.in_flight.values()):
                        break  # its record is still being made
                    # its record was dropped (or failed): serve it as a compress of the same snapshot
                    req = dataclasses.replace(req, op="compress")
                    pending[0] = req
                need = device_bytes(req.op, req.side, req.eb)
                slot = self._free_slot()
                if slot is None or not self._fits(need):
                    if not self.in_flight and not self._fits(need):
                        if self.records:  # make room by dropping kept records
                            rid, _ = self.records.popitem(last=False)
                            self.ex.drop_record(rid)
                            continue
                        raise RuntimeError("request %d needs %d bytes, more than the budget" % (req.id, need))
                    break
                pending.popleft()
                h = self.ex.submit(req, slot)
                self.in_flight[slot] = (req, h, need, now)
                self.bytes_in_flight += need
                self.peak_bytes = max(self.peak_bytes, self.bytes_in_flight + self._record_bytes())
                self.peak_concurrency = max(self.peak_concurrency, len(self.in_flight))
                admitted = True
            if not admitted:
                if pending and not self.in_flight:
                    wait = pending[0].t - (self.clock() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 1e-3))
                else:
                    time.sleep(idle_sleep)
        self.ex.finish()
        return self.done


def summarize(done: List[Done], wall_s: float) -> dict:
    lat = sorted(d.latency for d in done)
    if not lat:
        return {}

    def q(p):
        k = min(len(lat) - 1, max(0, int(math.ceil(p * len(lat))) - 1))
        return lat[k]

    tot = sum(d.bytes_in for d in done)
    return dict(n=len(done), p50_ms=1e3 * q(0.50), p99_ms=1e3 * q(0.99), max_ms=1e3 * lat[-1],
                mean_ms=1e3 * sum(lat) / len(lat), gbs=tot / wall_s / 1e9, wall_s=wall_s,
                n_compress=sum(d.op == "compress" for d in done),
                n_decompress=sum(d.op == "decompress" for d in done),
                failed=sum(d.status != 0 for d in done))


class FakeExecutor:
    """Host-only stand-in: a request takes `duration(req)` seconds of its slot."""

    def __init__(self, duration: Callable[[Request], float], clock: Callable[[], float] = time.perf_counter):
        self.duration = duration
        self.clock = clock
        self.t0 = None
        self.log = []
        self.records = set()

    def start(self):
        self.t0 = self.clock()

    def finish(self):
        pass

    def submit(self, req, slot):
        t = self.clock() - self.t0
        self.log.append(("submit", req.id, slot, t))
        return (req, t + self.duration(req))

    def poll(self, h):
        req, t_end = h
        if self.clock() - self.t0 >= t_end:
            return (t_end, 0)
        return None

    def release(self, h):
        self.log.append(("release", h[0].id))

    def record_bytes(self, req):
        self.records.add(req.id)
        return req.side ** 3 * 2

    def extra_bytes(self, h):
        return 0

    def drop_record(self, rid):
        self.records.discard(rid)


class GpuExecutor:
    """Requests on CUDA streams through the library's C ABI.

    A compress request materialises its snapshot (a side^3 block of a
    resident base field, one device copy on its stream standing in for the
    simulation writing it), then runs hi_compress; its record (codes,
    anchors, outliers, header) is kept for later decompress requests.  A
    decompress request runs hi_decompress of a kept record into a new field.
    Completion is a CUDA event after the last kernel.

    Buffers come from per-shape pools and go back once their last reader has
    completed: a kept record stays until it is dropped and no decompress of
    it is in flight."""

    def __init__(self, base, anchor_stride=16, keep_outputs=False, device=None):
        import torch

        from . import hi
        self.torch = torch
        self.hi = hi
        self.base = base  # resident float32 [B, B, B] field the snapshots come from
        self.A = anchor_stride
        self.dev = base.device if device is None else device
        self.streams = {}
        self.kept = {}      # compress id -> Buffers of its record
        self.readers = {}   # compress id -> decompress requests of it in flight
        self.dropped = set()
        self.outputs = {}   # request id -> result tensors (when keep_outputs)
        self.keep_outputs = keep_outputs
        self.t0_event = None
        self.pool = collections.defaultdict(list)  # (kind, shape, cap) -> free buffers
        self.params = {}
        self.launches = 0  # library kernels enqueued

    def start(self):
        self.t0_event = self.torch.cuda.Event(enable_timing=True)
        self.t0_event.record(self.torch.cuda.current_stream(self.dev))

    def finish(self):
        self.torch.cuda.synchronize(self.dev)

    def _stream(self, slot):
        if slot not in self.streams:
            self.streams[slot] = self.torch.cuda.Stream(device=self.dev)
        return self.streams[slot]

    def _get(self, key, make):
        free = self.pool[key]
        return free.pop() if free else make()

    def _put(self, key, obj):
        self.pool[key].append(obj)

    @staticmethod
    def _copy_record(b):
        """A copy of a finished record (tests compare it with the same request run alone)."""
        import types
        return types.SimpleNamespace(codes=b.codes.clone(), anchors=b.anchors.clone(), hist=b.hist.clone(),
                                     header=b.header.clone(), out_idx=b.out_idx.clone(),
                                     out_val=b.out_val.clone(), out_cap=b.out_cap, shape=b.shape)

    def _params(self, shape, eb):
        key = (shape, eb)
        if key not in self.params:
            self.params[key] = self.hi.make_params(shape, eb, "rel", self.A, autotune=True)
        return self.params[key]

    def snapshot_view(self, req):
        B = self.base.shape[0]
        s = req.side
        o = [(req.seed >> (8 * k)) % (B - s + 1) for k in range(3)]
        return self.base[o[0]:o[0] + s, o[1]:o[1] + s, o[2]:o[2] + s]

    def submit(self, req, slot):
        torch, hi = self.torch, self.hi
        st = self._stream(slot)
        shape = (req.side,) * 3
        with torch.cuda.stream(st):
            if req.op == "compress":
                cap = outlier_capacity(req.side, req.eb)
                x = self._get(("x", shape), lambda: torch.empty(shape, dtype=torch.float32, device=self.dev))
                x.copy_(self.snapshot_view(req))
                p = self._params(shape, req.eb)
                b = self._get(("rec", shape, cap),
                              lambda: hi.alloc(p, shape, self.dev, out_cap=cap, hist=True, recon=False))
                b.params = p
                hi.compress_into(x, b, stream=st)
                self.launches += 3  # set-up, range + auto-tune (one launch), predict-quantize
                hdr = self._get(("hdr",), lambda: torch.empty(hi.HEADER_BYTES, dtype=torch.uint8, pin_memory=True))
                hdr.copy_(b.header, non_blocking=True)
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(st)
                return dict(req=req, x=x, b=b, cap=cap, hdr=hdr, ev=ev, st=st, p=p)
            b = self.kept[req.source]
            self.readers[req.source] = self.readers.get(req.source, 0) + 1
            out = self._get(("out", shape), lambda: torch.empty(shape, dtype=torch.float32, device=self.dev))
            status = self._get(("st",), lambda: torch.zeros(1, dtype=torch.int32, device=self.dev))
            ws = self._get(("ws",), lambda: torch.empty(hi.DECOMPRESS_WS_BYTES, dtype=torch.uint8, device=self.dev))
            hi.decompress_into(b, out, status, stream=st, ws=ws)  # its own tile queue
            self.launches += 2  # outlier scatter, reconstruct
            sh = self._get(("sh",), lambda: torch.empty(1, dtype=torch.int32, pin_memory=True))
            sh.copy_(status, non_blocking=True)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(st)
            return dict(req=req, out=out, stat_t=status, sh=sh, ev=ev, ws=ws)

    def poll(self, h):
        if not h["ev"].query():
            return None
        t = self.t0_event.elapsed_time(h["ev"]) * 1e-3
        req = h["req"]
        if req.op == "compress":
            hd = self.hi.HiHeader.from_buffer_copy(h["hdr"].numpy().tobytes())
            st = int(hd.status)
            if st == self.hi.HI_ECAPACITY and not h.get("retried"):
                # more outliers than the first capacity: once more with the exact count
                torch, hi = self.torch, self.hi
                with torch.cuda.stream(h["st"]):
                    self._put(("rec", h["x"].shape, h["cap"]), h["b"])
                    b = hi.alloc(h["p"], h["x"].shape, self.dev, out_cap=int(hd.n_outliers), hist=True, recon=False)
                    hi.compress_into(h["x"], b, stream=h["st"])
                    self.launches += 3
                    h["hdr"].copy_(b.header, non_blocking=True)
                    h["ev"] = torch.cuda.Event(enable_timing=True)
                    h["ev"].record(h["st"])
                h["extra"] = 8 * max(0, int(hd.n_outliers) - int(h["b"].out_cap))
                h["b"] = b
                h["cap"] = None  # not a pooled size
                h["retried"] = True
                return None
        else:
            st = int(h["sh"].item())
        h["status"] = st
        return (t, st)

    def _recycle_record(self, rid):
        b = self.kept.pop(rid, None)
        self.dropped.discard(rid)
        self.readers.pop(rid, None)
        if b is not None and getattr(b, "pool_key", None) is not None:
            self._put(b.pool_key, b)

    def release(self, h):
        req = h["req"]
        shape = (req.side,) * 3
        if req.op == "compress":
            self._put(("x", shape), h["x"])
            self._put(("hdr",), h["hdr"])
            b = h["b"]
            b.pool_key = ("rec", shape, h["cap"]) if h["cap"] is not None else None
            if h.get("status", 1) == 0:
                self.kept[req.id] = b
            elif b.pool_key is not None:
                self._put(b.pool_key, b)
            if self.keep_outputs:
                self.outputs[req.id] = self._copy_record(b)
        else:
            if self.keep_outputs:
                self.outputs[req.id] = h["out"].clone()
            self._put(("out", shape), h["out"])
            self._put(("st",), h["stat_t"])
            self._put(("ws",), h["ws"])
            self._put(("sh",), h["sh"])
            left = self.readers.get(req.source, 1) - 1
            self.readers[req.source] = left
            if left == 0 and req.source in self.dropped:
                self._recycle_record(req.source)
        h.clear()

    def record_bytes(self, req):
        n = req.side ** 3
        return n + 8 * outlier_capacity(req.side, req.eb) + 4 * (n // 64 + 1) + 1024

    def extra_bytes(self, h):
        """Device bytes a request holds beyond device_bytes(): a capacity re-run's larger outlier arrays."""
        return int(h.get("extra", 0))

    def drop_record(self, rid):
        if self.readers.get(rid, 0) > 0:
            self.dropped.add(rid)  # recycled when its last decompress completes
        else:
            self._recycle_record(rid)


def make_requests(n=2000, rate=200.0, seed=5, lo=64, hi=512):
    """The serving workload: Poisson arrivals, half compress, half decompress
    of an earlier compress result, cubic sides log-uniform in [lo, hi], rel
    eb from {1e-2, 1e-3, 1e-4, 1e-5}."""
    from . import fields
    reqs = []
    last_compress = []
    for r in fields.request_stream(n, rate=rate, seed=seed, lo=lo, hi=hi):
        op = r["op"]
        src = -1
        side = r["side"]
        if op == "decompress":
            if last_compress:
                src = last_compress[-1 - r["seed"] % min(len(last_compress), 8)]  # one of the last 8
                side = next(q.side for q in reqs if q.id == src)
            else:
                op = "compress"
        req = Request(id=r["id"], t=r["t"], op=op, side=side, eb=r["eb"], seed=r["seed"], source=src)
        if op == "compress":
            last_compress.append(req.id)
        reqs.append(req)
    return reqs
