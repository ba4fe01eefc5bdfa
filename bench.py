"""Benchmark: interpolation predict/quantize + reconstruct on GB300.

One step = one compression (header set-up, value range, auto-tune on 0.2% of
the blocks, fused predict-quantize with outlier compaction and code
histogram) plus one decompression (outlier scatter, level-by-level
reconstruction) of a 512^3 float32 log-normal Gaussian random field
(P(k) ~ k^-3) at value-range-relative error bound 1e-3, anchor stride 16.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints ONE JSON line (rank 0).  ``value`` = input bytes (4 B per point, all
ranks) per second of device time for compress + decompress; the per-stage
CUDA-event times give the predict-quantize and reconstruct throughputs and
the HBM roofline fraction of the dominant kernel.  ``--impl reference`` times
the CPU oracle (the reference arm of this benchmark) on host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SHAPE = (512, 512, 512)
EB = 1e-3
A = 16
SEED = 1
WORKLOAD = "512^3 float32 log-normal GRF P(k)~k^-3 (seed 1), rel eb 1e-3, anchor stride 16, auto-tuned levels"
METRIC = "compress / decompress input GB/s per GB300 at rel eb 1e-3 (% HBM peak), bit-exact"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, period_ms=50):
        self.index = index
        self.period_ms = period_ms
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", str(self.period_ms)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.06)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        if self.proc is None:
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [v.strip() for v in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return dict(sm_mhz=None, sm_max_mhz=mx, reasons=sorted(reasons), samples=0)
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=mx, reasons=sorted(reasons), samples=len(sm))


def traffic_record(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    r = rec.get(kernel)
    if not r:
        return None
    if r.get("source_sha") != kernel_source_sha():
        return None
    return r.get("bytes_per_launch")


def kernel_source_sha():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2507_11165_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


# ---------------------------------------------------------------------------
# reference arm / CPU baseline: the oracle, as it stands, on host cores
# ---------------------------------------------------------------------------
def oracle_roundtrip(x, A=None, eb=None, levels=None, workers=1):
    """The oracle's compress + decompress of ``x`` (relative bound): range and
    eps, auto-tune unless ``levels`` (interp[L], order[L,3]) are given,
    predict-quantize, outlier/histogram collection, reconstruction.  With
    workers > 1 the block loops of compress and decompress run on that many
    host threads (same routine, disjoint blocks)."""
    import oracle
    A = A or globals()["A"]
    eb = eb or EB
    cst = oracle.eps_constants(x, oracle.REL, eb)
    if levels is None:
        err = oracle.tune_errors(x, A)
        interp, order = oracle.tune_select(x.shape, A, err)
    else:
        interp, order = levels
    if workers > 1:
        out = oracle.compress_parallel(x, A, interp, order, cst, workers)
    else:
        out = oracle.compress(x, A, interp, order, cst)
    col = oracle.collect(x, out["codes"], A)
    if workers > 1:
        y = oracle.decompress_parallel(x.shape, A, interp, order, cst["ebx2_f"], out["codes"], out["anchors"],
                                       col["out_idx"], col["out_val"], workers)
    else:
        y = oracle.decompress(x.shape, A, interp, order, cst["ebx2_f"], out["codes"], out["anchors"],
                              col["out_idx"], col["out_val"])
    return out, y, (interp, order)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def cpu_baseline(x, planes):
    """Oracle compress + decompress of the first ``planes`` planes (bounded
    sample), on every host core (blocks over threads) and on one thread."""
    import numpy as np
    sub = np.ascontiguousarray(x[:planes])
    cores = host_cores()
    t0 = time.perf_counter()
    out, y, cfg = oracle_roundtrip(sub, workers=cores)
    dt_all = time.perf_counter() - t0
    t0 = time.perf_counter()
    out1, y1, cfg1 = oracle_roundtrip(sub)
    dt = time.perf_counter() - t0
    same = bool(np.array_equal(out["codes"], out1["codes"]) and np.array_equal(y.view(np.uint32), y1.view(np.uint32)))
    what = "compress+decompress of planes [0,%d) of the workload field (%d x %d x %d), C oracle" % (
        planes, planes, x.shape[1], x.shape[2])
    return dict(value=4.0 * sub.size / dt_all / 1e9, unit="GB/s", cores=cores, kind="oracle",
                sample=what + ", blocks of the compress and decompress loops over %d host threads (range, "
                              "auto-tune and outlier collection on one)" % cores,
                seconds=dt_all, threads_equal_single=same,
                single_thread=dict(value=4.0 * sub.size / dt / 1e9, unit="GB/s", cores=1, seconds=dt,
                                   sample=what + ", one thread")), out1


def run_reference(args):
    """The reference arm: the oracle, as it stands, on every host core (the
    block loops of compress and decompress over threads), each step one
    compress + decompress of planes [0, ref_planes) of the workload field
    (the whole field by default); one single-threaded step is timed beside."""
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return
    from paper_2507_11165_gb300 import fields
    import numpy as np
    x = fields.lognormal_grf(SHAPE, seed=SEED)
    planes = min(args.ref_planes, SHAPE[0])
    sub = np.ascontiguousarray(x[:planes])
    cores = host_cores()
    for w in range(max(1, args.warmup)):
        t0 = time.perf_counter()
        oracle_roundtrip(sub, workers=cores)
        tw = time.perf_counter() - t0
        if w == 0 and args.steps * tw > 150.0:
            # keep the timed steps to about 150 s: fewer planes per step (a bounded sample)
            planes = max(17, int(planes * 150.0 / (args.steps * tw)))
            sub = np.ascontiguousarray(x[:planes])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_roundtrip(sub, workers=cores)
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    t0 = time.perf_counter()
    oracle_roundtrip(sub)
    t1 = time.perf_counter() - t0
    v = 4.0 * sub.size / t / 1e9
    whole = planes == SHAPE[0]
    what = ("compress+decompress of the whole %d^3 field per step" % SHAPE[0]) if whole else (
        "compress+decompress of planes [0,%d) (%d x %d x %d) per step" % (planes, planes, SHAPE[1], SHAPE[2]))
    line = dict(metric=METRIC, value=v, unit="GB/s", impl="reference", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=t * 1e3, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f32", data="synthetic",
                config=dict(workload=WORKLOAD, sample="whole field" if whole else "planes [0,%d) per step" % planes),
                cpu_baseline=dict(value=v, unit="GB/s", cores=cores, kind="oracle",
                                  sample=what + ", C oracle with its block loops over %d host threads" % cores,
                                  single_thread=dict(value=4.0 * sub.size / t1 / 1e9, unit="GB/s", cores=1,
                                                     seconds=t1, sample=what + ", one thread, one step")),
                e2e=dict(value=v, unit="GB/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# The other single-GPU workloads, measured in the default run beside the headline
# ---------------------------------------------------------------------------
def field_line(x_host, eb, A_, dev, levels=None, reps=20, cpu=True):
    """One field at a relative bound: compress and decompress through the
    public calls (every launch of each), CUDA events, median of ``reps``, L2
    flushed (a 256 MiB write) before every timed call; quality and entropy
    size estimate; the oracle's result compared bit for bit and the oracle
    timed on every host core and on one thread.  ``levels``: fixed
    (interp, order) per level, or None for the auto-tuner."""
    import numpy as np
    import torch
    from paper_2507_11165_gb300 import hi
    x = torch.from_numpy(x_host).to(dev)
    N = x_host.size
    p = hi.make_params(x.shape, eb, "rel", A_, autotune=levels is None, levels=levels)
    b = hi.alloc(p, x.shape, dev, out_cap=N, hist=True, recon=False)  # every point may be an outlier
    out = torch.empty_like(x)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        hi.compress_into(x, b)
        hi.decompress_into(b, out, st)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(reps)]
    for r in ev:
        flush.fill_(1)
        r[0].record(stream)
        hi.compress_into(x, b)
        r[1].record(stream)
        flush.fill_(2)
        r[2].record(stream)
        hi.decompress_into(b, out, st)
        r[3].record(stream)
    torch.cuda.synchronize()
    c_ms = statistics.median(r[0].elapsed_time(r[1]) for r in ev)
    d_ms = statistics.median(r[2].elapsed_time(r[3]) for r in ev)
    h = hi.read_header(b.header)
    assert h.status == 0 and int(st.item()) == 0, (h.status, int(st.item()))
    hist = b.hist.cpu().numpy().view(np.uint32)
    est = hi.estimate_cr(hist, int(h.n_outliers), int(h.n_anchors), N)
    err = (out - x).abs().max().item()
    mse = float(((out.double() - x.double()) ** 2).mean().item())
    vrange = float(h.vmax) - float(h.vmin)
    line = dict(shape=list(x_host.shape), eb=eb, anchor_stride=A_,
                levels=[(int(h.level[l].interp), list(h.level[l].order)) for l in range(h.n_levels)],
                tuned=levels is None, compress_ms=c_ms, decompress_ms=d_ms,
                compress_gbs=4.0 * N / (c_ms * 1e-3) / 1e9, decompress_gbs=4.0 * N / (d_ms * 1e-3) / 1e9,
                n_outliers=int(h.n_outliers), entropy_bits=est["entropy_bits"], cr_est=est["cr"],
                max_err_over_eps=err / h.eps,
                psnr_db=20 * math.log10(vrange) - 10 * math.log10(mse) if mse > 0 else None,
                gpu_launches_per_call={"compress": 3, "decompress": 2},
                l2="256 MiB written between timed calls")
    if cpu:
        import oracle
        olv = None
        if levels is not None:
            olv = (np.array([lv[0] for lv in levels], dtype=np.uint8),
                   np.array([lv[1] for lv in levels], dtype=np.uint8))
        cores = host_cores()
        t0 = time.perf_counter()
        ref, y, _ = oracle_roundtrip(x_host, A=A_, eb=eb, levels=olv, workers=cores)
        t_all = time.perf_counter() - t0
        t0 = time.perf_counter()
        oracle_roundtrip(x_host, A=A_, eb=eb, levels=olv)
        t_one = time.perf_counter() - t0
        line["bit_exact_vs_oracle"] = bool(
            np.array_equal(b.codes.cpu().numpy().reshape(x_host.shape), ref["codes"])
            and np.array_equal(out.cpu().numpy().view(np.uint32), y.view(np.uint32)))
        line["oracle"] = dict(kind="oracle", what="compress + decompress of the whole field", unit="GB/s",
                              all_cores=dict(cores=cores, value=4.0 * N / t_all / 1e9, seconds=t_all),
                              one_thread=dict(cores=1, value=4.0 * N / t_one / 1e9, seconds=t_one))
    del b, out, flush, x
    torch.cuda.empty_cache()
    return line


def other_workloads(args, dev, x512_host):
    """Config 0 (64^3 bumps, A = 8, cubic, latency), config 2 (the 2D and the
    stratified 3D field at 1e-3 and 1e-4), the bound sweep of the 512^3 field
    (1e-2, 1e-4), the batched workload and the serving loop."""
    import torch
    from paper_2507_11165_gb300 import fields, hi
    res = {}
    x0 = fields.bumps_field((64, 64, 64), seed=0)
    c0 = field_line(x0, 1e-3, 8, dev, levels=[(hi.CUBIC, (0, 1, 2))] * 3, reps=50)
    c0["latency_us"] = dict(compress=1e3 * c0["compress_ms"], decompress=1e3 * c0["decompress_ms"])
    res["config0_64cube_bumps_A8_cubic_rel1e-3"] = c0
    x2a = fields.fronts_2d((1800, 3600), seed=2)
    x2b = fields.stratified_3d((100, 500, 500), seed=3)
    for eb in (1e-3, 1e-4):
        res["config2a_1800x3600_fronts_rel%g" % eb] = field_line(x2a, eb, 16, dev)
        res["config2b_100x500x500_stratified_rel%g" % eb] = field_line(x2b, eb, 16, dev)
    for eb in (1e-2, 1e-4):
        res["config1_512cube_grf_rel%g" % eb] = field_line(x512_host, eb, 16, dev, reps=10, cpu=False)
    if not args.no_batch:
        try:
            res["batch"] = batch_line(args)
        except Exception as e:  # keep the headline line even if a side workload fails
            res["batch"] = dict(error=repr(e))
        torch.cuda.empty_cache()
    if not args.no_serve:
        try:
            res["serve"] = serve_line(args, base=torch.from_numpy(x512_host).to(dev))
        except Exception as e:
            res["serve"] = dict(error=repr(e))
        torch.cuda.empty_cache()
    return res


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2507_11165_gb300 import fields, hi

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    x_host = fields.lognormal_grf(SHAPE, seed=SEED)
    N = x_host.size
    x = torch.from_numpy(x_host).to(dev)
    p = hi.make_params(SHAPE, EB, "rel", A, autotune=2 if args.md else True)
    b = hi.alloc(p, SHAPE, dev, hist=True, recon=False)
    out = torch.empty(SHAPE, dtype=torch.float32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)

    def step():
        hi.compress_into(x, b)
        hi.decompress_into(b, out, status)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    h = hi.read_header(b.header)
    assert h.status == 0 and int(status.item()) == 0, (h.status, int(status.item()))

    # per-stage events on a bounded number of steps inside the timed region
    n_ev = min(args.steps, 256)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(8)] for _ in range(n_ev)]
    for row in ev:  # torch creates the CUDA event on its first record
        for e in row:
            e.record(stream)
    torch.cuda.synchronize()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_start.record(stream)
        for k in range(args.steps):
            if k < n_ev:
                hi.set_stage_events(ev[k])
            elif k == n_ev:
                hi.set_stage_events(None)
            step()
        t_end.record(stream)
        torch.cuda.synchronize()
    hi.set_stage_events(None)
    if ws > 1:
        dist.barrier()
    ms = t_start.elapsed_time(t_end) / args.steps
    if ws > 1:
        tt = torch.tensor([ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    stage_names = ["setup", "range", "autotune", "predict_quantize", "scatter", "reconstruct"]
    pairs = [(0, 1), (1, 2), (2, 3), (3, 4), (5, 6), (6, 7)]
    st = {n: sum(e[a].elapsed_time(e[b_]) for e in ev) / n_ev for n, (a, b_) in zip(stage_names, pairs)}

    # results of the last step: quality and size
    h = hi.read_header(b.header)
    assert h.status == 0 and int(status.item()) == 0
    hist = b.hist.cpu().numpy().view(np.uint32)
    est = hi.estimate_cr(hist, int(h.n_outliers), int(h.n_anchors), N)
    err = (out - x).abs().max().item()
    mse = float(((out.double() - x.double()) ** 2).mean().item())
    vrange = float(h.vmax) - float(h.vmin)
    psnr = 20 * math.log10(vrange) - 10 * math.log10(mse) if mse > 0 else float("inf")

    bytes_in = 4.0 * N
    n_out = int(h.n_outliers)
    n_anc = int(h.n_anchors)
    alg = {"predict_quantize": 4.0 * N + N + 4.0 * n_anc + 8.0 * n_out,
           "reconstruct": N + 4.0 * n_anc + 4.0 * N}
    peak, peak_kind = peaks()
    dom = max(("predict_quantize", "reconstruct"), key=lambda k: st[k])
    achieved = alg[dom] / (st[dom] * 1e-3) / 1e9
    kname = {"predict_quantize": "k_compress", "reconstruct": "k_decompress"}[dom]
    traffic = traffic_record(kname)

    # quantization-code reordering (Sec. 5.2.2, Eq. 3) of this step's codes and back, each timed on
    # its own (not part of the step: decompression reads the row-major codes); 2N bytes per direction
    seq = torch.empty(N, dtype=torch.uint8, device=dev)
    back = torch.empty(N, dtype=torch.uint8, device=dev)
    for _ in range(3):
        hi.reorder_codes(b.codes, p, out=seq, stream=stream)
        hi.unreorder_codes(seq, p, out=back, stream=stream)
    rev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(10)]
    for e in rev:
        e[0].record(stream)
        hi.reorder_codes(b.codes, p, out=seq, stream=stream)
        e[1].record(stream)
        hi.unreorder_codes(seq, p, out=back, stream=stream)
        e[2].record(stream)
    torch.cuda.synchronize()
    assert torch.equal(back, b.codes)
    f_ms = statistics.median(e[0].elapsed_time(e[1]) for e in rev)
    i_ms = statistics.median(e[1].elapsed_time(e[2]) for e in rev)
    rows_path = SHAPE[-1] % 16 == 0 and SHAPE[-1] <= 4096  # staged rows (buffers from torch: aligned)
    reorder = dict(kernel="k_reorder_rows" if rows_path else "k_reorder", forward_ms=f_ms, inverse_ms=i_ms,
                   alg_bytes=2 * N,
                   traffic_fwd=traffic_record("k_reorder_rows_fwd") if rows_path else None,
                   traffic_inv=traffic_record("k_reorder_rows_inv") if rows_path else None,
                   forward_gbs=2 * N / (f_ms * 1e-3) / 1e9, inverse_gbs=2 * N / (i_ms * 1e-3) / 1e9,
                   forward_frac=2 * N / (f_ms * 1e-3) / 1e9 / peak, inverse_frac=2 * N / (i_ms * 1e-3) / 1e9 / peak)
    # the forward reordering written by predict-quantize itself (hi_compress_seq: each tile row's codes
    # also go to their places in the sequence from the kernel's registers), against hi_compress followed
    # by hi_reorder_codes; both whole compressions (range, auto-tune, predict-quantize)
    seq2 = torch.empty(N, dtype=torch.uint8, device=dev)
    fused = hi.compress_seq_fused(p, b.codes.data_ptr(), seq2.data_ptr())
    for _ in range(3):
        hi.compress_seq_into(x, b, seq2, stream=stream)
        hi.compress_into(x, b, stream=stream)
        hi.reorder_codes(b.codes, p, out=seq, stream=stream)
    fev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(10)]
    for e in fev:
        e[0].record(stream)
        hi.compress_seq_into(x, b, seq2, stream=stream)
        e[1].record(stream)
        hi.compress_into(x, b, stream=stream)
        hi.reorder_codes(b.codes, p, out=seq, stream=stream)
        e[2].record(stream)
    torch.cuda.synchronize()
    cs_ms = statistics.median(e[0].elapsed_time(e[1]) for e in fev)
    cr_ms = statistics.median(e[1].elapsed_time(e[2]) for e in fev)
    reorder["compress_seq"] = dict(api="hi_compress_seq", fused_in_kernel=fused, compress_seq_ms=cs_ms,
                                   compress_then_reorder_ms=cr_ms, saved_ms=cr_ms - cs_ms,
                                   bit_exact_vs_separate=bool(torch.equal(seq, seq2)))
    del seq2
    # throughput-mode lossless pipeline TCMS1-BIT1-RRE1 (Sec. 5.2.3) on the reordered codes: a real
    # compressed size beside the entropy estimate; timed on its own, not part of the step
    hi.reorder_codes(b.codes, p, out=seq, stream=stream)
    codec = hi.TpCodec(N, dev)
    for _ in range(2):
        codec.encode_into(seq, stream=stream)
        torch.cuda.synchronize()
        s_len = int(codec.len.item())
        codec.decode_into(codec.stream_buf, s_len, back, stream=stream)
    tev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(5)]
    for e in tev:
        e[0].record(stream)
        codec.encode_into(seq, stream=stream)
        e[1].record(stream)
        codec.decode_into(codec.stream_buf, s_len, back, stream=stream)
        e[2].record(stream)
    torch.cuda.synchronize()
    assert int(codec.status.item()) == 0 and torch.equal(back, seq) and int(codec.len.item()) == s_len
    te_ms = statistics.median(e[0].elapsed_time(e[1]) for e in tev)
    td_ms = statistics.median(e[1].elapsed_time(e[2]) for e in tev)
    n_out_tp = int(hi.read_header(b.header).n_outliers)
    rec_bytes = s_len + 8 * n_out_tp + 4 * int(b.anchors.numel()) + hi.HEADER_BYTES
    lossless_tp = dict(pipeline="TCMS1-BIT1-RRE1", kernels=["k_tp_encode_chunks", "k_tp_scan", "k_tp_gather",
                                                            "k_tp_decode_chunks"],
                       encode_ms=te_ms, decode_ms=td_ms, encode_gbs_of_codes=N / (te_ms * 1e-3) / 1e9,
                       decode_gbs_of_codes=N / (td_ms * 1e-3) / 1e9, stream_bytes=s_len,
                       codes_ratio=N / s_len, record_bytes=rec_bytes, cr=4.0 * N / rec_bytes,
                       launches_encode=3, launches_decode=2)
    # compression-ratio-mode lossless pipeline HF-RRE4-TCMS8-RZE1 (Sec. 5.2.3) on the same codes
    crc = hi.CrCodec(N, dev)
    for _ in range(2):
        crc.encode_into(seq, stream=stream)
        torch.cuda.synchronize()
        c_len = int(crc.len.item())
        crc.decode_into(crc.stream_buf, c_len, back, stream=stream)
    cev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(5)]
    for e in cev:
        e[0].record(stream)
        crc.encode_into(seq, stream=stream)
        e[1].record(stream)
        crc.decode_into(crc.stream_buf, c_len, back, stream=stream)
        e[2].record(stream)
    torch.cuda.synchronize()
    assert int(crc.status.item()) == 0 and torch.equal(back, seq) and int(crc.len.item()) == c_len
    ce_ms = statistics.median(e[0].elapsed_time(e[1]) for e in cev)
    cd_ms = statistics.median(e[1].elapsed_time(e[2]) for e in cev)
    rec_cr = c_len + 8 * n_out_tp + 4 * int(b.anchors.numel()) + hi.HEADER_BYTES
    lossless_cr = dict(pipeline="HF-RRE4-TCMS8-RZE1",
                       kernels=["k_cr_hist", "k_cr_codebook", "k_hf_count", "k_cr_scan_words", "k_hf_encode",
                                "k_cr_lc_encode", "k_cr_scan_payloads", "k_cr_gather", "k_cr_dec_scan",
                                "k_cr_lc_decode", "k_hf_decode"],
                       encode_ms=ce_ms, decode_ms=cd_ms, encode_gbs_of_codes=N / (ce_ms * 1e-3) / 1e9,
                       decode_gbs_of_codes=N / (cd_ms * 1e-3) / 1e9, stream_bytes=c_len, codes_ratio=N / c_len,
                       record_bytes=rec_cr, cr=4.0 * N / rec_cr, launches_encode=8, launches_decode=3)
    del seq, back, codec, crc

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    e2e = None
    b2 = None
    if not args.no_e2e:
        xh = torch.from_numpy(x_host).pin_memory()
        codes_h = torch.empty(N, dtype=torch.uint8).pin_memory()
        anch_h = torch.empty(b.anchors.numel(), dtype=torch.float32).pin_memory()
        oidx_h = torch.empty(b.out_cap, dtype=torch.int32).pin_memory()
        oval_h = torch.empty(b.out_cap, dtype=torch.float32).pin_memory()
        hdr_h = torch.empty(hi.HEADER_BYTES, dtype=torch.uint8).pin_memory()
        y_h = torch.empty(SHAPE, dtype=torch.float32).pin_memory()
        xd = torch.empty_like(x)
        b2 = hi.alloc(p, SHAPE, dev, hist=True, recon=False)
        io = {"h2d": 0, "d2h": 0}

        def e2e_step():
            # host field -> device -> compressed record on the host -> device -> host field
            xd.copy_(xh, non_blocking=True)
            hi.compress_into(xd, b)
            hdr = hi.read_header(b.header)  # the record's size is known only now
            k = min(int(hdr.n_outliers), b.out_cap)
            codes_h.copy_(b.codes, non_blocking=True)
            anch_h.copy_(b.anchors, non_blocking=True)
            hdr_h.copy_(b.header, non_blocking=True)
            if k:
                oidx_h[:k].copy_(b.out_idx[:k], non_blocking=True)
                oval_h[:k].copy_(b.out_val[:k], non_blocking=True)
            b2.codes.copy_(codes_h, non_blocking=True)
            b2.anchors.copy_(anch_h, non_blocking=True)
            b2.header.copy_(hdr_h, non_blocking=True)
            if k:
                b2.out_idx[:k].copy_(oidx_h[:k], non_blocking=True)
                b2.out_val[:k].copy_(oval_h[:k], non_blocking=True)
            hi.decompress_into(b2, out, status)
            y_h.copy_(out, non_blocking=True)
            return k

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        ke = max(3, min(args.steps, 20))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ks = []
        for _ in range(ke):
            ks.append(e2e_step())
        e1.record(stream)
        torch.cuda.synchronize()
        serial_ms = e0.elapsed_time(e1) / ke
        assert torch.equal(y_h.to(dev), out)

        # the same steps with two fields in flight on three streams: a field's upload and compression;
        # the previous field's record to the host and back and its reconstruction; the download of the
        # reconstructed field (uploads and downloads share the link in opposite directions); the host
        # still reads each record's header before copying its outliers
        s_c, s_d, s_y = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        D = 2  # steps in flight (three measured the same)
        xds = [xd] + [torch.empty_like(x) for _ in range(D - 1)]
        bbs = [b] + [hi.alloc(p, SHAPE, dev, out_cap=b.out_cap, hist=True, recon=False) for _ in range(D - 1)]
        outs = [out] + [torch.empty_like(out) for _ in range(D - 1)]
        hdr_hs = [hdr_h] + [torch.empty(hi.HEADER_BYTES, dtype=torch.uint8).pin_memory() for _ in range(D - 1)]
        y_hs = [y_h] + [torch.empty(SHAPE, dtype=torch.float32).pin_memory() for _ in range(D - 1)]
        ev_hdr, ev_free, ev_dec, ev_yfree = ([torch.cuda.Event() for _ in range(D)] for _ in range(4))

        def front(k):
            i = k % D
            with torch.cuda.stream(s_c):
                s_c.wait_event(ev_free[i])  # the record of D steps back has left these buffers
                xds[i].copy_(xh, non_blocking=True)
                hi.compress_into(xds[i], bbs[i], stream=s_c)
                hdr_hs[i].copy_(bbs[i].header, non_blocking=True)
                ev_hdr[i].record(s_c)

        def back(k):
            i = k % D
            ev_hdr[i].synchronize()
            kk = min(int(hi.HiHeader.from_buffer_copy(hdr_hs[i].numpy().tobytes()).n_outliers), bbs[i].out_cap)
            bb = bbs[i]
            with torch.cuda.stream(s_d):
                s_d.wait_event(ev_hdr[i])
                codes_h.copy_(bb.codes, non_blocking=True)
                anch_h.copy_(bb.anchors, non_blocking=True)
                if kk:
                    oidx_h[:kk].copy_(bb.out_idx[:kk], non_blocking=True)
                    oval_h[:kk].copy_(bb.out_val[:kk], non_blocking=True)
                ev_free[i].record(s_d)
                b2.codes.copy_(codes_h, non_blocking=True)
                b2.anchors.copy_(anch_h, non_blocking=True)
                b2.header.copy_(hdr_hs[i], non_blocking=True)
                if kk:
                    b2.out_idx[:kk].copy_(oidx_h[:kk], non_blocking=True)
                    b2.out_val[:kk].copy_(oval_h[:kk], non_blocking=True)
                s_d.wait_event(ev_yfree[i])  # the field of D steps back has left outs[i]
                hi.decompress_into(b2, outs[i], status, stream=s_d)
                ev_dec[i].record(s_d)
            with torch.cuda.stream(s_y):
                s_y.wait_event(ev_dec[i])
                y_hs[i].copy_(outs[i], non_blocking=True)
                ev_yfree[i].record(s_y)
            return kk

        def pipelined(nsteps, ev_a=None, ev_b=None):
            if ev_a is not None:
                ev_a.record(s_c)
                s_d.wait_event(ev_a)
                s_y.wait_event(ev_a)
            kl = []
            for k in range(min(D - 1, nsteps)):
                front(k)
            for k in range(D - 1, nsteps):
                front(k)
                kl.append(back(k - D + 1))
            for k in range(max(0, nsteps - D + 1), nsteps):
                kl.append(back(k))
            if ev_b is not None:
                ev_b.record(s_y)  # after the last step's download, which waited for all its other work
            return kl

        torch.cuda.synchronize()
        pipelined(D)
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ks = pipelined(ke, p0, p1)
        torch.cuda.synchronize()
        ems = p0.elapsed_time(p1) / ke
        assert int(status.item()) == 0
        assert torch.equal(y_hs[(ke - 1) % D].to(dev), outs[(ke - 1) % D])
        kmean = sum(ks) / len(ks)
        h2d = 4 * N + (N + 4 * b.anchors.numel() + hi.HEADER_BYTES + 8 * kmean)
        d2h = (N + 4 * b.anchors.numel() + hi.HEADER_BYTES + 8 * kmean) + hi.HEADER_BYTES + 4 * N
        if ws > 1:
            tt = torch.tensor([ems, serial_ms], device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            ems, serial_ms = float(tt[0].item()), float(tt[1].item())
        # the link alone, same pinned buffers: the field up, the field down, and both at once on two
        # streams (10 repetitions each, median); the step's copies cannot beat these
        def copy_ms(up, down):
            ts = []
            for _ in range(10):
                a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record(s_c)
                s_d.wait_event(a)
                if up:
                    with torch.cuda.stream(s_c):
                        xds[0].copy_(xh, non_blocking=True)
                if down:
                    with torch.cuda.stream(s_d):
                        y_hs[0].copy_(outs[0], non_blocking=True)
                s_c.wait_stream(s_d)
                z.record(s_c)
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(z))
            return statistics.median(ts)
        up_ms, down_ms, both_ms = copy_ms(True, False), copy_ms(False, True), copy_ms(True, True)
        link = dict(h2d_gbs=4 * N / (up_ms * 1e-3) / 1e9, d2h_gbs=4 * N / (down_ms * 1e-3) / 1e9,
                    both_gbs=8 * N / (both_ms * 1e-3) / 1e9, bytes=4 * N,
                    step_copy_bound_ms=(h2d + d2h) / (8 * N / (both_ms * 1e-3)) * 1e3,
                    how="512 MiB pinned host <-> device with cudaMemcpyAsync (torch copy_), up, down, and both "
                        "at once on two streams; medians of 10")
        e2e = dict(value=ws * bytes_in / (ems * 1e-3) / 1e9, unit="GB/s", ms_per_step=ems, link=link,
                   h2d_bytes_per_step=int(h2d), d2h_bytes_per_step=int(d2h),
                   how="per step: the field from pinned host memory, hi_compress, the record to pinned host "
                       "memory (header read on the host first), back to the device, hi_decompress, the field "
                       "to the host; two steps in flight on three streams (upload + compress, record round trip + "
                       "reconstruct, download)",
                   serial=dict(value=ws * bytes_in / (serial_ms * 1e-3) / 1e9, ms_per_step=serial_ms,
                               how="the same step one at a time on one stream"))
        del b2, xh, codes_h, anch_h, oidx_h, oval_h, hdr_h, y_h, xd, xds, bbs, outs, hdr_hs, y_hs

    others = None
    if rank == 0 and ws == 1 and not args.no_extra:
        torch.cuda.empty_cache()
        others = other_workloads(args, dev, x_host)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:  # the oracle leg: one process on one GPU only
        cpu, ref = cpu_baseline(x_host, args.cpu_planes)
        if args.cpu_planes == SHAPE[0]:
            # same field, same eb: the oracle's codes must equal this run's, bit for bit
            cpu["codes_match_gpu"] = bool(np.array_equal(b.codes.cpu().numpy().reshape(SHAPE), ref["codes"]))

    if rank == 0:
        clocks = clk.summary()
        line = dict(
            metric=METRIC, value=ws * bytes_in / (ms * 1e-3) / 1e9, unit="GB/s", n_gpus=ws, steps=args.steps,
            warmup=args.warmup, ms_per_step=ms, higher_is_better=True, scaling="weak", vs_baseline=None,
            dtype="f32", data="synthetic",
            config=dict(workload=WORKLOAD, shape=list(SHAPE), eb_mode="rel", eb=EB, anchor_stride=A,
                        l2="input 512 MiB and outputs exceed the 126 MB L2: no flush between steps",
                        step="compress (setup, range + autotune in one launch, predict_quantize) + decompress (scatter, "
                             "reconstruct)", parallelism="replicas" if ws > 1 else "single"),
            compress_gbs=bytes_in / ((st["setup"] + st["range"] + st["autotune"] + st["predict_quantize"])
                                     * 1e-3) / 1e9,
            decompress_gbs=bytes_in / ((st["scatter"] + st["reconstruct"]) * 1e-3) / 1e9,
            predict_quantize_gbs=bytes_in / (st["predict_quantize"] * 1e-3) / 1e9,
            reconstruct_gbs=bytes_in / (st["reconstruct"] * 1e-3) / 1e9,
            stage_ms=st,
            roofline=dict(bound="hbm", kernel=kname, achieved=achieved, peak=peak, unit="GB/s",
                          frac=achieved / peak, traffic=traffic, peak_kind=peak_kind,
                          alg_bytes_per_launch=alg[dom],
                          other={k: dict(achieved=alg[k] / (st[k] * 1e-3) / 1e9,
                                         frac=alg[k] / (st[k] * 1e-3) / 1e9 / peak) for k in alg}),
            quality=dict(max_abs_err=err, eps=h.eps, max_err_over_eps=err / h.eps, psnr_db=psnr,
                         n_outliers=n_out, entropy_bits=est["entropy_bits"], cr_est=est["cr"],
                         bit_rate=est["bit_rate"],
                         levels=[(int(h.level[l].interp), list(h.level[l].order)) for l in range(h.n_levels)]),
            reorder=reorder,
            lossless_tp=lossless_tp,
            lossless_cr=lossless_cr,
            e2e=e2e,
            gpu_launches=5 * args.steps,  # setup, range + auto-tune (one launch), predict-quantize, scatter, reconstruct
            cpu_baseline=cpu,
            clocks=clocks,
            other_workloads=others,
        )
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def _gen_field(spec):
    from paper_2507_11165_gb300 import fields
    return fields.make_field(spec)


def make_batch_inputs(n_fields, seed=4):
    """The batched workload's fields, generated on the host cores (spawned
    workers: no CUDA context is inherited)."""
    import concurrent.futures as cf
    import multiprocessing as mp

    from paper_2507_11165_gb300 import fields
    specs = fields.batch_specs(n_fields, seed=seed)
    workers = max(1, min(16, (os.cpu_count() or 1)))
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        arrs = list(ex.map(_gen_field, specs, chunksize=4))
    return specs, arrs


BATCH_METRIC = "batched compress input GB/s per GB300 (256 fields, rel eb 1e-2/1e-3/1e-4), bit-exact vs per-field"


def run_batch(args):
    print(json.dumps(batch_line(args)), flush=True)


def batch_line(args):
    """Batched workload: 256 fields with sides log-uniform in [32, 256], rel eb
    per field from {1e-2, 1e-3, 1e-4}, auto-tuned levels; one step = one
    hi_compress_batch (four launches for all fields) replayed from a captured
    CUDA graph, after the launch-shape tuner picked the CTA shape.  Beside it:
    the plain per-field path (256 hi_compress calls) on the same buffers."""
    import numpy as np
    import torch

    specs, arrs = make_batch_inputs(args.batch_fields)
    from paper_2507_11165_gb300 import hi

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    xs = [torch.from_numpy(a).to(dev) for a in arrs]
    ebs = [s["eb"] for s in specs]
    Ns = [a.size for a in arrs]
    N = sum(Ns)
    # outlier capacity = field size: no field can overflow at any bound
    bat = hi.Batch(xs, ebs, "rel", anchor_stride=A, autotune=True, out_caps=Ns, hist=True, recon=False, outs=True)
    shape_ms = bat.tune_launch(reps=3)
    # plain path: one hi_compress per field, its own buffers
    plain = []
    for x, eb, n in zip(xs, ebs, Ns):
        p = hi.make_params(x.shape, eb, "rel", A, autotune=True)
        plain.append(hi.alloc(p, x.shape, dev, out_cap=n, hist=True, recon=False))

    def plain_step():
        for x, b in zip(xs, plain):
            hi.compress_into(x, b)

    for _ in range(max(args.warmup, 3)):
        bat.compress()
        plain_step()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bat.compress()
    for _ in range(max(args.warmup, 3)):
        g.replay()
    torch.cuda.synchronize()

    # per-stage times on a few graph-free runs
    n_ev = 5
    sev = [[torch.cuda.Event(enable_timing=True) for _ in range(8)] for _ in range(n_ev)]
    for row in sev:
        for e in row:
            e.record(stream)
    torch.cuda.synchronize()
    for row in sev:
        hi.set_stage_events(row)
        bat.compress()
    hi.set_stage_events(None)
    torch.cuda.synchronize()
    stage = {nm: sum(r[a].elapsed_time(r[b_]) for r in sev) / n_ev
             for nm, (a, b_) in zip(["setup", "range", "autotune", "predict_quantize"], [(0, 1), (1, 2), (2, 3), (3, 4)])}

    steps = args.steps
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    with ClockSampler(0) as clk:
        ev[0].record(stream)
        for _ in range(steps):
            g.replay()
        ev[1].record(stream)
        torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / steps
    ksteps = max(3, min(steps, 10))
    ev[2].record(stream)
    for _ in range(ksteps):
        plain_step()
    ev[3].record(stream)
    torch.cuda.synchronize()
    ms_plain = ev[2].elapsed_time(ev[3]) / ksteps

    # batched reconstruction (two launches for all fields, replayed from a graph) against one
    # hi_decompress per field into the same outputs
    gd = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gd):
        bat.decompress()
    pst = torch.zeros(1, dtype=torch.int32, device=dev)

    def plain_dstep():
        for b, y in zip(bat.buffers, bat.outs):
            hi.decompress_into(b, y, pst)

    for _ in range(max(args.warmup, 3)):
        gd.replay()
        plain_dstep()
    torch.cuda.synchronize()
    dev_ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    dev_ev[0].record(stream)
    for _ in range(steps):
        gd.replay()
    dev_ev[1].record(stream)
    for _ in range(ksteps):
        plain_dstep()
    dev_ev[2].record(stream)
    gd.replay()
    dev_ev[3].record(stream)
    torch.cuda.synchronize()
    d_ms = dev_ev[0].elapsed_time(dev_ev[1]) / steps
    d_ms_plain = dev_ev[1].elapsed_time(dev_ev[2]) / ksteps
    d_ok = int(bat.dstatus.item()) == 0 and int(pst.item()) == 0
    d_exact = True
    refs = [torch.empty_like(y) for y in bat.outs]
    for b, r in zip(bat.buffers, refs):
        hi.decompress_into(b, r, pst)
    torch.cuda.synchronize()
    for y, r in zip(bat.outs, refs):
        d_exact = d_exact and torch.equal(y.view(torch.int32), r.view(torch.int32))
    del refs

    # every field: the batch's record equals the plain path's
    g.replay()
    torch.cuda.synchronize()
    mismatched = []
    n_out = 0
    n_anc = 0
    for i, (bb, pb) in enumerate(zip(bat.buffers, plain)):
        hb_, hp_ = hi.read_header(bb.header), hi.read_header(pb.header)
        ok = bytes(hb_) == bytes(hp_) and hb_.status == 0
        ok = ok and torch.equal(bb.codes, pb.codes) and torch.equal(bb.hist, pb.hist)
        ok = ok and torch.equal(bb.anchors[: int(hb_.n_anchors)], pb.anchors[: int(hp_.n_anchors)])
        k = int(hb_.n_outliers)
        ok = ok and torch.equal(torch.sort(bb.out_idx[:k])[0], torch.sort(pb.out_idx[:k])[0])
        if not ok:
            mismatched.append(i)
        n_out += k
        n_anc += int(hb_.n_anchors)
    exact = not mismatched
    bytes_in = 4.0 * N
    alg = 4.0 * N + (4.0 * N + N + 4.0 * n_anc + 8.0 * n_out)  # range read + predict-quantize
    peak, peak_kind = peaks()
    achieved = alg / (ms * 1e-3) / 1e9
    line = dict(
        metric=BATCH_METRIC, value=bytes_in / (ms * 1e-3) / 1e9, unit="GB/s", n_gpus=1, steps=steps,
        warmup=args.warmup, ms_per_step=ms, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
        data="synthetic",
        config=dict(workload="%d fields, sides log-uniform in [32, 256] per axis (seed 4), bumps / log-normal GRF "
                             "alternating, rel eb per field from {1e-2, 1e-3, 1e-4}, anchor stride 16, auto-tuned "
                             "levels" % len(xs),
                    points=N, input_bytes=int(bytes_in),
                    step="hi_compress_batch (setup, range, autotune, predict_quantize for all fields) replayed "
                         "from a CUDA graph",
                    l2="%.2f GB of input exceeds the 126 MB L2: no flush" % (bytes_in / 1e9)),
        launch_shape=dict(threads=bat.shape[0], buffers=bat.shape[1],
                          tuner_ms={"%dx%d" % k: v for k, v in shape_ms.items()}),
        plain_path=dict(value=bytes_in / (ms_plain * 1e-3) / 1e9, ms_per_step=ms_plain,
                        launches=4 * len(xs), how="one hi_compress per field, same stream"),
        speedup_vs_plain=ms_plain / ms,
        bit_exact_vs_plain=bool(exact),
        decompress=dict(value=bytes_in / (d_ms * 1e-3) / 1e9, ms_per_step=d_ms, launches=2,
                        how="hi_decompress_batch (outlier scatter + one persistent reconstruction) from a CUDA graph",
                        plain_path=dict(value=bytes_in / (d_ms_plain * 1e-3) / 1e9, ms_per_step=d_ms_plain,
                                        launches=2 * len(xs), how="one hi_decompress per field, same stream"),
                        speedup_vs_plain=d_ms_plain / d_ms, bit_exact_vs_plain=bool(d_exact), status_ok=bool(d_ok)),
        mismatched_fields=mismatched,
        stage_ms=stage,
        n_outliers=n_out,
        roofline=dict(bound="hbm", achieved=achieved, peak=peak, unit="GB/s", frac=achieved / peak,
                      peak_kind=peak_kind, alg_bytes_per_step=alg,
                      note="whole step: range read 4 B/pt + predict-quantize 5 B/pt"),
        gpu_launches=4 * steps,  # setup, range + auto-tune, gather, predict-quantize
        clocks=clk.summary(),
    )
    return line


SERVE_METRIC = "serving: sustained input GB/s with p50/p99 latency (ms), Poisson 200 req/s, 40 GB budget"


def run_serve(args):
    print(json.dumps(serve_line(args)), flush=True)


def serve_line(args, base=None):
    """Serving workload: Poisson arrivals (200 / s), half compress of a
    snapshot, half decompress of an earlier record; cubic sides log-uniform
    in [64, 512]; rel eb from {1e-2, 1e-3, 1e-4, 1e-5}; admitted by slot
    (8 streams) and a 40 GB device budget.  Snapshots are side^3 blocks of a
    resident 512^3 field.  Also: the same requests all arriving at once
    (saturation), and one slot only (no overlap) on the timed stream.  One
    untimed burst of the whole stream first: the process is warm."""
    import numpy as np
    import torch

    from paper_2507_11165_gb300 import fields, hi, serve

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    if base is None:
        base = torch.from_numpy(fields.lognormal_grf(SHAPE, seed=SEED)).to(dev)
    reqs = serve.make_requests(n=args.serve_requests, rate=200.0, seed=5, lo=64, hi=SHAPE[0])
    warm = serve.make_requests(n=16, rate=1e6, seed=6, lo=64, hi=SHAPE[0])

    def one(requests, slots, budget=40 * 10 ** 9):
        ex = serve.GpuExecutor(base)
        sv = serve.Server(ex, slots=slots, budget_bytes=budget)
        t0 = time.perf_counter()
        done = sv.run(requests)
        wall = time.perf_counter() - t0
        s = serve.summarize(done, wall)
        s.update(peak_concurrency=sv.peak_concurrency, peak_bytes=sv.peak_bytes, slots=slots, launches=ex.launches)
        return s

    burst = [serve.Request(r.id, 0.0, r.op, r.side, r.eb, r.seed, r.source) for r in reqs]
    one(warm, 8)
    one(burst, 8)  # a warm process: the allocator holds blocks of every size the stream asks for
    with ClockSampler(0) as clk:
        main = one(reqs, 8)
    sat = one(burst, 8)
    single = one(reqs, 1)
    offered = sum(4 * r.side ** 3 for r in reqs) / max(r.t for r in reqs) / 1e9
    line = dict(
        metric=SERVE_METRIC, value=main["gbs"], unit="GB/s", n_gpus=1, steps=len(reqs), warmup=len(warm),
        ms_per_step=1e3 * main["wall_s"] / len(reqs), higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype="f32", data="synthetic",
        config=dict(workload="%d requests, Poisson 200/s (seed 5), 50%% compress / 50%% decompress of an earlier "
                             "record, cubic sides log-uniform in [64, 512], rel eb from {1e-2,1e-3,1e-4,1e-5}, "
                             "anchor stride 16, auto-tuned levels" % len(reqs),
                    slots=8, budget_gb=40, snapshots="side^3 blocks of a resident 512^3 log-normal GRF",
                    step="one request (value = input bytes of all requests / wall time of the run)"),
        p50_ms=main["p50_ms"], p99_ms=main["p99_ms"], max_ms=main["max_ms"], offered_gbs=offered,
        served=main, saturated=sat, one_slot=single,
        gpu_launches=main["launches"],  # compress 3 (+3 on a capacity re-run), decompress 2 per request
        clocks=clk.summary(),
    )
    return line


SHARD_METRIC = "sharded compress: input GB/s of one field split along d0 over the ranks (whole-job, max over ranks)"


def run_shard(args):
    """One field split along d0 over the ranks of the job (torchrun, NCCL):
    every rank holds its read planes on its GPU and runs
    shard.compress_distributed (value-range all-reduce, auto-tune rows of the
    global sample blocks, its owned part with global indices); one step is
    that whole call (host wall clock between barriers, max over ranks).  At
    N = 1 the single rank holds the whole field; rank 0 also checks the
    merged record against hi_compress of the whole field when N = 1."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2507_11165_gb300 import fields, hi, shard

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl")
    x_np = fields.lognormal_grf(SHAPE, seed=SEED)
    plan = shard.shard_bounds(SHAPE[0], A, ws)
    sh = plan[rank] if rank < len(plan) else None
    x_local = torch.from_numpy(np.ascontiguousarray(x_np[sh["own_lo"]:sh["read_hi"]] if sh else x_np[:0])).to(dev)
    ex = shard.GpuShardExecutor(dev)

    def step():
        return shard.compress_distributed(x_local, SHAPE, EB, A, ex, mode="rel", autotune=True)

    for _ in range(max(1, args.warmup)):
        part = step()
    steps = max(1, min(args.steps, 10))
    times = []
    with ClockSampler(local) as clk:
        for _ in range(steps):
            if ws > 1:
                dist.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            part = step()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
    t = statistics.median(times)
    if ws > 1:
        tt = torch.tensor([t], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    exact = None
    if ws == 1:
        c = hi.compress(torch.from_numpy(x_np).to(dev), EB, "rel", A, autotune=True, out_cap=x_np.size // 8)
        m = shard.merge_parts([part])
        exact = bool(np.array_equal(m["codes"].numpy().reshape(SHAPE), c.codes.cpu().numpy().reshape(SHAPE)))
    if rank == 0:
        line = dict(
            metric=SHARD_METRIC, value=4.0 * x_np.size / t / 1e9, unit="GB/s", n_gpus=ws, steps=steps,
            warmup=max(1, args.warmup), ms_per_step=1e3 * t, higher_is_better=True, scaling="strong",
            vs_baseline=None, dtype="f32", data="synthetic",
            config=dict(workload=WORKLOAD + ", split along d0 over the ranks", shards=len(plan),
                        parallelism="shard%d" % ws,
                        step="shard.compress_distributed: range all-reduce, auto-tune rows all-reduce, own part "
                             "(host wall clock, results on the device)"),
            bit_exact_vs_whole_field=exact,
            gpu_launches=None,
            clocks=clk.summary(),
        )
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


OOC_METRIC = "out-of-core compress: input GB/s of a host-resident field, two shards on the device"


def run_ooc(args):
    """A field held in pinned host memory compressed on one GPU two shards at
    a time (value ranges, then each shard with its halo plane at the field's
    eps, the next shard uploading meanwhile), merged into host arrays; the
    record is checked against the whole field compressed on the device."""
    import numpy as np
    import torch

    from paper_2507_11165_gb300 import fields, hi, shard

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    x_np = fields.lognormal_grf(SHAPE, seed=SEED)
    x_host = torch.from_numpy(x_np).pin_memory()
    blocks = 4
    c = hi.compress(torch.from_numpy(x_np).to(dev), EB, "rel", A, autotune=True, out_cap=x_np.size // 8)
    levels = [(int(c.h.level[l].interp), tuple(int(v) for v in c.h.level[l].order)) for l in range(c.h.n_levels)]
    ref_codes = c.codes.cpu().numpy().reshape(SHAPE)
    ref_hist = c.hist.cpu().numpy().view(np.uint32).astype(np.int64)
    del c
    torch.cuda.empty_cache()
    for _ in range(max(1, args.warmup)):
        shard.compress_out_of_core(x_host, EB, A, levels, shard_blocks=blocks)
    steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        for _ in range(steps):
            m = shard.compress_out_of_core(x_host, EB, A, levels, shard_blocks=blocks)
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) / steps
    exact = bool(np.array_equal(m["codes"], ref_codes)) and bool(np.array_equal(m["hist"], ref_hist))
    nb0 = (SHAPE[0] - 1 + A - 1) // A
    line = dict(
        metric=OOC_METRIC, value=4.0 * x_np.size / wall / 1e9, unit="GB/s", n_gpus=1, steps=steps,
        warmup=max(1, args.warmup), ms_per_step=1e3 * wall, higher_is_better=True, scaling="weak",
        vs_baseline=None, dtype="f32", data="synthetic",
        config=dict(workload=WORKLOAD + ", held in pinned host memory", shards=-(-nb0 // blocks),
                    shard_planes=blocks * A + 1, levels="the whole-field auto-tuner's choice",
                    step="value ranges of the shards + compression of each shard, results copied to host arrays "
                         "(host wall clock)"),
        bit_exact_vs_whole_field=exact,
        # per shard: set-up + range (hi_value_range), then set-up + predict-quantize (absolute bound)
        gpu_launches=steps * (-(-nb0 // blocks)) * 4,
        clocks=clk.summary(),
    )
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="single: only the headline field (no other workloads)")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--cpu-planes", type=int, default=512)
    ap.add_argument("--ref-planes", type=int, default=512)
    ap.add_argument("--workload", default="single", choices=["single", "batch", "serve", "ooc", "shard"],
                    help="single: the 512^3 field (default); batch: 256 fields in one batched launch per stage; "
                         "serve: a Poisson request stream through the continuous-batching loop")
    ap.add_argument("--batch-fields", type=int, default=256)
    ap.add_argument("--eb", type=float, default=None, help="single: another relative bound (the sweep 1e-2 / 1e-4)")
    ap.add_argument("--md", action="store_true",
                    help="single: auto-tune over the 1D sequences and the multi-dimensional scheme")
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--shape", type=int, default=None,
                    help="cube side of a smaller field of the same recipe (profiling captures)")
    args = ap.parse_args()
    global SHAPE, WORKLOAD, EB
    if args.eb:
        EB = args.eb
        WORKLOAD = WORKLOAD.replace("rel eb 1e-3", "rel eb %g" % EB)
    if args.md:
        WORKLOAD = WORKLOAD.replace("auto-tuned levels", "auto-tuned levels incl. the multi-dimensional scheme")
    if args.shape:
        SHAPE = (args.shape,) * 3
        WORKLOAD = WORKLOAD.replace("512^3", "%d^3" % args.shape)
        args.cpu_planes = min(args.cpu_planes, args.shape)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "ooc":
        run_ooc(args)
    elif args.workload == "shard":
        run_shard(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
