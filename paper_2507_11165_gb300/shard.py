"""One field split into shards along its slowest dim (d0), at block
boundaries: the layout for several ranks (or several passes of one GPU) to
compress one field and reproduce the single-field record exactly.

Blocks share their faces (Sec. 5.1.1), and a block's points depend only on
its own (A+1)^3 points, so shard k, owning the blocks [t_lo, t_hi) along d0,
reads the planes [t_lo A, min(t_hi A, n0 - 1)]: its own planes plus the next
shard's first plane (its blocks' upper face), which it recomputes exactly as
the next shard does and does not output.  Across shards only three things
are exchanged:
  * value-range-relative bound: the min and the max of the finite values
    (eps then follows on every rank from the global range),
  * auto-tune: the per-sample error sums of the global sample blocks each
    rank holds, summed in global sample order on every rank,
  * outliers: counts and lists, concatenated in rank order.
"""
from __future__ import annotations

import math
from typing import List


def shard_bounds(n0: int, A: int, parts: int) -> List[dict]:
    """Shard k: blocks [t_lo, t_hi) along d0, owned planes [own_lo, own_hi),
    read planes [own_lo, read_hi).  Blocks are split as evenly as possible
    (the first shards take one more); fewer shards when there are fewer
    blocks than parts."""
    nb0 = 1 if n0 == 1 else (n0 - 1 + A - 1) // A
    parts = max(1, min(parts, nb0))
    base, extra = divmod(nb0, parts)
    out = []
    t = 0
    for k in range(parts):
        t_hi = t + base + (1 if k < extra else 0)
        last = k == parts - 1
        own_hi = n0 if last else t_hi * A
        read_hi = n0 if last else min(t_hi * A, n0 - 1) + 1
        out.append(dict(k=k, t_lo=t, t_hi=t_hi, own_lo=t * A, own_hi=own_hi, read_hi=read_hi, last=last))
        t = t_hi
    return out


def sample_blocks(shape, A: int) -> List[int]:
    """Row-major ids of the auto-tuner's sample blocks of the whole field
    (Sec. 5.1.3): every (n_blocks / m)-th block, m = max(1, round(0.002 N /
    A^d))."""
    dims = (1,) * (3 - len(shape)) + tuple(int(s) for s in shape)
    nb = [1 if n == 1 else (n - 1 + A - 1) // A for n in dims]
    nt = nb[0] * nb[1] * nb[2]
    d = sum(1 for n in dims if n > 1)
    m = int(math.floor(0.002 * math.prod(dims) / (A ** d) + 0.5))
    m = min(max(m, 1), nt)
    stride = nt // m
    return [k * stride for k in range(m)]


def local_block(gid: int, shape, A: int, sh: dict) -> int:
    """Row-major id, within shard sh, of global block gid (which it must hold)."""
    dims = (1,) * (3 - len(shape)) + tuple(int(s) for s in shape)
    nb1 = 1 if dims[1] == 1 else (dims[1] - 1 + A - 1) // A
    nb2 = 1 if dims[2] == 1 else (dims[2] - 1 + A - 1) // A
    t0, rem = divmod(gid, nb1 * nb2)
    if not sh["t_lo"] <= t0 < sh["t_hi"]:
        raise ValueError("block %d is not in shard %d" % (gid, sh["k"]))
    return (t0 - sh["t_lo"]) * nb1 * nb2 + rem


def compress_in_sequence(x, eb: float, A: int, parts: int, levels, mode: str = "rel"):
    """Compress the 3D device field x shard by shard on one GPU, as separate
    ranks would, and merge: returns dict(codes, anchors, out_idx, out_val,
    hist, eps, eb_f, ebx2_f, r_f) of the whole field (outliers in shard
    order).  `levels` fixes the per-level configuration (the auto-tuner's
    choice needs the global sample blocks; see sample_blocks)."""
    import torch

    from . import hi

    n0, n1, n2 = x.shape
    plan = shard_bounds(n0, A, parts)
    # global range: each shard's own planes through the library's range stage
    vmin, vmax = math.inf, -math.inf
    if mode == "rel":
        for sh in plan:
            xs = x[sh["own_lo"]:sh["own_hi"]].contiguous()
            if not bool(torch.isfinite(xs).any()):
                continue  # no finite value: nothing to add to the range
            c = hi.compress(xs, eb, "rel", A, autotune=False, levels=levels, out_cap=xs.numel())
            vmin, vmax = min(vmin, float(c.h.vmin)), max(vmax, float(c.h.vmax))
    if vmin > vmax:
        vmin = vmax = 0.0
    eps = hi.resolve_eps(mode, eb, vmin, vmax)["eps"]
    codes, anchors, oidx, oval = [], [], [], []
    hist = torch.zeros(256, dtype=torch.int64, device=x.device)
    cst = None
    for sh in plan:
        xs = x[sh["own_lo"]:sh["read_hi"]].contiguous()
        c = hi.compress(xs, eps, "abs", A, autotune=False, levels=levels, out_cap=xs.numel())
        cst = c.h
        nown = sh["own_hi"] - sh["own_lo"]
        cd = c.codes
        codes.append(cd[:nown])
        ash = ((xs.shape[0] - 1) // A + 1, (n1 - 1) // A + 1, (n2 - 1) // A + 1)
        an = c.anchors.view(ash)
        anchors.append(an if sh["last"] else an[:-1])
        idx, val = c.outliers
        idx = idx.to(torch.int64)
        keep = idx < nown * n1 * n2
        oidx.append(idx[keep] + sh["own_lo"] * n1 * n2)
        oval.append(val[keep])
        h = c.hist.to(torch.int64)
        if not sh["last"]:  # take off the read-only plane's non-anchor codes
            top = cd[nown].reshape(-1).to(torch.int64)
            amask = torch.zeros((n1, n2), dtype=torch.bool, device=x.device)
            amask[::A, ::A] = True
            top = top[~amask.reshape(-1)]
            h = h - torch.bincount(top, minlength=256)
        hist += h
    return dict(codes=torch.cat(codes, 0), anchors=torch.cat(anchors, 0).reshape(-1),
                out_idx=torch.cat(oidx), out_val=torch.cat(oval), hist=hist, eps=eps,
                eb_f=cst.eb_f, ebx2_f=cst.ebx2_f, r_f=cst.r_f, vmin=vmin, vmax=vmax)


def compress_out_of_core(x_host, eb: float, A: int, levels, mode: str = "rel", shard_blocks: int = 8,
                         device=None):
    """Compress a 3D float32 field held in host memory (a CPU tensor; pinned
    memory lets the copies overlap the kernels) on one GPU, a shard of
    ``shard_blocks`` block planes along d0 (plus the next shard's first
    plane) at a time: the device holds two shards, never the field.  The
    shards' value ranges (hi_value_range) give the field's eps first; then
    each shard is compressed at that absolute bound while the next one is
    uploaded.  Returns host arrays equal to a whole-field compression with
    the same level configuration: dict(codes, anchors, out_idx, out_val,
    hist, eps, eb_f, ebx2_f, r_f, vmin, vmax)."""
    import numpy as np
    import torch

    from . import hi

    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    n0, n1, n2 = (int(v) for v in x_host.shape)
    plane = n1 * n2
    nb0 = 1 if n0 == 1 else (n0 - 1 + A - 1) // A
    plan = shard_bounds(n0, A, max(1, -(-nb0 // max(1, shard_blocks))))
    max_planes = max(sh["read_hi"] - sh["own_lo"] for sh in plan)
    comp = torch.cuda.current_stream(dev)
    copy = torch.cuda.Stream(dev)
    bufs = [torch.empty(max_planes * plane, dtype=torch.float32, device=dev) for _ in range(2)]
    ready = [torch.cuda.Event() for _ in range(2)]
    free = [torch.cuda.Event() for _ in range(2)]
    for e in free:
        e.record(comp)
    flat = x_host.reshape(-1)

    def upload(i, lo, hi_):
        k = i % 2
        copy.wait_event(free[k])
        with torch.cuda.stream(copy):
            n = (hi_ - lo) * plane
            bufs[k][:n].copy_(flat[lo * plane:hi_ * plane], non_blocking=True)
            ready[k].record(copy)
        return bufs[k][:n].view(hi_ - lo, n1, n2)

    # pass 1: the field's value range from the shards' own planes
    vmin, vmax = math.inf, -math.inf
    if mode == "rel":
        ws = torch.empty(hi.RANGE_WS_BYTES, dtype=torch.uint8, device=dev)
        parts = []
        nxt = upload(0, plan[0]["own_lo"], plan[0]["own_hi"])
        for i, sh in enumerate(plan):
            xs = nxt
            comp.wait_event(ready[i % 2])
            p = hi.make_params(tuple(xs.shape), eb, "rel", A, autotune=False, levels=levels)
            hdr = torch.empty(hi.HEADER_BYTES, dtype=torch.uint8, device=dev)
            hi.value_range_into(xs, p, hdr, ws)
            parts.append((hdr, torch.isfinite(xs).any()))  # a shard without finite values adds nothing
            free[i % 2].record(comp)
            if i + 1 < len(plan):
                nxt = upload(i + 1, plan[i + 1]["own_lo"], plan[i + 1]["own_hi"])
        for hdr, fin in parts:
            if bool(fin.item()):
                h = hi.read_header(hdr)
                vmin, vmax = min(vmin, float(h.vmin)), max(vmax, float(h.vmax))
        if vmin > vmax:
            vmin = vmax = 0.0
    eps = hi.resolve_eps(mode, eb, vmin, vmax)["eps"]

    # pass 2: each shard with its halo plane at the absolute bound eps
    codes = np.empty(n0 * plane, dtype=np.uint8)
    anchors, oidx, oval = [], [], []
    hist = np.zeros(256, dtype=np.int64)
    amask = torch.zeros((n1, n2), dtype=torch.bool, device=dev)
    amask[::A, ::A] = True
    cst = None
    nxt = upload(0, plan[0]["own_lo"], plan[0]["read_hi"])
    for i, sh in enumerate(plan):
        xs = nxt
        comp.wait_event(ready[i % 2])
        p = hi.make_params(tuple(xs.shape), eps, "abs", A, autotune=False, levels=levels)
        cap = max(1024, xs.numel() // 16)
        b = hi.alloc(p, tuple(xs.shape), dev, out_cap=cap, hist=True, recon=False)
        hi.compress_into(xs, b)
        h = hi.read_header(b.header)  # also orders the results before the next upload reuses the buffer
        if h.status == hi.HI_ECAPACITY:  # more outliers than the first guess: once more with the count
            b = hi.alloc(p, tuple(xs.shape), dev, out_cap=int(h.n_outliers), hist=True, recon=False)
            hi.compress_into(xs, b)
            h = hi.read_header(b.header)
        if h.status != 0:
            raise hi.HiError(h.status, "shard %d" % sh["k"])
        free[i % 2].record(comp)
        if i + 1 < len(plan):
            nxt = upload(i + 1, plan[i + 1]["own_lo"], plan[i + 1]["read_hi"])
        cst = h
        nown = sh["own_hi"] - sh["own_lo"]
        codes[sh["own_lo"] * plane:sh["own_hi"] * plane] = b.codes[:nown * plane].cpu().numpy()
        ash = ((xs.shape[0] - 1) // A + 1, (n1 - 1) // A + 1, (n2 - 1) // A + 1)
        an = b.anchors[:int(np.prod(ash))].view(ash)
        anchors.append((an if sh["last"] else an[:-1]).cpu().numpy())
        k = int(h.n_outliers)
        idx = b.out_idx[:k].to(torch.int64) & 0xFFFFFFFF
        keep = idx < nown * plane
        oidx.append((idx[keep] + sh["own_lo"] * plane).cpu().numpy())
        oval.append(b.out_val[:k][keep].cpu().numpy())
        hs = b.hist.to(torch.int64)
        if not sh["last"]:  # the halo plane's non-anchor codes belong to the next shard
            top = b.codes[nown * plane:(nown + 1) * plane].view(n1, n2).to(torch.int64)
            hs = hs - torch.bincount(top[~amask], minlength=256)
        hist += hs.cpu().numpy()
    torch.cuda.current_stream(dev).synchronize()
    return dict(codes=codes.reshape(n0, n1, n2), anchors=np.concatenate(anchors, 0).reshape(-1),
                out_idx=np.concatenate(oidx), out_val=np.concatenate(oval), hist=hist, eps=eps,
                eb_f=cst.eb_f, ebx2_f=cst.ebx2_f, r_f=cst.r_f, vmin=vmin, vmax=vmax)

