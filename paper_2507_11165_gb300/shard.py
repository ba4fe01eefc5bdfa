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



# ---------------------------------------------------------------------------
# One field over several ranks (torch.distributed): each rank holds the read
# planes of its shard and compresses them; only the three exchanges of the
# module docstring cross ranks.
# ---------------------------------------------------------------------------
def _coll_device(group):
    import torch
    import torch.distributed as dist
    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else \
        torch.device("cpu")


def compress_distributed(x_local, shape, eb: float, A: int, executor, group=None, mode: str = "rel",
                         autotune: bool = True, levels=None, md: bool = False):
    """Compress one 3D field split over the ranks of ``group`` along d0
    (shard_bounds(shape[0], A, world), shard k on rank k); ``x_local`` is
    this rank's read planes [own_lo, read_hi) (empty on ranks past the last
    shard).  ``executor`` runs the steps on this rank's data (GpuShardExecutor
    for the library; any object with its five methods).  Exchanged: the
    min / max of the finite values (one all-reduce), every sample block's
    auto-tune error row (one all-reduce; each row comes from the one rank
    that holds the block), nothing else.  Returns this rank's part of the
    whole-field record: dict(shard, codes [own planes], anchors [its anchor
    planes], out_idx (global, int64), out_val, hist (of its own non-anchor
    points), levels, eps, vmin, vmax); merge_parts() of all ranks' parts in
    rank order is the single-field record."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from . import hi

    if len(shape) != 3:
        raise ValueError("compress_distributed takes 3D fields")
    n0, n1, n2 = (int(v) for v in shape)
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    plan = shard_bounds(n0, A, world)
    sh = plan[rank] if rank < len(plan) else None
    cdev = _coll_device(group) if world > 1 else torch.device("cpu")
    if sh is not None and tuple(x_local.shape) != (sh["read_hi"] - sh["own_lo"], n1, n2):
        raise ValueError("x_local must hold planes [%d, %d)" % (sh["own_lo"], sh["read_hi"]))

    # 1. the field's value range -> eps (Eq. 1, relative bound)
    vmin = vmax = 0.0
    if mode == "rel":
        r = executor.value_range(x_local[: sh["own_hi"] - sh["own_lo"]]) if sh is not None else None
        t = torch.tensor([r[0] if r else math.inf, -r[1] if r else math.inf], dtype=torch.float64, device=cdev)
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
        vmin, vmax = float(t[0]), -float(t[1])
        if vmin > vmax:  # no finite value anywhere
            vmin = vmax = 0.0
    cst = hi.resolve_eps(mode, eb, vmin, vmax)

    # 2. auto-tune over the whole field's sample blocks (Sec. 5.1.3)
    if autotune:
        gids = sample_blocks(shape, A)
        nb12 = ((n1 - 1 + A - 1) // A) * ((n2 - 1 + A - 1) // A)
        mine = [k for k, g in enumerate(gids) if sh is not None and sh["t_lo"] <= g // nb12 < sh["t_hi"]]
        L, nc = executor.tune_dims(shape, A, md)
        full = torch.zeros((len(gids), L, nc), dtype=torch.float64, device=cdev)
        if mine:
            rows = executor.block_errors(x_local, A, [local_block(gids[k], shape, A, sh) for k in mine], md)
            full[mine] = torch.as_tensor(np.asarray(rows, dtype=np.float64), device=cdev)
        if world > 1:
            dist.all_reduce(full, op=dist.ReduceOp.SUM, group=group)  # x + 0 = x: every row exact
        levels = executor.select(shape, A, full.cpu().numpy(), md)
    elif levels is None:
        raise ValueError("levels are needed without autotune")

    out = dict(shard=sh, levels=[(int(i), tuple(int(v) for v in o)) for i, o in levels], eps=cst["eps"],
               vmin=vmin, vmax=vmax)
    if sh is None:
        return out
    # 3. this shard at the field's absolute bound, then its owned part
    part = executor.compress(x_local, cst, A, out["levels"])
    nown = sh["own_hi"] - sh["own_lo"]
    codes = part["codes"].reshape(-1, n1, n2)
    anchors = part["anchors"].reshape(-1, (n1 - 1) // A + 1, (n2 - 1) // A + 1)
    idx = torch.as_tensor(part["out_idx"]).to(torch.int64)
    val = torch.as_tensor(part["out_val"])
    keep = idx < nown * n1 * n2
    hist = torch.as_tensor(part["hist"]).to(torch.int64).clone()
    if not sh["last"]:  # the read-only plane's non-anchor codes belong to the next shard
        top = torch.as_tensor(codes[nown]).to(torch.int64)
        amask = torch.zeros((n1, n2), dtype=torch.bool, device=top.device)
        amask[::A, ::A] = True
        hist -= torch.bincount(top[~amask], minlength=256).to(hist.device)
    out.update(codes=codes[:nown], anchors=anchors if sh["last"] else anchors[:-1],
               out_idx=idx[keep] + sh["own_lo"] * n1 * n2, out_val=val[keep], hist=hist)
    return out


def merge_parts(parts):
    """The whole-field record from the ranks' parts (rank order)."""
    import torch
    parts = [p for p in parts if p.get("shard") is not None]
    cat = lambda k: torch.cat([torch.as_tensor(p[k]).cpu() for p in parts], 0)
    return dict(codes=cat("codes"), anchors=cat("anchors").reshape(-1), out_idx=cat("out_idx"),
                out_val=cat("out_val"), hist=sum(torch.as_tensor(p["hist"]).cpu() for p in parts),
                levels=parts[0]["levels"], eps=parts[0]["eps"])


class GpuShardExecutor:
    """The steps of compress_distributed on this rank's GPU, through the C ABI."""

    def __init__(self, device=None):
        import torch
        self.dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)

    def value_range(self, x_own):
        """(vmin, vmax) of the finite values of the owned planes, or None (hi_value_range)."""
        import torch

        from . import hi
        x_own = x_own.to(self.dev).contiguous()
        if x_own.numel() == 0 or not bool(torch.isfinite(x_own).any()):
            return None
        p = hi.make_params(tuple(x_own.shape), 1e-3, "rel", 16, autotune=False, levels=[(hi.LINEAR, (0, 1, 2))] * 4)
        hdr = torch.empty(hi.HEADER_BYTES, dtype=torch.uint8, device=self.dev)
        ws = torch.empty(max(8, hi.query(p)["ws_bytes"]), dtype=torch.uint8, device=self.dev)
        hi.value_range_into(x_own, p, hdr, ws)
        h = hi.read_header(hdr)
        return float(h.vmin), float(h.vmax)

    def tune_dims(self, shape, A, md):
        from . import hi
        e = hi.autotune_dims(shape, A, md)
        return e[1], e[2]

    def block_errors(self, x_read, A, local_ids, md):
        """Auto-tune error rows [len(local_ids), L, ncfg] of blocks of the read planes: each block as a field of
        its own, whose one sample is the whole block (the same rows the whole field's tuner computes)."""
        import numpy as np

        from . import hi
        x_read = x_read.to(self.dev)
        n = x_read.shape
        nb = [1 if v == 1 else (v - 1 + A - 1) // A for v in n]
        rows = []
        for b in local_ids:
            t0, r = divmod(int(b), nb[1] * nb[2])
            t1, t2 = divmod(r, nb[2])
            blk = x_read[t0 * A: min(t0 * A + A, n[0] - 1) + 1, t1 * A: min(t1 * A + A, n[1] - 1) + 1,
                         t2 * A: min(t2 * A + A, n[2] - 1) + 1].contiguous()
            rows.append(hi.tune_errors(blk, A, md)[0])
        return np.stack(rows)

    def select(self, shape, A, err, md):
        from . import hi
        return hi.autotune_select(shape, A, err, md)

    def compress(self, x_read, cst, A, levels):
        """The read planes at the field's absolute bound: codes, anchors, outliers (local), histogram."""
        from . import hi
        x_read = x_read.to(self.dev).contiguous()
        c = hi.compress(x_read, cst["eps"], "abs", A, autotune=False, levels=levels, out_cap=x_read.numel())
        idx, val = c.outliers
        return dict(codes=c.codes, anchors=c.anchors[: int(c.h.n_anchors)], out_idx=idx, out_val=val, hist=c.hist)
