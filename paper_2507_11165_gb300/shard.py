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


def eps_from_range(eb_mode: str, eb: float, vmin: float, vmax: float) -> float:
    """The absolute bound (Eq. 1): eb, or eb * (vmax - vmin) for the
    value-range-relative bound (eb when the range is 0), in IEEE double as
    the library derives it on the device."""
    if eb_mode == "abs":
        return float(eb)
    r = float(vmax) - float(vmin)
    return float(eb) * r if r > 0.0 else float(eb)


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
    eps = eps_from_range(mode, eb, vmin, vmax)
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
