"""One field split along d0 over two gloo ranks (CPU), each driving the
oracle on its blocks: the exchanged range, auto-tune errors and outliers
reproduce the single-field record bit for bit.  Plus the shard layout."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2507_11165_gb300 import fields, hi, shard

SHAPE = (101, 80, 80)  # 13 blocks along d0 at A = 8, the last one ragged; 3 auto-tune samples
A = 8
EB = 1e-4


def test_shard_bounds_cover_the_field():
    for n0, A_, parts in [(101, 8, 2), (101, 8, 3), (17, 16, 4), (513, 16, 8), (1, 8, 2), (9, 8, 1)]:
        b = shard.shard_bounds(n0, A_, parts)
        assert b[0]["own_lo"] == 0 and b[-1]["own_hi"] == n0
        for a, c in zip(b, b[1:]):
            assert a["own_hi"] == c["own_lo"] and a["t_hi"] == c["t_lo"]
            assert a["read_hi"] == a["own_hi"] + 1  # the next shard's first plane, read only
            assert a["own_lo"] % A_ == 0 and a["own_hi"] % A_ == 0
        sizes = [s["t_hi"] - s["t_lo"] for s in b]
        assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _owned(sh, x, ref, col, n1, n2):
    nown = sh["own_hi"] - sh["own_lo"]
    codes = ref["codes"][:nown]
    ash = ((ref["codes"].shape[0] - 1) // A + 1, (n1 - 1) // A + 1, (n2 - 1) // A + 1)
    an = ref["anchors"].reshape(ash)
    an = an if sh["last"] else an[:-1]
    keep = col["out_idx"] < nown * n1 * n2
    idx = col["out_idx"][keep].astype(np.int64) + sh["own_lo"] * n1 * n2
    val = col["out_val"][keep]
    hist = col["hist"].astype(np.int64)
    if not sh["last"]:  # the read-only plane's non-anchor codes are the next shard's
        top = ref["codes"][nown].copy()
        mask = np.ones((n1, n2), dtype=bool)
        mask[::A, ::A] = False
        hist -= np.bincount(top[mask].reshape(-1), minlength=256)
    return codes, an, idx, val, hist


def _worker(rank, world, port, outdir):
    import oracle

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    x = fields.lognormal_grf(SHAPE, seed=21)  # every rank makes the same field and keeps its planes
    n1, n2 = SHAPE[1], SHAPE[2]
    sh = shard.shard_bounds(SHAPE[0], A, world)[rank]
    xs = np.ascontiguousarray(x[sh["own_lo"]:sh["read_hi"]])
    own = x[sh["own_lo"]:sh["own_hi"]]
    fin = own[np.isfinite(own)]
    mn = torch.tensor([float(fin.min())], dtype=torch.float64)
    mx = torch.tensor([float(fin.max())], dtype=torch.float64)
    dist.all_reduce(mn, op=dist.ReduceOp.MIN)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    cst = oracle.eps_constants(np.array([mn.item(), mx.item()], dtype=np.float32), 1, EB)
    assert cst["eps"] == hi.resolve_eps("rel", EB, mn.item(), mx.item())["eps"]
    # auto-tune: the errors of the global sample blocks this rank holds, then
    # every sample's errors on every rank, summed in global sample order
    gids = shard.sample_blocks(SHAPE, A)
    nb12 = ((n1 - 1 + A - 1) // A) * ((n2 - 1 + A - 1) // A)
    mine = [k for k, g in enumerate(gids) if sh["t_lo"] <= g // nb12 < sh["t_hi"]]
    L = oracle.n_levels(A)
    nc = len(oracle.tune_configs(SHAPE))
    full = torch.zeros((len(gids), L, nc), dtype=torch.float64)
    if mine:
        e = oracle.tune_errors_tiles(xs, A, [shard.local_block(gids[k], SHAPE, A, sh) for k in mine])
        for j, k in enumerate(mine):
            full[k] = torch.from_numpy(e[j])
    dist.all_reduce(full, op=dist.ReduceOp.SUM)  # each sample's row is non-zero on one rank only
    tot = torch.zeros((L, nc), dtype=torch.float64)
    for k in range(len(gids)):
        tot = tot + full[k]
    interp, order = oracle.tune_select(SHAPE, A, tot.numpy())
    ref = oracle.compress(xs, A, interp, order, cst)
    col = oracle.collect(xs, ref["codes"], A)
    part = _owned(sh, x, ref, col, n1, n2)
    parts = [None] * world
    dist.all_gather_object(parts, (part, interp, order, len(mine)))
    if rank == 0:
        codes = np.concatenate([p[0][0] for p in parts], 0)
        anchors = np.concatenate([p[0][1] for p in parts], 0).reshape(-1)
        idx = np.concatenate([p[0][2] for p in parts])
        val = np.concatenate([p[0][3] for p in parts])
        hist = sum(p[0][4] for p in parts)
        np.savez(os.path.join(outdir, "merged.npz"), codes=codes, anchors=anchors, idx=idx, val=val, hist=hist,
                 interp=interp, order=order, held=np.array([p[3] for p in parts]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_reproduce_the_single_field_record(oracle_mod, tmp_path):
    mp.start_processes(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, start_method="spawn")
    m = np.load(os.path.join(str(tmp_path), "merged.npz"))
    x = fields.lognormal_grf(SHAPE, seed=21)
    cst = oracle_mod.eps_constants(x, 1, EB)
    err = oracle_mod.tune_errors(x, A)
    interp, order = oracle_mod.tune_select(SHAPE, A, err)
    ref = oracle_mod.compress(x, A, interp, order, cst)
    col = oracle_mod.collect(x, ref["codes"], A)
    assert len(shard.sample_blocks(SHAPE, A)) == oracle_mod.tune_samples(SHAPE, A) >= 2
    assert all(h >= 1 for h in m["held"])  # both ranks held sample blocks
    assert np.array_equal(m["interp"], interp) and np.array_equal(m["order"], order)
    assert np.array_equal(m["codes"], ref["codes"])
    assert np.array_equal(m["anchors"].view(np.uint32), ref["anchors"].view(np.uint32))
    o = np.argsort(m["idx"])
    assert np.array_equal(m["idx"][o], col["out_idx"].astype(np.int64))
    assert np.array_equal(m["val"][o].view(np.uint32), col["out_val"].view(np.uint32))
    assert np.array_equal(m["hist"], col["hist"].astype(np.int64))
    assert col["n_out"] > 0
