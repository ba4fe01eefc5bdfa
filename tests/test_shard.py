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


class OracleExecutor:
    """compress_distributed's steps on the CPU oracle (test infrastructure)."""

    def __init__(self):
        import oracle
        self.o = oracle

    def value_range(self, x_own):
        fin = np.asarray(x_own)[np.isfinite(x_own)]
        return (float(fin.min()), float(fin.max())) if fin.size else None

    def tune_dims(self, shape, A_, md):
        return self.o.n_levels(A_), len(self.o.tune_configs(shape))

    def block_errors(self, x_read, A_, ids, md):
        return self.o.tune_errors_tiles(np.ascontiguousarray(x_read), A_, ids)

    def select(self, shape, A_, err, md):
        tot = np.zeros(err.shape[1:], dtype=np.float64)
        for k in range(err.shape[0]):  # samples summed in global order
            tot = tot + err[k]
        interp, order = self.o.tune_select(shape, A_, tot)
        return [(int(i), tuple(int(v) for v in o)) for i, o in zip(interp, order)]

    def compress(self, x_read, cst, A_, levels):
        consts = dict(eb_f=np.float32(cst["eb_f"]), ebx2_f=np.float32(cst["ebx2_f"]), r_f=np.float32(cst["r_f"]),
                      vmin=np.float32(0), vmax=np.float32(0), eps=cst["eps"])
        interp = np.array([l[0] for l in levels], dtype=np.uint8)
        order = np.array([l[1] for l in levels], dtype=np.uint8)
        x = np.ascontiguousarray(x_read)
        ref = self.o.compress(x, A_, interp, order, consts)
        col = self.o.collect(x, ref["codes"], A_)
        return dict(codes=ref["codes"], anchors=ref["anchors"], out_idx=col["out_idx"], out_val=col["out_val"],
                    hist=col["hist"])


def _worker(rank, world, port, outdir):
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    x = fields.lognormal_grf(SHAPE, seed=21)  # every rank makes the same field and keeps its planes
    sh = shard.shard_bounds(SHAPE[0], A, world)[rank]
    part = shard.compress_distributed(np.ascontiguousarray(x[sh["own_lo"]:sh["read_hi"]]), SHAPE, EB, A,
                                      OracleExecutor())
    gids = shard.sample_blocks(SHAPE, A)
    nb12 = ((SHAPE[1] - 1 + A - 1) // A) * ((SHAPE[2] - 1 + A - 1) // A)
    held = sum(sh["t_lo"] <= g // nb12 < sh["t_hi"] for g in gids)
    parts = [None] * world
    dist.all_gather_object(parts, (part, held))
    if rank == 0:
        m = shard.merge_parts([p[0] for p in parts])
        np.savez(os.path.join(outdir, "merged.npz"), codes=m["codes"].numpy(), anchors=m["anchors"].numpy(),
                 idx=m["out_idx"].numpy(), val=m["out_val"].numpy(), hist=m["hist"].numpy(),
                 interp=np.array([l[0] for l in m["levels"]]), order=np.array([l[1] for l in m["levels"]]),
                 held=np.array([p[1] for p in parts]), eps=np.array([p[0]["eps"] for p in parts]))
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
    assert all(e == cst["eps"] for e in m["eps"])
    assert np.array_equal(m["codes"], ref["codes"])
    assert np.array_equal(m["anchors"].view(np.uint32), ref["anchors"].view(np.uint32))
    o = np.argsort(m["idx"])
    assert np.array_equal(m["idx"][o], col["out_idx"].astype(np.int64))
    assert np.array_equal(m["val"][o].view(np.uint32), col["out_val"].view(np.uint32))
    assert np.array_equal(m["hist"], col["hist"].astype(np.int64))
    assert col["n_out"] > 0
