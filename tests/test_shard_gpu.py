"""One GPU compressing a field shard by shard (as separate ranks would, each
with the global bound) and merging: the same record as compressing the
field whole."""
import os

import numpy as np
import pytest
import torch

from paper_2507_11165_gb300 import fields, shard

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_11165_gb300 import hi as hi_mod
    hi_mod.lib()
    return hi_mod


@pytest.mark.parametrize("shape,A,parts,eb", [((150, 64, 72), 16, 3, 1e-3), ((101, 40, 36), 8, 2, 1e-5),
                                              ((33, 20, 48), 16, 2, 1e-4)])
def test_shards_in_sequence_equal_the_whole_field(hi, shape, A, parts, eb):
    x = torch.from_numpy(fields.lognormal_grf(shape, seed=31)).cuda()
    L = A.bit_length() - 1
    levels = [(1 if l % 2 == 0 else 0, (0, 1, 2) if l % 3 else (2, 0, 1)) for l in range(L)]
    m = shard.compress_in_sequence(x, eb, A, parts, levels)
    c = hi.compress(x, eb, "rel", A, autotune=False, levels=levels, out_cap=x.numel())
    assert m["eps"] == c.h.eps
    assert np.float32(m["eb_f"]) == np.float32(c.h.eb_f) and np.float32(m["r_f"]) == np.float32(c.h.r_f)
    assert torch.equal(m["codes"], c.codes)
    assert torch.equal(m["anchors"].view(torch.int32), c.anchors.view(torch.int32))
    idx, val = c.outliers
    oa, ob = torch.argsort(m["out_idx"]), torch.argsort(idx.to(torch.int64))
    assert torch.equal(m["out_idx"][oa], idx.to(torch.int64)[ob])
    assert torch.equal(m["out_val"][oa].view(torch.int32), val[ob].view(torch.int32))
    assert torch.equal(m["hist"], c.hist.to(torch.int64))
    if eb <= 1e-5:
        assert c.n_outliers > 0


@pytest.mark.parametrize("shape,A,blocks,eb,mode,nan_slab", [((150, 64, 72), 16, 2, 1e-3, "rel", True),
                                                             ((101, 40, 36), 8, 3, 1e-5, "rel", False),
                                                             ((70, 33, 52), 16, 1, 1e-3, "abs", False),
                                                             ((40, 17, 20), 16, 8, 1e-3, "rel", False)])
def test_out_of_core_equals_the_whole_field(hi, shape, A, blocks, eb, mode, nan_slab):
    """A host-resident field compressed two shards at a time on the device
    (value ranges first, then each shard with its halo plane at the field's
    eps) gives the whole-field record; a shard with no finite value at all
    leaves the range alone and re-runs with the exact outlier count."""
    xn = fields.lognormal_grf(shape, seed=32)
    xn[5, 3, 7] = np.inf
    xn[-1, -2, -3] = np.nan
    if nan_slab:
        xn[:blocks * A] = np.nan
    L = A.bit_length() - 1
    levels = [(l % 2, (2, 1, 0) if l % 2 else (0, 2, 1)) for l in range(L)]
    m = shard.compress_out_of_core(torch.from_numpy(xn).pin_memory(), eb, A, levels, mode=mode, shard_blocks=blocks)
    c = hi.compress(torch.from_numpy(xn).cuda(), eb, mode, A, autotune=False, levels=levels, out_cap=xn.size)
    assert c.h.status == 0
    assert m["eps"] == c.h.eps
    assert np.float32(m["eb_f"]) == np.float32(c.h.eb_f) and np.float32(m["r_f"]) == np.float32(c.h.r_f)
    assert np.array_equal(m["codes"], c.codes.cpu().numpy().reshape(shape))
    assert np.array_equal(m["anchors"].view(np.uint32), c.anchors.cpu().numpy().view(np.uint32))
    idx, val = c.outliers
    idx = idx.cpu().numpy().view(np.uint32).astype(np.int64)
    val = val.cpu().numpy()
    oa, ob = np.argsort(m["out_idx"]), np.argsort(idx)
    assert np.array_equal(m["out_idx"][oa], idx[ob])
    assert np.array_equal(m["out_val"][oa].view(np.uint32), val[ob].view(np.uint32))
    assert np.array_equal(m["hist"], c.hist.cpu().numpy().view(np.uint32).astype(np.int64))


@pytest.mark.parametrize("shape", [(64, 48, 40), (1, 1, 1000), (7, 300)])
def test_value_range_matches_oracle(hi, oracle_mod, shape):
    """hi_value_range: the min and max over the finite values and the
    constants derived from them, as the oracle derives them (Eq. 1,
    relative bound); an all-non-finite part reports 0 and 0."""
    xn = fields.lognormal_grf(shape, seed=41)
    flat = xn.reshape(-1)
    flat[::97] = np.nan
    flat[5] = -np.inf
    flat[11] = np.inf
    x = torch.from_numpy(xn).cuda()
    p = hi.make_params(shape, 1e-3, "rel", 16, autotune=False)
    ws = torch.empty(hi.RANGE_WS_BYTES, dtype=torch.uint8, device="cuda")
    hdr = torch.empty(hi.HEADER_BYTES, dtype=torch.uint8, device="cuda")
    hi.value_range_into(x, p, hdr, ws)
    h = hi.read_header(hdr)
    fin = flat[np.isfinite(flat)]
    assert np.float32(h.vmin) == fin.min() and np.float32(h.vmax) == fin.max()
    cst = oracle_mod.eps_constants(xn, 1, 1e-3)
    assert h.eps == cst["eps"]
    assert np.float32(h.eb_f) == cst["eb_f"] and np.float32(h.ebx2_f) == cst["ebx2_f"]
    assert np.float32(h.r_f) == cst["r_f"]
    hi.value_range_into(torch.full(shape, float("nan"), device="cuda"), p, hdr, ws)
    h = hi.read_header(hdr)
    assert float(h.vmin) == 0.0 and float(h.vmax) == 0.0
    small = torch.empty(hi.RANGE_WS_BYTES - 8, dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError):
        hi.value_range_into(x, p, hdr, small)


def _dist_worker(rank, world, port, outdir):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2507_11165_gb300 import fields, shard
    torch.cuda.set_device(0)  # both ranks on one GPU: their kernels never wait on each other
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    shape = (101, 80, 72)
    x = fields.lognormal_grf(shape, seed=23)
    sh = shard.shard_bounds(shape[0], 16, world)[rank]
    xl = torch.from_numpy(np.ascontiguousarray(x[sh["own_lo"]:sh["read_hi"]])).cuda()
    part = shard.compress_distributed(xl, shape, 1e-3, 16, shard.GpuShardExecutor())
    part = {k: (v.cpu() if torch.is_tensor(v) else v) for k, v in part.items()}
    parts = [None] * world
    dist.all_gather_object(parts, part)
    if rank == 0:
        m = shard.merge_parts(parts)
        torch.save(m, os.path.join(outdir, "merged.pt"))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.gpu
def test_distributed_ranks_reproduce_hi_compress(tmp_path):
    import socket

    import numpy as np
    import torch
    import torch.multiprocessing as mp

    from paper_2507_11165_gb300 import fields, hi
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_dist_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    m = torch.load(os.path.join(str(tmp_path), "merged.pt"))
    x = torch.from_numpy(fields.lognormal_grf((101, 80, 72), seed=23)).cuda()
    c = hi.compress(x, 1e-3, "rel", 16, autotune=True, out_cap=x.numel())
    levels = [(int(c.h.level[l].interp), tuple(int(v) for v in c.h.level[l].order)) for l in range(c.h.n_levels)]
    assert m["levels"] == levels
    assert m["eps"] == c.h.eps
    assert torch.equal(m["codes"].reshape(-1), c.codes.cpu().reshape(-1))
    assert torch.equal(m["anchors"].reshape(-1).view(torch.int32), c.anchors.cpu().reshape(-1).view(torch.int32))
    idx, val = c.outliers
    o1, o2 = torch.argsort(m["out_idx"]), torch.argsort(idx.cpu().to(torch.int64))
    assert torch.equal(m["out_idx"][o1], idx.cpu().to(torch.int64)[o2])
    assert torch.equal(m["out_val"][o1].view(torch.int32), val.cpu()[o2].view(torch.int32))
    assert torch.equal(m["hist"], c.hist.cpu().to(torch.int64))
    assert len(idx) > 0
