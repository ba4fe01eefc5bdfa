"""Batched compression (many fields, one launch per stage): every field's
results equal those of a single-field compression of it, bit for bit, under
every launch shape, and when the batch is replayed from a captured CUDA
graph.  Two fields are also checked against the oracle directly."""
import numpy as np
import pytest
import torch

from paper_2507_11165_gb300 import fields
from tests.test_gpu_parity import check_against_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_11165_gb300 import hi as hi_mod
    hi_mod.lib()
    return hi_mod


# shape, eb, mode: spans full and ragged tiles, 1D/2D fields, a fastest dim
# that is not a multiple of 4 (plain loads instead of TMA), the absolute
# bound, a constant field and a bound tight enough for many outliers
MIX16 = [
    ((37, 45, 70), 1e-3, "rel"), ((64, 64, 64), 1e-2, "abs"), ((33, 33, 33), 1e-4, "rel"),
    ((20, 300), 1e-3, "rel"), ((1000,), 1e-3, "rel"), ((17, 17, 17), 1e-3, "rel"),
    ((50, 47, 63), 1e-3, "rel"), ((40, 40, 40), 1e-3, "rel"), ((48, 40, 52), 1e-6, "rel"),
    ((100, 20, 16), 1e-3, "rel"), ((1, 129, 64), 1e-4, "rel"), ((81, 97, 112), 1e-3, "rel"),
]


def _mk(shape, seed):
    if len(shape) == 3 and min(shape) >= 8:
        return fields.lognormal_grf(shape, seed=seed) if seed % 2 else fields.bumps_field(shape, seed=seed)
    return fields.bumps_field(shape, seed=seed)


def _inputs(mix, seed0=0):
    xs = []
    for i, (shape, eb, mode) in enumerate(mix):
        x = _mk(shape, seed0 + i)
        if shape == (40, 40, 40):
            x[:] = 2.5  # constant field
        xs.append(torch.from_numpy(x).cuda())
    return xs


def _single(hi, x, eb, mode, A, autotune, cap):
    p = hi.make_params(x.shape, eb, mode, A, autotune)
    b = hi.alloc(p, x.shape, "cuda", out_cap=cap, hist=True, recon=True)
    hi.compress_into(x, b)
    return b


def _same(hi, a, b):
    ha, hb = hi.read_header(a.header), hi.read_header(b.header)
    assert bytes(ha) == bytes(hb)
    assert torch.equal(a.codes, b.codes)
    assert torch.equal(a.anchors, b.anchors)
    assert torch.equal(a.hist, b.hist)
    assert torch.equal(a.recon.view(torch.int32), b.recon.view(torch.int32))
    n = min(int(ha.n_outliers), a.out_cap)
    ia, ib = a.out_idx[:n].cpu().numpy(), b.out_idx[:n].cpu().numpy()
    va, vb = a.out_val[:n].cpu().numpy(), b.out_val[:n].cpu().numpy()
    oa, ob = np.argsort(ia, kind="stable"), np.argsort(ib, kind="stable")
    assert np.array_equal(ia[oa], ib[ob])
    assert np.array_equal(va[oa].view(np.uint32), vb[ob].view(np.uint32))
    return ha


def _batch_vs_single(hi, mix, A, autotune, xs=None):
    xs = _inputs(mix) if xs is None else xs
    caps = [x.numel() for x in xs]
    bat = hi.Batch(xs, [m[1] for m in mix], [m[2] for m in mix], anchor_stride=A, autotune=autotune,
                   out_caps=caps, recon=True)
    bat.compress()
    torch.cuda.synchronize()
    singles = [_single(hi, x, m[1], m[2], A, autotune, caps[i]) for i, (x, m) in enumerate(zip(xs, mix))]
    torch.cuda.synchronize()
    for s, b in zip(singles, bat.buffers):
        h = _same(hi, s, b)
        assert h.status == 0
    return bat, singles, xs


def test_batch_equals_single_A16(hi):
    bat, singles, xs = _batch_vs_single(hi, MIX16, 16, True)
    assert bat.plan.total_samples > 0 and bat.plan.total_chunks > 0
    assert bat.plan.all_tma == 0  # fields whose fastest dim is not a multiple of 4 use plain loads
    assert int(hi.read_header(bat.buffers[8].header).n_outliers) > 1000


def test_batch_equals_single_A8_fixed_levels(hi):
    mix = [((64, 64, 64), 1e-3, "rel"), ((30, 41, 52), 1e-4, "rel"), ((9, 9, 9), 1e-3, "abs"),
           ((200, 72), 1e-3, "rel"), ((45, 23, 88), 1e-2, "rel")]
    _batch_vs_single(hi, mix, 8, False)


def test_batch_equals_single_multidimensional(hi):
    """Auto-tune over the 1D sequences and the multi-dimensional scheme
    (autotune = 2): the batched kernel runs the same levels per field."""
    mix = [((37, 45, 70), 1e-3, "rel"), ((64, 64, 64), 1e-3, "rel"), ((33, 33, 33), 1e-4, "rel"),
           ((20, 300), 1e-3, "rel"), ((81, 97, 112), 1e-3, "rel"), ((50, 47, 63), 1e-2, "rel")]
    bat, singles, xs = _batch_vs_single(hi, mix, 16, 2)
    picked = set()
    for b in bat.buffers:
        h = hi.read_header(b.header)
        picked |= {int(h.level[l].interp) for l in range(4)}
    assert picked & {hi.MD_LINEAR, hi.MD_CUBIC}  # the scheme was chosen somewhere


def test_batch_against_oracle(oracle_mod, hi):
    mix = [((37, 45, 70), 1e-3, "rel"), ((33, 33, 33), 1e-4, "rel")]
    xs = _inputs(mix, seed0=20)
    bat = hi.Batch(xs, [1e-3, 1e-4], "rel", anchor_stride=16, autotune=True, out_caps=[x.numel() for x in xs],
                   recon=True)
    bat.compress()
    for x, b in zip(xs, bat.buffers):
        h = hi.read_header(b.header)
        interp = np.array([h.level[l].interp for l in range(4)], dtype=np.uint8)
        order = np.array([tuple(h.level[l].order) for l in range(4)], dtype=np.uint8)
        check_against_oracle(oracle_mod, hi, x.cpu().numpy(), 16, h.eb, 1, interp, order, b, h)


def test_launch_shapes_give_identical_results(hi):
    mix = [m for m in MIX16 if m[0][-1] % 4 == 0]  # every field staged by TMA: all four shapes apply
    xs = _inputs(mix, seed0=40)
    bat = hi.Batch(xs, [m[1] for m in mix], [m[2] for m in mix], anchor_stride=16, autotune=True,
                   out_caps=[x.numel() for x in xs], recon=True)
    assert bat.plan.all_tma == 1
    ref = None
    for th, bu in hi.BATCH_SHAPES:
        bat.set_shape(th, bu)
        for b in bat.buffers:  # stale outputs must not survive
            b.codes.fill_(7)
            b.recon.fill_(-1.0)
        bat.compress()
        torch.cuda.synchronize()
        snap = [(b.codes.clone(), b.recon.clone(), b.hist.clone(), b.anchors.clone(), bytes(hi.read_header(b.header)))
                for b in bat.buffers]
        if ref is None:
            ref = snap
            continue
        for r, s in zip(ref, snap):
            for a, c in zip(r[:4], s[:4]):
                assert torch.equal(a, c)
            assert r[4] == s[4]
    times = bat.tune_launch(reps=2)
    assert len(times) == 4 and bat.shape in times


def test_batch_graph_replay(hi):
    mix = MIX16[:6]
    xs = _inputs(mix, seed0=60)
    caps = [x.numel() for x in xs]
    bat = hi.Batch(xs, [m[1] for m in mix], [m[2] for m in mix], anchor_stride=16, autotune=True, out_caps=caps,
                   recon=True)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        bat.compress()  # first launch outside the capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bat.compress()
    for rep in range(2):  # new data in the same buffers, then replay
        new = _inputs(mix, seed0=80 + 10 * rep)
        for x, y in zip(xs, new):
            x.copy_(y)
        g.replay()
        torch.cuda.synchronize()
        for i, (x, m) in enumerate(zip(xs, mix)):
            _same(hi, _single(hi, x, m[1], m[2], 16, True, caps[i]), bat.buffers[i])


def test_batch_workload_sample(hi):
    """32 fields of the 256-field workload recipe (sides log-uniform in [32, 256])."""
    specs, arrs = fields.batch_fields(32, seed=4)
    xs = [torch.from_numpy(a).cuda() for a in arrs]
    mix = [(s["shape"], s["eb"], "rel") for s in specs]
    _batch_vs_single(hi, mix, 16, True, xs=xs)


def _decompress_single(hi, b, shape):
    out = torch.empty(shape, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    hi.decompress_into(b, out, st)
    torch.cuda.synchronize()
    return out, int(st.item())


@pytest.mark.parametrize("A", [16, 8])
def test_batched_decompress_equals_single(hi, A):
    """hi_decompress_batch of a batch (1D/2D/3D, ragged and whole tiles,
    plain loads, a constant field, many outliers) gives every field the
    output of hi_decompress of it alone, bit for bit, and the compressor's
    own reconstruction."""
    xs = _inputs(MIX16)
    caps = [x.numel() for x in xs]
    bat = hi.Batch(xs, [m[1] for m in MIX16], [m[2] for m in MIX16], anchor_stride=A, autotune=A == 16,
                   levels=None if A == 16 else (hi.CUBIC, (0, 1, 2)), out_caps=caps, recon=True, outs=True)
    bat.compress()
    bat.decompress()
    torch.cuda.synchronize()
    assert int(bat.dstatus.item()) == 0
    for x, b, y in zip(xs, bat.buffers, bat.outs):
        ref, st = _decompress_single(hi, b, x.shape)
        assert st == 0
        assert torch.equal(y.view(torch.int32), ref.view(torch.int32))
        assert torch.equal(y.reshape(-1).view(torch.int32), b.recon.reshape(-1).view(torch.int32))


def test_batched_decompress_against_oracle(oracle_mod, hi):
    """Two fields of a batch reconstructed by hi_decompress_batch against the
    oracle's decompression of the batch's own records."""
    mix = [((37, 45, 70), 1e-3, "rel"), ((33, 33, 33), 1e-4, "rel")]
    xs = _inputs(mix)
    bat = hi.Batch(xs, [m[1] for m in mix], "rel", anchor_stride=16, autotune=True, out_caps=[x.numel() for x in xs],
                   outs=True)
    bat.compress()
    bat.decompress()
    torch.cuda.synchronize()
    for x, b, y in zip(xs, bat.buffers, bat.outs):
        h = hi.read_header(b.header)
        L = int(h.n_levels)
        interp = np.array([h.level[l].interp for l in range(L)], dtype=np.uint8)
        order = np.array([list(h.level[l].order) for l in range(L)], dtype=np.uint8)
        k = int(h.n_outliers)
        ref = oracle_mod.decompress(tuple(x.shape), 16, interp, order, float(h.ebx2_f), b.codes.cpu().numpy(),
                                    b.anchors[: int(h.n_anchors)].cpu().numpy(), b.out_idx[:k].cpu().numpy(),
                                    b.out_val[:k].cpu().numpy())
        assert np.array_equal(y.cpu().numpy().view(np.uint32), ref.view(np.uint32))


def test_batched_decompress_graph_replay_and_capacity(hi):
    """The reconstruction replayed from a captured CUDA graph follows new
    records; a field whose outliers overflow its capacity is left unwritten
    and reports HI_ECAPACITY while the others are reconstructed."""
    mix = [((40, 44, 48), 1e-3, "rel"), ((30, 31, 32), 1e-7, "rel"), ((64, 64, 64), 1e-3, "rel")]
    xs = _inputs(mix, seed0=7)
    caps = [xs[0].numel(), 64, xs[2].numel()]  # the tight bound overflows 64 slots
    bat = hi.Batch(xs, [m[1] for m in mix], "rel", anchor_stride=16, autotune=True, out_caps=caps, outs=True)
    for y in bat.outs:
        y.fill_(-7.0)
    bat.compress()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bat.decompress()
    g.replay()
    torch.cuda.synchronize()
    assert int(bat.dstatus.item()) == hi.HI_ECAPACITY
    assert bool((bat.outs[1] == -7.0).all())
    for i in (0, 2):
        ref, st = _decompress_single(hi, bat.buffers[i], xs[i].shape)
        assert st == 0 and torch.equal(bat.outs[i].view(torch.int32), ref.view(torch.int32))
    # new inputs, recompress, replay the captured reconstruction
    for i in (0, 2):
        xs[i].copy_(torch.from_numpy(fields.lognormal_grf(tuple(xs[i].shape), seed=40 + i)).cuda())
    bat.compress()
    g.replay()
    torch.cuda.synchronize()
    for i in (0, 2):
        ref, st = _decompress_single(hi, bat.buffers[i], xs[i].shape)
        assert st == 0 and torch.equal(bat.outs[i].view(torch.int32), ref.view(torch.int32))
        h = hi.read_header(bat.buffers[i].header)
        assert float((bat.outs[i] - xs[i]).abs().max()) < h.eps
