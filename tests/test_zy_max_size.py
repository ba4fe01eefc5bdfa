"""A field past 2^31 points (the library takes N < 2^32; outlier indices are
32-bit): compress, decompress, reorder and the lossless stage at that size,
with the index arithmetic of every kernel exercised above 2^31.

520 x 2048 x 2048 = 2,181,038,080 points (8.7 GB of float32), built on the
device from seeded smooth modes plus noise, with planted spikes before and
beyond index 2^31.  Checks: sampled blocks (all corners, blocks beyond
2^31, random ones) equal the oracle run on each block's own box -- a
block's result depends only on its (A+1)^3 points, extents and the level
configuration; the spikes are outliers at their exact indices with their
exact values; the error bound over the whole field; histogram totals;
decompression; the code reordering and lossless stream roundtrip."""
import numpy as np
import pytest
import torch

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SHAPE = (520, 2048, 2048)
A = 16
EB = 1e-3
SPIKES = [((519, 2047, 2047), 1.0e4), ((515, 100, 5), -3.0e3), ((300, 1000, 777), 2.5e3), ((0, 0, 1), 7.0e2)]


@pytest.fixture(scope="module")
def hi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, _ = torch.cuda.mem_get_info()
    if free < 40 * 2 ** 30:
        pytest.skip("needs 40 GiB of device memory")
    from paper_2507_11165_gb300 import hi as hi_mod
    hi_mod.lib()
    return hi_mod


def _field(dev):
    n0, n1, n2 = SHAPE
    g = torch.Generator(device=dev).manual_seed(11)
    i = torch.arange(n0, device=dev, dtype=torch.float32)[:, None, None]
    j = torch.arange(n1, device=dev, dtype=torch.float32)[None, :, None]
    k = torch.arange(n2, device=dev, dtype=torch.float32)[None, None, :]
    x = torch.sin(0.031 * i + 0.5) * torch.cos(0.017 * j) + 0.6 * torch.sin(0.023 * k + 0.011 * j)
    x = x.contiguous()
    x.add_(torch.randn(SHAPE, generator=g, device=dev, dtype=torch.float32), alpha=0.002)
    for (a, b, c), v in SPIKES:
        x[a, b, c] = v
    return x


def test_past_2_31_points(hi, oracle_mod):
    N = int(np.prod(SHAPE))
    assert 2 ** 31 < N < 2 ** 32
    dev = torch.device("cuda", 0)
    x = _field(dev)
    p = hi.make_params(SHAPE, EB, "abs", A, autotune=True)
    b = hi.alloc(p, SHAPE, dev, out_cap=1 << 20, hist=True, recon=False)
    hi.compress_into(x, b)
    h = hi.read_header(b.header)
    assert h.status == 0

    # outliers: every spike, at its index, with its value
    n_out = int(h.n_outliers)
    idx = b.out_idx[:n_out].cpu().numpy().view(np.uint32).astype(np.int64)
    val = b.out_val[:n_out].cpu().numpy()
    found = dict(zip(idx.tolist(), val.tolist()))
    for (a, bb, c), v in SPIKES:
        gi = (a * SHAPE[1] + bb) * SHAPE[2] + c
        assert gi in found and found[gi] == np.float32(v)
    assert any(gi >= 2 ** 31 for gi in found)
    codes_at = b.codes[torch.from_numpy(idx).to(dev)]
    assert int((codes_at != 0).sum().item()) == 0

    # histogram totals
    hist = b.hist.cpu().numpy().view(np.uint32).astype(np.int64)
    assert hist.sum() == N - int(h.n_anchors)
    assert hist[0] == n_out

    # sampled blocks against the oracle on their own boxes
    L = 4
    interp = np.array([h.level[l].interp for l in range(L)], dtype=np.uint8)
    order = np.array([tuple(h.level[l].order) for l in range(L)], dtype=np.uint8)
    cst = oracle_mod.eps_constants(np.zeros(8, dtype=np.float32), 0, EB)
    assert np.float32(h.eb_f) == cst["eb_f"] and np.float32(h.r_f) == cst["r_f"]
    nb = [(n - 1 + A - 1) // A for n in SHAPE]
    rng = np.random.default_rng(3)
    picks = {(t0, t1, t2) for t0 in (0, nb[0] - 1) for t1 in (0, nb[1] - 1) for t2 in (0, nb[2] - 1)}
    picks |= {(nb[0] - 2, 77, 12), (32, 64, 100), (32, 1, 126)}  # just below 2^31 (planes 496..), beyond it (512..)
    picks |= {tuple(int(rng.integers(0, n)) for n in nb) for _ in range(6)}
    codes = b.codes.view(SHAPE)
    for t in sorted(picks):
        o = [t[d] * A for d in range(3)]
        e = [min(A, SHAPE[d] - 1 - o[d]) for d in range(3)]
        own = [e[d] + 1 if t[d] == nb[d] - 1 else A for d in range(3)]
        box = x[o[0]:o[0] + e[0] + 1, o[1]:o[1] + e[1] + 1, o[2]:o[2] + e[2] + 1].cpu().numpy()
        ref = oracle_mod.compress(box, A, interp, order, cst)
        got = codes[o[0]:o[0] + own[0], o[1]:o[1] + own[1], o[2]:o[2] + own[2]].cpu().numpy()
        assert np.array_equal(got, ref["codes"][:own[0], :own[1], :own[2]]), t

    # decompression within the bound everywhere (outliers exact)
    y = torch.empty_like(x)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    hi.decompress_into(b, y, st)
    assert int(st.item()) == 0
    ebf = float(np.float32(h.eb_f))
    for s in range(0, SHAPE[0], 65):
        d = (x[s:s + 65] - y[s:s + 65]).abs()
        assert float(d.max().item()) < ebf
    for (a, bb, c), v in SPIKES:
        assert float(y[a, bb, c].item()) == np.float32(v)
    del y

    # code reordering and the lossless stage at this size
    seq = hi.reorder_codes(b.codes, p)
    back = hi.unreorder_codes(seq, p)
    assert torch.equal(back, b.codes)
    del back
    na = int(h.n_anchors)
    assert int((seq[:na] != 128).sum().item()) == 0  # the anchors lead the sequence
    codec = hi.TpCodec(N, dev)
    codec.encode_into(seq)
    torch.cuda.synchronize()
    n_stream = int(codec.len.item())
    assert n_stream < N
    out = torch.zeros_like(seq)
    codec.decode_into(codec.stream_buf, n_stream, out)
    torch.cuda.synchronize()
    assert int(codec.status.item()) == 0 and torch.equal(out, seq)
