"""GPU parity of the compression-ratio-mode lossless pipeline HF-RRE4-TCMS8-RZE1
(Sec. 5.2.3) through the C ABI: the stream bytes equal the oracle's byte for
byte (code book, Huffman blocks, chunk payloads, tables), each side decodes
the other's stream, decoding returns the input; the reordered codes of
fields at three bounds and of the full 512^3 benchmark field; corrupt
streams are reported."""
import numpy as np
import pytest
import torch

from paper_2507_11165_gb300 import fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_11165_gb300 import hi as hi_mod
    hi_mod.lib()
    return hi_mod


def _gpu_encode(hi, data):
    codec = hi.CrCodec(data.size, "cuda")
    d = torch.from_numpy(np.ascontiguousarray(data)).cuda()
    codec.encode_into(d)
    torch.cuda.synchronize()
    n = int(codec.len.item())
    return codec, codec.stream_buf[:n].cpu().numpy()


def _gpu_decode(hi, codec, stream, n):
    sd = torch.from_numpy(np.ascontiguousarray(stream)).cuda()
    out = torch.zeros(max(n, 1), dtype=torch.uint8, device="cuda")
    codec.status.zero_()
    codec.decode_into(sd, stream.size, out)
    torch.cuda.synchronize()
    return out[:n].cpu().numpy(), int(codec.status.item())


def _code_like(rng, n, sigma=1.5):
    d = (128 + np.round(rng.laplace(0, sigma, size=n))).clip(1, 255).astype(np.uint8)
    if n > 400:
        d[n // 3: n // 3 + 300] = 128
        d[::97] = rng.integers(0, 256, size=d[::97].size, dtype=np.uint8)
    return d


CASES = [0, 1, 5, 63, 4095, 4096, 4097, 16384, 50001, 262144 + 77, 1 << 20]


@pytest.mark.parametrize("n", CASES)
@pytest.mark.parametrize("kind", ["code", "const", "random", "two"])
def test_stream_matches_oracle(hi, oracle_mod, n, kind):
    rng = np.random.default_rng(n + 11)
    if kind == "code":
        d = _code_like(rng, n)
    elif kind == "const":
        d = np.full(n, 128, dtype=np.uint8)
    elif kind == "two":
        d = np.where(rng.random(n) < 0.3, 127, 129).astype(np.uint8)
    else:
        d = rng.integers(0, 256, size=n, dtype=np.uint8)
    ref = oracle_mod.cr_encode(d)
    codec, s = _gpu_encode(hi, d)
    assert s.size == ref.size and np.array_equal(s, ref)
    back, st = _gpu_decode(hi, codec, ref, n)
    assert st == 0 and np.array_equal(back, d)


def test_skewed_histogram_length_limit(hi, oracle_mod):
    """Fibonacci-like symbol counts force the 16-bit length limit."""
    fib = [1, 1]
    while len(fib) < 26:
        fib.append(fib[-1] + fib[-2])
    d = np.concatenate([np.full(c, 100 + i, dtype=np.uint8) for i, c in enumerate(fib)])
    d = np.random.default_rng(3).permutation(d)
    ref = oracle_mod.cr_encode(d)
    assert 12 < int(ref[32:288].max()) <= 16  # unlimited, the deepest code would take 25 bits
    codec, s = _gpu_encode(hi, d)
    assert np.array_equal(s, ref)
    back, st = _gpu_decode(hi, codec, s, d.size)
    assert st == 0 and np.array_equal(back, d)


def test_reordered_codes_of_a_field(hi, oracle_mod):
    shape, A = (70, 66, 90), 16
    x = fields.lognormal_grf(shape, seed=9)
    for eb in (1e-2, 1e-3, 1e-4):
        p = hi.make_params(shape, eb, "rel", A, autotune=True)
        b = hi.alloc(p, shape, "cuda", out_cap=x.size, hist=True, recon=False)
        hi.compress_into(torch.from_numpy(x).cuda(), b)
        seq = hi.reorder_codes(b.codes, p)
        torch.cuda.synchronize()
        sq = seq.cpu().numpy()
        codec, s = _gpu_encode(hi, sq)
        assert np.array_equal(s, oracle_mod.cr_encode(sq))
        back, st = _gpu_decode(hi, codec, s, sq.size)
        assert st == 0 and np.array_equal(back, sq)


def test_full_size_field(hi, oracle_mod):
    """The 512^3 benchmark field at rel 1e-3: the whole stream against the
    oracle's, and smaller than the throughput-mode stream."""
    shape = (512, 512, 512)
    x = torch.from_numpy(fields.lognormal_grf(shape, seed=1)).cuda()
    p = hi.make_params(shape, 1e-3, "rel", 16, autotune=True)
    b = hi.alloc(p, shape, "cuda", out_cap=x.numel() // 8, hist=True, recon=False)
    hi.compress_into(x, b)
    del x
    seq = hi.reorder_codes(b.codes, p)
    codec = hi.CrCodec(seq.numel(), "cuda")
    codec.encode_into(seq)
    torch.cuda.synchronize()
    n = int(codec.len.item())
    s = codec.stream_buf[:n].cpu().numpy()
    sq = seq.cpu().numpy()
    assert np.array_equal(s, oracle_mod.cr_encode(sq))
    out = torch.zeros_like(seq)
    codec.decode_into(codec.stream_buf, n, out)
    torch.cuda.synchronize()
    assert int(codec.status.item()) == 0 and torch.equal(out, seq)
    assert n < oracle_mod.tp_encode(sq).size


def test_corrupt_streams(hi, oracle_mod):
    rng = np.random.default_rng(1)
    d = _code_like(rng, 70000)
    codec, s = _gpu_encode(hi, d)
    # wrong length
    codec2 = hi.CrCodec(69999, "cuda")
    _, st = _gpu_decode(hi, codec2, s, 69999)
    assert st == hi.HI_ECORRUPT
    # a chunk size that points past the end of the stream
    nb = (d.size + 4095) // 4096
    tab = 288 + 4 * nb + (6 * nb + 3) // 4 * 4
    bad = s.copy()
    bad[tab:tab + 4] = np.frombuffer(np.uint32(1 << 24).tobytes(), dtype=np.uint8)
    _, st = _gpu_decode(hi, codec, bad, d.size)
    assert st == hi.HI_ECORRUPT
    # a code length above 16
    bad = s.copy()
    bad[32 + 128] = 17
    _, st = _gpu_decode(hi, codec, bad, d.size)
    assert st == hi.HI_ECORRUPT
    # truncated payloads
    _, st = _gpu_decode(hi, codec, s[: s.size // 2 // 16 * 16], d.size)
    assert st == hi.HI_ECORRUPT
    # a starting point of a block that is not where its symbol 1024 begins
    bad = s.copy()
    sp = 288 + 4 * nb + 2 * 3 * 5  # block 5's first starting point
    bad[sp:sp + 2] = np.frombuffer(np.uint16(int(np.frombuffer(bytes(s[sp:sp + 2]), np.uint16)[0]) + 1).tobytes(),
                                   dtype=np.uint8)
    _, st = _gpu_decode(hi, codec, bad, d.size)
    assert st == hi.HI_ECORRUPT


def test_rejects_bad_args(hi):
    import ctypes
    L = hi.lib()
    mx, ws = hi.cr_query(1000)
    data = torch.zeros(1000, dtype=torch.uint8, device="cuda")
    out = torch.zeros(mx + 16, dtype=torch.uint8, device="cuda")
    w = torch.zeros(ws, dtype=torch.uint8, device="cuda")
    ln = torch.zeros(1, dtype=torch.int64, device="cuda")

    def P(t, off=0):
        return ctypes.c_void_p(t.data_ptr() + off)

    assert L.hi_cr_encode(P(data), 1000, P(out), mx - 1, P(ln), P(w), ws, None) == hi.HI_EINVAL
    assert L.hi_cr_encode(P(data), 1000, P(out), mx, P(ln), P(w), ws - 16, None) == hi.HI_EINVAL
    assert L.hi_cr_encode(P(data), 1000, P(out, 4), mx, P(ln), P(w), ws, None) == hi.HI_EINVAL
    assert L.hi_cr_encode(P(out, 16), 1000, P(out), mx, P(ln), P(w), ws, None) == hi.HI_EINVAL  # overlap
    assert L.hi_cr_decode(P(out), 8, P(data), 1000, None, P(w), ws, None) == hi.HI_EINVAL
    assert L.hi_cr_decode(P(out, 4), mx, P(data), 1000, None, P(w), ws, None) == hi.HI_EINVAL
    torch.cuda.synchronize()
