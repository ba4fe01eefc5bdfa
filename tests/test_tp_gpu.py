"""GPU parity of the throughput-mode lossless pipeline TCMS1-BIT1-RRE1
(Sec. 5.2.3) through the C ABI: the stream bytes equal the oracle's byte for
byte, each side decodes the other's stream, and decoding returns the input;
the full 512^3 field's reordered codes at the benchmark's bound in full;
corrupt streams are reported, not decoded."""
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
    codec = hi.TpCodec(data.size, "cuda")
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


def _code_like(rng, n, sigma=1.2):
    d = (128 + np.round(rng.normal(0, sigma, size=n))).clip(1, 255).astype(np.uint8)
    if n > 200:
        d[n // 3: n // 3 + 150] = 128
        d[::101] = rng.integers(0, 256, size=d[::101].size, dtype=np.uint8)
    return d


CASES = [0, 1, 63, 64, 65, 127, 1000, 16383, 16384, 16385, 50000, 262144 + 77]


@pytest.mark.parametrize("n", CASES)
@pytest.mark.parametrize("kind", ["code", "const", "random"])
def test_stream_matches_oracle(hi, oracle_mod, n, kind):
    rng = np.random.default_rng(n + 7)
    if kind == "code":
        d = _code_like(rng, n)
    elif kind == "const":
        d = np.full(n, 128, dtype=np.uint8)
    else:
        d = rng.integers(0, 256, size=n, dtype=np.uint8)
    ref = oracle_mod.tp_encode(d)
    codec, s = _gpu_encode(hi, d)
    assert np.array_equal(s, ref)
    back, st = _gpu_decode(hi, codec, ref, n)
    assert st == 0 and np.array_equal(back, d)
    assert np.array_equal(oracle_mod.tp_decode(s, n), d)


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
        assert np.array_equal(s, oracle_mod.tp_encode(sq))
        back, st = _gpu_decode(hi, codec, s, sq.size)
        assert st == 0 and np.array_equal(back, sq)


def test_full_size_field(hi, oracle_mod):
    """The 512^3 benchmark field at rel 1e-3: the whole stream against the oracle's."""
    shape = (512, 512, 512)
    x = torch.from_numpy(fields.lognormal_grf(shape, seed=1)).cuda()
    p = hi.make_params(shape, 1e-3, "rel", 16, autotune=True)
    b = hi.alloc(p, shape, "cuda", out_cap=x.numel() // 8, hist=True, recon=False)
    hi.compress_into(x, b)
    del x
    seq = hi.reorder_codes(b.codes, p)
    codec = hi.TpCodec(seq.numel(), "cuda")
    codec.encode_into(seq)
    torch.cuda.synchronize()
    n = int(codec.len.item())
    s = codec.stream_buf[:n].cpu().numpy()
    sq = seq.cpu().numpy()
    assert np.array_equal(s, oracle_mod.tp_encode(sq))
    out = torch.zeros_like(seq)
    codec.decode_into(codec.stream_buf, n, out)
    torch.cuda.synchronize()
    assert int(codec.status.item()) == 0 and torch.equal(out, seq)


@pytest.mark.parametrize("n", [100, 16384 + 640, 50000])
def test_unaligned_input_and_output(hi, oracle_mod, n):
    """Input and output at odd byte offsets (the byte-wise load and store
    paths): the same stream as the oracle's, and the input back."""
    rng = np.random.default_rng(n)
    d = _code_like(rng, n)
    big = torch.zeros(n + 16, dtype=torch.uint8, device="cuda")
    big[3:3 + n] = torch.from_numpy(d).cuda()
    codec = hi.TpCodec(n, "cuda")
    codec.encode_into(big[3:3 + n])
    torch.cuda.synchronize()
    ln = int(codec.len.item())
    s = codec.stream_buf[:ln].cpu().numpy()
    assert np.array_equal(s, oracle_mod.tp_encode(d))
    out = torch.zeros(n + 16, dtype=torch.uint8, device="cuda")
    codec.status.zero_()
    codec.decode_into(codec.stream_buf, ln, out[5:5 + n])
    torch.cuda.synchronize()
    assert int(codec.status.item()) == 0
    assert np.array_equal(out[5:5 + n].cpu().numpy(), d)
    assert int(out[:5].sum()) == 0 and int(out[5 + n:].sum()) == 0


def test_corrupt_streams(hi, oracle_mod):
    rng = np.random.default_rng(1)
    d = _code_like(rng, 40000)
    codec, s = _gpu_encode(hi, d)
    # wrong length
    codec2 = hi.TpCodec(39999, "cuda")
    _, st = _gpu_decode(hi, codec2, s, 39999)
    assert st == hi.HI_ECORRUPT
    # a size-table entry that points past the end
    bad = s.copy()
    bad[16:20] = np.frombuffer(np.uint32(16384 + 4096).tobytes(), dtype=np.uint8)
    _, st = _gpu_decode(hi, codec, bad, d.size)
    assert st == hi.HI_ECORRUPT
    # truncated payloads
    _, st = _gpu_decode(hi, codec, s[: s.size // 2 // 16 * 16], d.size)
    assert st == hi.HI_ECORRUPT


def test_rejects_bad_args(hi):
    import ctypes
    L = hi.lib()
    mx, ws = hi.tp_query(1000)
    data = torch.zeros(1000, dtype=torch.uint8, device="cuda")
    out = torch.zeros(mx + 16, dtype=torch.uint8, device="cuda")
    w = torch.zeros(ws, dtype=torch.uint8, device="cuda")
    ln = torch.zeros(1, dtype=torch.int64, device="cuda")

    def P(t, off=0):
        return ctypes.c_void_p(t.data_ptr() + off)

    assert L.hi_tp_encode(P(data), 1000, P(out), mx - 1, P(ln), P(w), ws, None) == hi.HI_EINVAL
    assert L.hi_tp_encode(P(data), 1000, P(out), mx, P(ln), P(w), ws - 16, None) == hi.HI_EINVAL
    assert L.hi_tp_encode(P(data), 1000, P(out, 4), mx, P(ln), P(w), ws, None) == hi.HI_EINVAL
    assert L.hi_tp_encode(P(out, 16), 1000, P(out), mx, P(ln), P(w), ws, None) == hi.HI_EINVAL  # overlap
    assert L.hi_tp_decode(P(out), 8, P(data), 1000, None, P(w), ws, None) == hi.HI_EINVAL
    assert L.hi_tp_decode(P(out, 4), mx, P(data), 1000, None, P(w), ws, None) == hi.HI_EINVAL
    torch.cuda.synchronize()
