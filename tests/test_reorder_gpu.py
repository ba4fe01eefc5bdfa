"""GPU parity of the quantization-code reordering (Sec. 5.2.2, Eq. 3),
through the C ABI (hi_reorder_codes / hi_unreorder_codes).

Small and ragged shapes: byte-exact against the oracle, both directions.
Full-size shapes: the whole permutation is read back from the GPU (the four
byte planes of a point-index field reordered one by one) and checked
against the properties that fix it uniquely -- levels non-increasing along
the sequence, row-major order within a level, every point exactly once.
"""
import numpy as np
import pytest
import torch

from paper_2507_11165_gb300 import fields

pytestmark = pytest.mark.gpu

CASES = [((9, 9, 9), 8), ((10, 7, 13), 8), ((17, 17, 17), 16), ((33, 20, 5), 16), ((12, 30), 4),
         ((21,), 4), ((5, 1, 19), 8), ((2, 3, 4), 2), ((1, 1, 1), 8), ((40,), 32), ((70, 45, 1100), 16),
         ((3, 2500), 8), ((5000,), 2), ((65, 64, 63), 32), ((1, 1, 3000), 16),
         # rows of 16-byte multiples (at most 4096): the staged-row path
         ((9, 9, 16), 8), ((33, 20, 48), 16), ((12, 64), 4), ((5, 7, 4096), 32), ((2, 3, 16), 2),
         ((1, 1, 16), 16), ((3, 5, 32), 2), ((16,), 16), ((40, 1, 160), 8), ((31, 17, 4080), 16)]


@pytest.fixture(scope="module")
def hi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_11165_gb300 import hi as hi_mod
    hi_mod.lib()
    return hi_mod


@pytest.mark.parametrize("shape,A", CASES)
def test_reorder_matches_oracle(hi, oracle_mod, shape, A):
    rng = np.random.default_rng(sum(shape) * 31 + A)
    c = rng.integers(0, 256, size=shape, dtype=np.uint8)
    p = hi.make_params(shape, 1e-3, "rel", A, autotune=False)
    cd = torch.from_numpy(c).cuda()
    seq = hi.reorder_codes(cd, p)
    back = hi.unreorder_codes(seq, p)
    torch.cuda.synchronize()
    ref = oracle_mod.reorder_codes(c, A)
    assert np.array_equal(seq.cpu().numpy(), ref)
    assert np.array_equal(back.cpu().numpy().reshape(shape), c)
    # the inverse alone, from the oracle's sequence
    back2 = hi.unreorder_codes(torch.from_numpy(ref).cuda(), p)
    assert np.array_equal(back2.cpu().numpy().reshape(shape), oracle_mod.unreorder_codes(ref, shape, A))


@pytest.mark.parametrize("shape,A", [((9, 9, 16), 8), ((33, 20, 48), 16), ((10, 7, 13), 8)])
def test_reorder_unaligned_buffers(hi, oracle_mod, shape, A):
    """Buffers off a 16-byte boundary take the general path: same sequence."""
    rng = np.random.default_rng(7)
    c = rng.integers(0, 256, size=shape, dtype=np.uint8)
    n = c.size
    p = hi.make_params(shape, 1e-3, "rel", A, autotune=False)
    src = torch.zeros(n + 8, dtype=torch.uint8, device="cuda")
    dst = torch.zeros(n + 8, dtype=torch.uint8, device="cuda")
    src[3:3 + n] = torch.from_numpy(c.reshape(-1)).cuda()
    hi.reorder_codes(src[3:3 + n], p, out=dst[5:5 + n])
    back = torch.zeros(n + 8, dtype=torch.uint8, device="cuda")
    hi.unreorder_codes(dst[5:5 + n], p, out=back[1:1 + n])
    torch.cuda.synchronize()
    assert np.array_equal(dst[5:5 + n].cpu().numpy(), oracle_mod.reorder_codes(c, A))
    assert np.array_equal(back[1:1 + n].cpu().numpy().reshape(shape), c)


def test_reorder_of_compressed_codes(hi, oracle_mod):
    """The codes of a real compression, reordered: the oracle's sequence, and
    its first n_anchors bytes are the anchors' code (128)."""
    shape, A = (49, 40, 66), 16
    x = fields.lognormal_grf(shape, seed=5)
    p = hi.make_params(shape, 1e-3, "rel", A, autotune=True)
    b = hi.alloc(p, shape, "cuda", out_cap=x.size, hist=True, recon=False)
    hi.compress_into(torch.from_numpy(x).cuda(), b)
    seq = hi.reorder_codes(b.codes, p)
    torch.cuda.synchronize()
    codes = b.codes.cpu().numpy().reshape(shape)
    s = seq.cpu().numpy()
    assert np.array_equal(s, oracle_mod.reorder_codes(codes, A))
    na = int(np.prod([(n - 1) // A + 1 for n in shape]))
    assert np.all(s[:na] == 128)


def _levels(shape, A):
    L = A.bit_length() - 1
    d = (1,) * (3 - len(shape)) + tuple(shape)
    g = np.zeros(d, dtype=np.int64)
    g |= np.arange(d[0], dtype=np.int64)[:, None, None]
    g |= np.arange(d[1], dtype=np.int64)[None, :, None]
    g |= np.arange(d[2], dtype=np.int64)[None, None, :]
    g = g.reshape(-1)
    lv = np.full(g.size, L, dtype=np.int8)
    nz = g != 0
    low = g[nz] & -g[nz]  # lowest set bit
    lv[nz] = np.minimum(np.log2(low).astype(np.int8), L)
    return lv


@pytest.mark.parametrize("shape,A", [((512, 512, 512), 16), ((100, 500, 500), 16), ((1800, 3600), 16),
                                     ((257, 300, 301), 8)])
def test_full_size_permutation(hi, shape, A):
    N = int(np.prod(shape))
    p = hi.make_params(shape, 1e-3, "rel", A, autotune=False)
    idx = torch.arange(N, dtype=torch.int32, device="cuda")
    perm = torch.zeros(N, dtype=torch.int64, device="cuda")
    for k in range(4):
        plane = ((idx >> (8 * k)) & 0xFF).to(torch.uint8)
        seq = hi.reorder_codes(plane, p)
        back = hi.unreorder_codes(seq, p)
        assert torch.equal(back, plane)
        perm |= seq.to(torch.int64) << (8 * k)
    del idx, plane, seq, back
    perm = perm.cpu().numpy()
    assert np.array_equal(np.bincount(perm, minlength=N), np.ones(N, dtype=np.int64))
    lv = _levels(shape, A)[perm]
    assert np.all(np.diff(lv) <= 0)  # coarser levels first
    same = np.diff(lv) == 0
    assert np.all(np.diff(perm)[same] > 0)  # row-major within a level


def test_rejects_overlap_and_bad_args(hi):
    p = hi.make_params((8, 8, 8), 1e-3, "rel", 8, autotune=False)
    buf = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError):
        hi.reorder_codes(buf[:512], p, out=buf[100:612])
    q = hi.make_params((8, 8, 8), 1e-3, "rel", 8, autotune=False)
    q.anchor_stride = 12
    with pytest.raises(RuntimeError):
        hi.reorder_codes(buf[:512], q, out=buf[512:])


SEQ_CASES = [((64, 64, 64), 16, True), ((32, 48, 64), 16, True), ((24, 40, 32), 8, True), ((1, 64, 128), 16, True),
             ((40, 48, 64), 16, True), ((33, 48, 64), 16, True), ((17, 9, 32), 8, True),
             ((1, 1, 4096), 16, True), ((37, 45, 70), 16, False), ((16, 16, 48), 16, False), ((33, 20, 48), 16, False),
             ((9, 9, 9), 8, False)]


@pytest.mark.parametrize("shape,A,fused", SEQ_CASES)
def test_compress_seq_matches_oracle(hi, oracle_mod, shape, A, fused):
    """hi_compress_seq: the same record as hi_compress, and the oracle's
    reordering of its codes in d_seq, whether the predict-quantize kernel
    writes the sequence itself (fused) or a reordering pass follows it."""
    x = torch.from_numpy(fields.lognormal_grf(shape, seed=sum(shape) + A)).cuda()
    p = hi.make_params(shape, 1e-3, "rel", A, autotune=True)
    a = hi.alloc(p, shape, "cuda", out_cap=x.numel(), hist=True, recon=True)
    b = hi.alloc(p, shape, "cuda", out_cap=x.numel(), hist=True, recon=True)
    seq = torch.full((x.numel(),), 7, dtype=torch.uint8, device="cuda")
    assert hi.compress_seq_fused(p, b.codes.data_ptr(), seq.data_ptr()) == fused
    hi.compress_into(x, a)
    hi.compress_seq_into(x, b, seq)
    torch.cuda.synchronize()
    assert torch.equal(a.codes, b.codes) and torch.equal(a.hist, b.hist)
    assert torch.equal(a.recon.view(torch.int32), b.recon.view(torch.int32))
    assert bytes(hi.read_header(a.header)) == bytes(hi.read_header(b.header))
    codes = b.codes.cpu().numpy().reshape(shape)
    assert np.array_equal(seq.cpu().numpy(), oracle_mod.reorder_codes(codes, A))


def test_compress_seq_full_size(hi):
    """The benchmark field (512^3, A = 16), fused: d_seq equals the separate
    reordering of the kernel's own codes (whose permutation the full-size
    test above checks), with outliers and a capacity re-run in between."""
    shape = (512, 512, 512)
    x = torch.from_numpy(fields.lognormal_grf(shape, seed=1)).cuda()
    p = hi.make_params(shape, 1e-4, "rel", 16, autotune=True)
    b = hi.alloc(p, shape, "cuda", out_cap=1 << 16, hist=True, recon=False)
    seq = torch.empty(x.numel(), dtype=torch.uint8, device="cuda")
    assert hi.compress_seq_fused(p, b.codes.data_ptr(), seq.data_ptr())
    hi.compress_seq_into(x, b, seq)
    torch.cuda.synchronize()
    h = hi.read_header(b.header)
    assert h.status == hi.HI_ECAPACITY  # the codes (and the sequence) stay valid
    ref = hi.reorder_codes(b.codes, p)
    torch.cuda.synchronize()
    assert torch.equal(seq, ref)
    assert int((seq == 0).sum()) == int(h.n_outliers)
