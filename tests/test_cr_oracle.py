"""Pins of the oracle's compression-ratio-mode lossless pipeline
HF-RRE4-TCMS8-RZE1 (Sec. 5.2.3).  The paper names the stages (Huffman
coding, repeat elimination on 4-byte symbols with a recursively compressed
bitmap, the magnitude-sign transform (w << 1) ^ (w >> 63) on 8-byte words,
zero elimination on bytes); the tie rule of the code construction, the
16-bit length limit, the 4096-symbol blocks and the container are this
library's reading.  Pins: Huffman lengths against the Kraft equality and a
brute-force optimum on small alphabets, the tie rule on hand examples, the
length limit, streams worked out by hand from the format, the transform
against the paper's formula on Python integers, and lossless roundtrip.
"""
import itertools
import struct

import numpy as np
import pytest

import oracle


def _freq(d):
    f = np.zeros(256, dtype=np.uint64)
    for k, v in d.items():
        f[k] = v
    return f


def _cost(freq, ln):
    return sum(int(freq[v]) * int(ln[v]) for v in range(256))


def _brute_optimum(weights):
    """Minimal sum w_i l_i over length vectors with sum 2^-l_i <= 1 (any prefix code)."""
    k = len(weights)
    best = None
    for ls in itertools.product(range(1, k), repeat=k):
        if sum(2.0 ** -l for l in ls) <= 1.0 + 1e-12:
            c = sum(w * l for w, l in zip(weights, ls))
            best = c if best is None else min(best, c)
    return best


@pytest.mark.parametrize("seed", range(12))
def test_huffman_lengths_optimal_and_complete(seed):
    """On 2..6 symbols the lengths meet the Kraft equality (a full tree) and
    reach the brute-force minimum of the coded size."""
    rng = np.random.default_rng(seed)
    k = 2 + seed % 5
    syms = rng.choice(256, size=k, replace=False)
    w = rng.integers(1, 50, size=k)
    f = _freq(dict(zip(syms.tolist(), w.tolist())))
    ln = oracle.hf_lengths(f)
    assert all(ln[s] > 0 for s in syms) and int(np.count_nonzero(ln)) == k
    assert sum(2.0 ** -int(ln[s]) for s in syms) == 1.0
    assert _cost(f, ln) == _brute_optimum(w.tolist())


def test_huffman_tie_rule_by_hand():
    """Weights a:1, b:1, c:2 (a < b < c): a and b merge first (node 3, weight
    2); then c (weight 2, leaf index 2) ranks before node 3 (weight 2, index
    3): c gets 1 bit, a and b 2 bits.  Weights 2, 2, 2, 2: two pairs of
    leaves, then the two internal nodes: all 2 bits.  Weights 1, 1, 1: the
    first two leaves merge, the last leaf is 1 bit."""
    ln = oracle.hf_lengths(_freq({10: 1, 20: 1, 30: 2}))
    assert (ln[10], ln[20], ln[30]) == (2, 2, 1)
    ln = oracle.hf_lengths(_freq({1: 2, 2: 2, 3: 2, 4: 2}))
    assert (ln[1], ln[2], ln[3], ln[4]) == (2, 2, 2, 2)
    ln = oracle.hf_lengths(_freq({5: 1, 6: 1, 7: 1}))
    assert (ln[5], ln[6], ln[7]) == (2, 2, 1)
    ln = oracle.hf_lengths(_freq({200: 7}))
    assert ln[200] == 1 and int(np.count_nonzero(ln)) == 1
    assert int(np.count_nonzero(oracle.hf_lengths(np.zeros(256, dtype=np.uint64)))) == 0


def test_huffman_length_limit():
    """Fibonacci weights over 30 symbols make a 29-deep tree; the limited
    lengths stay within 16, still form a complete prefix code, and give
    shorter (or equal) codes to more frequent symbols."""
    fib = [1, 1]
    while len(fib) < 30:
        fib.append(fib[-1] + fib[-2])
    f = _freq({i: fib[i] for i in range(30)})
    ln = oracle.hf_lengths(f)
    assert int(ln[:30].max()) <= 16 and int(np.count_nonzero(ln)) == 30
    assert sum(2.0 ** -int(ln[i]) for i in range(30)) == 1.0
    for i in range(29):
        assert ln[i + 1] <= ln[i]
    # unlimited, the same weights give lengths 29, 29, 28, ..., 1
    f2 = _freq({i: fib[i] for i in range(17)})
    ln2 = oracle.hf_lengths(f2)
    assert [int(ln2[i]) for i in range(17)] == [16, 16] + list(range(15, 0, -1))


def _header(n, nb, H, nc):
    return struct.pack("<QIIQII", n, 4096, nb, H, 16384, nc)


def test_single_symbol_stream_by_hand():
    """8 codes of 128: one symbol, 1-bit code 0; 8 zero bits pad to one word
    (H = 4 bytes, one chunk).  RRE4: the word equals word -1 = 0, bitmap
    00, no kept words (m1 = 1); TCMS8: no whole word; RZE1 of the byte 00:
    one level, kept as is.  Payload 00 padded to 16."""
    s = oracle.cr_encode(np.full(8, 128, dtype=np.uint8))
    ln = bytearray(256)
    ln[128] = 1
    want = _header(8, 1, 4, 1) + bytes(ln) + struct.pack("<I", 1) + struct.pack("<HHH", 8, 8, 8) + bytes(2)
    want += struct.pack("<II", 16, 1)
    want += bytes(320 - len(want)) + bytes(16)
    assert bytes(s) == want
    assert np.array_equal(oracle.cr_decode(s, 8), np.full(8, 128, dtype=np.uint8))


def test_two_symbol_stream_by_hand():
    """128 codes of 127 and 129: two symbols get 1-bit codes 0 (127) and
    1 (129), so the HF bytes are the symbol bits, MSB first: 16 bytes, four
    words, the first two equal (69 69 69 69) and the last two (96 96 96 96).
    RRE4: words 0 and 2 differ from their predecessor, bitmap 05, kept w0
    and w2: r = 05 | w0 | w2 (9 bytes).  TCMS8 on r[0:8] read as a
    little-endian int64 t: (t << 1) ^ (t >> 63), the paper's formula; r[8]
    stays.  RZE1 over the 9 bytes: one level (<= 64), stored as is; 9 <= 16
    bytes, so not raw."""
    bits = [0, 1, 1, 0, 1, 0, 0, 1] * 8 + [1, 0, 0, 1, 0, 1, 1, 0] * 8  # 128 symbols
    d = np.array([129 if b else 127 for b in bits], dtype=np.uint8)
    s = oracle.cr_encode(d)
    r = bytes([5]) + bytes([0b01101001] * 4) + bytes([0b10010110] * 4)
    t = int.from_bytes(r[:8], "little", signed=True)
    u = ((t << 1) ^ (t >> 63)) & (2 ** 64 - 1)
    payload = u.to_bytes(8, "little") + r[8:]
    ln = bytearray(256)
    ln[127] = ln[129] = 1
    want = _header(128, 1, 16, 1) + bytes(ln) + struct.pack("<I", 4) + struct.pack("<HHH", 128, 128, 128) + bytes(2)
    want += struct.pack("<II", 16, 9)
    want += bytes(320 - len(want)) + payload + bytes(16 - len(payload))
    assert bytes(s) == want
    assert np.array_equal(oracle.cr_decode(s, 128), d)


def test_tcms8_sign_magnitude_order():
    """The magnitude-sign order the transform gives: 0, -1, 1, -2, 2 map to
    0, 1, 2, 3, 4 (the formula on Python integers), and negative words
    (high byte >= 0x80) come out odd: seen through a stream whose RRE4
    output starts with a negative little-endian word."""
    f = lambda w: ((w << 1) ^ (w >> 63)) & (2 ** 64 - 1)
    assert [f(w) for w in (0, -1, 1, -2, 2)] == [0, 1, 2, 3, 4]


def test_random_bytes_stored_raw():
    """Uniform random bytes: every length is 8 bits, the HF bytes are the
    input bytes, nothing repeats or is zero often enough: the chunk is raw."""
    rng = np.random.default_rng(1)
    d = rng.permutation(np.repeat(np.arange(256, dtype=np.uint8), 64))  # 16384 bytes, every symbol 64 times
    s = oracle.cr_encode(d)
    n, hb, nb, H, cc, nc = struct.unpack("<QIIQII", bytes(s[:32]))
    assert (n, nb, H, nc) == (16384, 4, 16384, 1)
    assert all(v == 8 for v in s[32:288])
    assert struct.unpack("<12H", bytes(s[288 + 16:288 + 40])) == (8192, 16384, 24576) * 4
    size, m1 = struct.unpack("<II", bytes(s[288 + 40:288 + 48]))
    assert size == 0x80000000 | 16384 and m1 == 0
    assert np.array_equal(oracle.cr_decode(s, d.size), d)


@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 4095, 4096, 4097, 16384, 40000, 70001])
def test_roundtrip_lengths(n):
    rng = np.random.default_rng(n)
    d = np.clip(np.round(rng.laplace(128.0, 1.2, n)), 1, 255).astype(np.uint8)
    d[rng.random(n) < 0.01] = 0
    s = oracle.cr_encode(d)
    assert np.array_equal(oracle.cr_decode(s, n), d)


def test_reordered_codes_smaller_than_throughput_mode():
    """On the reordered codes of a 64^3 field the CR-mode stream is smaller
    than the throughput-mode stream (the paper's reason for the CR mode)."""
    from paper_2507_11165_gb300 import fields
    x = fields.lognormal_grf((64, 64, 64), seed=1)
    r = oracle.full_compress(x, 16, *oracle.levels(4, oracle.LINEAR, (0, 1, 2)), oracle.REL, 1e-3)
    seq = oracle.reorder_codes(r["codes"], 16)
    s = oracle.cr_encode(seq)
    assert np.array_equal(oracle.cr_decode(s, seq.size), seq)
    assert s.size < oracle.tp_encode(seq).size


@pytest.mark.parametrize("n", [5000, 4096 * 3 + 1500, 4096 + 1024, 4096 + 1023])
def test_block_starting_points(n):
    """The table of starting points: for every block, the bit offsets of its
    symbols 1024, 2048 and 3072 (the running sum of the code lengths), or
    its bit count where the block is shorter; a wrong entry makes the
    stream corrupt."""
    rng = np.random.default_rng(n)
    d = np.clip(np.round(rng.laplace(128.0, 2.0, n)), 0, 255).astype(np.uint8)
    s = oracle.cr_encode(d)
    freq = np.bincount(d, minlength=256).astype(np.uint64)
    ln = oracle.hf_lengths(freq).astype(np.int64)
    nb = (n + 4095) // 4096
    sub = struct.unpack("<%dH" % (3 * nb), bytes(s[288 + 4 * nb:288 + 4 * nb + 6 * nb]))
    for b in range(nb):
        blk = d[4096 * b:4096 * (b + 1)].astype(np.int64)
        cum = np.concatenate([[0], np.cumsum(ln[blk])])
        for j in (1, 2, 3):
            want = int(cum[min(1024 * j, blk.size)])
            assert sub[3 * b + j - 1] == want, (b, j)
    assert np.array_equal(oracle.cr_decode(s, n), d)
    bad = s.copy()
    off = 288 + 4 * nb + 2 * 0
    bad[off] ^= 1
    with pytest.raises(Exception):
        oracle.cr_decode(bad, n)
