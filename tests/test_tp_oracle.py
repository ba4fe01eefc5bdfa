"""Pins of the oracle's throughput-mode lossless pipeline TCMS1-BIT1-RRE1
(Sec. 5.2.3).  The paper names the stages; the container (16 KiB chunks,
bit planes MSB first, RRE recursing on its bitmap down to 64 bytes, raw
fallback) is this library's reading.  Pins: the TCMS transform against the
paper's formula evaluated on Python integers, streams worked out by hand
from the format for a constant chunk and for single set bits, the raw
fallback, and lossless roundtrip on lengths around every boundary.
"""
import struct

import numpy as np
import pytest

import oracle


def _hdr(n, nchunks):
    h = struct.pack("<QII", n, 16384, nchunks)
    return h


def test_tcms_matches_paper_formula():
    """(w << 1) ^ (w >> (width - 1)) on the two's complement value, 8 bits:
    code 128 (the zero residual) -> 0xff, 127 -> 0xfe, 129 -> 0xfd."""
    for b in range(256):
        w = b - 256 if b >= 128 else b
        want = ((w << 1) ^ (w >> 7)) & 0xFF
        data = np.full(64, b, dtype=np.uint8)
        # a single chunk of 64 equal bytes: 8 planes of 8 bytes, each 0x00 or 0xff
        s = oracle.tp_encode(data)
        payload = s[32:32 + 64]
        planes = [int(payload[8 * p]) for p in range(8)]
        got = sum(((planes[p] & 1) << (7 - p)) for p in range(8))
        assert got == want, b
    assert [((w << 1) ^ (w >> 7)) & 0xFF for w in (-128, 127, -127)] == [0xFF, 0xFE, 0xFD]


def test_constant_chunk_by_hand():
    """16384 codes of 128: every shuffled byte is 0xff; RRE keeps one 0xff
    (bitmap 01 00..), then 01 00 (bitmap 03 00..), then 03 00, leaving a
    32-byte top level 03 00..; payload 32 + 2 + 2 + 1 = 37 -> 48 bytes."""
    s = oracle.tp_encode(np.full(16384, 128, dtype=np.uint8))
    want = bytearray(_hdr(16384, 1) + struct.pack("<I", 48))
    want += bytes(32 - len(want))
    payload = bytes([3]) + bytes(31) + bytes([3, 0]) + bytes([1, 0]) + bytes([0xFF])
    want += payload + bytes(48 - len(payload))
    assert bytes(s) == bytes(want)
    assert np.array_equal(oracle.tp_decode(s, 16384), np.full(16384, 128, dtype=np.uint8))


def test_single_bits_by_hand():
    """64 bytes, element 0 = 0x40 (TCMS 0x80: plane 0, bit 0 of byte 0),
    element 9 = 0x20 (TCMS 0x40: plane 1, byte 1 of that plane, bit 1);
    one 64-byte level, stored as is."""
    d = np.zeros(64, dtype=np.uint8)
    d[0], d[9] = 0x40, 0x20
    s = oracle.tp_encode(d)
    u = bytearray(64)
    u[0] = 0x01
    u[8 + 1] = 0x02
    want = bytearray(_hdr(64, 1) + struct.pack("<I", 64))
    want += bytes(32 - len(want))
    want += u
    assert bytes(s) == bytes(want)


def test_random_chunk_is_stored_raw():
    rng = np.random.default_rng(0)
    d = rng.integers(0, 256, size=20000, dtype=np.uint8)
    s = oracle.tp_encode(d)
    n0, ch, nc = struct.unpack("<QII", bytes(s[:16]))
    assert (n0, ch, nc) == (20000, 16384, 2)
    sizes = struct.unpack("<II", bytes(s[16:24]))
    assert sizes[0] == 0x80000000 | 16384 and sizes[1] == 0x80000000 | 3616
    assert bytes(s[32:32 + 16384]) == d[:16384].tobytes()
    assert np.array_equal(oracle.tp_decode(s, 20000), d)


@pytest.mark.parametrize("n", [0, 1, 63, 64, 65, 127, 16383, 16384, 16385, 40000, 100003])
def test_roundtrip_lengths(n):
    rng = np.random.default_rng(n)
    # code-like bytes: mostly 128 +- small, some runs, some rare large values
    d = (128 + np.round(rng.normal(0, 1.2, size=n))).clip(1, 255).astype(np.uint8)
    if n > 100:
        d[n // 3: n // 3 + 50] = 128
        d[::97] = rng.integers(0, 256, size=d[::97].size, dtype=np.uint8)
    s = oracle.tp_encode(d)
    assert s.size <= oracle.tp_bound(n)
    assert np.array_equal(oracle.tp_decode(s, n), d)


def test_reordered_codes_compress():
    from paper_2507_11165_gb300 import fields
    x = fields.lognormal_grf((64, 64, 64), seed=2)
    out = oracle.full_compress(x, 16, *oracle.levels(4, oracle.CUBIC, (0, 1, 2)), oracle.REL, 1e-2)
    seq = oracle.reorder_codes(out["codes"], 16)
    s = oracle.tp_encode(seq)
    assert np.array_equal(oracle.tp_decode(s, seq.size), seq)
    assert s.size < 0.5 * seq.size


def test_corrupt_stream_rejected():
    d = np.full(1000, 128, dtype=np.uint8)
    s = oracle.tp_encode(d)
    with pytest.raises(oracle.OracleError):
        oracle.tp_decode(s[:20], 1000)
    with pytest.raises(oracle.OracleError):
        oracle.tp_decode(s, 999)
