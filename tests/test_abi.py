"""The C-ABI library builds, loads and exports every entry point include/*.h
declares; host-only calls (sizes, validation, status text) work without a GPU."""
import ctypes
import glob
import os
import re

import pytest

from paper_2507_11165_gb300 import build as hb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    hb.build()
    from paper_2507_11165_gb300 import hi
    return hi


def declared_symbols():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names += re.findall(r"HI_API\s+[\w\s\*]+?\b(hi_\w+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 8
    L = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert set(lib.SYMBOLS) <= set(names)


def test_struct_layouts(lib):
    assert ctypes.sizeof(lib.HiHeader) == 168
    assert ctypes.sizeof(lib.HiParams) == 80


def test_host_calls_without_gpu(lib):
    assert lib.lib().hi_version() == 1
    assert lib.status_str(lib.HI_ECAPACITY) == "outlier capacity exceeded"
    q = lib.query(lib.make_params((512, 512, 512), 1e-3, "rel", 16))
    assert q["n_points"] == 512 ** 3 and q["n_anchors"] == 32 ** 3 and q["n_blocks"] == 32 ** 3
    q = lib.query(lib.make_params((1800, 3600), 1e-3, "rel", 16))
    assert q["n_anchors"] == 113 * 225 and q["n_blocks"] == 113 * 225
    q = lib.query(lib.make_params((100, 500, 500), 1e-3, "rel", 16))
    assert q["n_blocks"] == 7 * 32 * 32 and q["n_anchors"] == 7 * 32 * 32
    for bad in [dict(anchor_stride=12), dict(anchor_stride=64), dict(eb=-1.0), dict(eb=float("inf"))]:
        p = lib.make_params((9, 9, 9), 1e-3, "rel", 8)
        for k, v in bad.items():
            setattr(p, k, v)
        with pytest.raises(lib.HiError):
            lib.query(p)
    p = lib.make_params((70000, 70000), 1e-3, "rel", 16)  # 4.9e9 points: beyond uint32 indices
    with pytest.raises(lib.HiError):
        lib.query(p)
    p = lib.make_params((9, 9, 9), 1e-3, "rel", 8, autotune=False)
    p.level[0].interp = 7
    with pytest.raises(lib.HiError):
        lib.query(p)


def test_batch_host_validation(lib):
    import ctypes as C
    assert C.sizeof(lib.HiBatchField) == 160 and C.sizeof(lib.HiBatchPlan) == 120
    L = lib.lib()
    arr = (lib.HiBatchField * 3)()
    arr[0].p = lib.make_params((40, 50, 60), 1e-3, "rel", 16)
    arr[1].p = lib.make_params((64, 64), 1e-3, "abs", 16)
    arr[2].p = lib.make_params((1000,), 1e-3, "rel", 16)
    ws = C.c_size_t()
    assert L.hi_batch_query(3, arr, C.byref(ws)) == lib.HI_OK
    # 256 B counters + 3 field records + prefixes + tickets + two range partials + auto-tune sums
    assert ws.value % 256 == 0 and ws.value > 256 + 3 * 256
    assert L.hi_batch_query(0, arr, C.byref(ws)) == lib.HI_EINVAL
    arr[1].p = lib.make_params((64, 64), 1e-3, "abs", 8)  # mixed anchor strides
    assert L.hi_batch_query(3, arr, C.byref(ws)) == lib.HI_EINVAL
    for i in range(3):
        arr[i].p.anchor_stride = 4  # batches take A = 8 or 16
    assert L.hi_batch_query(3, arr, C.byref(ws)) == lib.HI_EINVAL
    plan = lib.HiBatchPlan()
    arr[0].p = lib.make_params((40, 50, 60), 1e-3, "rel", 16)
    assert L.hi_batch_prepare(1, arr, 3, None, 0, C.byref(plan), None) == lib.HI_EINVAL  # bad tuning
    assert L.hi_batch_prepare(1, arr, 0, None, 0, C.byref(plan), None) == lib.HI_EINVAL  # no workspace


def test_lossless_query_without_gpu(lib):
    """Sizes of both lossless pipelines are host-only; the stream bounds cover
    the oracle's streams, from constant to uniformly random bytes."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(0)
    for n in (0, 1, 4096, 100000):
        mx, ws = lib.cr_query(n)
        mt, wt = lib.tp_query(n)
        assert ws > 0 and wt > 0
        for d in (np.full(n, 128, dtype=np.uint8), rng.integers(0, 256, size=n, dtype=np.uint8)):
            assert oracle.cr_encode(d).size <= mx
            assert oracle.tp_encode(d).size <= mt


def test_compress_seq_fused_decision(lib):
    """hi_compress_seq writes the reordered codes from the predict-quantize
    kernel only where every run of a tile row starts at a multiple of its
    length (A = 8 or 16, n2 a multiple of A, a 16-byte aligned sequence);
    elsewhere it reorders after the kernel."""
    a, b = 0x100000, 0x900000  # addresses only: nothing is dereferenced
    fused = [((512, 512, 512), 16), ((64, 64, 64), 16), ((32, 48, 64), 16), ((24, 40, 32), 8), ((384, 384, 384), 16),
             ((1, 64, 128), 16), ((1, 1, 4096), 16)]
    separate = [((37, 45, 70), 16), ((100, 500, 500), 16), ((16, 16, 48), 16), ((64, 64, 64), 32),
                ((64, 64, 64), 4), ((1800, 3600), 16), ((9, 9, 9), 8)]
    for shape, A in fused:
        p = lib.make_params(shape, 1e-3, "rel", A)
        assert lib.compress_seq_fused(p, a, b), (shape, A)
        assert not lib.compress_seq_fused(p, a, b + 8), (shape, A)  # sequence off a 16-byte boundary
        assert lib.compress_seq_fused(p, a + 4, b), (shape, A)  # the codes' own alignment does not matter
    for shape, A in separate:
        assert not lib.compress_seq_fused(lib.make_params(shape, 1e-3, "rel", A), a, b), (shape, A)


def test_compress_seq_fused_rule_random_shapes(lib):
    """The same decision on 300 random shapes against a restatement of the
    rule: A = 8 or 16, n2 a multiple of A, and on every level l < log2 A
    the coarser-point count, the fastest-dim extent, the all-even points of a
    plane and of a row of the stride-2^l subgrid all multiples of A >> l."""
    import numpy as np
    rng = np.random.default_rng(3)

    def rule(shape, A):
        n = (1,) * (3 - len(shape)) + tuple(shape)
        if A not in (8, 16) or n[2] % A:
            return False
        sub = list(n)
        for l in range(A.bit_length() - 1):
            c = A >> l
            h1, h2 = (sub[1] + 1) // 2, (sub[2] + 1) // 2
            pre = ((sub[0] + 1) // 2) * h1 * h2
            if pre % c or sub[2] % c or (h1 * h2) % c or h2 % c:
                return False
            sub = [(s + 1) // 2 for s in sub]
        return True

    hits = 0
    for _ in range(300):
        A = int(rng.choice([4, 8, 16, 32]))
        shape = tuple(int(v) for v in rng.choice([1, 2, 3, 5, 8, 16, 24, 32, 40, 48, 64, 96, 100, 128], size=3))
        if max(shape) < 2:
            continue
        p = lib.make_params(shape, 1e-3, "rel", A)
        want = rule(shape, A)
        hits += want
        assert lib.compress_seq_fused(p, 0x100000, 0x900000) == want, (shape, A)
    assert hits > 20


def test_header_is_plain_c(tmp_path):
    """include/hi.h is a C header: it compiles as strict C99 with no C++ and
    no torch types (the boundary is plain pointers and sizes)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_hi.c"
    src.write_text('#include "hi.h"\nint main(void) { return (int)sizeof(hi_header) == 0; }\n')
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                        "-I" + os.path.join(ROOT, "include"), "-I" + cuda_inc, str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
