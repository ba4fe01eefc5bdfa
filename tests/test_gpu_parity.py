"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bit-exact on codes, anchors, reconstructed values, the outlier set (compared
after sorting by index: the order of the list is unspecified), the histogram
and the float32 quantizer constants.  Sizes span several blocks and ragged
tails; the last tests run the full-size workloads with sampled blocks.
"""
import functools

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


def _levels_from(interp, order):
    return [(int(interp[l]), tuple(int(v) for v in order[l])) for l in range(len(interp))]


def run_gpu(hi, x, A, eb, mode, interp=None, order=None, autotune=False, out_cap=None, recon=True,
            x_dev=None):
    levels = None if interp is None else _levels_from(interp, order)
    p = hi.make_params(x.shape, eb, mode, A, autotune, levels)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda() if x_dev is None else x_dev
    cap = x.size if out_cap is None else out_cap
    b = hi.alloc(p, x.shape, "cuda", out_cap=cap, hist=True, recon=recon)
    hi.compress_into(xd, b)
    h = hi.read_header(b.header)
    return p, b, h


def gpu_outliers(b, h):
    k = min(int(h.n_outliers), b.out_cap)
    idx = b.out_idx[:k].cpu().numpy().view(np.uint32)
    val = b.out_val[:k].cpu().numpy()
    o = np.argsort(idx, kind="stable")
    return idx[o], val[o]


def check_against_oracle(oracle, hi, x, A, eb, mode, interp, order, b, h, recon=True):
    cst = oracle.eps_constants(x, mode, eb)
    assert h.status == 0, hi.status_str(h.status)
    assert h.magic == hi.MAGIC
    assert np.float32(h.eb_f) == cst["eb_f"] and np.float32(h.ebx2_f) == cst["ebx2_f"]
    assert np.float32(h.r_f) == cst["r_f"]
    assert h.eps == cst["eps"]
    ref = oracle.compress(x, A, interp, order, cst)
    col = oracle.collect(x, ref["codes"], A)
    codes = b.codes.cpu().numpy().reshape(x.shape)
    mism = np.count_nonzero(codes != ref["codes"])
    assert mism == 0, "codes differ at %d points" % mism
    na = int(h.n_anchors)
    assert np.array_equal(b.anchors[:na].cpu().numpy().view(np.uint32), ref["anchors"].view(np.uint32))
    if recon:
        r = b.recon.cpu().numpy().reshape(x.shape)
        assert np.array_equal(r.view(np.uint32), ref["recon"].view(np.uint32))
    assert int(h.n_outliers) == col["n_out"]
    idx, val = gpu_outliers(b, h)
    assert np.array_equal(idx, col["out_idx"])
    assert np.array_equal(val.view(np.uint32), col["out_val"].view(np.uint32))
    assert np.array_equal(b.hist.cpu().numpy().view(np.uint32), col["hist"])
    return ref, col, cst


CASES = [
    # shape, A, eb, mode, interp/order spec
    ((64, 64, 64), 8, 1e-3, 1, "cubic012"),          # the 64^3 unit-scale workload
    ((70, 45, 53), 16, 1e-3, 1, "random"),
    ((33, 33, 33), 16, 1e-4, 1, "random"),
    ((40, 36, 44), 8, 1e-2, 1, "random"),
    ((17, 17, 17), 16, 1e-3, 0, "linear"),
    ((31, 29, 30), 4, 1e-3, 1, "random"),
    ((20, 22, 36), 2, 1e-3, 1, "random"),
    ((50, 40, 70), 32, 1e-3, 1, "random"),
    ((257, 301), 16, 1e-3, 1, "random"),             # 2D, ragged
    ((1, 129, 64), 16, 1e-4, 1, "random"),
    ((1000,), 16, 1e-3, 1, "random"),                # 1D
    ((5, 1, 19), 8, 1e-3, 1, "random"),
    ((2, 3, 4), 2, 1e-3, 1, "random"),
    ((1, 1, 1), 8, 1e-3, 1, "random"),
    ((37, 41, 43), 16, 1e-3, 1, "random"),           # n2 % 4 != 0: plain-load path
    ((48, 48, 52), 16, 1e-5, 1, "random"),           # many outliers
    # the multi-dimensional scheme (Sec. 5.1.2), mixed with 1D levels
    ((70, 45, 53), 16, 1e-3, 1, "md"),
    ((33, 33, 33), 16, 1e-4, 1, "md"),
    ((40, 36, 44), 8, 1e-2, 1, "md"),
    ((257, 301), 16, 1e-3, 1, "md"),
    ((37, 41, 43), 16, 1e-3, 1, "md"),               # plain-load path
    ((31, 29, 30), 4, 1e-3, 1, "md"),
    ((50, 40, 70), 32, 1e-3, 1, "md"),
    ((64, 64, 64), 8, 1e-3, 1, "md_all"),
]


def _field(shape, seed):
    if len(shape) == 3 and min(shape) >= 8:
        return fields.lognormal_grf(shape, seed=seed) if seed % 2 else fields.bumps_field(shape, seed=seed)
    return fields.bumps_field(shape, seed=seed)


def _cfg(oracle, shape, A, spec, rng):
    L = oracle.n_levels(A)
    if spec == "cubic012":
        return oracle.levels(L, oracle.CUBIC, (0, 1, 2))
    if spec == "linear":
        return oracle.levels(L, oracle.LINEAR, (2, 1, 0))
    if spec == "md_all":
        return oracle.levels(L, oracle.MD_CUBIC, (0, 1, 2))
    n3 = (1,) * (3 - len(shape)) + tuple(shape)
    act = [d for d in range(3) if n3[d] > 1]
    interp = rng.integers(0, 2, size=L).astype(np.uint8)
    order = np.zeros((L, 3), dtype=np.uint8)
    for l in range(L):
        order[l] = list(rng.permutation(act)) + [d for d in range(3) if d not in act]
        if spec == "md" and rng.uniform() < 0.6:
            interp[l] = oracle.MD_LINEAR + int(rng.integers(0, 2))
    return interp, order


@pytest.mark.parametrize("case", range(len(CASES)))
def test_compress_decompress_parity(oracle_mod, hi, case):
    shape, A, eb, mode, spec = CASES[case]
    rng = np.random.default_rng(100 + case)
    x = _field(shape, case)
    interp, order = _cfg(oracle_mod, shape, A, spec, rng)
    p, b, h = run_gpu(hi, x, A, eb, mode, interp, order)
    ref, col, cst = check_against_oracle(oracle_mod, hi, x, A, eb, mode, interp, order, b, h)
    # reconstruction: GPU decompress == oracle decompress == compressor's recon (Eq. 1)
    out = torch.empty(b.shape, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    hi.decompress_into(b, out, st)
    assert int(st.item()) == 0
    y = out.cpu().numpy()
    odec = oracle_mod.decompress(x.shape, A, interp, order, cst["ebx2_f"], ref["codes"], ref["anchors"],
                                 col["out_idx"], col["out_val"])
    assert np.array_equal(y.view(np.uint32), odec.view(np.uint32))
    assert np.array_equal(y.view(np.uint32), ref["recon"].view(np.uint32))
    fin = np.isfinite(x)
    assert np.all(np.abs(y[fin].astype(np.float64) - x[fin]) < cst["eps"])


def test_nonfinite_and_constant(oracle_mod, hi):
    x = fields.bumps_field((33, 34, 35), seed=3)
    x[3, 5, 7] = np.nan
    x[10, 1, 2] = np.inf
    x[32, 33, 34] = -np.inf
    L = 4
    it, od = oracle_mod.levels(L)
    p, b, h = run_gpu(hi, x, 16, 1e-3, 1, it, od)
    check_against_oracle(oracle_mod, hi, x, 16, 1e-3, 1, it, od, b, h)
    c = np.full((20, 21, 22), 3.25, dtype=np.float32)
    p, b, h = run_gpu(hi, c, 8, 1e-4, 1, *oracle_mod.levels(3))
    check_against_oracle(oracle_mod, hi, c, 8, 1e-4, 1, *oracle_mod.levels(3), b, h)
    assert np.all(b.codes.cpu().numpy() == 128)


def test_tiny_eb_all_outliers_and_capacity(oracle_mod, hi):
    x = fields.bumps_field((30, 31, 33), seed=5)
    it, od = oracle_mod.levels(3)
    p, b, h = run_gpu(hi, x, 8, 1e-30, 1, it, od)
    check_against_oracle(oracle_mod, hi, x, 8, 1e-30, 1, it, od, b, h)
    n_anchor = int(np.prod(oracle_mod.anchor_dims(x.shape, 8)))
    assert int(h.n_outliers) == x.size - n_anchor
    # capacity too small: status reports it, the count is exact, codes stay valid
    p, b2, h2 = run_gpu(hi, x, 8, 1e-30, 1, it, od, out_cap=100)
    assert h2.status == hi.HI_ECAPACITY and int(h2.n_outliers) == x.size - n_anchor
    assert torch.equal(b2.codes, b.codes)
    # decompress refuses a truncated record
    out = torch.empty(b2.shape, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    hi.decompress_into(b2, out, st)
    assert int(st.item()) == hi.HI_ECAPACITY


def test_misaligned_views(oracle_mod, hi):
    """Sub-views that are not 16-byte aligned take the plain-load path, same bytes."""
    x = fields.lognormal_grf((40, 40, 40), seed=9)
    it, od = oracle_mod.levels(4)
    base = torch.from_numpy(np.concatenate([np.zeros(1, np.float32), x.reshape(-1)])).cuda()
    xd = base[1:]
    p, b, h = run_gpu(hi, x, 16, 1e-3, 1, it, od, x_dev=xd)
    check_against_oracle(oracle_mod, hi, x, 16, 1e-3, 1, it, od, b, h)


def test_invalid_arguments(hi):
    import ctypes
    x = torch.zeros((9, 9, 9), device="cuda")
    p = hi.make_params(x.shape, 1e-3, "rel", 8, False)
    b = hi.alloc(p, x.shape, "cuda")
    for bad in [dict(anchor_stride=12), dict(eb=0.0), dict(eb=float("nan")), dict(eb_mode=7)]:
        q = hi.make_params(x.shape, 1e-3, "rel", 8, False)
        for k, v in bad.items():
            setattr(q, k, v)
        rc = hi.lib().hi_compress(ctypes.byref(q), hi._ptr(x), hi._ptr(b.codes), hi._ptr(b.anchors),
                                  hi._ptr(b.out_idx), hi._ptr(b.out_val), b.out_cap, None, None,
                                  hi._ptr(b.header), hi._ptr(b.ws), b.ws.numel(), hi._stream(None))
        assert rc == hi.HI_EINVAL
    q = hi.make_params(x.shape, 1e-3, "rel", 8, False)
    q.level[1].order[2] = 1  # not a permutation
    assert hi.lib().hi_compress(ctypes.byref(q), hi._ptr(x), hi._ptr(b.codes), hi._ptr(b.anchors), None, None, 0,
                                None, None, hi._ptr(b.header), hi._ptr(b.ws), b.ws.numel(),
                                hi._stream(None)) == hi.HI_EINVAL
    # workspace too small
    assert hi.lib().hi_compress(ctypes.byref(p), hi._ptr(x), hi._ptr(b.codes), hi._ptr(b.anchors), None, None, 0,
                                None, None, hi._ptr(b.header), hi._ptr(b.ws), 16,
                                hi._stream(None)) == hi.HI_ENOMEM


def test_corrupt_outlier_index(oracle_mod, hi):
    x = fields.bumps_field((24, 24, 24), seed=2)
    p, b, h = run_gpu(hi, x, 8, 1e-5, 1, *oracle_mod.levels(3))
    assert int(h.n_outliers) > 0
    b.out_idx[0] = 24 ** 3 + 5  # outside the field
    out = torch.empty(b.shape, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    hi.decompress_into(b, out, st)
    assert int(st.item()) == hi.HI_ECORRUPT


def test_determinism(hi):
    x = torch.from_numpy(fields.lognormal_grf((96, 80, 72), seed=4)).cuda()
    res = []
    for _ in range(3):
        c = hi.compress(x, 1e-4, "rel", 16, autotune=True, recon=True)
        idx, val = c.outliers
        o = torch.argsort(idx)
        res.append((c.codes.clone(), c.recon.clone(), c.hist.clone(), idx[o].clone(), val[o].clone(),
                    c.info()["levels"]))
    for r in res[1:]:
        for a, b in zip(res[0][:5], r[:5]):
            assert torch.equal(a, b)
        assert r[5] == res[0][5]


# --------------------------------------------------------------------------
# Auto-tune (Sec. 5.1.3)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("shape,A,md", [((64, 64, 64), 8, False), ((96, 112, 80), 16, False), ((300, 500), 16, False),
                                        ((5000,), 8, False), ((100, 120, 90), 4, False), ((96, 112, 80), 16, True),
                                        ((300, 500), 16, True), ((64, 64, 64), 8, True)])
def test_autotune_parity(oracle_mod, hi, shape, A, md):
    """md: candidates include the multi-dimensional scheme (autotune = 2)."""
    x = fields.lognormal_grf(shape, seed=7) if len(shape) == 3 else fields.bumps_field(shape, seed=7)
    p, b, h = run_gpu(hi, x, A, 1e-3, 1, autotune=2 if md else True)
    assert h.status == 0
    gerr = hi.autotune_errors(b)  # [m, L, ncfg]
    oerr = oracle_mod.tune_errors(x, A, md=md)  # [L, ncfg]
    assert gerr.shape[0] == oracle_mod.tune_samples(shape, A)
    tot = gerr.sum(axis=0)
    np.testing.assert_allclose(tot, oerr, rtol=1e-9, atol=1e-12)
    cfgs = oracle_mod.tune_configs(shape, md=md)
    L = oracle_mod.n_levels(A)
    for l in range(L):
        chosen = (int(h.level[l].interp), tuple(h.level[l].order))
        c = cfgs.index(chosen)
        assert oerr[l, c] <= oerr[l].min() * (1 + 1e-6) + 1e-300
    # the rest of the pipeline with the chosen configuration is bit-exact
    interp = np.array([h.level[l].interp for l in range(L)], dtype=np.uint8)
    order = np.array([tuple(h.level[l].order) for l in range(L)], dtype=np.uint8)
    check_against_oracle(oracle_mod, hi, x, A, 1e-3, 1, interp, order, b, h)


# --------------------------------------------------------------------------
# Mixed-shape workloads at full size (1800 x 3600 and 100 x 500 x 500)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("which,eb", [("2d", 1e-3), ("2d", 1e-4), ("3d", 1e-3), ("3d", 1e-4)])
def test_mixed_shapes_full(oracle_mod, hi, which, eb):
    x = fields.fronts_2d() if which == "2d" else fields.stratified_3d()
    A = 16
    p, b, h = run_gpu(hi, x, A, eb, 1, autotune=True)
    L = 4
    interp = np.array([h.level[l].interp for l in range(L)], dtype=np.uint8)
    order = np.array([tuple(h.level[l].order) for l in range(L)], dtype=np.uint8)
    check_against_oracle(oracle_mod, hi, x, A, eb, 1, interp, order, b, h)


# --------------------------------------------------------------------------
# 512^3 at the benchmark's launch configuration: sampled blocks
# --------------------------------------------------------------------------
def _sample_tiles(nb, rng, k=48):
    nbt = int(np.prod(nb))
    corners = []
    for t0 in (0, nb[0] - 1):
        for t1 in (0, nb[1] - 1):
            for t2 in (0, nb[2] - 1):
                corners.append((t0 * nb[1] + t1) * nb[2] + t2)
    rand = rng.choice(nbt, size=k, replace=False)
    return np.unique(np.concatenate([corners, rand])).astype(np.int64)


def _tile_mask(shape, A, tiles, nb):
    """Points owned by the listed blocks."""
    m = np.zeros(shape, dtype=bool)
    for t in tiles:
        t0, t1, t2 = t // (nb[1] * nb[2]), (t // nb[2]) % nb[1], t % nb[2]
        sl = []
        for d, td in enumerate((t0, t1, t2)):
            lo = td * A
            hi_ = shape[d] if td == nb[d] - 1 else lo + A
            sl.append(slice(lo, hi_))
        m[tuple(sl)] = True
    return m


@functools.lru_cache(maxsize=1)
def _grf512():
    return fields.lognormal_grf((512, 512, 512), seed=1)


@pytest.mark.slow
@pytest.mark.parametrize("eb", [1e-2, 1e-3, 1e-4])
def test_full_512_sampled(oracle_mod, hi, eb):
    shape, A = (512, 512, 512), 16
    x = _grf512()
    p, b, h = run_gpu(hi, x, A, eb, 1, autotune=True, recon=True)
    assert h.status == 0
    cst = oracle_mod.eps_constants(x, 1, eb)
    assert np.float32(h.eb_f) == cst["eb_f"] and np.float32(h.r_f) == cst["r_f"]
    L = 4
    interp = np.array([h.level[l].interp for l in range(L)], dtype=np.uint8)
    order = np.array([tuple(h.level[l].order) for l in range(L)], dtype=np.uint8)
    nb = oracle_mod.block_grid(shape, A)
    tiles = _sample_tiles(nb, np.random.default_rng(int(eb * 1e6)))
    ref = oracle_mod.compress(x, A, interp, order, cst, tiles=tiles)
    mask = _tile_mask(shape, A, tiles, nb)
    codes = b.codes.cpu().numpy().reshape(shape)
    assert np.array_equal(codes[mask], ref["codes"][mask])
    recon = b.recon.cpu().numpy().reshape(shape)
    assert np.array_equal(recon[mask].view(np.uint32), ref["recon"][mask].view(np.uint32))
    # properties that hold at any size
    err = np.abs(recon.astype(np.float64) - x)
    assert err.max() < cst["eps"]
    hist = b.hist.cpu().numpy().view(np.uint32).astype(np.int64)
    assert hist.sum() == x.size - int(h.n_anchors)
    assert hist[0] == int(h.n_outliers) == int(np.count_nonzero(codes == 0)) - 0
    idx, val = gpu_outliers(b, h)
    assert np.array_equal(idx, np.flatnonzero(codes.reshape(-1) == 0).astype(np.uint32))
    assert np.array_equal(val.view(np.uint32), x.reshape(-1)[idx].view(np.uint32))
    # decompress == compressor's reconstruction, bit for bit
    out = torch.empty(shape, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    hi.decompress_into(b, out, st)
    assert int(st.item()) == 0
    assert torch.equal(out.view(torch.int32).reshape(-1), b.recon.view(torch.int32))
