"""hi_compress_static_ws: the compress entry point that allocates nothing and
uses the library's fixed per-device scratch.  Its results must equal those of
hi_compress with a caller workspace, call after call.

The file name sorts last so that the GPU test also runs after every other
test of the suite (the scratch then has been through other calls' kernels)."""
import ctypes

import numpy as np
import pytest

from paper_2507_11165_gb300 import build as hb
from paper_2507_11165_gb300 import fields


@pytest.fixture(scope="module")
def hi():
    hb.build()
    from paper_2507_11165_gb300 import hi as mod
    return mod


def test_static_scratch_size_limits(hi):
    """The limits the header states, through hi_query (host only)."""
    lim = hi.STATIC_WS_BYTES
    for shape in [(10 ** 7,), (3162, 3162), (215, 215, 215)]:
        for A in (2, 4, 8, 16, 32):
            assert hi.query(hi.make_params(shape, 1e-3, "rel", A))["ws_bytes"] <= lim, (shape, A)
    for shape in [(1024, 2048, 2047), (512, 512, 512), (1625, 1625, 1625)]:
        assert hi.query(hi.make_params(shape, 1e-3, "rel", 16))["ws_bytes"] <= lim, shape


def test_static_scratch_rejects_large_field(hi):
    """A field whose workspace exceeds the fixed scratch is refused on the host
    before anything is enqueued or any pointer is looked at."""
    p = hi.make_params((10 ** 8,), 1e-3, "rel", 2)
    assert hi.query(p)["ws_bytes"] > hi.STATIC_WS_BYTES
    rc = hi.lib().hi_compress_static_ws(ctypes.byref(p), None, None, None, None, None, 0, None, None, None, None)
    assert rc == hi.HI_ENOMEM
    assert hi.status_str(rc) == "workspace too small"


def _same(hi, torch, ref, got):
    torch.cuda.synchronize()
    hr, hg = hi.read_header(ref.header), hi.read_header(got.header)
    assert bytes(hr) == bytes(hg)
    assert hr.status == 0
    assert torch.equal(ref.codes, got.codes)
    assert torch.equal(ref.anchors, got.anchors)
    assert torch.equal(ref.hist, got.hist)
    assert torch.equal(ref.recon, got.recon)
    n = int(hr.n_outliers)
    ia, va = ref.out_idx[:n].cpu().numpy(), ref.out_val[:n].cpu().numpy()
    ib, vb = got.out_idx[:n].cpu().numpy(), got.out_val[:n].cpu().numpy()
    oa, ob = np.argsort(ia, kind="stable"), np.argsort(ib, kind="stable")
    assert np.array_equal(ia[oa], ib[ob])
    assert np.array_equal(va[oa].view(np.uint32), vb[ob].view(np.uint32))
    return n


@pytest.mark.gpu
def test_static_ws_equals_compress_two_calls_in_a_row(hi):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    cases = [((70, 81, 96), 11, 1e-3, 16), ((48, 65, 128), 12, 1e-5, 16)]
    outliers = []
    for k, (shape, seed, eb, A) in enumerate(cases):
        x = torch.from_numpy(fields.lognormal_grf(shape, seed=seed)).to(dev)
        p = hi.make_params(shape, eb, "rel", A, autotune=True)
        n = hi.query(p)["n_points"]
        ref = hi.alloc(p, shape, dev, out_cap=n, hist=True, recon=True)
        got = hi.alloc(p, shape, dev, out_cap=n, hist=True, recon=True)
        for t in (got.codes, got.hist, got.out_idx):
            t.fill_(0x5A)
        got.anchors.fill_(float("nan"))
        got.recon.fill_(float("nan"))
        hi.compress_into(x, ref)
        torch.cuda.synchronize()
        if k == 0:
            hi.compress_static_ws_into(x, got)  # first call on the device: set-up
        else:
            free0 = torch.cuda.mem_get_info(dev)[0]
            hi.compress_static_ws_into(x, got)
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info(dev)[0] == free0  # nothing allocated
        outliers.append(_same(hi, torch, ref, got))
    assert outliers[1] > 0  # the tight bound exercises the outlier path
