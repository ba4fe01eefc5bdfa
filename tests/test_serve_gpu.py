"""The serving loop on the GPU: requests overlap on several streams under a
tight memory budget, and every result equals, bit for bit, the result of the
same request run alone."""
import numpy as np
import pytest
import torch

from paper_2507_11165_gb300 import fields, serve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_11165_gb300 import hi as hi_mod
    hi_mod.lib()
    return hi_mod


def _same_record(hi, a, b):
    ha, hb = hi.read_header(a.header), hi.read_header(b.header)
    assert bytes(ha) == bytes(hb) and ha.status == 0
    assert torch.equal(a.codes, b.codes)
    assert torch.equal(a.anchors, b.anchors)
    assert torch.equal(a.hist, b.hist)
    n = int(ha.n_outliers)
    ia, ib = a.out_idx[:n].cpu().numpy(), b.out_idx[:n].cpu().numpy()
    va, vb = a.out_val[:n].cpu().numpy(), b.out_val[:n].cpu().numpy()
    oa, ob = np.argsort(ia, kind="stable"), np.argsort(ib, kind="stable")
    assert np.array_equal(ia[oa], ib[ob]) and np.array_equal(va[oa].view(np.uint32), vb[ob].view(np.uint32))


def test_results_alone_equal_results_in_the_mix(hi):
    base = torch.from_numpy(fields.lognormal_grf((128, 128, 128), seed=11)).cuda()
    reqs = serve.make_requests(n=32, rate=4000.0, seed=7, lo=24, hi=100)
    budget = 3 * serve.device_bytes("compress", 100, 1e-5)
    ex = serve.GpuExecutor(base, keep_outputs=True)
    sv = serve.Server(ex, slots=4, budget_bytes=budget, keep_records=4)  # records are recycled too
    done = sv.run(reqs)
    assert len(done) == len(reqs) and all(d.status == 0 for d in done)
    assert sv.peak_concurrency >= 2  # work overlapped on the device
    assert sv.peak_bytes <= budget
    by_id = {r.id: r for r in reqs}
    alone = {}
    for d in sorted(done, key=lambda d: d.id):
        req = by_id[d.id]
        if d.op == "compress":
            x = ex.snapshot_view(req).contiguous()
            p = hi.make_params(x.shape, req.eb, "rel", 16, autotune=True)
            n = x.numel()
            b = hi.alloc(p, x.shape, "cuda", out_cap=serve.outlier_capacity(req.side, req.eb), hist=True,
                         recon=False)
            hi.compress_into(x, b)
            h = hi.read_header(b.header)
            if h.status == hi.HI_ECAPACITY:  # as the server does: again with the exact capacity
                b = hi.alloc(p, x.shape, "cuda", out_cap=int(h.n_outliers), hist=True, recon=False)
                hi.compress_into(x, b)
            torch.cuda.synchronize()
            alone[d.id] = b
            _same_record(hi, b, ex.outputs[d.id])
    n_dec = 0
    for d in done:
        if d.op != "decompress":
            continue
        req = by_id[d.id]
        b = alone[req.source]
        out = torch.empty(b.shape, dtype=torch.float32, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        hi.decompress_into(b, out, st)
        assert int(st.item()) == 0
        assert torch.equal(out.view(torch.int32), ex.outputs[d.id].view(torch.int32))
        n_dec += 1
    assert n_dec > 0
    # buffers were reused across requests (the pools served later requests)
    assert sum(len(v) for v in ex.pool.values()) > 0
