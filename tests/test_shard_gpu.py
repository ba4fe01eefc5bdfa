"""One GPU compressing a field shard by shard (as separate ranks would, each
with the global bound) and merging: the same record as compressing the
field whole."""
import numpy as np
import pytest
import torch

from paper_2507_11165_gb300 import fields, shard

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_11165_gb300 import hi as hi_mod
    hi_mod.lib()
    return hi_mod


@pytest.mark.parametrize("shape,A,parts,eb", [((150, 64, 72), 16, 3, 1e-3), ((101, 40, 36), 8, 2, 1e-5),
                                              ((33, 20, 48), 16, 2, 1e-4)])
def test_shards_in_sequence_equal_the_whole_field(hi, shape, A, parts, eb):
    x = torch.from_numpy(fields.lognormal_grf(shape, seed=31)).cuda()
    L = A.bit_length() - 1
    levels = [(1 if l % 2 == 0 else 0, (0, 1, 2) if l % 3 else (2, 0, 1)) for l in range(L)]
    m = shard.compress_in_sequence(x, eb, A, parts, levels)
    c = hi.compress(x, eb, "rel", A, autotune=False, levels=levels, out_cap=x.numel())
    assert m["eps"] == c.h.eps
    assert np.float32(m["eb_f"]) == np.float32(c.h.eb_f) and np.float32(m["r_f"]) == np.float32(c.h.r_f)
    assert torch.equal(m["codes"], c.codes)
    assert torch.equal(m["anchors"].view(torch.int32), c.anchors.view(torch.int32))
    idx, val = c.outliers
    oa, ob = torch.argsort(m["out_idx"]), torch.argsort(idx.to(torch.int64))
    assert torch.equal(m["out_idx"][oa], idx.to(torch.int64)[ob])
    assert torch.equal(m["out_val"][oa].view(torch.int32), val[ob].view(torch.int32))
    assert torch.equal(m["hist"], c.hist.to(torch.int64))
    if eb <= 1e-5:
        assert c.n_outliers > 0
