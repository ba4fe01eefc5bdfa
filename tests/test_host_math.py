"""Host-side method arithmetic behind the C ABI (no GPU): the entropy-based
size estimate (hi_estimate_cr) and the eps of a value range (hi_resolve_eps)
equal the oracle's on the same inputs."""
import math

import numpy as np
import pytest

from paper_2507_11165_gb300 import build as hb


@pytest.fixture(scope="module")
def hi():
    hb.build()
    from paper_2507_11165_gb300 import hi
    return hi


def _hists():
    rng = np.random.default_rng(7)
    out = []
    h = np.full(256, 10, dtype=np.uint32)  # uniform: 8 bits
    out.append((h, 0, 0, 2560))
    h = np.zeros(256, dtype=np.uint32)
    h[128] = 1000  # one symbol: 0 bits
    out.append((h, 5, 7, 1012))
    h = np.zeros(256, dtype=np.uint32)
    h[[127, 129]] = 4  # two equal symbols: 1 bit
    out.append((h, 0, 0, 8))
    for k in range(20):  # peaked around 128 like real code histograms, and spread ones
        w = rng.uniform(0.5, 30.0)
        p = np.exp(-np.abs(np.arange(256) - 128) / w)
        h = rng.multinomial(int(rng.integers(10 ** 3, 10 ** 8)), p / p.sum()).astype(np.uint32)
        out.append((h, int(rng.integers(0, 10 ** 4)), int(rng.integers(1, 10 ** 5)), int(h.sum()) + 8))
    return out


def test_estimate_cr_matches_oracle(hi, oracle_mod):
    for hb_ in (0, hi.HEADER_BYTES):
        for h, n_out, n_anc, n in _hists():
            a = hi.estimate_cr(h, n_out, n_anc, n, header_bytes=hb_)
            b = oracle_mod.entropy_cr(h, n_out, n_anc, n, header_bytes=hb_)
            assert a["est_bytes"] == b["est_bytes"]
            assert math.isclose(a["entropy_bits"], b["entropy_bits"], rel_tol=1e-12, abs_tol=1e-15)
            assert math.isclose(a["cr"], b["cr"], rel_tol=1e-12)


def test_estimate_cr_closed_forms(hi):
    h = np.full(256, 10, dtype=np.uint32)
    e = hi.estimate_cr(h, 0, 0, 2560, header_bytes=0)
    assert abs(e["entropy_bits"] - 8.0) < 1e-12 and e["est_bytes"] == 2560 and e["cr"] == 4.0
    h = np.zeros(256, dtype=np.uint32)
    h[[127, 129]] = 4
    e = hi.estimate_cr(h, 1, 2, 8, header_bytes=3)
    assert e["entropy_bits"] == 1.0 and e["est_bytes"] == 1 + 8 + 8 + 3
    with pytest.raises(hi.HiError):
        hi.estimate_cr(h, 0, 0, 0)


def test_resolve_eps_matches_oracle(hi, oracle_mod):
    rng = np.random.default_rng(3)
    cases = [(-1.0, 3.0), (2.0, 2.0), (0.0, 1e-30), (-3.4e38, 3.4e38), (1e-20, 1e-19)]
    cases += [tuple(sorted(rng.normal(0, 10 ** rng.uniform(-6, 6), 2).astype(np.float32))) for _ in range(40)]
    for vmin, vmax in cases:
        x = np.array([vmin, vmax], dtype=np.float32)
        for mode, om, eb in (("rel", oracle_mod.REL, 1e-3), ("rel", oracle_mod.REL, 1e-5),
                             ("abs", oracle_mod.ABS, 0.25)):
            try:
                ref = oracle_mod.eps_constants(x, om, eb)
            except Exception:
                with pytest.raises(hi.HiError):
                    hi.resolve_eps(mode, eb, float(x[0]), float(x[1]))
                continue
            got = hi.resolve_eps(mode, eb, float(x[0]), float(x[1]))
            assert got["eps"] == ref["eps"]
            for k in ("eb_f", "ebx2_f", "r_f"):
                assert np.float32(got[k]).view(np.uint32) == np.float32(ref[k]).view(np.uint32), (k, vmin, vmax)


def test_resolve_eps_rejects(hi):
    for args in (("rel", 0.0, 0.0, 1.0), ("rel", float("nan"), 0.0, 1.0), (7, 1e-3, 0.0, 1.0)):
        with pytest.raises(hi.HiError):
            hi.resolve_eps(*args)


def test_autotune_select_matches_oracle(hi, oracle_mod):
    rng = np.random.default_rng(11)
    for shape, A in (((40, 70, 90), 16), ((300, 500), 16), ((5000,), 8), ((65, 65, 65), 8)):
        m, L, nc = hi.autotune_dims(shape, A)
        assert nc == len(oracle_mod.tune_configs(shape)) and L == oracle_mod.n_levels(A)
        for trial in range(6):
            # integer error sums: every order of summation is exact, so the argmin is the oracle's
            err = rng.integers(0, 50 if trial % 2 else 4, size=(m, L, nc)).astype(np.float64)
            got = hi.autotune_select(shape, A, err)
            interp, order = oracle_mod.tune_select(shape, A, err.sum(axis=0))
            assert got == [(int(i), tuple(int(v) for v in o)) for i, o in zip(interp, order)]
    with pytest.raises(hi.HiError):
        hi.autotune_select((40, 70, 90), 16, np.zeros(3))  # short array
