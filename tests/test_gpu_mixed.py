"""Reduced-precision (FP32-table) layers against the FP64 oracle.

Losses, terms, the ELT combination and the occurrence terms run in binary32;
each trial is still summed exactly.  The bar is relative 1e-5 per trial with
a 1 USD absolute floor.  As for the FP64 path, the relative error is taken
against max(|o|, S_o), S_o the oracle's pre-aggregate sum: binary32 rounding
of the event losses moves S by ~1e-7 S, and the aggregate clamp passes that
change through unchanged however much of S the retention removes.
"""
import numpy as np
import pytest

import ara_synth as S
import oracle

pytestmark = pytest.mark.gpu

REL, FLOOR = 1e-5, 1.0


def assert_reduced_parity(g, o, presum, what="ylt"):
    err = np.abs(np.asarray(g) - o)
    bound = np.maximum(REL * np.maximum(np.abs(o), presum), FLOOR)
    i = int(np.argmax(err / bound))
    assert err[i] <= bound[i], f"{what}: trial {i} gpu={g[i]!r} oracle={o[i]!r} presum={presum[i]!r}"
    return float(np.max(err / np.maximum(np.maximum(np.abs(o), presum), 1e-300)))


@pytest.fixture
def engine():
    from paper_1412_4556_b300 import Engine
    e = Engine(0)
    yield e
    e.close()


def test_fp32_layers_against_fp64_oracle(engine):
    from paper_1412_4556_b300 import ARA_FP32_TABLE
    w = S.batched(n_layers=6, n_trials=3_000, lam=300.0, catalog_size=200_000, n_pool=40)
    engine.load_yet_from(w.yet)
    first = engine.load_pool(w.pool)
    hs = [engine.define_layer([first + j for j in L.elts], L.occ_ret, L.occ_lim, L.agg_ret, L.agg_lim,
                              precision=ARA_FP32_TABLE) for L in w.layers]
    batch = engine.layers_ylt(hs)
    for i, (h, lay) in enumerate(zip(hs, w.layers)):
        single = engine.layer_ylt(h)
        np.testing.assert_array_equal(batch[i], single)
        o, pre = oracle.layer_ylt(w.yet, w.pool, lay, mode="memo")
        assert_reduced_parity(single, o, pre, what=f"layer {i}")
        # the per-event table holds binary32 values
        tab = engine.event_table(h)
        np.testing.assert_array_equal(tab, tab.astype(np.float32).astype(np.float64))
        tab64 = oracle.event_table(w.yet.catalog_size, w.pool, lay)
        # each binary32 operation and input rounding is off by <= 2^-24 of the
        # combined loss x <= value + OccR (or of OccL when it caps the value)
        bound = 2e-7 * (len(lay.elts) + 4) * (tab64 + lay.occ_ret) + 1e-3
        assert np.all(np.abs(tab - tab64) <= bound)
        # PML/TVaR move by at most the largest per-trial error
        rps = [10.0, 100.0]
        pml_o, tvar_o = oracle.pml_tvar(o, rps)
        pml_g, tvar_g = engine.pml_tvar(single, rps)
        # (plus the rounding of the oracle's sequential tail sum)
        bound = np.max(np.abs(single - o)) + 1e-12 * np.abs(tvar_o)
        assert np.all(np.abs(pml_g - pml_o) <= bound) and np.all(np.abs(tvar_g - tvar_o) <= bound)


def test_fp32_and_fp64_layers_mix_in_one_batch(engine):
    from paper_1412_4556_b300 import ARA_FP32_TABLE, ARA_FP64
    w = S.batched(n_layers=4, n_trials=2_000, lam=200.0, catalog_size=150_000, n_pool=30)
    engine.load_yet_from(w.yet)
    first = engine.load_pool(w.pool)
    precs = [ARA_FP64, ARA_FP32_TABLE, ARA_FP32_TABLE, ARA_FP64]
    hs = [engine.define_layer([first + j for j in L.elts], L.occ_ret, L.occ_lim, L.agg_ret, L.agg_lim,
                              precision=p) for L, p in zip(w.layers, precs)]
    batch = engine.layers_ylt(hs)
    for i, h in enumerate(hs):
        np.testing.assert_array_equal(batch[i], engine.layer_ylt(h))


@pytest.mark.parametrize("n_layers", [3, 9])
def test_fp32_layers_four_per_pass(engine, n_layers):
    """FP32-table layers go four to a YET pass (4 x 8-byte entries = one L2
    sector): every grouping (4 + 4 + 1, 2 + 1) gives the single-layer bits."""
    from paper_1412_4556_b300 import ARA_FP32_TABLE
    w = S.batched(n_layers=n_layers, n_trials=2_500, lam=150.0, catalog_size=120_000, n_pool=30)
    engine.load_yet_from(w.yet)
    first = engine.load_pool(w.pool)
    hs = [engine.define_layer([first + j for j in L.elts], L.occ_ret, L.occ_lim, L.agg_ret, L.agg_lim,
                              precision=ARA_FP32_TABLE) for L in w.layers]
    batch = engine.layers_ylt(hs)
    for i, (h, lay) in enumerate(zip(hs, w.layers)):
        single = engine.layer_ylt(h)
        np.testing.assert_array_equal(batch[i].view(np.uint64), single.view(np.uint64))
        o, pre = oracle.layer_ylt(w.yet, w.pool, lay, mode="memo")
        assert_reduced_parity(single, o, pre, what=f"layer {i}")
    rev = engine.layers_ylt(hs[::-1], n_trials=777)
    for i, h in enumerate(hs[::-1]):
        np.testing.assert_array_equal(rev[i], batch[hs.index(h)][:777])
