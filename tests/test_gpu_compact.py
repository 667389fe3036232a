"""The compact (sorted, difference-coded) id stream of ara_compact_yet: every
YLT it feeds is bit for bit the YLT of the stored layout, for single layers,
batched passes (pairs of FP64 layers, fours of FP32-table layers) and plans,
with trials that stay in the stored layout (long or sparse trials) mixed in;
the Year Event Loss Table keeps the stored order; a reload drops it."""
import math

import numpy as np
import pytest

import ara_synth as S
import oracle
from parity import assert_fp64_parity
from test_gpu_parity import LENGTHS, _custom_pool, _custom_yet

pytestmark = pytest.mark.gpu


@pytest.fixture
def engine():
    from paper_1412_4556_b300 import Engine
    e = Engine(0)
    yield e
    e.close()


def _layers(engine, first, precs):
    from paper_1412_4556_b300 import ARA_FP32_TABLE, ARA_FP64
    specs = [S.Layer([0, 1, 2, 3], 1e3, 5e6, 1e4, 1e8), S.Layer([2, 0], 0.0, math.inf, 0.0, math.inf),
             S.Layer([3, 2, 1], 5e5, 1e6, 2e6, 3e6), S.Layer([0, 2], 250.0, 2e7, 1.2345e-30, 7.77e-29 + 3e6),
             S.Layer([1, 3], 10.0, 1e7, 0.0, math.inf), S.Layer([0], 0.0, 1e6, 5e5, 2e8)]
    hs = [engine.define_layer([first + j for j in L.elts], L.occ_ret, L.occ_lim, L.agg_ret, L.agg_lim,
                              precision=ARA_FP32_TABLE if p else ARA_FP64)
          for L, p in zip(specs, precs)]
    return specs, hs


@pytest.mark.parametrize("catalog", [3, 2_049, 1_000_003, 2_000_000])
def test_compact_stream_is_bit_identical(engine, catalog):
    from paper_1412_4556_b300 import Plan
    sizes = [min(catalog, s) for s in (1, 300, 200_000, 7)]
    pool = _custom_pool(catalog, sizes, 21)
    hot = [0, catalog - 1, catalog // 2] + [int(x) for x in pool.ids[:50]]
    # ragged lengths around every tile edge, trials around the shared-memory
    # staging limit (1536 events) and longer (up to 20,000 events), and very
    # short trials (far-apart sorted ids)
    lengths = LENGTHS * 3 + [1535, 1536, 1537, 8192, 8193, 20_000, 2, 3, 9, 17] * 3
    yet = _custom_yet(catalog, lengths, catalog + 7, hot)
    engine.load_yet_from(yet)
    first = engine.load_pool(pool)
    specs, hs = _layers(engine, first, [0, 0, 1, 1, 1, 0])
    before = [engine.layer_ylt(h) for h in hs]
    batch_before = engine.layers_ylt(hs)
    yelt_before, omax_before = engine.layer_yelt(hs[0])
    engine.compact_yet()
    engine.compact_yet()  # a second call is a no-op
    for h, b in zip(hs, before):
        np.testing.assert_array_equal(engine.layer_ylt(h).view(np.uint64), b.view(np.uint64))
        n = 77
        np.testing.assert_array_equal(engine.layer_ylt(h, n_trials=n), b[:n])
    np.testing.assert_array_equal(engine.layers_ylt(hs).view(np.uint64), batch_before.view(np.uint64))
    np.testing.assert_array_equal(engine.layers_ylt(hs[::-1]), batch_before[::-1])
    with Plan(engine, hs, [10.0, 50.0]) as p:
        y = np.empty_like(batch_before)
        p.run(ylt_out=y)
    np.testing.assert_array_equal(y, batch_before)
    yelt, omax = engine.layer_yelt(hs[0])
    np.testing.assert_array_equal(yelt, yelt_before)
    np.testing.assert_array_equal(omax, omax_before)
    o, pre = oracle.layer_ylt(yet, pool, specs[0], mode="memo")
    assert_fp64_parity(before[0], o, pre)


def test_paper_shaped_compact_and_reload(engine):
    w = S.paper_scale(n_trials=20_000, catalog_size=2_000_000)
    lay = w.layers[0]
    engine.load_yet_from(w.yet)
    first = engine.load_pool(w.pool)
    h = engine.define_layer([first + j for j in lay.elts], lay.occ_ret, lay.occ_lim, lay.agg_ret, lay.agg_lim)
    ref = engine.layer_ylt(h)
    engine.compact_yet()
    np.testing.assert_array_equal(engine.layer_ylt(h), ref)
    # a reload drops the compact stream; the new YET prices correctly
    w2 = S.paper_scale(seed=99, n_trials=5_000, catalog_size=2_000_000)
    engine.load_yet_from(w2.yet)
    o, pre = oracle.layer_ylt(w2.yet, w.pool, lay, mode="memo")
    assert_fp64_parity(engine.layer_ylt(h), o, pre)
    engine.compact_yet()
    assert_fp64_parity(engine.layer_ylt(h), o, pre)


def test_compact_is_a_no_op_for_wide_catalogs(engine):
    catalog = 5_000_000
    pool = _custom_pool(catalog, [300, 20_000], 4)
    yet = _custom_yet(catalog, LENGTHS * 2, 3)
    engine.load_yet_from(yet)
    first = engine.load_pool(pool)
    h = engine.define_layer([first, first + 1], 100.0, 1e7, 1e3, 1e9)
    ref = engine.layer_ylt(h)
    engine.compact_yet()
    np.testing.assert_array_equal(engine.layer_ylt(h), ref)


def test_service_on_a_compacted_yet(engine):
    """Service batches price one-layer passes from the compact stream and
    multi-layer passes from the stored layout; every result equals the same
    request priced on the stored layout."""
    from paper_1412_4556_b300 import ARA_FP32_TABLE, ARA_FP64, Service
    w = S.batched(n_layers=1, n_trials=20_000, lam=300.0, catalog_size=300_000, n_pool=24)
    reqs = S.service_requests(n_requests=16, rate_per_s=1000.0, n_pool=24, trial_choices=(2_000, 20_000))
    rps = (10.0, 100.0)

    def run(compact):
        engine.load_yet_from(w.yet)
        if compact:
            engine.compact_yet()
        first = engine.load_pool(w.pool)
        with Service(engine, rps, slots=2, max_batch=4) as svc:
            ts = [svc.submit([first + j for j in rq.layer.elts], rq.layer.occ_ret, rq.layer.occ_lim,
                             rq.layer.agg_ret, rq.layer.agg_lim, rq.n_trials,
                             precision=ARA_FP32_TABLE if i % 2 else ARA_FP64, want_ylt=True)
                  for i, rq in enumerate(reqs)]
            return [svc.wait(t) for t in ts]

    stored, compacted = run(False), run(True)
    for a, b in zip(stored, compacted):
        assert a.ok and b.ok
        np.testing.assert_array_equal(b.ylt.view(np.uint64), a.ylt.view(np.uint64))
        np.testing.assert_array_equal(b.pml, a.pml)
        np.testing.assert_array_equal(b.tvar, a.tvar)
