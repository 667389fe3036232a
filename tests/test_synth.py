"""Seeded input generator: determinism, shapes and the documented distributions."""
import numpy as np

import ara_synth as S


def test_yet_is_deterministic_and_thread_independent():
    a = S.make_yet(7, 1000, 500, 30.0, threads=1)
    b = S.make_yet(7, 1000, 500, 30.0, threads=4)
    np.testing.assert_array_equal(a.offsets, b.offsets)
    np.testing.assert_array_equal(a.ids, b.ids)
    np.testing.assert_array_equal(a.ts, b.ts)
    c = S.make_yet(8, 1000, 500, 30.0)
    assert not np.array_equal(a.ids[:100], c.ids[:100])


def test_yet_layout():
    y = S.make_yet(1, 10_000, 2_000, 100.0)
    assert y.offsets[0] == 0 and np.all(np.diff(y.offsets) >= 0)
    assert y.ids.dtype == np.int32 and y.ids.min() >= 0 and y.ids.max() < 10_000
    assert abs(np.diff(y.offsets).mean() - 100.0) < 2.0
    for t in range(0, 2_000, 97):
        seg = y.ts[y.offsets[t]:y.offsets[t + 1]]
        assert np.all(np.diff(seg) >= 0) and (seg.size == 0 or (seg[0] >= 0 and seg[-1] < 365))
    # uniform over the year: mean 182.5, each month-sized bin about 1/12
    assert abs(float(y.ts.mean()) - 182.5) < 1.0
    h, _ = np.histogram(y.ts, bins=12, range=(0.0, 365.0))
    assert np.all(np.abs(h / h.sum() - 1.0 / 12.0) < 0.005)


def test_elt_pool_distinct_ids_and_terms():
    w = S.tiny()
    p = w.pool
    assert p.n_elts == 4
    for j in range(4):
        ids, losses = p.elt(j)
        assert len(np.unique(ids)) == ids.size == 1000
        assert np.all(losses > 0)
    # lognormal(12, 1.5): the median of log-losses is near 12
    assert abs(np.median(np.log(p.losses)) - 12.0) < 0.15
    assert w.layers[0].occ_ret == 1e5 and w.layers[0].agg_lim == 1e8


def test_batched_layers_and_requests():
    w = S.batched(n_layers=8, n_trials=200, lam=20.0, catalog_size=50_000, n_pool=40)
    assert len(w.layers) == 8
    for L in w.layers:
        assert 1 <= len(L.elts) <= 32 and len(set(L.elts)) == len(L.elts)
        assert 1e4 <= L.occ_ret <= 1e6 and 1e7 <= L.agg_lim <= 1e9
    reqs = S.service_requests(n_requests=50, n_pool=40)
    assert all(2 <= len(r.layer.elts) <= 32 for r in reqs)
    assert all(r.n_trials in (100_000, 250_000, 1_000_000) for r in reqs)
    assert np.all(np.diff([r.arrival_s for r in reqs]) >= 0)
