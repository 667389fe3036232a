"""Batched layers (several layers in one pass over the YET) against the
single-layer path and the oracle, and batched PML/TVaR."""
import numpy as np
import pytest

import ara_synth as S
import oracle
from parity import assert_fp64_parity

pytestmark = pytest.mark.gpu


@pytest.fixture
def engine():
    from paper_1412_4556_b300 import Engine
    e = Engine(0)
    yield e
    e.close()


def define_all(engine, w):
    first = engine.load_pool(w.pool)
    return [engine.define_layer([first + j for j in L.elts], L.occ_ret, L.occ_lim, L.agg_ret,
                                L.agg_lim) for L in w.layers]


@pytest.mark.parametrize("n_layers", [1, 2, 7])
def test_batched_equals_single_layer_and_oracle(engine, n_layers):
    w = S.batched(n_layers=n_layers, n_trials=3_000, lam=300.0, catalog_size=200_000, n_pool=40)
    engine.load_yet_from(w.yet)
    hs = define_all(engine, w)
    batch = engine.layers_ylt(hs)
    assert batch.shape == (n_layers, w.yet.n_trials)
    for i, (h, lay) in enumerate(zip(hs, w.layers)):
        single = engine.layer_ylt(h)
        np.testing.assert_array_equal(batch[i].view(np.uint64), single.view(np.uint64))
        o, pre = oracle.layer_ylt(w.yet, w.pool, lay, mode="memo")
        assert_fp64_parity(batch[i], o, pre, what=f"layer {i}")
    # a prefix, and the reversed order (different pairs)
    pre_batch = engine.layers_ylt(hs[::-1], n_trials=1234)
    for i, h in enumerate(hs[::-1]):
        np.testing.assert_array_equal(pre_batch[i], batch[hs.index(h)][:1234])


def test_batched_device_output_and_pml_tvar(engine):
    import torch
    w = S.batched(n_layers=5, n_trials=4_000, lam=200.0, catalog_size=100_000, n_pool=30)
    engine.load_yet_from(w.yet)
    hs = define_all(engine, w)
    out = torch.empty((len(hs), w.yet.n_trials), dtype=torch.float64, device="cuda")
    engine.layers_ylt(hs, out=out)
    torch.cuda.synchronize()
    host = engine.layers_ylt(hs)
    np.testing.assert_array_equal(out.cpu().numpy(), host)
    rps = [10.0, 100.0, 400.0]
    pml_b, tvar_b = engine.pml_tvar_batch(out, rps)
    for i in range(len(hs)):
        p, t = engine.pml_tvar(host[i], rps)
        np.testing.assert_array_equal(pml_b[i], p)
        np.testing.assert_array_equal(tvar_b[i], t)
        po, to = oracle.pml_tvar(host[i], rps)
        np.testing.assert_array_equal(p, po)
        np.testing.assert_allclose(t, to, rtol=1e-13, atol=0)


def test_batched_rejects_bad_handles(engine):
    from paper_1412_4556_b300 import AraError
    w = S.batched(n_layers=2, n_trials=100, lam=20.0, catalog_size=100_000, n_pool=10)
    engine.load_yet_from(w.yet)
    hs = define_all(engine, w)
    with pytest.raises(AraError) as ei:
        engine.layers_ylt([hs[0], 99])
    assert ei.value.name == "ARA_E_NOT_FOUND"
    with pytest.raises(AraError):
        engine.layers_ylt(hs, n_trials=101)
