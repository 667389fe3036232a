"""Pricing plans (one CUDA graph per fixed list of layers, with the launch-shape
autotuner) against the direct calls they replace."""
import numpy as np
import pytest

import ara_synth as S
import oracle
from parity import assert_fp64_parity

pytestmark = pytest.mark.gpu

RPS = [10.0, 100.0, 250.0]


@pytest.fixture
def engine():
    from paper_1412_4556_b300 import Engine
    e = Engine(0)
    yield e
    e.close()


def setup(engine, n_layers=7, n_trials=4_000, precisions=None):
    from paper_1412_4556_b300 import ARA_FP32_TABLE, ARA_FP64
    w = S.batched(n_layers=n_layers, n_trials=n_trials, lam=250.0, catalog_size=250_000, n_pool=40)
    engine.load_yet_from(w.yet)
    first = engine.load_pool(w.pool)
    precisions = precisions or [ARA_FP64 if i % 2 == 0 else ARA_FP32_TABLE for i in range(n_layers)]
    hs = [engine.define_layer([first + j for j in L.elts], L.occ_ret, L.occ_lim, L.agg_ret, L.agg_lim,
                              precision=p) for L, p in zip(w.layers, precisions)]
    return w, hs, precisions


@pytest.mark.parametrize("autotune", [True, False])
def test_plan_equals_direct_calls(engine, autotune):
    from paper_1412_4556_b300 import ARA_FP64, Plan
    w, hs, precs = setup(engine)
    direct = engine.layers_ylt(hs)
    pml_d, tvar_d = engine.pml_tvar_batch(direct, RPS)
    with Plan(engine, hs, RPS, autotune=autotune) as plan:
        for _ in range(2):
            y = np.empty_like(direct)
            pml, tvar = plan.run(ylt_out=y)
            np.testing.assert_array_equal(y.view(np.uint64), direct.view(np.uint64))
            np.testing.assert_array_equal(pml, pml_d)
            np.testing.assert_array_equal(tvar, tvar_d)
        passes = plan.passes()
        # one replay: the folds' clear and batch, one launch per pass (the
        # folds write each multi-layer pass's table: no interleave), selection
        assert plan.kernel_launches() == 2 + len(passes) + 10
    # every layer in exactly one pass, of its own entry width
    pos = sorted(i for *_, ps in passes for i in ps)
    assert pos == list(range(len(hs)))
    for eb, g, lpt, u, pf, th, ps in passes:
        assert len(ps) == g and all((eb == 16) == (precs[i] == ARA_FP64) for i in ps)
        assert (eb, g) in ((16, 1), (16, 2), (8, 1), (8, 2), (8, 4))
        assert lpt in (16, 32) and u in (1, 2) and pf in (0, 1) and th in (768, 1024)
    if not autotune:
        # the largest groups: 4 FP64 layers -> 2 passes of 2; 3 FP32-table layers -> 2 + 1
        assert sorted((eb, g) for eb, g, *_ in passes) == [(8, 1), (8, 2), (16, 2), (16, 2)]
    for i, (lay, p) in enumerate(zip(w.layers, precs)):
        if p == ARA_FP64 and i < 3:
            o, pre = oracle.layer_ylt(w.yet, w.pool, lay, mode="memo")
            assert_fp64_parity(direct[i], o, pre, what=f"layer {i}")


def test_plan_with_the_interleave_step(engine, monkeypatch):
    """The path a plan takes when its passes' tables cannot be allocated: the
    layers fold into their own tables and the graph interleaves them; same
    bits as the direct calls."""
    from paper_1412_4556_b300 import Plan
    monkeypatch.setenv("ARA_PLAN_INTERLEAVE", "1")
    w, hs, precs = setup(engine)
    direct = engine.layers_ylt(hs)
    pml_d, tvar_d = engine.pml_tvar_batch(direct, RPS)
    with Plan(engine, hs, RPS, autotune=False) as plan:
        y = np.empty_like(direct)
        pml, tvar = plan.run(ylt_out=y)
        passes = plan.passes()
        multi = sum(1 for _, g, *_ in passes if g > 1)
        assert multi > 0
        assert plan.kernel_launches() == 2 + len(passes) + multi + 10
    np.testing.assert_array_equal(y.view(np.uint64), direct.view(np.uint64))
    np.testing.assert_array_equal(pml, pml_d)
    np.testing.assert_array_equal(tvar, tvar_d)


def test_plan_device_output_prefix_and_streams(engine):
    import torch
    from paper_1412_4556_b300 import Plan
    w, hs, _ = setup(engine, n_layers=5)
    n = 1_234
    direct = engine.layers_ylt(hs, n_trials=n)
    s = torch.cuda.Stream()
    with Plan(engine, hs, [10.0], n_trials=n) as plan:
        out = torch.empty((len(hs), n), dtype=torch.float64, device="cuda")
        plan.run(ylt_out=out, stream=s, want_pml=False)
        s.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), direct)


def test_plan_invalidated_by_release_and_reload(engine):
    from paper_1412_4556_b300 import AraError, Plan
    w, hs, _ = setup(engine, n_layers=3)
    plan = Plan(engine, hs, RPS)
    plan.run()
    engine.release_layer(hs[1])
    with pytest.raises(AraError) as ei:
        plan.run()
    assert ei.value.name == "ARA_E_STATE"
    plan.close()
    plan2 = Plan(engine, [hs[0], hs[2]], RPS)
    plan2.run()
    engine.load_yet_from(w.yet)  # a reload invalidates every plan
    with pytest.raises(AraError) as ei:
        plan2.run()
    assert ei.value.name == "ARA_E_STATE"
    with pytest.raises(AraError) as ei:
        Plan(engine, [hs[0], 99], RPS)
    assert ei.value.name == "ARA_E_NOT_FOUND"
    # closing the engine closes its live plans
    Plan(engine, [hs[0]], RPS)
    engine.close()
    assert not engine._plans


def test_plan_with_many_layers_groups_each_layer_once(engine):
    """200 layers (beyond 128 the grouping compares layers on a sample of the
    bitmap words): every layer in exactly one pass, the plan's bits equal the
    direct call's, and the first FP64 layers match the oracle."""
    from paper_1412_4556_b300 import ARA_FP64, Plan
    n = 200
    w, hs, precs = setup(engine, n_layers=n, n_trials=1_500)
    direct = engine.layers_ylt(hs)
    with Plan(engine, hs, RPS, autotune=False) as plan:
        y = np.empty_like(direct)
        plan.run(ylt_out=y)
        passes = plan.passes()
    np.testing.assert_array_equal(y.view(np.uint64), direct.view(np.uint64))
    pos = sorted(i for *_, ps in passes for i in ps)
    assert pos == list(range(n))
    # 100 FP64 layers in 50 pairs, 100 FP32-table layers in 25 fours
    assert sum(1 for eb, g, *rest in passes if eb == 16 and g == 2) == 50
    assert sum(1 for eb, g, *rest in passes if eb == 8 and g == 4) == 25
    for i in [i for i, p in enumerate(precs) if p == ARA_FP64][:2]:
        o, pre = oracle.layer_ylt(w.yet, w.pool, w.layers[i], mode="memo")
        assert_fp64_parity(direct[i], o, pre, what=f"layer {i}")
