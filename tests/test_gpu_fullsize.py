"""Full-size parity: every trial of the paper-scale workloads against the FP64
oracle, in the launch configurations the benchmark times.

* one layer over 16 ELTs, 1,000,000 trials x Poisson(1000) events (~1e9
  occurrences): the YLT from the compact id stream, every trial against the
  memoised oracle at relative 1e-12 (reading R9), and PML/TVaR at return
  periods 100/250/500 from the engine's YLT against the oracle's PML/TVaR
  from the oracle's YLT;
* 64 batched FP64 layers of 1-32 ELTs over the same YET shape: all
  64 x 1,000,000 trial losses from the plan (one CUDA graph) against the
  oracle, PML/TVaR of each layer likewise;
* the same 64 layers with FP32 tables: every trial at 1e-5 with a 1 USD
  floor, PML/TVaR within the largest per-trial error.

The oracle runs memoised Algorithm 1 (same bits as the literal loop) on all
host cores.  Each test prints its error report (pytest -s shows it).
"""
import json

import numpy as np
import pytest

import ara_synth as S
import oracle

pytestmark = pytest.mark.gpu


def _report(name, d):
    print(f"\n{name}: {json.dumps(d)}")


@pytest.fixture(scope="module")
def paper_full():
    w = S.paper_scale()
    o, pre = oracle.layer_ylt(w.yet, w.pool, w.layers[0], mode="memo")
    return w, o, pre


def test_paper_scale_every_trial(paper_full):
    """1,000,000 trials, one layer over 16 ELTs: every trial and PML/TVaR."""
    from paper_1412_4556_b300 import Engine
    w, o, pre = paper_full
    layer = w.layers[0]
    with Engine(0) as e:
        e.load_yet_from(w.yet)
        first = e.load_pool(w.pool)
        L = e.define_layer([first + j for j in layer.elts], layer.occ_ret, layer.occ_lim, layer.agg_ret,
                           layer.agg_lim)
        stored = e.layer_ylt(L)
        e.compact_yet()  # the benchmark prices from the compact id stream
        g = e.layer_ylt(L)
        pml_g, tvar_g = e.pml_tvar(g, w.return_periods)
        # the selection alone, on the oracle's own YLT
        pml_x, tvar_x = e.pml_tvar(o, w.return_periods)
    np.testing.assert_array_equal(g.view(np.uint64), stored.view(np.uint64))
    rep = oracle.compare_fp64(g, o, pre)
    assert rep["trials"] == 1_000_000
    assert rep["trials_over_r9_bar"] == 0, rep
    pml_o, tvar_o = oracle.pml_tvar(o, w.return_periods)
    pt = oracle.compare_pml_tvar(pml_g, tvar_g, pml_o, tvar_o, w.return_periods, g.size, rep["max_abs_err"])
    assert pt["within_bound"], pt
    np.testing.assert_array_equal(pml_x, pml_o)
    k = np.floor(g.size / np.asarray(w.return_periods))
    np.testing.assert_allclose(tvar_x, tvar_o, rtol=float((k.max() + 1) * 2.0 ** -53), atol=0)
    _report("config 1 YLT", rep)
    _report("config 1 PML/TVaR", pt)


@pytest.fixture(scope="module")
def batched_full():
    """The 64-layer workload and the oracle's YLTs of all its layers (shared
    by the FP64 and FP32-table tests)."""
    w = S.batched()
    o, pre = oracle.layers_ylt(w.yet, w.pool, w.layers, mode="memo")
    pml_o = np.empty((len(w.layers), len(w.return_periods)))
    tvar_o = np.empty_like(pml_o)
    for i in range(len(w.layers)):
        pml_o[i], tvar_o[i] = oracle.pml_tvar(o[i], w.return_periods)
    return w, o, pre, pml_o, tvar_o


def _plan_ylts(w, precision):
    from paper_1412_4556_b300 import Engine, Plan
    with Engine(0) as e:
        e.load_yet_from(w.yet)
        e.compact_yet()
        first = e.load_pool(w.pool)
        hs = [e.define_layer([first + j for j in L.elts], L.occ_ret, L.occ_lim, L.agg_ret, L.agg_lim,
                             precision=precision) for L in w.layers]
        y = np.empty((len(hs), w.yet.n_trials))
        with Plan(e, hs, w.return_periods, autotune=True) as plan:
            pml, tvar = plan.run(ylt_out=y)
        # the calls path gives the plan's bits
        y2 = e.layers_ylt(hs[:3])
    np.testing.assert_array_equal(y2.view(np.uint64), y[:3].view(np.uint64))
    return y, pml, tvar


def test_batched_64_fp64_layers_every_trial(batched_full):
    """64 FP64 layers x 1,000,000 trials from the plan, every value."""
    from paper_1412_4556_b300 import ARA_FP64
    w, o, pre, pml_o, tvar_o = batched_full
    y, pml, tvar = _plan_ylts(w, ARA_FP64)
    worst, over, plain_over, pt_ok = 0.0, 0, 0, True
    per_layer = []
    for i in range(len(w.layers)):
        rep = oracle.compare_fp64(y[i], o[i], pre[i])
        pt = oracle.compare_pml_tvar(pml[i], tvar[i], pml_o[i], tvar_o[i], w.return_periods, y.shape[1],
                                     rep["max_abs_err"])
        assert rep["trials_over_r9_bar"] == 0, (i, rep)
        assert pt["within_bound"], (i, pt)
        worst = max(worst, rep["max_rel_err_r9"])
        over += rep["trials_over_r9_bar"]
        plain_over += rep["trials_over_plain_bar"]
        per_layer.append(max(pt["pml_rel_err"] + pt["tvar_rel_err"]))
    _report("config 2 YLTs", {"layers": len(w.layers), "trials_per_layer": int(y.shape[1]),
                              "max_rel_err_r9": worst, "trials_over_r9_bar": over,
                              "trials_over_plain_bar": plain_over,
                              "max_rel_pml_tvar_err": max(per_layer)})


def test_batched_64_fp32_table_layers_every_trial(batched_full):
    """The same 64 layers with FP32 tables (config 3) against the FP64 oracle:
    every trial within 1e-5 (1 USD floor), PML/TVaR within the largest
    per-trial error."""
    from paper_1412_4556_b300 import ARA_FP32_TABLE
    w, o, pre, pml_o, tvar_o = batched_full
    y, pml, tvar = _plan_ylts(w, ARA_FP32_TABLE)
    worst, over, plain_over, pt_worst = 0.0, 0, 0, 0.0
    for i in range(len(w.layers)):
        rep = oracle.compare_reduced(y[i], o[i], pre[i])
        pt = oracle.compare_pml_tvar(pml[i], tvar[i], pml_o[i], tvar_o[i], w.return_periods, y.shape[1],
                                     rep["max_abs_err"])
        assert rep["trials_over_bar"] == 0, (i, rep)
        assert pt["within_bound"], (i, pt)
        worst = max(worst, rep["max_err_over_bar"])
        over += rep["trials_over_bar"]
        plain_over += rep["trials_over_plain_bar"]
        pt_worst = max(pt_worst, max(pt["pml_rel_err"] + pt["tvar_rel_err"]))
    _report("config 3 YLTs", {"layers": len(w.layers), "trials_per_layer": int(y.shape[1]),
                              "max_err_over_bar": worst, "trials_over_bar": over,
                              "trials_over_plain_bar": plain_over, "max_rel_pml_tvar_err": pt_worst})
