"""Seeded random instances through every pricing path, against the oracle.

Each instance draws a catalog size (including 1, the 21-bit packing boundary
and catalogs above it), ELTs of random sizes (including empty ones) with
lognormal losses of random scale plus exact zeros and very large losses,
deductibles and limits including 0 and +inf, layer terms including 0, +inf
and retentions off any fixed-point grid, and a YET of random trial lengths
(empty trials, long trials and repeated hot events).  Every layer is priced
through ara_layer_ylt on the stored and on the compact id stream, through
ara_layers_ylt and a plan (FP64 and FP32-table layers mixed), and through the
YELT; each result is checked against the FP64 oracle at its precision's bar
(reading R9), and PML/TVaR against the oracle's.
"""
import math

import numpy as np
import pytest

import ara_synth as S
import oracle

pytestmark = pytest.mark.gpu

CATALOGS = [1, 2, 37, 4_096, 65_537, (1 << 21) - 2, (1 << 21) - 1, 1 << 21, 3_000_001]


def _instance(seed):
    rng = np.random.default_rng(seed)
    catalog = int(CATALOGS[seed % len(CATALOGS)])
    n_elts = int(rng.integers(1, 9))
    sizes = [int(min(catalog, rng.choice([0, 1, 5, 300, 5_000, 40_000]))) for _ in range(n_elts)]
    off = np.zeros(n_elts + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    ids, losses = [], []
    for s in sizes:
        ids.append(rng.choice(catalog, s, replace=False).astype(np.int32))
        lo = rng.lognormal(rng.uniform(2, 14), rng.uniform(0.1, 2.5), s)
        if s:
            lo[rng.random(s) < 0.05] = 0.0                  # exact zero losses
            lo[rng.random(s) < 0.01] *= 1e6                 # very large ones
        losses.append(lo)
    ded = rng.choice([0.0, 10.0, 5e3, 1e5], n_elts)
    lim = rng.choice([math.inf, 1e6, 5e7, 1e12, 0.0], n_elts, p=[0.4, 0.2, 0.2, 0.15, 0.05])
    pool = S.ELTPool(off, np.concatenate(ids) if ids else np.zeros(0, np.int32),
                     np.concatenate(losses) if losses else np.zeros(0), ded, lim)
    n_trials = int(rng.integers(1, 1_500))
    lam = float(rng.choice([0.5, 10.0, 200.0]))
    counts = rng.poisson(lam, n_trials).astype(np.int64)
    counts[rng.random(n_trials) < 0.01] = int(rng.integers(2_000, 12_000))  # long trials
    counts[rng.random(n_trials) < 0.05] = 0                                # empty trials
    yoff = np.zeros(n_trials + 1, np.int64)
    yoff[1:] = np.cumsum(counts)
    yids = rng.integers(0, catalog, int(yoff[-1])).astype(np.int32)
    if yids.size and sizes[0]:
        hot = pool.ids[:min(3, sizes[0])]
        pos = rng.integers(0, yids.size, min(yids.size, 200))
        yids[pos] = hot[rng.integers(0, hot.size, pos.size)]
    yet = S.YET(catalog, yoff, yids)
    layers = []
    for _ in range(int(rng.integers(1, 6))):
        k = int(rng.integers(1, n_elts + 1))
        elts = [int(x) for x in rng.choice(n_elts, k, replace=False)]
        occ_ret = float(rng.choice([0.0, 1.0, 1e4, 1e5, 3.3e-7]))
        occ_lim = float(rng.choice([math.inf, 1e6, 2e7, 0.5]))
        agg_ret = float(rng.choice([0.0, 5e5, 1e7, 1.2345e-30]))
        agg_lim = float(rng.choice([math.inf, 1e8, 1e9, 7.77e-29 + 3e6]))
        layers.append(S.Layer(elts, occ_ret, occ_lim, agg_ret, agg_lim))
    return yet, pool, layers


def _check(g, o, pre, fp32, what):
    rep = (oracle.compare_reduced if fp32 else oracle.compare_fp64)(g, o, pre)
    over = rep["trials_over_bar"] if fp32 else rep["trials_over_r9_bar"]
    assert over == 0, (what, rep)
    return rep


@pytest.mark.parametrize("seed", range(120))
def test_random_instance_every_path(seed):
    from paper_1412_4556_b300 import ARA_FP32_TABLE, ARA_FP64, Engine, Plan
    yet, pool, layers = _instance(seed)
    precs = [ARA_FP32_TABLE if (seed + i) % 3 == 2 else ARA_FP64 for i in range(len(layers))]
    rps = [1.0, 2.0, 7.0] if yet.n_trials >= 7 else [1.0]
    with Engine(0) as e:
        e.load_yet_from(yet)
        first = e.load_pool(pool)
        hs = [e.define_layer([first + j for j in L.elts], L.occ_ret, L.occ_lim, L.agg_ret, L.agg_lim, precision=p)
              for L, p in zip(layers, precs)]
        stored = [e.layer_ylt(h) for h in hs]
        batch = e.layers_ylt(hs)
        yelts = [e.layer_yelt(h) for h in hs]
        e.compact_yet()
        compact = [e.layer_ylt(h) for h in hs]
        with Plan(e, hs, rps, autotune=(seed % 2 == 0)) as plan:
            y_plan = np.empty((len(hs), yet.n_trials))
            pml_plan, tvar_plan = plan.run(ylt_out=y_plan)
    for i, (L, p) in enumerate(zip(layers, precs)):
        fp32 = p == ARA_FP32_TABLE
        # every path gives the same bits
        for name, y in (("batched", batch[i]), ("compact", compact[i]), ("plan", y_plan[i])):
            np.testing.assert_array_equal(y.view(np.uint64), stored[i].view(np.uint64), err_msg=f"{name} layer {i}")
        o, pre = oracle.layer_ylt(yet, pool, L, mode="memo")
        rep = _check(stored[i], o, pre, fp32, f"seed {seed} layer {i}")
        assert np.all(stored[i] >= 0.0) and np.all(stored[i] <= L.agg_lim)
        # the YELT's trial maxima and increments
        inc, occ_max = yelts[i]
        o_inc, out_off, o_max, _, _ = oracle.layer_yelt(yet, pool, L)
        tol_rel, tol_floor = (1e-5, 1.0) if fp32 else (1e-12, 0.0)
        trial_of = np.repeat(np.arange(yet.n_trials), np.diff(out_off))
        assert np.all(np.abs(inc - o_inc) <= np.maximum(tol_rel * pre[trial_of], tol_floor)), f"seed {seed} yelt {i}"
        assert np.all(np.abs(occ_max - o_max) <= np.maximum(tol_rel * pre, tol_floor))
        # PML/TVaR of the plan against the oracle's
        p_o, t_o = oracle.pml_tvar(o, rps)
        pt = oracle.compare_pml_tvar(pml_plan[i], tvar_plan[i], p_o, t_o, rps, yet.n_trials, rep["max_abs_err"])
        assert pt["within_bound"], (seed, i, pt)
