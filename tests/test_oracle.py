"""Pins for the FP64 oracle (CPU only).

The oracle is checked against things other than itself:
  * a hand-worked instance derived from the paper's definitions
    (tests/golden/hand_worked.json, Section III, Algorithm 1),
  * closed forms (a trial repeating one event; neutral terms),
  * a library routine (numpy bincount) for the special case where every
    financial term is neutral and the YLT is a plain segmented sum,
  * library sorting for PML/TVaR,
  * invariants the method fixes (bounds, monotonicity, permutation
    invariance, telescoping of the aggregate increments),
  * brute force over every trial of a 3-event catalog against exact
    rational arithmetic of the total-then-clamp form.
"""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from hypothesis import given, settings, strategies as st, HealthCheck

import oracle
from ara_synth import YET, ELTPool, Layer

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_worked.json")


def _f(x):
    return math.inf if x == "inf" else float(x)


def hand_instance(neutral=False):
    g = json.load(open(GOLDEN))
    ids, losses, off, ded, lim = [], [], [0], [], []
    for e in g["elts"]:
        ids += e["ids"]
        losses += e["losses"]
        off.append(len(ids))
        ded.append(e["deductible"])
        lim.append(e["limit"])
    if neutral:
        n = g["neutral_terms"]
        ded = [n["deductible"]] * len(ded)
        lim = [_f(n["limit"])] * len(lim)
    pool = ELTPool(np.array(off, np.int64), np.array(ids, np.int32), np.array(losses),
                   np.array(ded), np.array(lim, dtype=np.float64))
    L = g["layer"]
    if neutral:
        n = g["neutral_terms"]
        layer = Layer(L["elts"], n["occ_ret"], _f(n["occ_lim"]), n["agg_ret"], _f(n["agg_lim"]))
    else:
        layer = Layer(L["elts"], L["occ_ret"], L["occ_lim"], L["agg_ret"], L["agg_lim"])
    trials = g["trials"]
    offsets = np.zeros(len(trials) + 1, np.int64)
    offsets[1:] = np.cumsum([len(t) for t in trials])
    yet = YET(g["catalog_size"], offsets, np.array([e for t in trials for e in t], np.int32))
    return g, yet, pool, layer


def test_hand_worked_ylt():
    g, yet, pool, layer = hand_instance()
    for mode in ("literal", "memo"):
        ylt, pre = oracle.layer_ylt(yet, pool, layer, mode=mode, threads=2)
        assert ylt.tolist() == g["ylt"]
        assert pre.tolist() == g["presum"]


def test_hand_worked_event_table():
    g, yet, pool, layer = hand_instance()
    assert oracle.event_table(3, pool, layer).tolist() == g["event_table"]


def test_hand_worked_trace():
    g, yet, pool, layer = hand_instance()
    occ, agg, inc, tl, ps = oracle.trial_trace(3, np.array(g["trials"][0]), pool, layer)
    t = g["trace_trial0"]
    assert occ.tolist() == t["occ"]
    assert agg.tolist() == t["agg"]
    assert inc.tolist() == t["inc"]
    assert tl == g["ylt"][0] and ps == g["presum"][0]


def test_hand_worked_neutral_terms():
    g, yet, pool, layer = hand_instance(neutral=True)
    ylt, _ = oracle.layer_ylt(yet, pool, layer)
    assert ylt[0] == g["neutral_terms"]["ylt_trial0"]


def test_hand_worked_pml_tvar():
    g = json.load(open(GOLDEN))["pml_tvar"]
    pml, tvar = oracle.pml_tvar(np.array(g["ylt"]), g["return_periods"])
    assert pml.tolist() == g["pml"]
    assert tvar.tolist() == g["tvar"]


def test_pml_tvar_rejects_bad_return_periods():
    with pytest.raises(oracle.OracleError):
        oracle.pml_tvar(np.ones(10), [20.0])     # floor(10/20) = 0
    with pytest.raises(oracle.OracleError):
        oracle.pml_tvar(np.ones(10), [0.5])      # RP < 1
    with pytest.raises(oracle.OracleError):
        oracle.pml_tvar(np.ones(10), [float("nan")])


def _random_instance(seed, catalog=500, n_trials=300, lam=40, n_elts=4, elt_size=120,
                     integer=False, neutral=False):
    rng = np.random.default_rng(seed)
    counts = rng.poisson(lam, n_trials)
    counts[:3] = [0, 1, 0]                     # empty and single-event trials
    offsets = np.zeros(n_trials + 1, np.int64)
    offsets[1:] = np.cumsum(counts)
    ids = rng.integers(0, catalog, offsets[-1]).astype(np.int32)
    e_ids, e_loss, e_off = [], [], [0]
    for j in range(n_elts):
        e_ids.append(rng.choice(catalog, elt_size, replace=False))
        l = rng.lognormal(8, 1.5, elt_size)
        e_loss.append(np.round(l) if integer else l)
        e_off.append(e_off[-1] + elt_size)
    ded = np.round(rng.uniform(0, 2000, n_elts)) if not neutral else np.zeros(n_elts)
    lim = np.round(rng.uniform(5e3, 5e4, n_elts)) if not neutral else np.full(n_elts, np.inf)
    pool = ELTPool(np.array(e_off, np.int64), np.concatenate(e_ids).astype(np.int32),
                   np.concatenate(e_loss), ded, lim)
    if neutral:
        layer = Layer(list(range(n_elts)), 0.0, np.inf, 0.0, np.inf)
    else:
        layer = Layer(list(range(n_elts)), 500.0, 3e4, 2e4, 2e5)
    return YET(catalog, offsets, ids), pool, layer


def _dat_sum(pool, layer, catalog):
    """Raw combined loss per event via numpy.add.at (terms neutral)."""
    raw = np.zeros(catalog)
    for j in layer.elts:
        ids, losses = pool.elt(j)
        np.add.at(raw, ids, losses)
    return raw


def test_neutral_terms_reduce_to_segmented_sum():
    """With zero retentions and infinite limits the YLT is a segmented sum of
    raw event losses: numpy.bincount over the trial index of each occurrence."""
    yet, pool, layer = _random_instance(1, neutral=True)
    raw = _dat_sum(pool, layer, yet.catalog_size)
    trial_of = np.repeat(np.arange(yet.n_trials), np.diff(yet.offsets))
    ref = np.bincount(trial_of, weights=raw[yet.ids], minlength=yet.n_trials)
    for mode in ("literal", "memo"):
        ylt, pre = oracle.layer_ylt(yet, pool, layer, mode=mode)
        np.testing.assert_allclose(ylt, ref, rtol=1e-13, atol=0)
        np.testing.assert_array_equal(ylt, pre)


def test_mean_trial_loss_with_neutral_layer_terms_is_poisson_mean_times_catalog_mean():
    """Statistical sanity on the tiny workload: with neutral occurrence and
    aggregate terms a trial's loss sums about Poisson(100) uniform draws of
    the per-event combined ELT loss C, so the mean over 1,000 trials lies
    within a few standard errors of 100 x mean(C) (C computed here with
    NumPy from the ELTs, not by the oracle)."""
    import ara_synth as S
    w = S.tiny()
    pool = w.pool
    layer = Layer(w.layers[0].elts, 0.0, math.inf, 0.0, math.inf)
    c = np.zeros(w.yet.catalog_size)
    for j in layer.elts:
        a, b = pool.offsets[j], pool.offsets[j + 1]
        c[pool.ids[a:b]] += np.minimum(np.maximum(pool.losses[a:b] - pool.deductibles[j], 0.0), pool.limits[j])
    ylt, _ = oracle.layer_ylt(w.yet, pool, layer)
    expect = 100.0 * c.mean()
    stderr = math.sqrt(100.0 * np.mean(c * c) / ylt.size)
    assert abs(ylt.mean() - expect) < 5.0 * stderr, (ylt.mean(), expect, stderr)
    # and the draws themselves average lambda per trial
    assert abs(np.diff(w.yet.offsets).mean() - 100.0) < 5.0 * math.sqrt(100.0 / ylt.size)


def test_literal_and_memo_modes_are_bit_identical():
    yet, pool, layer = _random_instance(2)
    a, pa = oracle.layer_ylt(yet, pool, layer, mode="literal", threads=3)
    b, pb = oracle.layer_ylt(yet, pool, layer, mode="memo", threads=1)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(pa, pb)


def test_trial_subset_matches_full_run():
    yet, pool, layer = _random_instance(3)
    full, _ = oracle.layer_ylt(yet, pool, layer)
    sel = np.array([7, 0, 299, 3, 3], np.int64)
    sub, _ = oracle.layer_ylt(yet, pool, layer, trials=sel)
    np.testing.assert_array_equal(sub, full[sel])


def test_many_layer_call_equals_one_call_per_layer():
    """The many-layer entry (the YET checked once, each layer's memo built on
    several threads) gives each layer the bits of its own call, whatever the
    thread count, with the hand-worked layer among them."""
    yet, pool, layer = _random_instance(4, catalog=70_000, n_trials=200)
    other = Layer([2, 0], 100.0, 1e4, 0.0, 5e4)
    g, hy, hp, hl = hand_instance()
    layers = [layer, other, Layer([1], 0.0, math.inf, 0.0, math.inf)]
    y, p = oracle.layers_ylt(yet, pool, layers, threads=5)
    assert y.shape == (3, yet.n_trials)
    for i, L in enumerate(layers):
        a, pa = oracle.layer_ylt(yet, pool, L, mode="literal", threads=2)
        np.testing.assert_array_equal(y[i].view(np.uint64), a.view(np.uint64))
        np.testing.assert_array_equal(p[i].view(np.uint64), pa.view(np.uint64))
    sel = np.array([5, 1, 199], np.int64)
    ys, _ = oracle.layers_ylt(yet, pool, layers, trials=sel, mode="literal", threads=1)
    np.testing.assert_array_equal(ys, y[:, sel])
    hy_out, _ = oracle.layers_ylt(hy, hp, [hl, hl])
    assert hy_out[0].tolist() == g["ylt"] and hy_out[1].tolist() == g["ylt"]


def test_comparison_forms():
    """The R9 gate divides by max(|o|, S_o); the plain form by |o|; the
    reduced-precision gate is max(1e-5 max(|o|, S_o), 1 USD)."""
    o = np.array([0.0, 1.0, 100.0, 0.0])
    pre = np.array([0.0, 1e6, 100.0, 5.0])
    g = np.array([0.0, 1.0 + 1e-7, 100.0, 1e-12])
    r = oracle.compare_fp64(g, o, pre)
    assert r["trials_over_r9_bar"] == 0             # 1e-7 / 1e6 and 1e-12 / 5 pass the gate
    assert r["trials_over_plain_bar"] == 2          # 1e-7 / 1 and 1e-12 / 0 fail the plain form
    assert r["bitwise_equal_trials"] == 2
    r = oracle.compare_fp64(np.array([1.0]), np.array([0.0]), np.array([0.0]))
    assert r["trials_over_r9_bar"] == 1             # a loss where the oracle has no sum at all
    q = oracle.compare_reduced(np.array([0.5, 1e6 + 20.0, 3.0]), np.array([0.0, 1e6, 0.0]),
                               np.array([0.0, 1e6, 4e6]))
    assert q["trials_over_bar"] == 1                # 20 USD > 1e-5 * 1e6; 3 USD <= 1e-5 * 4e6
    assert q["trials_over_plain_bar"] == 2
    pt = oracle.compare_pml_tvar([10.0], [12.0], [10.5], [12.0], [100.0], 1000, 0.5)
    assert pt["within_bound"]
    pt = oracle.compare_pml_tvar([10.0], [12.0], [10.6], [12.0], [100.0], 1000, 0.5)
    assert not pt["within_bound"]


def test_closed_form_repeated_event():
    """A trial that repeats one event n times: loss = clamp(n*c - AggR, 0, AggL),
    with c the event's occurrence-net loss (integers, so exact)."""
    g, _, pool, layer = hand_instance()
    c = g["event_table"]
    for e in range(3):
        for n in range(0, 9):
            yet = YET(3, np.array([0, n], np.int64), np.full(n, e, np.int32))
            ylt, _ = oracle.layer_ylt(yet, pool, layer)
            want = min(max(n * c[e] - layer.agg_ret, 0.0), layer.agg_lim)
            assert ylt[0] == want, (e, n)


def test_pml_tvar_against_numpy_sort():
    rng = np.random.default_rng(5)
    y = rng.lognormal(10, 2, 10_000)
    y[:50] = 0.0
    y[50:80] = 7.5                              # ties
    rps = [1.0, 2.0, 100.0, 250.0, 500.0, 3.3]
    pml, tvar = oracle.pml_tvar(y, rps)
    s = np.sort(y)[::-1]
    for r, p, t in zip(rps, pml, tvar):
        k = int(math.floor(len(y) / r))
        assert p == s[k - 1]
        assert t == pytest.approx(math.fsum(s[:k]) / k, rel=1e-13)


# ---------------------------------------------------------------- invariants
small = dict(max_examples=60, deadline=None, suppress_health_check=[HealthCheck.too_slow])


@st.composite
def integer_instances(draw):
    catalog = draw(st.integers(1, 12))
    n_elts = draw(st.integers(1, 4))
    e_ids, e_loss, e_off = [], [], [0]
    for _ in range(n_elts):
        k = draw(st.integers(0, catalog))
        ids = draw(st.permutations(list(range(catalog))))[:k]
        e_ids += ids
        e_loss += [float(draw(st.integers(0, 1000))) for _ in ids]
        e_off.append(len(e_ids))
    ded = [float(draw(st.integers(0, 300))) for _ in range(n_elts)]
    lim = [float(draw(st.sampled_from([0, 50, 200, 700, 10**6]))) for _ in range(n_elts)]
    trials = draw(st.lists(st.lists(st.integers(0, catalog - 1), max_size=10), min_size=1,
                           max_size=8))
    terms = [float(draw(st.integers(0, 500))) for _ in range(4)]
    pool = ELTPool(np.array(e_off, np.int64), np.array(e_ids, np.int32),
                   np.array(e_loss, dtype=np.float64), np.array(ded), np.array(lim))
    layer = Layer(list(range(n_elts)), terms[0], terms[1] + 1.0, terms[2], terms[3] + 1.0)
    off = np.zeros(len(trials) + 1, np.int64)
    off[1:] = np.cumsum([len(t) for t in trials])
    yet = YET(catalog, off, np.array([e for t in trials for e in t], np.int32))
    return yet, pool, layer


def _with(layer, **kw):
    d = dict(elts=list(layer.elts), occ_ret=layer.occ_ret, occ_lim=layer.occ_lim,
             agg_ret=layer.agg_ret, agg_lim=layer.agg_lim)
    d.update(kw)
    return Layer(**d)


@given(integer_instances())
@settings(**small)
def test_trial_loss_bounded(inst):
    yet, pool, layer = inst
    ylt, pre = oracle.layer_ylt(yet, pool, layer, threads=1)
    assert np.all(ylt >= 0.0) and np.all(ylt <= layer.agg_lim)
    assert np.all(pre >= 0.0)


@given(integer_instances(), st.integers(0, 3), st.integers(1, 400))
@settings(**small)
def test_monotone_in_layer_terms(inst, which, bump):
    yet, pool, layer = inst
    base, _ = oracle.layer_ylt(yet, pool, layer, threads=1)
    name = ["occ_ret", "occ_lim", "agg_ret", "agg_lim"][which]
    bumped = _with(layer, **{name: getattr(layer, name) + bump})
    ylt, _ = oracle.layer_ylt(yet, pool, bumped, threads=1)
    if name.endswith("ret"):
        assert np.all(ylt <= base)
    else:
        assert np.all(ylt >= base)


@given(integer_instances(), st.integers(1, 400))
@settings(**small)
def test_monotone_in_elt_terms(inst, bump):
    yet, pool, layer = inst
    base, _ = oracle.layer_ylt(yet, pool, layer, threads=1)
    p2 = ELTPool(pool.offsets, pool.ids, pool.losses, pool.deductibles + bump, pool.limits)
    lower, _ = oracle.layer_ylt(yet, p2, layer, threads=1)
    assert np.all(lower <= base)
    p3 = ELTPool(pool.offsets, pool.ids, pool.losses, pool.deductibles, pool.limits + bump)
    higher, _ = oracle.layer_ylt(yet, p3, layer, threads=1)
    assert np.all(higher >= base)


@given(integer_instances(), st.randoms(use_true_random=False))
@settings(**small)
def test_permutation_invariance(inst, rnd):
    """Trial losses do not depend on the ELT order or the event order within a
    trial (exact here: integer values keep every sum exact)."""
    yet, pool, layer = inst
    base, _ = oracle.layer_ylt(yet, pool, layer, threads=1)
    elts = list(layer.elts)
    rnd.shuffle(elts)
    a, _ = oracle.layer_ylt(yet, pool, _with(layer, elts=elts), threads=1)
    np.testing.assert_array_equal(a, base)
    ids = yet.ids.copy()
    for t in range(yet.n_trials):
        seg = list(ids[yet.offsets[t]:yet.offsets[t + 1]])
        rnd.shuffle(seg)
        ids[yet.offsets[t]:yet.offsets[t + 1]] = seg
    b, _ = oracle.layer_ylt(YET(yet.catalog_size, yet.offsets, ids), pool, layer, threads=1)
    np.testing.assert_array_equal(b, base)


@given(integer_instances())
@settings(**small)
def test_increments_telescope(inst):
    yet, pool, layer = inst
    ylt, _ = oracle.layer_ylt(yet, pool, layer, threads=1)
    for t in range(yet.n_trials):
        ids = yet.ids[yet.offsets[t]:yet.offsets[t + 1]]
        occ, agg, inc, tl, _ = oracle.trial_trace(yet.catalog_size, ids, pool, layer)
        assert tl == ylt[t]
        assert math.fsum(inc) == tl
        assert np.all(inc >= 0.0)          # the clamped running loss never decreases


def test_brute_force_three_event_catalog():
    """Every trial of length <= 6 over a 3-event catalog, against exact
    rationals of the total-then-clamp form (non-integer values)."""
    rng = np.random.default_rng(11)
    losses = rng.lognormal(6, 1.0, 6)
    pool = ELTPool(np.array([0, 2, 4, 6], np.int64), np.array([0, 1, 1, 2, 2, 0], np.int32),
                   losses, np.array([17.25, 3.5, 40.125]), np.array([700.5, 1e9, 333.0]))
    layer = Layer([2, 0, 1], 11.75, 900.0, 250.5, 1700.25)
    trials = [list(s) for m in range(7) for s in itertools.product(range(3), repeat=m)]
    off = np.zeros(len(trials) + 1, np.int64)
    off[1:] = np.cumsum([len(t) for t in trials])
    yet = YET(3, off, np.array([e for t in trials for e in t], np.int32))
    ylt, _ = oracle.layer_ylt(yet, pool, layer)

    F = Fraction

    def clamp(v, lo, hi):
        return min(max(v, lo), hi)

    occ = []
    for e in range(3):
        x = F(0)
        for j in layer.elts:
            ids, ls = pool.elt(j)
            hit = [F(float(l)) for i, l in zip(ids, ls) if i == e]
            l = hit[0] if hit else F(0)
            x += clamp(l - F(float(pool.deductibles[j])), F(0), F(float(pool.limits[j])))
        occ.append(clamp(x - F(layer.occ_ret), F(0), F(layer.occ_lim)))
    for t, tr in enumerate(trials):
        total = sum((occ[e] for e in tr), F(0))
        exact = clamp(total - F(layer.agg_ret), F(0), F(layer.agg_lim))
        # a sequential binary64 sum of m <= 6 non-negative terms is within
        # m ulps of the exact total; the clamps are 1-Lipschitz.
        assert abs(F(float(ylt[t])) - exact) <= F(8) * F(2) ** -52 * max(total, F(1)), tr


# ------------------------------------------------------------------ YELT (R11)
def test_hand_worked_yelt_and_oep():
    g, yet, pool, layer = hand_instance()
    y = g["yelt"]
    for mode in ("literal", "memo"):
        inc, out_off, occ_max, ylt, pre = oracle.layer_yelt(yet, pool, layer, mode=mode, threads=2)
        for i, want in enumerate(y["inc"]):
            assert inc[out_off[i]:out_off[i + 1]].tolist() == want
        assert occ_max.tolist() == y["occ_max"]
        assert ylt.tolist() == g["ylt"] and pre.tolist() == g["presum"]
    oep, oep_tvar = oracle.pml_tvar(occ_max, y["return_periods"])
    assert oep.tolist() == y["oep"] and oep_tvar.tolist() == y["oep_tvar"]
    # a subset in another order
    inc, out_off, occ_max, ylt, _ = oracle.layer_yelt(yet, pool, layer, trials=np.array([1, 0]))
    assert inc.tolist() == y["inc"][1] + y["inc"][0]
    assert occ_max.tolist() == [y["occ_max"][1], y["occ_max"][0]]


@given(integer_instances())
@settings(**small)
def test_yelt_telescopes_and_bounds_occurrence_loss(inst):
    """Integer losses: every running sum is exact, so the increments sum to the
    trial loss exactly; the largest increment is at most the trial loss and at
    least its share over the trial's events, and at most the occurrence limit."""
    yet, pool, layer = inst
    inc, out_off, occ_max, ylt, _ = oracle.layer_yelt(yet, pool, layer, threads=2)
    ylt_ref, _ = oracle.layer_ylt(yet, pool, layer, threads=1)
    np.testing.assert_array_equal(ylt, ylt_ref)
    for t in range(yet.n_trials):
        seg = inc[out_off[t]:out_off[t + 1]]
        assert math.fsum(seg) == ylt[t]
        assert np.all(seg >= 0.0)
        assert occ_max[t] <= ylt[t] and occ_max[t] <= layer.occ_lim
        if seg.size:
            assert occ_max[t] == seg.max() and occ_max[t] * seg.size >= ylt[t]
        else:
            assert occ_max[t] == 0.0


def test_yelt_brute_force_three_event_catalog():
    """Every trial of length <= 5 over a 3-event catalog: each increment
    against exact rationals of clamp(P_k) - clamp(P_{k-1})."""
    rng = np.random.default_rng(12)
    losses = rng.lognormal(6, 1.0, 6)
    pool = ELTPool(np.array([0, 2, 4, 6], np.int64), np.array([0, 1, 1, 2, 2, 0], np.int32),
                   losses, np.array([17.25, 3.5, 40.125]), np.array([700.5, 1e9, 333.0]))
    layer = Layer([2, 0, 1], 11.75, 900.0, 250.5, 1700.25)
    trials = [list(s) for m in range(6) for s in itertools.product(range(3), repeat=m)]
    off = np.zeros(len(trials) + 1, np.int64)
    off[1:] = np.cumsum([len(t) for t in trials])
    yet = YET(3, off, np.array([e for t in trials for e in t], np.int32))
    inc, out_off, occ_max, _, _ = oracle.layer_yelt(yet, pool, layer)
    F = Fraction

    def clamp(v, lo, hi):
        return min(max(v, lo), hi)

    occ = []
    for e in range(3):
        x = F(0)
        for j in layer.elts:
            ids, ls = pool.elt(j)
            hit = [F(float(l)) for i, l in zip(ids, ls) if i == e]
            x += clamp((hit[0] if hit else F(0)) - F(float(pool.deductibles[j])), F(0),
                       F(float(pool.limits[j])))
        occ.append(clamp(x - F(layer.occ_ret), F(0), F(layer.occ_lim)))
    for t, tr in enumerate(trials):
        P, prev, best = F(0), F(0), F(0)
        for k, e in enumerate(tr):
            P += occ[e]
            a = clamp(P - F(layer.agg_ret), F(0), F(layer.agg_lim))
            # the oracle's running sum is within k+1 ulps of P; both clamps are
            # 1-Lipschitz and the subtraction rounds once
            tol = F(16) * F(2) ** -52 * max(P, F(1))
            assert abs(F(float(inc[out_off[t] + k])) - (a - prev)) <= tol, (tr, k)
            best = max(best, a - prev)
            prev = a
        assert abs(F(float(occ_max[t])) - best) <= F(16) * F(2) ** -52 * max(prev + F(1), F(1))
