"""Year Event Loss Table (per-occurrence increments of the aggregate step) and
the Return Period Loss report (AEP and OEP), through the C ABI, against the
oracle's reading R11."""
import math

import numpy as np
import pytest

import ara_synth as S
import oracle
from test_gpu_parity import LENGTHS, _custom_pool, _custom_yet
from test_oracle import hand_instance

pytestmark = pytest.mark.gpu

# FP64 layers: each increment is a difference of two clamped running sums;
# both sides' running sums agree within ~1.7e-13 of the trial's
# pre-aggregate sum S (see parity.py), so an increment moves by at most twice
# that plus one rounding: gate at 1e-12 * S per occurrence, as for the YLT.
FP64_REL = 1e-12
# FP32-table layers: 1e-5 of S with a 1 USD floor, as for their YLT.
FP32_REL, FP32_FLOOR = 1e-5, 1.0


@pytest.fixture
def engine():
    from paper_1412_4556_b300 import Engine
    e = Engine(0)
    yield e
    e.close()


def assert_yelt_parity(g_inc, g_max, o_inc, out_off, o_max, pre, rel, floor=0.0, what=""):
    trial_of = np.repeat(np.arange(pre.size), np.diff(out_off))
    err = np.abs(np.asarray(g_inc) - o_inc)
    bound = np.maximum(rel * pre[trial_of], floor)
    if err.size:
        i = int(np.argmax(err - bound))
        assert err[i] <= bound[i], f"{what}: occurrence {i} (trial {trial_of[i]}) gpu={g_inc[i]!r} oracle={o_inc[i]!r}"
    err_m = np.abs(np.asarray(g_max) - o_max)
    bound_m = np.maximum(rel * pre, floor)
    i = int(np.argmax(err_m - bound_m))
    assert err_m[i] <= bound_m[i], f"{what}: trial {i} max gpu={g_max[i]!r} oracle={o_max[i]!r}"
    return float(err.max()) if err.size else 0.0, float(err_m.max())


def test_hand_worked_yelt_and_report(engine):
    g, yet, pool, layer = hand_instance()
    engine.load_yet_from(yet)
    first = engine.load_pool(pool)
    L = engine.define_layer([first + j for j in layer.elts], layer.occ_ret, layer.occ_lim,
                            layer.agg_ret, layer.agg_lim)
    inc, occ_max = engine.layer_yelt(L)
    y = g["yelt"]
    assert inc.tolist() == [v for t in y["inc"] for v in t]
    assert occ_max.tolist() == y["occ_max"]
    rep = engine.rpl_report(L, y["return_periods"])
    assert rep["oep"].tolist() == y["oep"] and rep["oep_tvar"].tolist() == y["oep_tvar"]
    pml, tvar = engine.pml_tvar(engine.layer_ylt(L), y["return_periods"])
    np.testing.assert_array_equal(rep["aep"], pml)
    np.testing.assert_array_equal(rep["aep_tvar"], tvar)


@pytest.mark.parametrize("catalog", [3, 2_049, 1_000_003, 5_000_000])
def test_ragged_trials_and_catalogs(engine, catalog):
    """Trial lengths around every tile edge; packed (catalog < 2^21) and plain
    id chunks; aggregate terms on and off the fixed-point grid."""
    sizes = [min(catalog, s) for s in (1, 300, 200_000, 7)]
    pool = _custom_pool(catalog, sizes, 5)
    hot = [0, catalog - 1, catalog // 2] + [int(x) for x in pool.ids[:50]]
    yet = _custom_yet(catalog, LENGTHS * 6, catalog + 1, hot)
    engine.load_yet_from(yet)
    first = engine.load_pool(pool)
    layers = [S.Layer([0, 1, 2, 3], 1e3, 5e6, 1e4, 1e8),
              S.Layer([2, 0], 0.0, math.inf, 0.0, math.inf),
              S.Layer([3, 2, 1], 5e5, 1e6, 2e6, 3e6),
              S.Layer([0, 2], 250.0, 2e7, 1.2345e-30, 7.77e-29 + 3e6)]
    for li, lay in enumerate(layers):
        L = engine.define_layer([first + j for j in lay.elts], lay.occ_ret, lay.occ_lim, lay.agg_ret,
                                lay.agg_lim)
        inc, occ_max = engine.layer_yelt(L)
        o_inc, out_off, o_max, o_ylt, pre = oracle.layer_yelt(yet, pool, lay)
        assert_yelt_parity(inc, occ_max, o_inc, out_off, o_max, pre, FP64_REL, what=f"layer {li}")
        assert np.all(inc >= 0.0)
        # each trial's increments add up to its YLT entry (up to the roundings
        # of the increments), and the largest is at most the trial loss
        ylt = engine.layer_ylt(L)
        lens = np.diff(out_off)
        sums = np.bincount(np.repeat(np.arange(lens.size), lens), weights=inc, minlength=lens.size)
        assert np.all(np.abs(sums - ylt) <= lens * 2.0 ** -52 * ylt + 1e-300)
        assert np.all(occ_max <= ylt)
        # a prefix of the YET, per-trial maxima only
        n = 41
        _, m41 = engine.layer_yelt(L, n_trials=n, want_yelt=False)
        np.testing.assert_array_equal(m41, occ_max[:n])


@pytest.mark.parametrize("catalog", [200_000, 3_000_000])
def test_fp32_table_layer(engine, catalog):
    """FP32-table layers (8-byte entries, 16-byte interleaved entries with
    output), with packed (catalog < 2^21) and plain id chunks."""
    from paper_1412_4556_b300 import ARA_FP32_TABLE
    w = S.batched(n_layers=3, n_trials=3_000, lam=200.0, catalog_size=catalog, n_pool=30)
    engine.load_yet_from(w.yet)
    first = engine.load_pool(w.pool)
    for lay in w.layers:
        L = engine.define_layer([first + j for j in lay.elts], lay.occ_ret, lay.occ_lim, lay.agg_ret,
                                lay.agg_lim, precision=ARA_FP32_TABLE)
        inc, occ_max = engine.layer_yelt(L)
        o_inc, out_off, o_max, _, pre = oracle.layer_yelt(w.yet, w.pool, lay)
        assert_yelt_parity(inc, occ_max, o_inc, out_off, o_max, pre, FP32_REL, FP32_FLOOR)


def test_rpl_report_against_oracle(engine):
    w = S.tiny(n_trials=5_000)
    lay = w.layers[0]
    engine.load_yet_from(w.yet)
    first = engine.load_pool(w.pool)
    L = engine.define_layer([first + j for j in lay.elts], lay.occ_ret, lay.occ_lim, lay.agg_ret, lay.agg_lim)
    rps = [1.0, 2.0, 10.0, 100.0, 250.0, 5_000.0]
    rep = engine.rpl_report(L, rps)
    pml, tvar = engine.pml_tvar(engine.layer_ylt(L), rps)
    np.testing.assert_array_equal(rep["aep"], pml)
    np.testing.assert_array_equal(rep["aep_tvar"], tvar)
    _, occ_max = engine.layer_yelt(L, want_yelt=False)
    p_own, t_own = engine.pml_tvar(occ_max, rps)
    np.testing.assert_array_equal(rep["oep"], p_own)
    np.testing.assert_array_equal(rep["oep_tvar"], t_own)
    _, _, o_max, _, pre = oracle.layer_yelt(w.yet, w.pool, lay)
    oep_o, oep_t_o = oracle.pml_tvar(o_max, rps)
    bound = np.max(np.abs(occ_max - o_max)) + 1e-12 * np.abs(oep_t_o)
    assert np.all(np.abs(rep["oep"] - oep_o) <= bound)
    assert np.all(np.abs(rep["oep_tvar"] - oep_t_o) <= bound)
    assert np.all(rep["oep"] <= rep["aep"])


def test_device_outputs(engine):
    import torch
    w = S.tiny(n_trials=2_000)
    lay = w.layers[0]
    engine.load_yet_from(w.yet)
    first = engine.load_pool(w.pool)
    L = engine.define_layer([first + j for j in lay.elts], lay.occ_ret, lay.occ_lim, lay.agg_ret, lay.agg_lim)
    host_inc, host_max = engine.layer_yelt(L)
    d_inc = torch.empty(host_inc.size, dtype=torch.float64, device="cuda")
    d_max = torch.empty(host_max.size, dtype=torch.float64, device="cuda")
    engine.layer_yelt(L, out=d_inc, occ_max=d_max)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(d_inc.cpu().numpy(), host_inc)
    np.testing.assert_array_equal(d_max.cpu().numpy(), host_max)


def test_invalid_arguments(engine):
    from paper_1412_4556_b300 import AraError
    w = S.tiny(n_trials=200)
    lay = w.layers[0]
    engine.load_yet_from(w.yet)
    first = engine.load_pool(w.pool)
    L = engine.define_layer([first + j for j in lay.elts], lay.occ_ret, lay.occ_lim, lay.agg_ret, lay.agg_lim)
    with pytest.raises(AraError) as ei:
        engine.rpl_report(L, [500.0])  # floor(200 / 500) = 0
    assert ei.value.name == "ARA_E_INVALID_ARG"
    with pytest.raises(AraError) as ei:
        engine.rpl_report(L + 7, [10.0])
    assert ei.value.name == "ARA_E_NOT_FOUND"
    with pytest.raises(AraError):
        engine.layer_yelt(L, n_trials=201)


def test_paper_scale_full_size_every_occurrence():
    """The full YELT of the paper-scale workload (~1e9 occurrences, 8 GB on
    the device): every increment and every trial maximum against the
    oracle's YELT, the YLT against the oracle's, and the AEP/OEP report
    against the oracle's return period losses."""
    import torch
    from paper_1412_4556_b300 import Engine
    w = S.paper_scale()
    lay = w.layers[0]
    with Engine(0) as e:
        e.load_yet_from(w.yet)
        first = e.load_pool(w.pool)
        L = e.define_layer([first + j for j in lay.elts], lay.occ_ret, lay.occ_lim, lay.agg_ret, lay.agg_lim)
        M = int(w.yet.offsets[-1])
        d_inc = torch.empty(M, dtype=torch.float64, device="cuda")
        d_max = torch.empty(w.yet.n_trials, dtype=torch.float64, device="cuda")
        e.layer_yelt(L, out=d_inc, occ_max=d_max)
        ylt = e.layer_ylt(L)
        rep = e.rpl_report(L, w.return_periods)
        torch.cuda.synchronize()
        g_inc = d_inc.cpu().numpy()
        occ_max = d_max.cpu().numpy()
        del d_inc
    o_inc, out_off, o_max, o_ylt, pre = oracle.layer_yelt(w.yet, w.pool, lay)
    np.testing.assert_array_equal(out_off, w.yet.offsets)
    # every occurrence, a block of trials at a time (bounded temporaries)
    step = 50_000
    for t0 in range(0, w.yet.n_trials, step):
        t1 = min(w.yet.n_trials, t0 + step)
        a, b = int(out_off[t0]), int(out_off[t1])
        assert_yelt_parity(g_inc[a:b], occ_max[t0:t1], o_inc[a:b], out_off[t0:t1 + 1] - a, o_max[t0:t1],
                           pre[t0:t1], FP64_REL, what=f"trials {t0}..{t1}")
    rep_y = oracle.compare_fp64(ylt, o_ylt, pre)
    assert rep_y["trials_over_r9_bar"] == 0, rep_y
    # AEP and OEP return period losses against the oracle's (1-Lipschitz in
    # the per-trial values)
    for key_p, key_t, g_vals, o_vals in (("aep", "aep_tvar", ylt, o_ylt), ("oep", "oep_tvar", occ_max, o_max)):
        p_o, t_o = oracle.pml_tvar(o_vals, w.return_periods)
        pt = oracle.compare_pml_tvar(rep[key_p], rep[key_t], p_o, t_o, w.return_periods, g_vals.size,
                                     float(np.max(np.abs(g_vals - o_vals))))
        assert pt["within_bound"], (key_p, pt)
    print(f"\nfull-size YELT: {M} occurrences, max |error| {float(np.max(np.abs(g_inc - o_inc))):.3e} USD")


def _inside_increments_check(yelt, table, yet):
    """Every increment is 0, or exactly the occurrence's event-table value
    (its running sum stayed inside the layer), or one of at most two per
    trial where the running sum crossed AggR or AggR + AggL."""
    v = table[yet.ids]
    same = (yelt == 0.0) | (yelt.view(np.uint64) == v.view(np.uint64))
    trial_of = np.repeat(np.arange(yet.n_trials), np.diff(yet.offsets))
    other = np.bincount(trial_of[~same], minlength=yet.n_trials)
    assert other.max() <= 2
    return int(np.count_nonzero(same & (yelt != 0.0)))


def test_inside_increments_are_the_event_table_values(engine):
    """The binary64 reading of in-layer increments (the event table, used
    when every table value is exactly on the grid) gives the bits the
    fixed-point difference gives."""
    w = S.paper_scale(n_trials=5_000, lam=200.0, catalog_size=200_000)
    L = w.layers[0]
    engine.load_yet_from(w.yet)
    first = engine.load_pool(w.pool)
    h = engine.define_layer([first + j for j in L.elts], L.occ_ret, L.occ_lim, L.agg_ret, 1.5e8)
    inc, occ_max = engine.layer_yelt(h)
    inside = _inside_increments_check(inc, engine.event_table(h), w.yet)
    assert inside > 100_000
    o_inc, out_off, o_max, _, pre = oracle.layer_yelt(w.yet, w.pool, S.Layer(L.elts, L.occ_ret, L.occ_lim,
                                                                               L.agg_ret, 1.5e8))
    assert_yelt_parity(inc, occ_max, o_inc, out_off, o_max, pre, FP64_REL, what="paper-shaped")


def test_tiny_losses_take_the_conversion_path(engine):
    """Losses far below the table's grid (rounded into the fixed-point
    table) make the binary64 table inexact: increments are then converted
    from the fixed-point entries, still within the parity bound."""
    catalog = 50_000
    pool = _custom_pool(catalog, [5_000, 20_000], 11, ded=[0.0, 0.0], lim=[1e12, 1e12])
    pool.losses[:2_500] *= 1e-25  # their last bits fall below the grid the large losses set
    yet = _custom_yet(catalog, LENGTHS * 4, 5)
    layer = S.Layer([0, 1], 0.0, math.inf, 1e3, 1e12)
    engine.load_yet_from(yet)
    first = engine.load_pool(pool)
    h = engine.define_layer([first, first + 1], layer.occ_ret, layer.occ_lim, layer.agg_ret, layer.agg_lim)
    inc, occ_max = engine.layer_yelt(h)
    o_inc, out_off, o_max, _, pre = oracle.layer_yelt(yet, pool, layer)
    assert_yelt_parity(inc, occ_max, o_inc, out_off, o_max, pre, FP64_REL, what="tiny losses")
    # events whose only loss is tiny are rounded in the fixed-point table, and
    # their increments follow the fixed-point sums, not the binary64 values
    tab = engine.event_table(h)
    tiny = (tab > 0.0) & (tab < 1e-15)
    hit = tiny[yet.ids] & (inc != 0.0)
    assert hit.sum() > 100
    assert np.any(inc[hit].view(np.uint64) != tab[yet.ids][hit].view(np.uint64))
