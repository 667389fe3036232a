"""CUDA engine vs the FP64 oracle, element by element, through the C ABI."""
import math

import numpy as np
import pytest

import ara_synth as S
import oracle
from parity import FP64_REL_TOL, assert_fp64_parity, load_workload
from test_oracle import hand_instance

pytestmark = pytest.mark.gpu


@pytest.fixture
def engine():
    from paper_1412_4556_b300 import Engine
    e = Engine(0)
    yield e
    e.close()


# ------------------------------------------------------------- exact cases
def test_hand_worked_instance_is_exact(engine):
    g, yet, pool, layer = hand_instance()
    engine.load_yet_from(yet)
    first = engine.load_pool(pool)
    L = engine.define_layer([first + j for j in layer.elts], layer.occ_ret, layer.occ_lim,
                            layer.agg_ret, layer.agg_lim)
    assert engine.layer_ylt(L).tolist() == g["ylt"]
    assert engine.event_table(L).tolist() == g["event_table"]
    p = g["pml_tvar"]
    pml, tvar = engine.pml_tvar(np.array(p["ylt"]), p["return_periods"])
    assert pml.tolist() == p["pml"] and tvar.tolist() == p["tvar"]
    _, gy, gp, gl = hand_instance(neutral=True)
    engine.load_yet_from(gy)
    f2 = engine.load_pool(gp)
    L2 = engine.define_layer([f2 + j for j in gl.elts], gl.occ_ret, gl.occ_lim, gl.agg_ret, gl.agg_lim)
    assert engine.layer_ylt(L2)[0] == g["neutral_terms"]["ylt_trial0"]


# ----------------------------------------------------------- tiny workload
def test_tiny_workload_parity(engine):
    w = S.tiny()
    layer = w.layers[0]
    (L,) = load_workload(engine, w)
    table = engine.event_table(L)
    np.testing.assert_array_equal(table.view(np.uint64),
                                  oracle.event_table(w.yet.catalog_size, w.pool, layer).view(np.uint64))
    o, pre = oracle.layer_ylt(w.yet, w.pool, layer)
    g = engine.layer_ylt(L)
    assert_fp64_parity(g, o, pre)
    # PML/TVaR: the selection is exact on a given YLT ...
    pml_o, tvar_o = oracle.pml_tvar(o, w.return_periods)
    pml_g, tvar_g = engine.pml_tvar(o, w.return_periods)
    np.testing.assert_array_equal(pml_g, pml_o)
    np.testing.assert_allclose(tvar_g, tvar_o, rtol=1e-13, atol=0)
    # ... and 1-Lipschitz in the trial losses.
    pml_gg, tvar_gg = engine.pml_tvar(g, w.return_periods)
    bound = np.max(np.abs(g - o)) + FP64_REL_TOL * np.abs(tvar_o)
    assert np.all(np.abs(pml_gg - pml_o) <= bound) and np.all(np.abs(tvar_gg - tvar_o) <= bound)


def test_paper_shaped_workload_20k_trials(engine):
    """Paper-scale catalog, ELTs and trial lengths; 20,000 trials (2e7 events)."""
    w = S.paper_scale(n_trials=20_000)
    layer = w.layers[0]
    (L,) = load_workload(engine, w)
    tab_g = engine.event_table(L)
    tab_o = oracle.event_table(w.yet.catalog_size, w.pool, layer)
    np.testing.assert_array_equal(tab_g.view(np.uint64), tab_o.view(np.uint64))
    o, pre = oracle.layer_ylt(w.yet, w.pool, layer, mode="memo")
    g = engine.layer_ylt(L)
    assert_fp64_parity(g, o, pre)
    # every return period of the workload (k = 200, 80, 40 of 20,000)
    pml_o, tvar_o = oracle.pml_tvar(o, w.return_periods)
    pml_g, tvar_g = engine.pml_tvar(o, w.return_periods)
    np.testing.assert_array_equal(pml_g, pml_o)
    np.testing.assert_allclose(tvar_g, tvar_o, rtol=1e-13, atol=0)
    # and from the engine's own YLT, within the largest per-trial error
    pml_e, tvar_e = engine.pml_tvar(g, w.return_periods)
    pt = oracle.compare_pml_tvar(pml_e, tvar_e, pml_o, tvar_o, w.return_periods, g.size,
                                 float(np.max(np.abs(g - o))))
    assert pt["within_bound"], pt


# -------------------------------------------------------------- edge cases
def _custom_yet(catalog, lengths, seed, hot=()):
    rng = np.random.default_rng(seed)
    off = np.zeros(len(lengths) + 1, np.int64)
    off[1:] = np.cumsum(lengths)
    ids = rng.integers(0, catalog, int(off[-1])).astype(np.int32)
    hot = list(hot)
    if hot and ids.size:
        pos = rng.integers(0, ids.size, min(ids.size, 64 * len(hot)))
        ids[pos] = np.array(hot, np.int32)[rng.integers(0, len(hot), pos.size)]
    return S.YET(catalog, off, ids)


def _custom_pool(catalog, sizes, seed, ded=None, lim=None):
    rng = np.random.default_rng(seed + 1)
    off = np.zeros(len(sizes) + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    ids, losses = [], []
    for s in sizes:
        ids.append(rng.choice(catalog, s, replace=False))
        losses.append(rng.lognormal(10, 2.0, s))
    n = len(sizes)
    ded = rng.uniform(0, 2e4, n) if ded is None else np.asarray(ded, float)
    lim = rng.uniform(1e5, 1e7, n) if lim is None else np.asarray(lim, float)
    return S.ELTPool(off, np.concatenate(ids).astype(np.int32) if ids else np.zeros(0, np.int32),
                     np.concatenate(losses) if losses else np.zeros(0), ded, lim)


LENGTHS = [0, 1, 2, 3, 4, 5, 31, 32, 33, 127, 128, 129, 255, 256, 257, 511, 512, 513, 1023, 1024,
           1025, 1500, 4099, 0, 0, 7, 2049, 8191]


@pytest.mark.parametrize("catalog", [3, 2_049, 1_000_003, 2_000_000, 5_000_000])
def test_ragged_trials_and_catalog_sizes(engine, catalog):
    """Trial lengths around every tile edge, catalogs below and above the
    shared-memory bitmap (exact and mixed-resolution layouts)."""
    sizes = [min(catalog, s) for s in (1, 300, 200_000, 7)]
    pool = _custom_pool(catalog, sizes, 3)
    hot = [0, catalog - 1, catalog // 2] + [int(x) for x in pool.ids[:50]]
    yet = _custom_yet(catalog, LENGTHS * 12, catalog, hot)
    engine.load_yet_from(yet)
    first = engine.load_pool(pool)
    layers = [S.Layer([0, 1, 2, 3], 1e3, 5e6, 1e4, 1e8),
              S.Layer([2, 0], 0.0, math.inf, 0.0, math.inf),
              S.Layer([3, 2, 1], 5e5, 1e6, 2e6, 3e6),
              S.Layer([1], 0.0, 0.0, 0.0, 1e9),
              # aggregate terms off the fixed-point grid: the FP64 clamp path
              S.Layer([0, 2], 250.0, 2e7, 1.2345e-30, 7.77e-29 + 3e6)]
    for lay in layers:
        L = engine.define_layer([first + j for j in lay.elts], lay.occ_ret, lay.occ_lim, lay.agg_ret,
                                lay.agg_lim)
        np.testing.assert_array_equal(engine.event_table(L).view(np.uint64),
                                      oracle.event_table(catalog, pool, lay).view(np.uint64))
        o, pre = oracle.layer_ylt(yet, pool, lay, mode="memo")
        assert_fp64_parity(engine.layer_ylt(L), o, pre)
        # a prefix of the YET
        n = 57
        assert_fp64_parity(engine.layer_ylt(L, n_trials=n), o[:n], pre[:n])


def test_empty_and_degenerate_inputs(engine):
    # a YET with trials but no events: every trial loss is 0
    yet = S.YET(10, np.zeros(6, np.int64), np.zeros(0, np.int32))
    engine.load_yet_from(yet)
    first = engine.load_pool(_custom_pool(10, [3, 0], 5))
    L = engine.define_layer([first, first + 1], 0, math.inf, 0, math.inf)
    assert engine.layer_ylt(L).tolist() == [0.0] * 5
    assert engine.layer_ylt(L, n_trials=0).shape == (0,)
    # a YET with no trials
    engine.load_yet_from(S.YET(10, np.zeros(1, np.int64), np.zeros(0, np.int32)))
    assert engine.layer_ylt(L).shape == (0,)
    # PML/TVaR: one trial, k = n, ties, all zeros
    pml, tvar = engine.pml_tvar(np.array([5.0]), [1.0])
    assert pml.tolist() == [5.0] and tvar.tolist() == [5.0]
    y = np.array([3.0, 3.0, 3.0, 1.0, 0.0, 0.0])
    pml, tvar = engine.pml_tvar(y, [1.0, 2.0, 6.0])
    assert pml.tolist() == [0.0, 3.0, 3.0] and tvar.tolist() == [10.0 / 6.0, 3.0, 3.0]
    pml, tvar = engine.pml_tvar(np.zeros(1000), [10.0, 1000.0])
    assert pml.tolist() == [0.0, 0.0] and tvar.tolist() == [0.0, 0.0]


def test_pml_tvar_many_return_periods_wide_range(engine):
    rng = np.random.default_rng(9)
    y = np.concatenate([rng.lognormal(12, 3.0, 200_000), np.zeros(5000), np.full(3000, 7.25e8)])
    rng.shuffle(y)
    rps = [1.0, 1.5, 2.0, 3.0, 10.0, 33.3, 100.0, 250.0, 500.0, 1000.0, 2500.0, 10_000.0, 50_000.0,
           100_000.0, 208_000.0, 7.0]
    pml_o, tvar_o = oracle.pml_tvar(y, rps)
    pml_g, tvar_g = engine.pml_tvar(y, rps)
    np.testing.assert_array_equal(pml_g, pml_o)
    np.testing.assert_allclose(tvar_g, tvar_o, rtol=1e-12, atol=0)


@pytest.mark.parametrize("rps", [[100.0], [100.0, 250.0, 500.0], [2.0, 7.0, 100.0, 999.0],
                                 [1.0, 2.0, 5.0, 10.0, 100.0], [float(r) for r in range(1, 17)]])
def test_pml_tvar_early_finish_and_ties(engine, rps):
    """The radix selection's shortcuts against the oracle, batched over
    layers that take different ones: distinct losses (a threshold's bucket
    ends with one key and the remaining passes return at once), at least k
    losses tied at the largest (the threshold is the largest after the
    second pass), a k-th largest shared by three trials below the top (no
    shortcut: every pass runs), all losses equal, and all zero."""
    rng = np.random.default_rng(31)
    n = 20_000
    distinct = rng.lognormal(14.0, 1.2, n)
    capped = np.minimum(rng.lognormal(16.0, 1.0, n), 2.5e7)          # thousands at the cap
    tied = rng.lognormal(14.0, 1.2, n)
    k = int(n // 100.0)
    tau = np.sort(tied)[::-1][k - 1]
    tied[np.argsort(-tied)[k - 3:k + 2]] = tau                     # the 100-year loss is shared
    equal = np.full(n, 123456.789)
    zero = np.zeros(n)
    ys = np.stack([distinct, capped, tied, equal, zero])
    pml_b, tvar_b = engine.pml_tvar_batch(ys, rps)
    for i, y in enumerate(ys):
        pml_o, tvar_o = oracle.pml_tvar(y, rps)
        np.testing.assert_array_equal(pml_b[i], pml_o, err_msg=f"layer {i}")
        np.testing.assert_allclose(tvar_b[i], tvar_o, rtol=1e-12, atol=0, err_msg=f"layer {i}")
        pml_1, tvar_1 = engine.pml_tvar(y, rps)                      # one layer alone: same bits
        np.testing.assert_array_equal(pml_1, pml_b[i])
        np.testing.assert_array_equal(tvar_1.view(np.uint64), tvar_b[i].view(np.uint64))


def test_result_independent_of_launch_shape(engine, monkeypatch):
    w = S.paper_scale(n_trials=3_000, catalog_size=300_000)
    (L,) = load_workload(engine, w)
    ref = None
    for u in ("1", "2"):
        for lpt in ("16", "32"):
            monkeypatch.setenv("ARA_YLT_UNROLL", u)
            monkeypatch.setenv("ARA_YLT_LPT", lpt)
            g = engine.layer_ylt(L)
            if ref is None:
                ref = g.copy()
            np.testing.assert_array_equal(g.view(np.uint64), ref.view(np.uint64))


def test_device_buffers_and_streams(engine):
    import torch
    w = S.tiny()
    layer = w.layers[0]
    dev = torch.device("cuda", 0)
    off = torch.from_numpy(w.yet.offsets).to(dev)
    ids = torch.from_numpy(w.yet.ids).to(dev)
    ts = torch.from_numpy(w.yet.ts).to(dev)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    engine.set_stream(s)
    engine.load_yet(w.yet.catalog_size, off, ids, ts)
    first = engine.load_pool(w.pool)
    L = engine.define_layer([first + j for j in layer.elts], layer.occ_ret, layer.occ_lim,
                            layer.agg_ret, layer.agg_lim)
    out = torch.empty(w.yet.n_trials, dtype=torch.float64, device=dev)
    engine.layer_ylt(L, out=out)
    s.synchronize()
    o, pre = oracle.layer_ylt(w.yet, w.pool, layer)
    assert_fp64_parity(out.cpu().numpy(), o, pre)
    pml, tvar = engine.pml_tvar(out, w.return_periods)
    pml_h, tvar_h = engine.pml_tvar(out.cpu().numpy(), w.return_periods)
    np.testing.assert_array_equal(pml, pml_h)
    np.testing.assert_array_equal(tvar, tvar_h)


def test_layer_reuse_after_yet_reload(engine):
    w = S.tiny()
    layer = w.layers[0]
    (L,) = load_workload(engine, w)
    w2 = S.tiny(seed=77, n_trials=1500)
    engine.load_yet_from(w2.yet)       # same catalog, new trials: the layer is re-folded
    o, pre = oracle.layer_ylt(w2.yet, w.pool, layer)
    assert_fp64_parity(engine.layer_ylt(L), o, pre)


# ------------------------------------------------------------ error paths
def test_invalid_inputs_are_rejected_with_status(engine):
    from paper_1412_4556_b300 import AraError
    def status(fn):
        with pytest.raises(AraError) as ei:
            fn()
        return ei.value.name

    bad = S.YET(10, np.array([0, 2, 3], np.int64), np.array([1, 10, 2], np.int32))
    assert status(lambda: engine.load_yet_from(bad)) == "ARA_E_EVENT_RANGE"
    assert status(lambda: engine.load_yet(10, np.array([0, 2, 1], np.int64),
                                          np.array([1, 2], np.int32))) == "ARA_E_INVALID_ARG"
    assert status(lambda: engine.load_yet(10, np.array([0, 3], np.int64), np.array([1, 2, 3], np.int32),
                                          np.array([1.0, 0.5, 2.0], np.float32))) == "ARA_E_INVALID_ARG"
    assert status(lambda: engine.load_pool(_custom_pool(10, [2], 1))) == "ARA_E_STATE"
    engine.load_yet_from(S.YET(10, np.array([0, 3], np.int64), np.array([1, 2, 3], np.int32),
                               np.array([0.5, 0.5, 2.0], np.float32)))
    dup = S.ELTPool(np.array([0, 2], np.int64), np.array([4, 4], np.int32), np.array([1.0, 2.0]),
                    np.array([0.0]), np.array([1.0]))
    assert status(lambda: engine.load_pool(dup)) == "ARA_E_DUP_EVENT"
    nan = S.ELTPool(np.array([0, 1], np.int64), np.array([4], np.int32), np.array([np.nan]),
                    np.array([0.0]), np.array([1.0]))
    assert status(lambda: engine.load_pool(nan)) == "ARA_E_INVALID_ARG"
    first = engine.load_pool(_custom_pool(10, [3], 2))
    assert status(lambda: engine.define_layer([first + 5], 0, 1, 0, 1)) == "ARA_E_NOT_FOUND"
    assert status(lambda: engine.define_layer([first, first], 0, 1, 0, 1)) == "ARA_E_INVALID_ARG"
    assert status(lambda: engine.define_layer([first], -1.0, 1, 0, 1)) == "ARA_E_INVALID_ARG"
    assert status(lambda: engine.define_layer([first], 0, float("nan"), 0, 1)) == "ARA_E_INVALID_ARG"
    L = engine.define_layer([first], 0, 1e9, 0, 1e9)
    assert status(lambda: engine.layer_ylt(L, n_trials=2)) == "ARA_E_INVALID_ARG"
    assert status(lambda: engine.layer_ylt(L + 7)) == "ARA_E_NOT_FOUND"
    assert status(lambda: engine.pml_tvar(np.ones(10), [11.0])) == "ARA_E_INVALID_ARG"
    assert status(lambda: engine.pml_tvar(np.array([1.0, -2.0]), [1.0])) == "ARA_E_INVALID_ARG"
    assert status(lambda: engine.pml_tvar(np.array([1.0, np.inf]), [1.0])) == "ARA_E_INVALID_ARG"
    engine.release_layer(L)
    assert status(lambda: engine.layer_ylt(L)) == "ARA_E_NOT_FOUND"
    # the context still works after every error
    L = engine.define_layer([first], 0, 1e9, 0, 1e9)
    assert engine.layer_ylt(L).shape == (1,)


def test_entry_points_refuse_another_gpus_memory(engine):
    """Device memory of a GPU other than the context's is refused with a
    status before anything is queued (its kernels could not read it); needs
    a second GPU."""
    import torch
    from paper_1412_4556_b300 import AraError
    if torch.cuda.device_count() < 2:
        pytest.skip("one GPU: no memory of another device to pass")
    w = S.tiny(n_trials=200)
    (L,) = load_workload(engine, w)
    other = torch.ones(200, dtype=torch.float64, device="cuda:1")
    for call in (lambda: engine.pml_tvar(other, [10.0]), lambda: engine.layer_ylt(L, out=other),
                 lambda: engine.ylt_tail(other, 5)):
        with pytest.raises(AraError) as ei:
            call()
        assert ei.value.name == "ARA_E_INVALID_ARG" and "another GPU" in str(ei.value)
    # the context still works
    assert engine.layer_ylt(L).shape == (200,)


# The full paper-scale workload (every trial against the oracle) is in
# test_gpu_fullsize.py.


@pytest.mark.parametrize("catalog", [(1 << 21) - 1, 1 << 21])
def test_packing_boundary_catalogs(engine, catalog):
    """The largest catalog whose ids (and the sentinel) pack into 21 bits, and
    the smallest that does not: both layouts give the oracle's YLT, and so
    does the compact stream of the first."""
    pool = _custom_pool(catalog, [40_000, 25_000, 5], 8)
    hot = [0, catalog - 1, catalog - 2] + [int(x) for x in pool.ids[:20]]
    yet = _custom_yet(catalog, LENGTHS * 4, 17, hot)
    engine.load_yet_from(yet)
    first = engine.load_pool(pool)
    lay = S.Layer([0, 1, 2], 1e3, 5e6, 1e4, 1e8)
    L = engine.define_layer([first + j for j in lay.elts], lay.occ_ret, lay.occ_lim, lay.agg_ret, lay.agg_lim)
    o, pre = oracle.layer_ylt(yet, pool, lay, mode="memo")
    y = engine.layer_ylt(L)
    assert_fp64_parity(y, o, pre)
    # the difference code's 21-bit bases and 8192-id buckets reach the top id
    # (a no-op for the plain layout of the larger catalog)
    engine.compact_yet()
    np.testing.assert_array_equal(engine.layer_ylt(L).view(np.uint64), y.view(np.uint64))


def test_layer_with_the_most_elts(engine):
    """A layer over 1,024 ELTs (the limit): the fold stays bit-identical to the
    oracle's ELT loop and the YLT matches; 1,025 ELTs are refused."""
    from paper_1412_4556_b300 import AraError
    catalog = 60_000
    pool = _custom_pool(catalog, [25 + (j % 17) for j in range(1025)], 9)
    yet = _custom_yet(catalog, LENGTHS * 2, 19)
    engine.load_yet_from(yet)
    first = engine.load_pool(pool)
    order = list(np.random.default_rng(2).permutation(1024))
    lay = S.Layer([int(j) for j in order], 2e3, 1e7, 5e4, 2e8)
    L = engine.define_layer([first + j for j in lay.elts], lay.occ_ret, lay.occ_lim, lay.agg_ret, lay.agg_lim)
    np.testing.assert_array_equal(engine.event_table(L).view(np.uint64),
                                  oracle.event_table(catalog, pool, lay).view(np.uint64))
    o, pre = oracle.layer_ylt(yet, pool, lay, mode="memo")
    assert_fp64_parity(engine.layer_ylt(L), o, pre)
    with pytest.raises(AraError) as ei:
        engine.define_layer(list(range(first, first + 1025)), 0.0, math.inf, 0.0, math.inf)
    assert ei.value.name == "ARA_E_INVALID_ARG"


def test_rejected_yet_keeps_the_previous_one(engine):
    """Offsets that fail their checks (found while the ids are being copied)
    leave the loaded YET and its layers usable; ids outside the catalog,
    found on the device after the copy, leave no YET."""
    from paper_1412_4556_b300 import AraError
    w = S.tiny()
    (L,) = load_workload(engine, w)
    ref = engine.layer_ylt(L)
    bad = w.yet.offsets.copy()
    bad[5], bad[6] = bad[6], bad[5] - 1  # decreasing
    with pytest.raises(AraError) as ei:
        engine.load_yet(w.yet.catalog_size, bad, w.yet.ids)
    assert ei.value.name == "ARA_E_INVALID_ARG"
    np.testing.assert_array_equal(engine.layer_ylt(L), ref)
    ids = w.yet.ids.copy()
    ids[7] = w.yet.catalog_size
    with pytest.raises(AraError) as ei:
        engine.load_yet(w.yet.catalog_size, w.yet.offsets, ids)
    assert ei.value.name == "ARA_E_EVENT_RANGE"
    with pytest.raises(AraError) as ei:
        engine.layer_ylt(L)
    assert ei.value.name == "ARA_E_STATE"
    engine.load_yet_from(w.yet)
    np.testing.assert_array_equal(engine.layer_ylt(L), ref)


def _split_at(lengths, pos, n_empty):
    """Split the trial that holds id position pos so that a trial ends exactly
    there, and put n_empty empty trials at the cut (the total is unchanged)."""
    off = np.concatenate([[0], np.cumsum(lengths)])
    t = int(np.searchsorted(off, pos, side="right")) - 1
    if off[t] == pos:
        return lengths[:t] + [0] * n_empty + lengths[t:]
    a = pos - int(off[t])
    return lengths[:t] + [a] + [0] * n_empty + [lengths[t] - a] + lengths[t + 1:]


@pytest.mark.parametrize("catalog", [2_000_000, 5_000_000])
def test_host_ids_load_in_pieces(engine, catalog):
    """Host ids of several times 2^24 entries are copied in pieces, and the
    trials each piece completes are chunked while the later pieces copy.  A
    trial spanning several pieces, trials that end exactly at a piece
    boundary with empty trials there, and empty trials at both ends give the
    bits of the same ids loaded from device memory (one chunking launch) and
    the oracle's YLT on sampled trials; a bad id in the first or the last
    piece is found."""
    import torch
    from paper_1412_4556_b300 import AraError
    rng = np.random.default_rng(31)
    # the long trial covers the first pieces whole (they complete no trial)
    lengths = [0, 0, (1 << 26) + 4_999] + [int(x) for x in rng.poisson(1000, 80_000)] + [0]
    M = sum(lengths)
    pieces = min(8, M >> 24)
    assert pieces == 8
    step = M // pieces
    lengths = _split_at(lengths, 5 * step, 3)
    lengths = _split_at(lengths, 6 * step, 1)
    assert sum(lengths) == M
    yet = _custom_yet(catalog, lengths, 41, hot=[0, catalog - 1])
    pool = _custom_pool(catalog, [50_000, 30_000, 20_000], 5)
    lay = S.Layer([0, 1, 2], 1e3, 5e6, 1e4, 1e9)
    dev = torch.device("cuda", 0)
    d_off, d_ids = torch.from_numpy(yet.offsets).to(dev), torch.from_numpy(yet.ids).to(dev)
    torch.cuda.synchronize()  # the engine's stream is not torch's
    engine.load_yet(catalog, d_off, d_ids)
    first = engine.load_pool(pool)
    L = engine.define_layer([first + j for j in lay.elts], lay.occ_ret, lay.occ_lim, lay.agg_ret, lay.agg_lim)
    ref = engine.layer_ylt(L)
    h_ids = torch.from_numpy(yet.ids).pin_memory()
    engine.load_yet(catalog, yet.offsets, h_ids.numpy())
    y = engine.layer_ylt(L)
    np.testing.assert_array_equal(y.view(np.uint64), ref.view(np.uint64))
    # device offsets with host ids: the pieces are sized from the offsets' last
    # entry, read back before the first piece starts
    engine.load_yet(catalog, d_off, h_ids.numpy())
    np.testing.assert_array_equal(engine.layer_ylt(L).view(np.uint64), ref.view(np.uint64))
    off = yet.offsets
    around = np.concatenate([np.searchsorted(off, b * step, side="right") + np.arange(-3, 3)
                             for b in range(1, pieces)])
    sel = np.unique(np.concatenate([around, [0, 1, 2, off.size - 2, int(np.argmax(np.diff(off)))],
                                    rng.choice(y.size, 300, replace=False)]))
    sel = sel[(sel >= 0) & (sel < y.size)]
    o, pre = oracle.layer_ylt(yet, pool, lay, trials=sel, mode="memo")
    assert_fp64_parity(y[sel], o, pre)
    for pos in (0, M - 1):
        ids = yet.ids.copy()
        ids[pos] = catalog
        with pytest.raises(AraError) as ei:
            engine.load_yet(catalog, yet.offsets, ids)
        assert ei.value.name == "ARA_E_EVENT_RANGE"
    engine.load_yet(catalog, yet.offsets, h_ids.numpy())
    np.testing.assert_array_equal(engine.layer_ylt(L).view(np.uint64), ref.view(np.uint64))


def test_pml_tvar_queued_matches_the_synchronous_form(engine):
    """ara_pml_tvar_async: several selections queued back to back on the
    engine's stream give the bits of ara_pml_tvar; losses that fail the check
    give NaN outputs; host pointers are refused."""
    import torch
    from paper_1412_4556_b300 import AraError
    w = S.tiny()
    rps = [10.0, 50.0, 100.0]
    (L,) = load_workload(engine, w)
    dev = torch.device("cuda", 0)
    base = torch.from_numpy(engine.layer_ylt(L)).to(dev)
    ylts = [base, base * 0.5, torch.flip(base, [0]), base[:777].contiguous()]
    outs = [torch.full((2 * len(rps),), -1.0, dtype=torch.float64, device=dev) for _ in ylts]
    torch.cuda.synchronize()
    for y, o in zip(ylts, outs):
        engine.pml_tvar_async(y, rps, o)
    torch.cuda.synchronize()
    for y, o in zip(ylts, outs):
        pml, tvar = engine.pml_tvar(y.cpu().numpy(), rps)
        got = o.cpu().numpy()
        np.testing.assert_array_equal(got[:3].view(np.uint64), pml.view(np.uint64))
        np.testing.assert_array_equal(got[3:].view(np.uint64), tvar.view(np.uint64))
    for bad_value in (float("nan"), -1.0, float("inf")):
        bad = base.clone()
        bad[5] = bad_value
        o = torch.zeros(2 * len(rps), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()  # the engine's stream is not torch's
        engine.pml_tvar_async(bad, rps, o)
        torch.cuda.synchronize()
        assert torch.isnan(o).all()
    # the next queued call is not affected by the failed one
    o = torch.zeros(2 * len(rps), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    engine.pml_tvar_async(base, rps, o)
    torch.cuda.synchronize()
    pml, _ = engine.pml_tvar(base.cpu().numpy(), rps)
    np.testing.assert_array_equal(o.cpu().numpy()[:3], pml)
    with pytest.raises(AraError) as ei:
        engine.pml_tvar_async(base.cpu().numpy(), rps, o)
    assert ei.value.name == "ARA_E_INVALID_ARG"
    with pytest.raises(AraError) as ei:
        engine.pml_tvar_async(base, [1e9], o)
    assert ei.value.name == "ARA_E_INVALID_ARG"
