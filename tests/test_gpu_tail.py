"""The exchange between trial shards (Section IV-C spreads one analysis'
trials over several GPUs): each shard's largest trial losses
(ara_ylt_tail), and PML/TVaR of the whole YLT from their union
(ara_pml_tvar_tail), bit for bit what ara_pml_tvar gives on the whole YLT
and within the parity bound of the oracle's."""
import math

import numpy as np
import pytest

import ara_synth as S
import oracle

pytestmark = pytest.mark.gpu

RPS = [10.0, 25.0, 50.0]


@pytest.fixture
def engine():
    from paper_1412_4556_b300 import Engine
    e = Engine(0)
    yield e
    e.close()


def layer_ylt(engine, n_trials=20_000):
    w = S.paper_scale(n_trials=n_trials, lam=200.0, catalog_size=200_000)
    engine.load_yet_from(w.yet)
    first = engine.load_pool(w.pool)
    L = w.layers[0]
    # an aggregate limit that about 4% of the trials reach: ties at it
    h = engine.define_layer([first + j for j in L.elts], L.occ_ret, L.occ_lim, L.agg_ret, 1.5e8)
    return w, engine.layer_ylt(h)


def check_tail(y, k, tail):
    """The k largest values as a multiset; the values above the k-th largest
    in index order, then copies of it."""
    tau = np.sort(y)[::-1][k - 1]
    above = y[y > tau]
    assert tail.shape == (k,)
    np.testing.assert_array_equal(tail[:above.size].view(np.uint64), above.view(np.uint64))
    assert np.all(tail[above.size:] == tau)
    np.testing.assert_array_equal(np.sort(tail), np.sort(y)[-k:])


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_tails_give_the_whole_ylt_pml_tvar(engine, world):
    w, y = layer_ylt(engine)
    n = y.size
    assert 100 < np.sum(y == 1.5e8) < n // 10  # ties at the aggregate limit
    pml, tvar = engine.pml_tvar(y, RPS)
    bounds = np.linspace(0, n, world + 1).astype(int)  # unequal shards for world = 3
    k_max = int(math.floor(n / min(RPS)))
    tails = []
    for a, b in zip(bounds[:-1], bounds[1:]):
        shard = y[a:b]
        k = min(shard.size, k_max)
        t = engine.ylt_tail(shard, k)
        check_tail(shard, k, t)
        tails.append(t)
    union = np.concatenate(tails)
    p2, t2 = engine.pml_tvar_tail(union, n, RPS)
    np.testing.assert_array_equal(p2, pml)
    np.testing.assert_array_equal(t2.view(np.uint64), tvar.view(np.uint64))
    # and the oracle's definition on the whole YLT (its tail sum is sequential)
    po, to = oracle.pml_tvar(y, RPS)
    np.testing.assert_array_equal(p2, po)
    assert np.all(np.abs(t2 - to) <= 1e-12 * np.abs(to))


def test_tail_edges_and_device_buffers(engine):
    import torch
    _, y = layer_ylt(engine, n_trials=5_000)
    for k in (1, 2, 37, y.size - 1, y.size):
        check_tail(y, k, engine.ylt_tail(y, k))
    zeros = np.zeros(1000)
    check_tail(zeros, 10, engine.ylt_tail(zeros, 10))
    d = torch.from_numpy(y).cuda()
    out = torch.empty(500, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()  # the engine's stream is not torch's
    engine.ylt_tail(d, 500, out=out)
    torch.cuda.synchronize()
    host = out.cpu().numpy()
    np.testing.assert_array_equal(host, engine.ylt_tail(y, 500))  # the same on every run and route
    p, t = engine.pml_tvar_tail(out, y.size, [y.size / 500.0])
    p0, t0 = engine.pml_tvar(y, [y.size / 500.0])
    assert p == p0 and t == t0


def test_tail_errors(engine):
    from paper_1412_4556_b300 import AraError
    y = np.linspace(0.0, 1e6, 1000)
    for k in (0, 1001):
        with pytest.raises(AraError) as ei:
            engine.ylt_tail(y, k)
        assert ei.value.name == "ARA_E_INVALID_ARG"
    bad = y.copy()
    bad[17] = np.nan
    with pytest.raises(AraError) as ei:
        engine.ylt_tail(bad, 10)
    assert ei.value.name == "ARA_E_INVALID_ARG"
    t = engine.ylt_tail(y, 10)
    with pytest.raises(AraError) as ei:  # floor(1000 / 50) = 20 largest needed, 10 given
        engine.pml_tvar_tail(t, 1000, [50.0])
    assert ei.value.name == "ARA_E_INVALID_ARG"
    with pytest.raises(AraError) as ei:
        engine.pml_tvar_tail(t, 5, [1.0])
    assert ei.value.name == "ARA_E_INVALID_ARG"
    p, tv = engine.pml_tvar_tail(t, 1000, [100.0])
    assert p[0] == y[-10] and tv[0] == pytest.approx(y[-10:].mean(), rel=1e-15)


@pytest.mark.parametrize("world", [2, 3])
def test_bench_shard_step_with_the_engine(world):
    """bench.py's per-rank step with the real engine, its ranks run one after
    the other on this GPU (one engine per rank; the all-gather is a device
    copy, nothing waits on another rank): PML/TVaR of the union of the shards
    equals the oracle's on the concatenated shard YLTs."""
    import torch

    import bench
    from paper_1412_4556_b300 import Engine
    rps = [100.0, 250.0, 500.0]
    shards = [S.paper_scale(seed=bench.shard_seed(S.DEFAULT_SEED, r), n_trials=4_000, lam=200.0,
                            catalog_size=200_000) for r in range(world)]
    n = shards[0].yet.n_trials
    k = bench.tail_size(n, world, rps)
    dev = torch.device("cuda", 0)
    tails = [None] * world
    res = None
    for rank in reversed(range(world)):  # rank 0 last: it gathers every tail
        w = shards[rank]
        with Engine(0) as eng:
            eng.load_yet_from(w.yet)
            first = eng.load_pool(w.pool)
            handles = [first + j for j in w.layers[0].elts]
            ylt_out = torch.empty(n, dtype=torch.float64, device=dev)
            tail_out = torch.empty(k, dtype=torch.float64, device=dev)
            gather_out = torch.empty(k * world, dtype=torch.float64, device=dev)

            def all_gather(out, inp, rank=rank):
                torch.cuda.synchronize()
                tails[rank] = inp.clone()
                if rank == 0:
                    out.copy_(torch.cat(tails))
                torch.cuda.synchronize()

            r = bench.shard_step(eng, handles, w.layers[0], ylt_out, k, tail_out, gather_out, n, rank, world,
                                 rps, all_gather)
            torch.cuda.synchronize()
            if rank == 0:
                res = r
            else:
                assert r is None
    pml, tvar = res
    ylts, errs = [], []
    for w in shards:
        o, pre = oracle.layer_ylt(w.yet, w.pool, w.layers[0])
        ylts.append(o)
        errs.append(oracle.compare_fp64(_engine_ylt(w), o, pre)["max_abs_err"])
    ref = np.concatenate(ylts)
    pml_o, tvar_o = oracle.pml_tvar(ref, rps)
    pt = oracle.compare_pml_tvar(pml, tvar, pml_o, tvar_o, rps, ref.size, max(errs))
    assert pt["within_bound"], pt


def _engine_ylt(w):
    """The shard's YLT from a fresh engine (the step released its layer)."""
    from paper_1412_4556_b300 import Engine
    with Engine(0) as eng:
        eng.load_yet_from(w.yet)
        first = eng.load_pool(w.pool)
        L = w.layers[0]
        h = eng.define_layer([first + j for j in L.elts], L.occ_ret, L.occ_lim, L.agg_ret, L.agg_lim)
        return eng.layer_ylt(h)
