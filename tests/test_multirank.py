"""Host logic of the multi-GPU path on CPU: gloo ranks each price their own
block of trials (as bench.py does under torchrun), all-gather their largest
losses (bench.tail_size of them, as ara_ylt_tail sends) and derive the
portfolio-wide PML/TVaR on rank 0.  The oracle and NumPy stand in for the
device kernels, so this runs without a GPU: PML/TVaR of the union padded
with zero losses to the whole trial count equal those of the whole YLT."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _shard(rank):
    import ara_synth as S
    import bench
    w = S.tiny(seed=bench.shard_seed(S.DEFAULT_SEED, rank), n_trials=300)
    return w


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    w = _shard(rank)
    ylt, _ = oracle.layer_ylt(w.yet, w.pool, w.layers[0], threads=1)
    import bench
    k = bench.tail_size(ylt.size, world, RPS)
    t = torch.from_numpy(np.sort(ylt)[-k:].copy())  # this shard's k largest
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t)
    if rank == 0:
        union = bench.merge_shard_tails([p.numpy() for p in parts])
        n_total = ylt.size * world
        padded = np.concatenate([union, np.zeros(n_total - union.size)])
        pml, tvar = oracle.pml_tvar(padded, RPS)
        out.put((union, pml, tvar))
    dist.barrier()
    dist.destroy_process_group()


RPS = [10.0, 30.0]


@pytest.mark.parametrize("world", [2, 3])
def test_shards_exchange_tails_and_merge(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    union, pml, tvar = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    import bench
    import oracle
    ref = []
    for r in range(world):
        w = _shard(r)
        ref.append(oracle.layer_ylt(w.yet, w.pool, w.layers[0], threads=1)[0])
    ref = np.concatenate(ref)
    k = bench.tail_size(ref.size // world, world, RPS)
    assert union.size == k * world and k == min(ref.size // world, ref.size // 10)
    pml_r, tvar_r = oracle.pml_tvar(ref, RPS)
    np.testing.assert_array_equal(pml, pml_r)
    np.testing.assert_array_equal(tvar, tvar_r)
    # the ranks priced different trials
    a, b = _shard(0), _shard(1)
    assert not np.array_equal(a.yet.ids[:200], b.yet.ids[:200])


class _CpuEngine:
    """Stands in for the CUDA engine where the step needs a GPU: layer_ylt by
    the oracle, ylt_tail and pml_tvar_tail by their documented definitions
    (the values above the k-th largest in index order, then copies of it;
    PML/TVaR of the union read as the whole YLT's k largest)."""

    def __init__(self, w):
        self.w = w
        self.layers = {}

    def define_layer(self, handles, occ_ret, occ_lim, agg_ret, agg_lim):
        import ara_synth as S
        h = len(self.layers) + 1
        self.layers[h] = S.Layer(list(handles), occ_ret, occ_lim, agg_ret, agg_lim)
        return h

    def release_layer(self, h):
        del self.layers[h]

    def layer_ylt(self, h, out):
        import oracle
        y, _ = oracle.layer_ylt(self.w.yet, self.w.pool, self.layers[h], threads=1)
        out.copy_(torch.from_numpy(y))
        return out

    def ylt_tail(self, ylt, k, out):
        y = ylt.numpy()
        tau = np.sort(y)[::-1][k - 1]
        above = y[y > tau]
        out.copy_(torch.from_numpy(np.concatenate([above, np.full(k - above.size, tau)])))
        return out

    def pml_tvar_tail(self, tail, n_total, rps):
        import oracle
        t = tail.numpy()
        return oracle.pml_tvar(np.concatenate([t, np.zeros(n_total - t.size)]), rps)


def _bench_step_worker(rank, world, port, out):
    """bench.shard_step end to end over gloo: the same tail size, buffers,
    all-gather and union pricing as the torchrun run of bench.py."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w = _shard(rank)
    eng = _CpuEngine(w)
    n = w.yet.n_trials
    k = bench.tail_size(n, world, RPS)
    ylt = torch.empty(n, dtype=torch.float64)
    tail = torch.empty(k, dtype=torch.float64)
    gathered = torch.empty(k * world, dtype=torch.float64)
    layer = w.layers[0]
    res = bench.shard_step(eng, layer.elts, layer, ylt, k, tail, gathered, n, rank, world, RPS,
                           lambda o, i: dist.all_gather_into_tensor(o, i))
    if rank == 0:
        out.put((gathered.numpy().copy(), res[0], res[1]))
    else:
        assert res is None
    assert not eng.layers  # the step released its layer
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_bench_shard_step_over_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_bench_step_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, pml, tvar = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    import bench
    import oracle
    ref = np.concatenate([oracle.layer_ylt(_shard(r).yet, _shard(r).pool, _shard(r).layers[0], threads=1)[0]
                          for r in range(world)])
    k = bench.tail_size(ref.size // world, world, RPS)
    assert gathered.size == k * world
    pml_r, tvar_r = oracle.pml_tvar(ref, RPS)
    np.testing.assert_array_equal(pml, pml_r)
    np.testing.assert_array_equal(tvar, tvar_r)
