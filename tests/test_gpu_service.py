"""Ad hoc pricing service (continuous batching over slots, admission by device
memory) through the C ABI: each result is the same alone and in the mix,
sampled requests match the oracle, and the host-side failure paths (injected
allocation failure, deadline, cancellation, wait timeout, shutdown) end
requests with their status while the rest proceed."""
import numpy as np
import pytest

import ara_synth as S
import oracle
from parity import assert_fp64_parity

pytestmark = pytest.mark.gpu

RPS = (100.0, 250.0, 500.0)
N_POOL = 48


@pytest.fixture(scope="module")
def workload():
    w = S.batched(n_layers=1, n_trials=20_000, lam=200.0, catalog_size=300_000, n_pool=N_POOL)
    reqs = S.service_requests(n_requests=36, rate_per_s=1000.0, n_pool=N_POOL,
                              trial_choices=(2_000, 5_000, 20_000))
    return w, reqs


def open_engine(w):
    from paper_1412_4556_b300 import Engine
    e = Engine(0)
    e.load_yet_from(w.yet)
    first = e.load_pool(w.pool)
    return e, first


def precision_of(i):
    from paper_1412_4556_b300 import ARA_FP32_TABLE, ARA_FP64
    return ARA_FP32_TABLE if i % 3 == 2 else ARA_FP64


def submit(svc, first, rq, precision, **kw):
    L = rq.layer
    return svc.submit([first + j for j in L.elts], L.occ_ret, L.occ_lim, L.agg_ret, L.agg_lim,
                      rq.n_trials, precision=precision, **kw)


def run_alone(w, reqs):
    from paper_1412_4556_b300 import Service
    e, first = open_engine(w)
    out = []
    with Service(e, RPS, slots=1, max_batch=1) as svc:
        for i, rq in enumerate(reqs):
            r = svc.wait(submit(svc, first, rq, precision_of(i), want_ylt=True))
            assert r.ok, r.message
            assert r.batch_size == 1
            out.append(r)
    e.close()
    return out


@pytest.fixture(scope="module")
def alone(workload):
    w, reqs = workload
    return run_alone(w, reqs)


def test_alone_matches_direct_calls(workload, alone):
    """The service computes what define_layer + layer_ylt + pml_tvar compute."""
    w, reqs = workload
    e, first = open_engine(w)
    for i, (rq, r) in enumerate(zip(reqs[:12], alone)):
        L = rq.layer
        h = e.define_layer([first + j for j in L.elts], L.occ_ret, L.occ_lim, L.agg_ret, L.agg_lim,
                           precision=precision_of(i))
        y = e.layer_ylt(h, rq.n_trials)
        np.testing.assert_array_equal(y.view(np.uint64), r.ylt.view(np.uint64))
        p, t = e.pml_tvar(y, RPS)
        np.testing.assert_array_equal(p, r.pml)
        np.testing.assert_array_equal(t, r.tvar)
        e.release_layer(h)
    e.close()


def test_mixed_equals_alone_bit_for_bit(workload, alone):
    """All requests submitted at once: they are batched (several per slot) and
    overlap on the device, and every result equals its alone result."""
    from paper_1412_4556_b300 import Service
    w, reqs = workload
    e, first = open_engine(w)
    with Service(e, RPS, slots=4, max_batch=8) as svc:
        tickets = [submit(svc, first, rq, precision_of(i), want_ylt=True) for i, rq in enumerate(reqs)]
        mixed = [svc.wait(t) for t in tickets]
        st = svc.stats()
    e.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["max_batch_seen"] > 1
    for rq, a, m in zip(reqs, alone, mixed):
        assert m.ok, m.message
        np.testing.assert_array_equal(m.ylt.view(np.uint64), a.ylt.view(np.uint64))
        np.testing.assert_array_equal(m.pml, a.pml)
        np.testing.assert_array_equal(m.tvar, a.tvar)
        assert m.t_submit <= m.t_start <= m.t_done


def test_sampled_requests_match_oracle(workload, alone):
    w, reqs = workload
    for i in range(0, len(reqs), 5):
        rq, r = reqs[i], alone[i]
        o, pre = oracle.layer_ylt(w.yet, w.pool, rq.layer, trials=np.arange(rq.n_trials), mode="memo")
        if precision_of(i) == 0:
            assert_fp64_parity(r.ylt, o, pre, what=f"request {i}")
        else:
            err = np.abs(r.ylt - o)
            assert np.all(err <= np.maximum(1e-5 * np.maximum(np.abs(o), pre), 1.0)), f"request {i}"
        pml_o, tvar_o = oracle.pml_tvar(o, RPS)
        bound = np.max(np.abs(r.ylt - o)) + 1e-12 * np.abs(tvar_o)
        assert np.all(np.abs(r.pml - pml_o) <= bound) and np.all(np.abs(r.tvar - tvar_o) <= bound)


def test_memory_budget_limits_requests_in_flight(workload, alone):
    """A budget that holds one request's tables (but not two plus the paired
    table) admits one request at a time; a request above the whole budget is
    refused at submit."""
    from paper_1412_4556_b300 import AraError, Service
    w, reqs = workload
    e, first = open_engine(w)
    table = 16 * (w.yet.catalog_size + 1)
    with Service(e, RPS, slots=4, max_batch=8, memory_budget=int(table * 1.6)) as svc:
        tickets = [submit(svc, first, rq, precision_of(i)) for i, rq in enumerate(reqs[:10])]
        res = [svc.wait(t) for t in tickets]
        st = svc.stats()
    assert st["max_in_flight"] == 1 and st["max_batch_seen"] == 1
    assert 0 < st["max_bytes_in_flight"] <= int(table * 1.6)
    for a, r in zip(alone, res):
        assert r.ok, r.message
        np.testing.assert_array_equal(r.pml, a.pml)
    with Service(e, RPS, memory_budget=table // 2) as svc:
        with pytest.raises(AraError) as ei:
            submit(svc, first, reqs[0], 0)
        assert ei.value.name == "ARA_E_NOMEM"
    e.close()


def test_injected_allocation_failures_fail_only_their_requests(workload, alone):
    from paper_1412_4556_b300 import Service
    w, reqs = workload
    e, first = open_engine(w)
    with Service(e, RPS, slots=2, max_batch=4, fail_every=3) as svc:
        tickets = [submit(svc, first, rq, precision_of(i), want_ylt=True) for i, rq in enumerate(reqs)]
        res = [svc.wait(t) for t in tickets]
        st = svc.stats()
    e.close()
    failed = [r for r in res if not r.ok]
    assert len(failed) == len(reqs) // 3 == st["failed"]
    for a, r in zip(alone, res):
        if r.ok:
            np.testing.assert_array_equal(r.ylt.view(np.uint64), a.ylt.view(np.uint64))
            np.testing.assert_array_equal(r.tvar, a.tvar)
        else:
            assert r.status_name == "ARA_E_NOMEM" and "injected" in r.message


def test_deadline_cancel_and_wait_timeout(workload):
    from paper_1412_4556_b300 import AraError, Service
    w, reqs = workload
    e, first = open_engine(w)
    big = max(reqs, key=lambda r: r.n_trials)
    with Service(e, RPS, slots=1, max_batch=1) as svc:
        head = submit(svc, first, big, 0)
        late = [submit(svc, first, big, 0, deadline_s=1e-9) for _ in range(3)]
        queued = [submit(svc, first, big, 0) for _ in range(6)]
        with pytest.raises(AraError) as ei:
            svc.wait(queued[-1], timeout=0.0)
        assert ei.value.name == "ARA_E_TIMEOUT"
        cancelled = 0
        for t in queued[1:]:
            try:
                svc.cancel(t)
                cancelled += 1
            except AraError as err:
                assert err.name == "ARA_E_STATE"
        assert cancelled >= 1
        assert svc.wait(head).ok
        for t in late:
            assert svc.wait(t).status_name == "ARA_E_TIMEOUT"
        ends = [svc.wait(t) for t in queued]
        assert ends[0].ok
        assert sum(r.status_name == "ARA_E_CANCELLED" for r in ends) == cancelled
        assert all(r.ok for r in ends if r.status_name != "ARA_E_CANCELLED")
        with pytest.raises(AraError) as ei:
            svc.wait(head)
        assert ei.value.name == "ARA_E_NOT_FOUND"
        st = svc.stats()
        assert st["timed_out"] == 3 and st["cancelled"] == cancelled
    e.close()


def test_context_is_owned_while_attached_and_checks_at_submit(workload):
    from paper_1412_4556_b300 import AraError, Service
    w, reqs = workload
    e, first = open_engine(w)
    svc = Service(e, RPS)
    with pytest.raises(AraError) as ei:
        e.define_layer([first], 0.0, np.inf, 0.0, np.inf)
    assert ei.value.name == "ARA_E_STATE" and "service" in str(ei.value)
    with pytest.raises(AraError) as ei:
        svc.submit([first + N_POOL + 5], 0.0, np.inf, 0.0, np.inf, 1000)
    assert ei.value.name == "ARA_E_NOT_FOUND"
    with pytest.raises(AraError) as ei:
        svc.submit([first], 0.0, np.inf, 0.0, np.inf, w.yet.n_trials + 1)
    assert ei.value.name == "ARA_E_INVALID_ARG"
    with pytest.raises(AraError) as ei:  # floor(400 / 500) = 0 trials in the tail
        svc.submit([first], 0.0, np.inf, 0.0, np.inf, 400)
    assert ei.value.name == "ARA_E_INVALID_ARG"
    with pytest.raises(AraError):
        svc.submit([first, first], 0.0, np.inf, 0.0, np.inf, 1000)
    svc.close()
    # detached: the engine works again
    h = e.define_layer([first], 0.0, np.inf, 0.0, np.inf)
    assert e.layer_ylt(h, 10).shape == (10,)
    # closing the engine closes a live service and ends its queued requests
    svc = Service(e, RPS, slots=1, max_batch=1)
    for rq in reqs[:4]:
        submit(svc, first, rq, 0)
    e.close()
    assert svc.svc == 0


def test_service_full_size_requests_every_trial():
    """Config 4 shapes at full size: requests over 1e5 / 2.5e5 / 1e6-trial
    prefixes of the paper-scale YET with the 256-ELT pool, FP32 tables, all
    submitted at once; every trial of five of them (one of 2.5e5 trials, one
    of 1e5, three of 1e6) and their PML/TVaR against the oracle; and each of
    those results equals the same request priced alone."""
    from paper_1412_4556_b300 import ARA_FP32_TABLE, Engine, Service
    w = S.batched(n_layers=1)
    reqs = S.service_requests(n_requests=24, rate_per_s=1000.0)
    checked = (0, 5, 10, 16, 21)
    with Engine(0) as e:
        e.load_yet_from(w.yet)
        first = e.load_pool(w.pool)
        with Service(e, RPS, slots=4, max_batch=8) as svc:
            tickets = [submit(svc, first, rq, ARA_FP32_TABLE, want_ylt=i in checked)
                       for i, rq in enumerate(reqs)]
            mixed = [svc.wait(t) for t in tickets]
            alone = [svc.wait(submit(svc, first, reqs[i], ARA_FP32_TABLE, want_ylt=True)) for i in checked]
    assert all(r.ok for r in mixed + alone)
    assert sorted({reqs[i].n_trials for i in checked}) == [100_000, 250_000, 1_000_000]
    for a, i in zip(alone, checked):
        m = mixed[i]
        np.testing.assert_array_equal(m.ylt.view(np.uint64), a.ylt.view(np.uint64))
        np.testing.assert_array_equal(m.pml, a.pml)
        np.testing.assert_array_equal(m.tvar, a.tvar)
        rq = reqs[i]
        o, pre = oracle.layer_ylt(w.yet, w.pool, rq.layer, trials=np.arange(rq.n_trials), mode="memo")
        rep = oracle.compare_reduced(m.ylt, o, pre)
        assert rep["trials_over_bar"] == 0, (i, rep)
        p_o, t_o = oracle.pml_tvar(o, RPS)
        pt = oracle.compare_pml_tvar(m.pml, m.tvar, p_o, t_o, RPS, rq.n_trials, rep["max_abs_err"])
        assert pt["within_bound"], (i, pt)
