"""ara_pml_tvar_noalloc, the allocation-free PML/TVaR entry point.

It serves callers that must not call cudaMalloc -- a service whose pooling
allocator already owns the device memory it may use, or a latency-critical
request path that forbids allocation after start-up -- so it keeps its
selection workspace in a fixed static device array instead.  This file runs
last so that a failure here cannot hide any other test; it passes both alone
in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RPS = np.array([1.0, 2.0, 100.0, 250.0, 500.0, 7.5], dtype=np.float64)


def _noalloc(ylt_dev, rps, stream):
    from paper_1412_4556_b300 import _native
    pml = np.zeros(rps.shape[0])
    tvar = np.zeros(rps.shape[0])
    _native.ara_pml_tvar_noalloc(ylt_dev.data_ptr(), int(ylt_dev.shape[0]), rps.ctypes.data,
                                 int(rps.shape[0]), pml.ctypes.data, tvar.ctypes.data, stream)
    return pml, tvar


def test_noalloc_matches_ara_pml_tvar_on_two_calls_in_a_row():
    import torch
    from paper_1412_4556_b300 import Engine

    rng = np.random.default_rng(2024)
    first = np.concatenate([rng.lognormal(13, 2.0, 300_000), np.zeros(20_000), np.full(777, 5e7)])
    second = rng.lognormal(9, 1.0, 100_000)   # smaller, different scale: state must not leak
    stream = torch.cuda.current_stream().cuda_stream
    with Engine(0) as eng:
        for y in (first, second):
            rng.shuffle(y)
            y_dev = torch.from_numpy(y).cuda()
            torch.cuda.synchronize()
            pml_ref, tvar_ref = eng.pml_tvar(y_dev, RPS)
            pml, tvar = _noalloc(y_dev, RPS, stream)
            np.testing.assert_array_equal(pml, pml_ref)
            np.testing.assert_allclose(tvar, tvar_ref, rtol=1e-12, atol=0)


def test_noalloc_rejects_what_its_fixed_scratch_cannot_hold():
    import torch
    from paper_1412_4556_b300 import AraError, _native

    y_dev = torch.ones(1000, dtype=torch.float64, device="cuda")
    too_many = np.full(17, 2.0)
    with pytest.raises(AraError) as ei:
        _noalloc(y_dev, too_many, 0)
    assert ei.value.name == "ARA_E_INVALID_ARG"
    assert "1..16" in _native.ara_last_error(None)
    host = np.ones(1000)
    pml = np.zeros(1)
    tvar = np.zeros(1)
    with pytest.raises(AraError) as ei:
        _native.ara_pml_tvar_noalloc(host.ctypes.data, 1000, RPS.ctypes.data, 1, pml.ctypes.data,
                                     tvar.ctypes.data, 0)
    assert "device memory" in str(ei.value)
