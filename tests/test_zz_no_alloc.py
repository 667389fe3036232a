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


def _noalloc_dev_out(ylt_dev, rps, stream):
    """The same call with device-resident outputs."""
    import torch
    from paper_1412_4556_b300 import _native
    pml = torch.zeros(rps.shape[0], dtype=torch.float64, device=ylt_dev.device)
    tvar = torch.zeros(rps.shape[0], dtype=torch.float64, device=ylt_dev.device)
    _native.ara_pml_tvar_noalloc(ylt_dev.data_ptr(), int(ylt_dev.shape[0]), rps.ctypes.data,
                                 int(rps.shape[0]), pml.data_ptr(), tvar.data_ptr(), stream)
    return pml.cpu().numpy(), tvar.cpu().numpy()


def _bits(a):
    return np.asarray(a, dtype=np.float64).view(np.uint64)


# 16 return periods fill the fixed scratch (its output and error words sit at
# the array's end); RP 1 selects every trial (k = n).
RPS16 = np.array([1.0, 1.5, 2.0, 3.0, 7.5, 10.0, 25.0, 50.0, 100.0, 200.0, 250.0, 400.0, 500.0, 750.0,
                  1000.0, 2500.0], dtype=np.float64)


@pytest.mark.parametrize("rps", [RPS, np.array([1.0]), RPS16], ids=["6rp", "1rp_k_eq_n", "16rp"])
@pytest.mark.parametrize("device_out", [False, True], ids=["host_out", "device_out"])
def test_noalloc_matches_ara_pml_tvar_on_two_calls_in_a_row(rps, device_out):
    import torch
    from paper_1412_4556_b300 import Engine

    rng = np.random.default_rng(2024)
    first = np.concatenate([rng.lognormal(13, 2.0, 300_000), np.zeros(20_000), np.full(777, 5e7)])
    second = rng.lognormal(9, 1.0, 100_000)   # smaller, different scale: state must not leak
    zeros = np.zeros(5_000)                    # a layer that never pays
    stream = torch.cuda.current_stream().cuda_stream
    call = _noalloc_dev_out if device_out else _noalloc
    with Engine(0) as eng:
        for y in (first, second, zeros):
            rng.shuffle(y)
            y_dev = torch.from_numpy(y).cuda()
            torch.cuda.synchronize()
            pml_ref, tvar_ref = eng.pml_tvar(y_dev, rps)
            pml, tvar = call(y_dev, rps, stream)
            np.testing.assert_array_equal(_bits(pml), _bits(pml_ref))
            np.testing.assert_array_equal(_bits(tvar), _bits(tvar_ref))
            if y is zeros:
                assert not pml.any() and not tvar.any()


def test_noalloc_refuses_another_gpus_memory_before_any_launch():
    """A YLT in another GPU's memory is refused on the host (the kernels on
    the current device could not read it); needs a second GPU."""
    import torch
    from paper_1412_4556_b300 import AraError, _native

    if torch.cuda.device_count() < 2:
        pytest.skip("one GPU: no memory of another device to pass")
    y_other = torch.ones(1000, dtype=torch.float64, device="cuda:1")
    torch.cuda.set_device(0)
    with pytest.raises(AraError) as ei:
        _noalloc(y_other, RPS[:1], 0)
    assert ei.value.name == "ARA_E_INVALID_ARG"
    assert "device 1" in _native.ara_last_error(None)


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
