"""B300 engine for the Year Loss Table of Aggregate Risk Analysis.

Varghese & Barker, "Are Clouds Ready to Accelerate Ad hoc Financial
Simulations?" (arXiv 1412.4556), Section III, Algorithm 1: for every layer and
trial, look each event of the trial up in the layer's ELTs, apply the ELT
terms, combine across ELTs, apply the occurrence terms, accumulate with the
aggregate terms, and report the trial loss; PML and TVaR follow from the YLT.

The computation runs in hand-written CUDA kernels behind the C ABI of
``include/ara.h`` (``libara_b300.so``).  :mod:`._native` binds each C entry
point under its own name; :class:`Engine` adds array marshalling for NumPy
arrays (host memory) and torch tensors (device memory).  PyTorch is only used
for device buffers and streams.
"""
from __future__ import annotations

from typing import Optional, Sequence, Tuple

import numpy as np

from . import _native
from ._native import (ARA_FP32_TABLE, ARA_FP64, ARA_TIMING_FOLD, ARA_TIMING_PML, ARA_TIMING_YELT,
                      ARA_TIMING_YLT, AraError)

__all__ = ["Engine", "Plan", "Service", "ServiceResult", "AraError", "ARA_FP64", "ARA_FP32_TABLE",
           "ARA_TIMING_YLT", "ARA_TIMING_FOLD", "ARA_TIMING_PML", "ARA_TIMING_YELT"]


def _is_tensor(a) -> bool:
    return type(a).__module__.startswith("torch")


def _arg(a, dtype, name: str):
    """(pointer, keep-alive object) for a NumPy array or a torch tensor."""
    if a is None:
        return 0, None
    if _is_tensor(a):
        import torch
        want = {np.int64: torch.int64, np.int32: torch.int32, np.float64: torch.float64,
                np.float32: torch.float32}[dtype]
        if a.dtype != want:
            raise TypeError(f"{name}: expected {want}, got {a.dtype}")
        if not a.is_contiguous():
            a = a.contiguous()
        return a.data_ptr(), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data, arr


class Engine:
    """One context of the CUDA engine on one GPU."""

    def __init__(self, device: int = 0, stream=None):
        self.ctx = _native.ara_create(device)
        self.device = device
        self._service = None
        self._plans = []
        self.catalog_size = 0
        self.n_trials = 0
        if stream is not None:
            self.set_stream(stream)

    # -------------------------------------------------------------- lifetime
    def close(self) -> None:
        if self._service is not None:
            self._service.close()
        for p in list(self._plans):
            p.close()
        if self.ctx:
            _native.ara_destroy(self.ctx)
            self.ctx = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream) -> None:
        """Queue later work on a torch.cuda.Stream (or a raw cudaStream_t int)."""
        handle = getattr(stream, "cuda_stream", stream)
        _native.ara_set_stream(self.ctx, int(handle or 0))

    # ------------------------------------------------------------------ data
    def load_yet(self, catalog_size: int, offsets, ids, ts=None) -> None:
        n_trials = int(offsets.shape[0]) - 1
        p_off, k1 = _arg(offsets, np.int64, "offsets")
        p_ids, k2 = _arg(ids, np.int32, "ids")
        p_ts, k3 = _arg(ts, np.float32, "ts")
        _native.ara_load_yet(self.ctx, int(catalog_size), n_trials, p_off, p_ids, p_ts)
        self._offsets_host = (offsets.detach().cpu().numpy() if _is_tensor(offsets)
                              else np.asarray(offsets, dtype=np.int64)).copy()
        self.catalog_size = int(catalog_size)
        self.n_trials = n_trials

    def load_yet_from(self, yet) -> None:
        """Load an :class:`ara_synth.YET`-like object (catalog_size, offsets, ids, ts)."""
        self.load_yet(yet.catalog_size, yet.offsets, yet.ids, yet.ts)

    def compact_yet(self) -> None:
        """Sorted, difference-coded id stream for later YLT passes (same results)."""
        _native.ara_compact_yet(self.ctx)

    def load_elts(self, offsets, ids, losses, deductibles, limits) -> int:
        n = int(np.asarray(offsets).shape[0]) - 1
        p = [_arg(offsets, np.int64, "offsets"), _arg(ids, np.int32, "ids"),
             _arg(losses, np.float64, "losses"), _arg(deductibles, np.float64, "deductibles"),
             _arg(limits, np.float64, "limits")]
        return _native.ara_load_elts(self.ctx, n, *[x[0] for x in p])

    def load_pool(self, pool) -> int:
        """Load an :class:`ara_synth.ELTPool`-like object; returns the first handle."""
        return self.load_elts(pool.offsets, pool.ids, pool.losses, pool.deductibles, pool.limits)

    def define_layer(self, elt_handles: Sequence[int], occ_ret: float, occ_lim: float,
                     agg_ret: float, agg_lim: float, precision: int = ARA_FP64) -> int:
        h = np.ascontiguousarray(elt_handles, dtype=np.int32)
        return _native.ara_define_layer(self.ctx, int(h.shape[0]), h.ctypes.data, occ_ret, occ_lim,
                                        agg_ret, agg_lim, precision)

    def release_layer(self, layer: int) -> None:
        _native.ara_release_layer(self.ctx, layer)

    # --------------------------------------------------------------- compute
    def layer_ylt(self, layer: int, n_trials: Optional[int] = None, out=None, stream=None):
        """YLT of one layer over the first n_trials trials.

        ``out`` may be a float64 NumPy array (host) or a CUDA torch tensor
        (device, filled asynchronously on the engine's stream); by default a
        new NumPy array is returned.
        """
        n = self.n_trials if n_trials is None else int(n_trials)
        if out is None:
            out = np.empty(n, dtype=np.float64)
        if int(out.shape[0]) < n:
            raise ValueError("out is shorter than n_trials")
        p, keep = _arg(out, np.float64, "out")
        if keep is not out:
            raise TypeError("out must be a contiguous float64 array or tensor")
        handle = getattr(stream, "cuda_stream", stream) if stream is not None else 0
        _native.ara_layer_ylt(self.ctx, layer, n, p, int(handle or 0))
        return out

    def layers_ylt(self, layers: Sequence[int], n_trials: Optional[int] = None, out=None, stream=None):
        """YLTs of several layers in one call: array [len(layers), n_trials]
        (NumPy by default, or a CUDA tensor given as ``out``)."""
        h = np.ascontiguousarray(layers, dtype=np.int32)
        n = self.n_trials if n_trials is None else int(n_trials)
        if out is None:
            out = np.empty((h.shape[0], n), dtype=np.float64)
        p, keep = _arg(out, np.float64, "out")
        if keep is not out:
            raise TypeError("out must be a contiguous float64 array or tensor")
        handle = getattr(stream, "cuda_stream", stream) if stream is not None else 0
        _native.ara_layers_ylt(self.ctx, int(h.shape[0]), h.ctypes.data, n, p, int(handle or 0))
        return out

    def pml_tvar_batch(self, ylts, return_periods: Sequence[float]):
        """PML and TVaR per layer of a [n_layers, n] YLT array: two [n_layers, n_rp] arrays."""
        p, keep = _arg(ylts, np.float64, "ylts")
        n_layers, n = int(ylts.shape[0]), int(ylts.shape[1])
        rps = np.ascontiguousarray(return_periods, dtype=np.float64)
        pml = np.zeros((n_layers, rps.shape[0]))
        tvar = np.zeros((n_layers, rps.shape[0]))
        _native.ara_pml_tvar_batch(self.ctx, p, n_layers, n, rps.ctypes.data, int(rps.shape[0]),
                                   pml.ctypes.data, tvar.ctypes.data)
        return pml, tvar

    def layer_yelt(self, layer: int, n_trials: Optional[int] = None, out=None, occ_max=None,
                   want_yelt: bool = True, stream=None):
        """Year Event Loss Table: (per-occurrence increments in the YET's CSR
        order, largest increment per trial).  ``out``/``occ_max`` may be
        float64 NumPy arrays or CUDA tensors; with ``want_yelt=False`` only
        the per-trial maxima are produced (the first value is then None)."""
        n = self.n_trials if n_trials is None else int(n_trials)
        if out is None and want_yelt:
            # (an n outside [0, n_trials] is rejected by the library)
            out = np.empty(int(self._offsets_host[min(max(n, 0), self.n_trials)]), dtype=np.float64)
        if occ_max is None:
            occ_max = np.empty(max(n, 0), dtype=np.float64)
        p1, k1 = _arg(out, np.float64, "out")
        p2, k2 = _arg(occ_max, np.float64, "occ_max")
        if (out is not None and k1 is not out) or k2 is not occ_max:
            raise TypeError("outputs must be contiguous float64 arrays or tensors")
        handle = getattr(stream, "cuda_stream", stream) if stream is not None else 0
        _native.ara_layer_yelt(self.ctx, layer, n, p1, p2, int(handle or 0))
        return out, occ_max

    def rpl_report(self, layer: int, return_periods: Sequence[float], n_trials: Optional[int] = None):
        """Return period losses: dict of aep, aep_tvar, oep, oep_tvar arrays."""
        n = self.n_trials if n_trials is None else int(n_trials)
        rps = np.ascontiguousarray(return_periods, dtype=np.float64)
        outs = [np.zeros(rps.shape[0]) for _ in range(4)]
        _native.ara_rpl_report(self.ctx, layer, n, rps.ctypes.data, int(rps.shape[0]),
                               *[o.ctypes.data for o in outs])
        return dict(zip(("aep", "aep_tvar", "oep", "oep_tvar"), outs))

    def event_table(self, layer: int, out=None):
        """The layer's per-event occurrence-net loss (float64, one per catalog event)."""
        if out is None:
            out = np.empty(self.catalog_size, dtype=np.float64)
        p, keep = _arg(out, np.float64, "out")
        if keep is not out:
            raise TypeError("out must be a contiguous float64 array or tensor")
        _native.ara_layer_event_table(self.ctx, layer, p)
        return out

    def pml_tvar(self, ylt, return_periods: Sequence[float]) -> Tuple[np.ndarray, np.ndarray]:
        p, keep = _arg(ylt, np.float64, "ylt")
        rps = np.ascontiguousarray(return_periods, dtype=np.float64)
        pml = np.zeros(rps.shape[0])
        tvar = np.zeros(rps.shape[0])
        _native.ara_pml_tvar(self.ctx, p, int(ylt.shape[0]), rps.ctypes.data, int(rps.shape[0]),
                             pml.ctypes.data, tvar.ctypes.data)
        return pml, tvar

    def pml_tvar_async(self, ylt, return_periods: Sequence[float], out):
        """PML and TVaR of a CUDA-tensor YLT queued on the engine's stream
        without waiting: ``out`` (a CUDA float64 tensor of 2 * len(return_periods)
        values) receives the PMLs, then the TVaRs, in stream order (quiet NaNs
        when the losses fail their check)."""
        p, keep = _arg(ylt, np.float64, "ylt")
        po, ko = _arg(out, np.float64, "out")
        if keep is not ylt or ko is not out:
            # a temporary copy could be freed before the queued work reads it
            raise TypeError("ylt and out must be contiguous float64 CUDA tensors")
        rps = np.ascontiguousarray(return_periods, dtype=np.float64)
        _native.ara_pml_tvar_async(self.ctx, p, int(ylt.shape[0]), rps.ctypes.data, int(rps.shape[0]), po)
        return out

    def ylt_tail(self, ylt, k: int, out=None):
        """The k largest values of a YLT (NumPy array or CUDA tensor): the
        values above the k-th largest in index order, then copies of it.
        ``out`` may be a float64 NumPy array or CUDA tensor of k values."""
        p, keep = _arg(ylt, np.float64, "ylt")
        if out is None:
            out = np.empty(int(k), dtype=np.float64)
        po, ko = _arg(out, np.float64, "out")
        if ko is not out:
            raise TypeError("out must be a contiguous float64 array or tensor")
        _native.ara_ylt_tail(self.ctx, p, int(ylt.shape[0]), int(k), po)
        return out

    def pml_tvar_tail(self, tail, n_total: int, return_periods: Sequence[float]):
        """PML and TVaR of a YLT of n_total trials from values of it that
        include its floor(n_total / RP) largest (e.g. shards' ylt_tail)."""
        p, keep = _arg(tail, np.float64, "tail")
        rps = np.ascontiguousarray(return_periods, dtype=np.float64)
        pml = np.zeros(rps.shape[0])
        tvar = np.zeros(rps.shape[0])
        _native.ara_pml_tvar_tail(self.ctx, p, int(tail.shape[0]), int(n_total), rps.ctypes.data,
                                  int(rps.shape[0]), pml.ctypes.data, tvar.ctypes.data)
        return pml, tvar

    # ----------------------------------------------------------- measurement
    def set_kernel_timing(self, enable: bool = True) -> None:
        _native.ara_set_kernel_timing(self.ctx, enable)

    def kernel_timing(self, channel: int = ARA_TIMING_YLT):
        """(launches, total milliseconds) recorded on a timing channel."""
        return _native.ara_kernel_timing(self.ctx, channel)


class Plan:
    """A fixed list of layers priced as one CUDA graph (see ``ara_plan_create``)."""

    def __init__(self, engine: Engine, layers: Sequence[int], return_periods: Sequence[float],
                 n_trials: Optional[int] = None, autotune: bool = True):
        h = np.ascontiguousarray(layers, dtype=np.int32)
        rps = np.ascontiguousarray(return_periods, dtype=np.float64)
        self.engine = engine
        self.n_layers = int(h.shape[0])
        self.n_trials = engine.n_trials if n_trials is None else int(n_trials)
        self.n_rp = int(rps.shape[0])
        self.plan = _native.ara_plan_create(engine.ctx, self.n_layers, h.ctypes.data, self.n_trials,
                                            rps.ctypes.data, self.n_rp, autotune)
        engine._plans.append(self)

    def run(self, ylt_out=None, stream=None, want_pml: bool = True):
        """Replay: (pml, tvar) arrays [n_layers, n_rp] (None with want_pml=False);
        ``ylt_out`` (NumPy array or CUDA tensor [n_layers, n_trials]) receives the YLTs."""
        p, keep = _arg(ylt_out, np.float64, "ylt_out")
        if ylt_out is not None and keep is not ylt_out:
            raise TypeError("ylt_out must be a contiguous float64 array or tensor")
        pml = np.zeros((self.n_layers, self.n_rp)) if want_pml else None
        tvar = np.zeros((self.n_layers, self.n_rp)) if want_pml else None
        handle = getattr(stream, "cuda_stream", stream) if stream is not None else 0
        _native.ara_plan_run(self.engine.ctx, self.plan, p, pml.ctypes.data if want_pml else 0,
                             tvar.ctypes.data if want_pml else 0, int(handle or 0))
        return pml, tvar

    def passes(self):
        return _native.ara_plan_passes(self.engine.ctx, self.plan)

    def kernel_launches(self) -> int:
        """Kernel launches one run replays (the kernel nodes of the plan's graph)."""
        return _native.ara_plan_kernel_launches(self.engine.ctx, self.plan)

    def close(self) -> None:
        if self.plan:
            _native.ara_plan_destroy(self.plan)
            self.plan = 0
            self.engine._plans.remove(self)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class ServiceResult:
    """Outcome of one pricing request (see ara_result)."""

    def __init__(self, r: "_native.Result", ylt):
        self.status = r.status
        self.status_name = _native.STATUS_NAMES.get(r.status, str(r.status))
        self.message = r.message.decode(errors="replace")
        self.batch_size = r.batch_size
        self.slot = r.slot
        n = r.n_return_periods
        self.pml = np.array(r.pml[:n])
        self.tvar = np.array(r.tvar[:n])
        self.t_submit, self.t_start, self.t_done = r.t_submit, r.t_start, r.t_done
        self.ylt = ylt

    @property
    def ok(self) -> bool:
        return self.status == _native.ARA_OK

    @property
    def latency(self) -> float:
        """Seconds from submit to the end of the request."""
        return self.t_done - self.t_submit


class Service:
    """Ad hoc pricing service on an :class:`Engine` (see ``ara_service_create``).

    While it runs, the engine's context belongs to the service's scheduler
    thread; other engine calls raise ``AraError(ARA_E_STATE)``.
    """

    def __init__(self, engine: Engine, return_periods: Sequence[float] = (100.0, 250.0, 500.0),
                 slots: int = 4, max_batch: int = 16, memory_budget: int = 0, fail_every: int = 0):
        if engine._service is not None:
            raise AraError(-8, "the engine already has a service")
        cfg = _native.ServiceConfig()
        cfg.slots, cfg.max_batch, cfg.memory_budget = int(slots), int(max_batch), int(memory_budget)
        rps = list(return_periods)
        if not 1 <= len(rps) <= 16:
            raise ValueError("1..16 return periods")
        cfg.n_return_periods = len(rps)
        for i, r in enumerate(rps):
            cfg.return_periods[i] = float(r)
        cfg.fail_every = int(fail_every)
        self.engine = engine
        self.return_periods = np.array(rps, dtype=np.float64)
        self.svc = _native.ara_service_create(engine.ctx, cfg)
        engine._service = self
        self._ylt = {}  # ticket -> host YLT buffer kept alive until the request is collected

    def submit(self, elt_handles: Sequence[int], occ_ret: float, occ_lim: float, agg_ret: float,
               agg_lim: float, n_trials: int, precision: int = ARA_FP64, deadline_s: float = 0.0,
               want_ylt: bool = False) -> int:
        h = np.ascontiguousarray(elt_handles, dtype=np.int32)
        rq = _native.Request()
        rq.n_elts = int(h.shape[0])
        rq.elt_handles = h.ctypes.data
        rq.occ_ret, rq.occ_lim, rq.agg_ret, rq.agg_lim = map(float, (occ_ret, occ_lim, agg_ret, agg_lim))
        rq.precision = int(precision)
        rq.n_trials = int(n_trials)
        rq.deadline_s = float(deadline_s)
        ylt = np.empty(int(n_trials), dtype=np.float64) if want_ylt else None
        rq.ylt_out = ylt.ctypes.data if ylt is not None else None
        ticket = _native.ara_service_submit(self.svc, rq)
        if ylt is not None:
            self._ylt[ticket] = ylt
        return ticket

    def wait(self, ticket: int, timeout: float = 600.0) -> ServiceResult:
        r = _native.ara_service_wait(self.svc, ticket, timeout)
        return ServiceResult(r, self._ylt.pop(ticket, None))

    def cancel(self, ticket: int) -> None:
        _native.ara_service_cancel(self.svc, ticket)

    def stats(self) -> dict:
        s = _native.ara_service_get_stats(self.svc)
        return {name: getattr(s, name) for name, _ in s._fields_}

    def close(self) -> None:
        if self.svc:
            _native.ara_service_destroy(self.svc)
            self.svc = 0
            self.engine._service = None
            self._ylt.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
