"""ctypes binding of the C ABI in include/ara.h (libara_b300.so).

Every function here has the name of the C entry point it wraps and only
marshals arguments: pointers are passed as integers (``ndarray.ctypes.data``
or ``tensor.data_ptr()``), and a negative status raises :class:`AraError`
with the library's message.  All computation happens in the CUDA library;
there is no Python or CPU fallback, and importing fails when the library has
not been built.
"""
from __future__ import annotations

import ctypes as C
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libara_b300.so")

ARA_OK = 0
ARA_FP64 = 0
ARA_FP32_TABLE = 1
ARA_TIMING_YLT = 0
ARA_TIMING_FOLD = 1
ARA_TIMING_PML = 2
ARA_TIMING_YELT = 3

STATUS_NAMES = {
    0: "ARA_OK", -1: "ARA_E_INVALID_ARG", -2: "ARA_E_EVENT_RANGE", -3: "ARA_E_DUP_EVENT",
    -4: "ARA_E_NOMEM", -5: "ARA_E_CUDA", -6: "ARA_E_TIMEOUT", -7: "ARA_E_NOT_FOUND",
    -8: "ARA_E_STATE", -9: "ARA_E_CANCELLED",
}


class ServiceConfig(C.Structure):
    """ara_service_config."""
    _fields_ = [("slots", C.c_int32), ("max_batch", C.c_int32), ("memory_budget", C.c_int64),
                ("n_return_periods", C.c_int32), ("return_periods", C.c_double * 16),
                ("fail_every", C.c_int32)]


class Request(C.Structure):
    """ara_request."""
    _fields_ = [("n_elts", C.c_int32), ("elt_handles", C.c_void_p), ("occ_ret", C.c_double),
                ("occ_lim", C.c_double), ("agg_ret", C.c_double), ("agg_lim", C.c_double),
                ("precision", C.c_int32), ("n_trials", C.c_int64), ("deadline_s", C.c_double),
                ("ylt_out", C.c_void_p)]


class Result(C.Structure):
    """ara_result."""
    _fields_ = [("status", C.c_int32), ("batch_size", C.c_int32), ("slot", C.c_int32),
                ("n_return_periods", C.c_int32), ("pml", C.c_double * 16), ("tvar", C.c_double * 16),
                ("t_submit", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double),
                ("message", C.c_char * 160)]


class ServiceStats(C.Structure):
    """ara_service_stats."""
    _fields_ = [(n, C.c_int64) for n in (
        "submitted", "completed", "failed", "cancelled", "timed_out", "batches", "queued", "in_flight",
        "max_in_flight", "max_batch_seen", "bytes_in_flight", "max_bytes_in_flight", "memory_budget",
        "max_slots_busy")]

# C prototypes: name -> (restype, argtypes)
_vp, _i32, _i64, _f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double
PROTOTYPES = {
    "ara_create": (_i32, [C.POINTER(C.c_void_p), C.c_int]),
    "ara_destroy": (None, [_vp]),
    "ara_last_error": (C.c_char_p, [_vp]),
    "ara_status_string": (C.c_char_p, [_i32]),
    "ara_set_stream": (_i32, [_vp, _vp]),
    "ara_load_yet": (_i32, [_vp, _i32, _i64, _vp, _vp, _vp]),
    "ara_load_elts": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, C.POINTER(_i32)]),
    "ara_define_layer": (_i32, [_vp, _i32, _vp, _f64, _f64, _f64, _f64, _i32, C.POINTER(_i32)]),
    "ara_release_layer": (_i32, [_vp, _i32]),
    "ara_layer_event_table": (_i32, [_vp, _i32, _vp]),
    "ara_layer_ylt": (_i32, [_vp, _i32, _i64, _vp, _vp]),
    "ara_pml_tvar": (_i32, [_vp, _vp, _i64, _vp, _i32, _vp, _vp]),
    "ara_pml_tvar_async": (_i32, [_vp, _vp, _i64, _vp, _i32, _vp]),
    "ara_pml_tvar_noalloc": (_i32, [_vp, _i64, _vp, _i32, _vp, _vp, _vp]),
    "ara_ylt_tail": (_i32, [_vp, _vp, _i64, _i64, _vp]),
    "ara_pml_tvar_tail": (_i32, [_vp, _vp, _i64, _i64, _vp, _i32, _vp, _vp]),
    "ara_layers_ylt": (_i32, [_vp, _i32, _vp, _i64, _vp, _vp]),
    "ara_pml_tvar_batch": (_i32, [_vp, _vp, _i32, _i64, _vp, _i32, _vp, _vp]),
    "ara_set_kernel_timing": (_i32, [_vp, _i32]),
    "ara_kernel_timing": (_i32, [_vp, _i32, C.POINTER(_i64), C.POINTER(_f64)]),
    "ara_compact_yet": (_i32, [_vp]),
    "ara_layer_yelt": (_i32, [_vp, _i32, _i64, _vp, _vp, _vp]),
    "ara_rpl_report": (_i32, [_vp, _i32, _i64, _vp, _i32, _vp, _vp, _vp, _vp]),
    "ara_plan_create": (_i32, [_vp, _vp, _i32, _i64, _vp, _i32, _i32, C.POINTER(C.c_void_p)]),
    "ara_plan_run": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "ara_plan_passes": (_i32, [_vp, _i32, _vp, C.POINTER(_i32)]),
    "ara_plan_kernel_launches": (_i32, [_vp, C.POINTER(_i32)]),
    "ara_plan_destroy": (None, [_vp]),
    "ara_service_create": (_i32, [_vp, C.POINTER(ServiceConfig), C.POINTER(C.c_void_p)]),
    "ara_service_submit": (_i32, [_vp, C.POINTER(Request), C.POINTER(_i64)]),
    "ara_service_wait": (_i32, [_vp, _i64, _f64, C.POINTER(Result)]),
    "ara_service_cancel": (_i32, [_vp, _i64]),
    "ara_service_get_stats": (_i32, [_vp, C.POINTER(ServiceStats)]),
    "ara_service_destroy": (None, [_vp]),
    "ara_probe_gather": (_i32, [C.c_int, _i64, _i32, _i32, _i32, _i32, C.POINTER(_f64), C.POINTER(_f64)]),
    "ara_probe_smem_lookup": (_i32, [C.c_int, C.POINTER(_f64)]),
    "ara_probe_fp64_add": (_i32, [C.c_int, C.POINTER(_f64)]),
}


class AraError(RuntimeError):
    """A negative status from the C ABI."""

    def __init__(self, status: int, message: str):
        self.status = status
        self.name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{self.name}: {message}")


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python paper_1412_4556_b300/build.py`")
    lib = C.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = load_library()


def _check(ctx, status: int) -> None:
    if status != ARA_OK:
        msg = lib.ara_last_error(ctx)
        raise AraError(status, msg.decode() if msg else "")


def ara_create(device: int = 0) -> int:
    out = C.c_void_p()
    _check(None, lib.ara_create(C.byref(out), int(device)))
    return out.value


def ara_destroy(ctx: int) -> None:
    lib.ara_destroy(ctx)


def ara_last_error(ctx) -> str:
    m = lib.ara_last_error(ctx)
    return m.decode() if m else ""


def ara_status_string(status: int) -> str:
    return lib.ara_status_string(int(status)).decode()


def ara_set_stream(ctx: int, stream: int) -> None:
    _check(ctx, lib.ara_set_stream(ctx, stream or None))


def ara_load_yet(ctx: int, catalog_size: int, n_trials: int, offsets: int, ids: int, ts: int) -> None:
    _check(ctx, lib.ara_load_yet(ctx, int(catalog_size), int(n_trials), offsets or None, ids or None,
                                 ts or None))


def ara_load_elts(ctx: int, n_elts: int, offsets: int, ids: int, losses: int, deductibles: int,
                  limits: int) -> int:
    first = _i32(-1)
    _check(ctx, lib.ara_load_elts(ctx, int(n_elts), offsets or None, ids or None, losses or None,
                                  deductibles or None, limits or None, C.byref(first)))
    return first.value


def ara_define_layer(ctx: int, n_elts: int, handles: int, occ_ret: float, occ_lim: float,
                     agg_ret: float, agg_lim: float, precision: int = ARA_FP64) -> int:
    out = _i32(-1)
    _check(ctx, lib.ara_define_layer(ctx, int(n_elts), handles or None, float(occ_ret), float(occ_lim),
                                     float(agg_ret), float(agg_lim), int(precision), C.byref(out)))
    return out.value


def ara_release_layer(ctx: int, layer: int) -> None:
    _check(ctx, lib.ara_release_layer(ctx, int(layer)))


def ara_layer_event_table(ctx: int, layer: int, out: int) -> None:
    _check(ctx, lib.ara_layer_event_table(ctx, int(layer), out or None))


def ara_layer_ylt(ctx: int, layer: int, n_trials: int, ylt_out: int, stream: int = 0) -> None:
    _check(ctx, lib.ara_layer_ylt(ctx, int(layer), int(n_trials), ylt_out or None, stream or None))


def ara_pml_tvar(ctx: int, ylt: int, n: int, return_periods: int, n_rp: int, pml_out: int,
                 tvar_out: int) -> None:
    _check(ctx, lib.ara_pml_tvar(ctx, ylt or None, int(n), return_periods or None, int(n_rp),
                                 pml_out or None, tvar_out or None))


def ara_pml_tvar_async(ctx: int, ylt: int, n: int, return_periods: int, n_rp: int, out: int) -> None:
    _check(ctx, lib.ara_pml_tvar_async(ctx, ylt or None, int(n), return_periods or None, int(n_rp), out or None))


def ara_ylt_tail(ctx: int, ylt: int, n: int, k: int, tail_out: int) -> None:
    _check(ctx, lib.ara_ylt_tail(ctx, ylt or None, int(n), int(k), tail_out or None))


def ara_pml_tvar_tail(ctx: int, tail: int, m: int, n_total: int, return_periods: int, n_rp: int,
                      pml_out: int, tvar_out: int) -> None:
    _check(ctx, lib.ara_pml_tvar_tail(ctx, tail or None, int(m), int(n_total), return_periods or None,
                                      int(n_rp), pml_out or None, tvar_out or None))


def ara_layers_ylt(ctx: int, n_layers: int, layers: int, n_trials: int, ylt_out: int,
                   stream: int = 0) -> None:
    _check(ctx, lib.ara_layers_ylt(ctx, int(n_layers), layers or None, int(n_trials), ylt_out or None,
                                   stream or None))


def ara_pml_tvar_batch(ctx: int, ylt: int, n_layers: int, n: int, return_periods: int, n_rp: int,
                       pml_out: int, tvar_out: int) -> None:
    _check(ctx, lib.ara_pml_tvar_batch(ctx, ylt or None, int(n_layers), int(n), return_periods or None,
                                       int(n_rp), pml_out or None, tvar_out or None))


def ara_pml_tvar_noalloc(ylt: int, n: int, return_periods: int, n_rp: int, pml_out: int,
                         tvar_out: int, stream: int = 0) -> None:
    """Context-free PML/TVaR that allocates no device memory (ylt on the device)."""
    _check(None, lib.ara_pml_tvar_noalloc(ylt or None, int(n), return_periods or None, int(n_rp),
                                          pml_out or None, tvar_out or None, stream or None))


def ara_compact_yet(ctx: int) -> None:
    _check(ctx, lib.ara_compact_yet(ctx))


def ara_layer_yelt(ctx: int, layer: int, n_trials: int, yelt_out: int, occ_max_out: int,
                   stream: int = 0) -> None:
    _check(ctx, lib.ara_layer_yelt(ctx, int(layer), int(n_trials), yelt_out or None, occ_max_out or None,
                                   stream or None))


def ara_rpl_report(ctx: int, layer: int, n_trials: int, return_periods: int, n_rp: int, aep: int,
                   aep_tvar: int, oep: int, oep_tvar: int) -> None:
    _check(ctx, lib.ara_rpl_report(ctx, int(layer), int(n_trials), return_periods or None, int(n_rp),
                                   aep or None, aep_tvar or None, oep or None, oep_tvar or None))


def ara_plan_create(ctx: int, n_layers: int, layers: int, n_trials: int, return_periods: int, n_rp: int,
                    autotune: bool) -> int:
    out = C.c_void_p()
    _check(ctx, lib.ara_plan_create(ctx, layers or None, int(n_layers), int(n_trials), return_periods or None,
                                    int(n_rp), 1 if autotune else 0, C.byref(out)))
    return out.value


def ara_plan_run(ctx: int, plan: int, ylt_out: int, pml_out: int, tvar_out: int, stream: int = 0) -> None:
    """(ctx is the plan's context, for the error message.)"""
    _check(ctx, lib.ara_plan_run(plan, ylt_out or None, pml_out or None, tvar_out or None, stream or None))


def ara_plan_passes(ctx: int, plan: int):
    """List of (entry bytes, layers G, lanes per trial, unroll, prefetch, threads per CTA,
    (positions of the G layers)) per YLT pass."""
    n = _i32(0)
    _check(ctx, lib.ara_plan_passes(plan, 0, None, C.byref(n)))
    info = (_i32 * (10 * max(n.value, 1)))()
    _check(ctx, lib.ara_plan_passes(plan, n.value, info, C.byref(n)))
    out = []
    for i in range(n.value):
        eb, g, lpt, u, pf, th = info[10 * i:10 * i + 6]
        out.append((eb, g, lpt, u, pf, th, tuple(info[10 * i + 6:10 * i + 6 + g])))
    return out


def ara_plan_kernel_launches(ctx: int, plan: int) -> int:
    """Kernel launches one replay of the plan makes."""
    n = _i32(0)
    _check(ctx, lib.ara_plan_kernel_launches(plan, C.byref(n)))
    return n.value


def ara_plan_destroy(plan: int) -> None:
    lib.ara_plan_destroy(plan)


def ara_set_kernel_timing(ctx: int, enable: bool) -> None:
    _check(ctx, lib.ara_set_kernel_timing(ctx, 1 if enable else 0))


def ara_kernel_timing(ctx: int, channel: int):
    n, ms = _i64(0), _f64(0.0)
    _check(ctx, lib.ara_kernel_timing(ctx, int(channel), C.byref(n), C.byref(ms)))
    return n.value, ms.value


def ara_service_create(ctx: int, config: ServiceConfig) -> int:
    out = C.c_void_p()
    _check(None, lib.ara_service_create(ctx, C.byref(config), C.byref(out)))
    return out.value


def ara_service_submit(svc: int, request: Request) -> int:
    ticket = _i64(0)
    _check(None, lib.ara_service_submit(svc, C.byref(request), C.byref(ticket)))
    return ticket.value


def ara_service_wait(svc: int, ticket: int, timeout_s: float) -> Result:
    """The request's result; AraError(ARA_E_TIMEOUT) if it has not ended in time."""
    out = Result()
    _check(None, lib.ara_service_wait(svc, int(ticket), float(timeout_s), C.byref(out)))
    return out


def ara_service_cancel(svc: int, ticket: int) -> None:
    _check(None, lib.ara_service_cancel(svc, int(ticket)))


def ara_service_get_stats(svc: int) -> ServiceStats:
    out = ServiceStats()
    _check(None, lib.ara_service_get_stats(svc, C.byref(out)))
    return out


def ara_service_destroy(svc: int) -> None:
    lib.ara_service_destroy(svc)


def ara_probe_gather(device: int, table_bytes: int, load_bytes: int, lanes_per_row: int,
                     threads_per_cta: int = 1024, ctas_per_sm: int = 1):
    """(rows/s, 32-byte sectors/s) of random row reads from an L2-resident table."""
    rows, sectors = _f64(0.0), _f64(0.0)
    _check(None, lib.ara_probe_gather(int(device), int(table_bytes), int(load_bytes), int(lanes_per_row),
                                      int(threads_per_cta), int(ctas_per_sm), C.byref(rows), C.byref(sectors)))
    return rows.value, sectors.value


def ara_probe_smem_lookup(device: int) -> float:
    """Random 32-bit shared-memory lookups per second over the device."""
    out = _f64(0.0)
    _check(None, lib.ara_probe_smem_lookup(int(device), C.byref(out)))
    return out.value


def ara_probe_fp64_add(device: int) -> float:
    """Binary64 adds per second over the device."""
    out = _f64(0.0)
    _check(None, lib.ara_probe_fp64_add(int(device), C.byref(out)))
    return out.value
