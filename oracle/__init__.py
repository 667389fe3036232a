"""FP64 CPU oracle for the Year Loss Table of Aggregate Risk Analysis.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the engine in
``paper_1412_4556_b300`` never does, and this package imports nothing from it.

The arithmetic lives in ``ara_oracle.c`` (plain C, binary64, built with
``-O2 -ffp-contract=off``), which follows Algorithm 1 of Varghese & Barker
(arXiv 1412.4556, Section III) loop by loop.  This module only compiles it
and marshals NumPy arrays into it.

Parity of secondary uncertainty (Section III, step 2) is unpinned: the paper
never defines it, so it is taken as the identity and not modelled.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ara_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libara_oracle.so")
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread", "-std=c11"]

_lib = None


class OracleError(RuntimeError):
    pass


def build(src: str = _SRC, out: str = _LIB, force: bool = False) -> str:
    """Compile the oracle with gcc (only when the source is newer)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, src, "-lm"])
        os.replace(tmp, out)
    return out


def load(path: Optional[str] = None):
    """Load (building first if needed) and type the oracle library."""
    global _lib
    if path is None and _lib is not None:
        return _lib
    lib = C.CDLL(path or build())
    p = C.c_void_p
    i32, i64, f64 = C.c_int32, C.c_int64, C.c_double
    lib.ara_oracle_layer_ylt.argtypes = [i32, i64, p, p, i32, p, p, p, p, p, f64, f64, f64, f64,
                                         i32, i32, p, i64, p, p]
    lib.ara_oracle_layer_ylt.restype = C.c_int
    lib.ara_oracle_layers_ylt.argtypes = [i32, i64, p, p, i32, p, p, p, p, p, p, p, p, p, p, i32, i32,
                                          p, i64, p, p]
    lib.ara_oracle_layers_ylt.restype = C.c_int
    lib.ara_oracle_layer_yelt.argtypes = [i32, i64, p, p, i32, p, p, p, p, p, f64, f64, f64, f64,
                                          i32, i32, p, i64, p, p, p, p, p]
    lib.ara_oracle_layer_yelt.restype = C.c_int
    lib.ara_oracle_trial_trace.argtypes = [i32, i64, p, i32, p, p, p, p, p, f64, f64, f64, f64,
                                           p, p, p, p, p]
    lib.ara_oracle_trial_trace.restype = C.c_int
    lib.ara_oracle_event_table.argtypes = [i32, i32, p, p, p, p, p, f64, f64, p]
    lib.ara_oracle_event_table.restype = C.c_int
    lib.ara_oracle_pml_tvar.argtypes = [p, i64, p, i32, p, p]
    lib.ara_oracle_pml_tvar.restype = C.c_int
    if path is None:
        _lib = lib
    return lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def _layer_elts(pool, elts: Sequence[int]):
    """Concatenate the layer's ELTs (in layer order) from a pool into CSR arrays."""
    ids, losses, off = [], [], [0]
    for j in elts:
        a, b = int(pool.offsets[j]), int(pool.offsets[j + 1])
        ids.append(pool.ids[a:b])
        losses.append(pool.losses[a:b])
        off.append(off[-1] + (b - a))
    ids = _c(np.concatenate(ids) if ids else np.zeros(0), np.int32)
    losses = _c(np.concatenate(losses) if losses else np.zeros(0), np.float64)
    ded = _c([pool.deductibles[j] for j in elts], np.float64)
    lim = _c([pool.limits[j] for j in elts], np.float64)
    return _c(off, np.int64), ids, losses, ded, lim


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise OracleError(f"{what} failed with status {rc}")


def layer_ylt(yet, pool, layer, trials: Optional[np.ndarray] = None, mode: str = "literal",
              threads: Optional[int] = None, lib=None) -> Tuple[np.ndarray, np.ndarray]:
    """Trial losses and pre-aggregate sums of one layer (Algorithm 1).

    ``trials``: optional subset of trial indices (the outputs follow its order).
    ``mode``: "literal" (ELT loop per occurrence) or "memo" (ELT loop once per
    catalog event; same bits).  Returns (ylt, presum), both float64.
    """
    lib = lib or load()
    off = _c(yet.offsets, np.int64)
    ids = _c(yet.ids, np.int32)
    e_off, e_ids, e_loss, ded, lim = _layer_elts(pool, layer.elts)
    sel = None if trials is None else _c(trials, np.int64)
    n = yet.n_trials if sel is None else sel.shape[0]
    ylt = np.zeros(n, dtype=np.float64)
    pre = np.zeros(n, dtype=np.float64)
    rc = lib.ara_oracle_layer_ylt(int(yet.catalog_size), int(yet.n_trials), _ptr(off), _ptr(ids),
                                  len(layer.elts), _ptr(e_off), _ptr(e_ids), _ptr(e_loss),
                                  _ptr(ded), _ptr(lim), float(layer.occ_ret), float(layer.occ_lim),
                                  float(layer.agg_ret), float(layer.agg_lim),
                                  1 if mode == "memo" else 0, int(threads or os.cpu_count() or 1),
                                  _ptr(sel), int(n), _ptr(ylt), _ptr(pre))
    _check(rc, "ara_oracle_layer_ylt")
    return ylt, pre


def layers_ylt(yet, pool, layers, trials: Optional[np.ndarray] = None, mode: str = "memo",
               threads: Optional[int] = None, lib=None) -> Tuple[np.ndarray, np.ndarray]:
    """Trial losses and pre-aggregate sums of several layers, layer by layer
    (Algorithm 1's loop over the layers of a Program), the YET checked once.
    Returns (ylt, presum), both float64 of shape (len(layers), n)."""
    lib = lib or load()
    off = _c(yet.offsets, np.int64)
    ids = _c(yet.ids, np.int32)
    sel = None if trials is None else _c(trials, np.int64)
    n = yet.n_trials if sel is None else sel.shape[0]
    nl = len(layers)
    parts = [_layer_elts(pool, L.elts) for L in layers]  # kept alive for the call
    ptrs = lambda k: (C.c_void_p * max(nl, 1))(*[_ptr(q[k]) for q in parts])  # noqa: E731
    n_elts = _c([len(L.elts) for L in layers], np.int32)
    terms = [_c([getattr(L, a) for L in layers], np.float64) for a in ("occ_ret", "occ_lim", "agg_ret", "agg_lim")]
    ylt = np.zeros((nl, n), dtype=np.float64)
    pre = np.zeros((nl, n), dtype=np.float64)
    rc = lib.ara_oracle_layers_ylt(int(yet.catalog_size), int(yet.n_trials), _ptr(off), _ptr(ids), nl,
                                   _ptr(n_elts), ptrs(0), ptrs(1), ptrs(2), ptrs(3), ptrs(4),
                                   *[_ptr(t) for t in terms], 1 if mode == "memo" else 0,
                                   int(threads or os.cpu_count() or 1), _ptr(sel), int(n), _ptr(ylt), _ptr(pre))
    _check(rc, "ara_oracle_layers_ylt")
    return ylt, pre


def layer_yelt(yet, pool, layer, trials: Optional[np.ndarray] = None, mode: str = "memo",
               threads: Optional[int] = None, lib=None):
    """Year Event Loss Table of one layer (reading R11).

    Returns (inc, out_off, occ_max, ylt, presum): the per-occurrence
    increments of the selected trials concatenated in list order (trial i at
    inc[out_off[i]:out_off[i+1]]), each trial's largest increment, its trial
    loss and its pre-aggregate sum.
    """
    lib = lib or load()
    off = _c(yet.offsets, np.int64)
    ids = _c(yet.ids, np.int32)
    e_off, e_ids, e_loss, ded, lim = _layer_elts(pool, layer.elts)
    sel = None if trials is None else _c(trials, np.int64)
    lens = np.diff(off) if sel is None else (off[sel + 1] - off[sel])
    n = lens.shape[0]
    out_off = np.zeros(n + 1, dtype=np.int64)
    out_off[1:] = np.cumsum(lens)
    inc = np.zeros(int(out_off[-1]), dtype=np.float64)
    occ_max, ylt, pre = (np.zeros(n, dtype=np.float64) for _ in range(3))
    rc = lib.ara_oracle_layer_yelt(int(yet.catalog_size), int(yet.n_trials), _ptr(off), _ptr(ids),
                                   len(layer.elts), _ptr(e_off), _ptr(e_ids), _ptr(e_loss),
                                   _ptr(ded), _ptr(lim), float(layer.occ_ret), float(layer.occ_lim),
                                   float(layer.agg_ret), float(layer.agg_lim),
                                   1 if mode == "memo" else 0, int(threads or os.cpu_count() or 1),
                                   _ptr(sel), int(n), _ptr(out_off), _ptr(inc), _ptr(occ_max),
                                   _ptr(ylt), _ptr(pre))
    _check(rc, "ara_oracle_layer_yelt")
    return inc, out_off, occ_max, ylt, pre


def trial_trace(catalog_size: int, ids: np.ndarray, pool, layer, lib=None):
    """Per-event trace of one trial: (occ, agg, inc, trial_loss, presum)."""
    lib = lib or load()
    ids = _c(ids, np.int32)
    e_off, e_ids, e_loss, ded, lim = _layer_elts(pool, layer.elts)
    n = ids.shape[0]
    occ, agg, inc = (np.zeros(n) for _ in range(3))
    tl, ps = C.c_double(0.0), C.c_double(0.0)
    rc = lib.ara_oracle_trial_trace(int(catalog_size), int(n), _ptr(ids), len(layer.elts),
                                    _ptr(e_off), _ptr(e_ids), _ptr(e_loss), _ptr(ded), _ptr(lim),
                                    float(layer.occ_ret), float(layer.occ_lim),
                                    float(layer.agg_ret), float(layer.agg_lim), _ptr(occ),
                                    _ptr(agg), _ptr(inc), C.byref(tl), C.byref(ps))
    _check(rc, "ara_oracle_trial_trace")
    return occ, agg, inc, tl.value, ps.value


def event_table(catalog_size: int, pool, layer, lib=None) -> np.ndarray:
    """Occurrence-net loss of every catalog event: FT2(sum_j FT1(DAT_j[e]))."""
    lib = lib or load()
    e_off, e_ids, e_loss, ded, lim = _layer_elts(pool, layer.elts)
    out = np.zeros(int(catalog_size), dtype=np.float64)
    rc = lib.ara_oracle_event_table(int(catalog_size), len(layer.elts), _ptr(e_off), _ptr(e_ids),
                                    _ptr(e_loss), _ptr(ded), _ptr(lim), float(layer.occ_ret),
                                    float(layer.occ_lim), _ptr(out))
    _check(rc, "ara_oracle_event_table")
    return out


def pml_tvar(ylt: np.ndarray, return_periods: Sequence[float], lib=None):
    """PML and TVaR at each return period (reading R5)."""
    lib = lib or load()
    y = _c(ylt, np.float64)
    rps = _c(return_periods, np.float64)
    pml = np.zeros(rps.shape[0])
    tvar = np.zeros(rps.shape[0])
    rc = lib.ara_oracle_pml_tvar(_ptr(y), int(y.shape[0]), _ptr(rps), int(rps.shape[0]),
                                 _ptr(pml), _ptr(tvar))
    _check(rc, "ara_oracle_pml_tvar")
    return pml, tvar


# ----------------------------------------------------------------- comparison
# Error forms for checking another implementation's results against the
# oracle's (pure NumPy on the two result arrays; no part of the method).
FP64_REL = 1e-12
REDUCED_REL, REDUCED_FLOOR = 1e-5, 1.0


def compare_fp64(g, o, presum) -> dict:
    """Per-trial errors of YLT g against the oracle's o.  The gate (reading R9)
    divides by max(|o|, S_o), S_o the oracle's pre-aggregate sum, because the
    aggregate clamp is 1-Lipschitz; the plain form |g - o| / |o| is reported
    beside it (a trial with o == 0 fails it when g != 0)."""
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    pre = np.asarray(presum, dtype=np.float64)
    err = np.abs(g - o)
    denom = np.maximum(np.abs(o), pre)
    r9 = np.where(denom > 0, err / np.where(denom > 0, denom, 1.0), np.where(err > 0, np.inf, 0.0))
    absn = np.abs(o)
    plain = np.where(absn > 0, err / np.where(absn > 0, absn, 1.0), np.where(err > 0, np.inf, 0.0))
    return {"trials": int(g.size), "max_rel_err_r9": float(r9.max()) if r9.size else 0.0,
            "trials_over_r9_bar": int(np.count_nonzero(r9 > FP64_REL)),
            "max_rel_err_plain": float(plain.max()) if plain.size else 0.0,
            "trials_over_plain_bar": int(np.count_nonzero(plain > FP64_REL)),
            "bitwise_equal_trials": int(np.count_nonzero(g.view(np.uint64) == o.view(np.uint64))),
            "max_abs_err": float(err.max()) if err.size else 0.0}


def compare_reduced(g, o, presum) -> dict:
    """The same for a reduced-precision YLT: the gate is |g - o| <=
    max(1e-5 * max(|o|, S_o), 1 USD); the plain form max(1e-5 * |o|, 1 USD)
    is reported beside it."""
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    pre = np.asarray(presum, dtype=np.float64)
    err = np.abs(g - o)
    bound = np.maximum(REDUCED_REL * np.maximum(np.abs(o), pre), REDUCED_FLOOR)
    plain = np.maximum(REDUCED_REL * np.abs(o), REDUCED_FLOOR)
    return {"trials": int(g.size), "max_err_over_bar": float((err / bound).max()) if err.size else 0.0,
            "trials_over_bar": int(np.count_nonzero(err > bound)),
            "max_err_over_plain_bar": float((err / plain).max()) if err.size else 0.0,
            "trials_over_plain_bar": int(np.count_nonzero(err > plain)),
            "max_rel_err": float(np.max(err / np.maximum(np.maximum(np.abs(o), pre), 1e-300))) if err.size else 0.0,
            "max_abs_err": float(err.max()) if err.size else 0.0}


def compare_pml_tvar(pml_g, tvar_g, pml_o, tvar_o, return_periods, n: int, max_trial_err: float) -> dict:
    """PML/TVaR of an implementation (from its own YLT of n trials) against
    the oracle's (from the oracle's YLT).  Order statistics and means of the
    k largest are 1-Lipschitz in the largest per-trial error; the oracle's
    sequential tail sum of k = floor(n / RP) terms carries at most (k - 1)
    roundings of 2^-53 of the sum, and each side's division one more, so the
    bound is max_trial_err + (k + 1) * 2^-53 * TVaR."""
    pml_g, tvar_g = np.asarray(pml_g, np.float64), np.asarray(tvar_g, np.float64)
    pml_o, tvar_o = np.asarray(pml_o, np.float64), np.asarray(tvar_o, np.float64)
    k = np.floor(n / np.asarray(return_periods, np.float64))
    bound = max_trial_err + (k + 1.0) * 2.0 ** -53 * np.abs(tvar_o)
    return {"return_periods": [float(r) for r in return_periods],
            "pml_abs_err": np.abs(pml_g - pml_o).tolist(), "tvar_abs_err": np.abs(tvar_g - tvar_o).tolist(),
            "pml_rel_err": (np.abs(pml_g - pml_o) / np.maximum(np.abs(pml_o), 1e-300)).tolist(),
            "tvar_rel_err": (np.abs(tvar_g - tvar_o) / np.maximum(np.abs(tvar_o), 1e-300)).tolist(),
            "bound": bound.tolist(),
            "within_bound": bool(np.all(np.abs(pml_g - pml_o) <= bound) and np.all(np.abs(tvar_g - tvar_o) <= bound))}
