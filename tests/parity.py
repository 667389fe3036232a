"""Shared helpers for the GPU parity tests (the oracle is the reference)."""
import numpy as np

# FP64 path: relative 1e-12 per trial.  The error is taken relative to
# max(|o|, S_o), S_o the oracle's pre-aggregate sum: the aggregate clamp is
# 1-Lipschitz, so an error in the sum can move the trial loss by at most the
# same amount, and a sum of n non-negative binary64 terms in any order is
# within (n-1) * 2^-53 * S of the exact sum.  The engine rounds the exact sum
# once; the oracle's sequential sum carries up to (n-1) roundings, so for
# trials of up to ~1500 events the two differ by at most ~1.7e-13 * S.
FP64_REL_TOL = 1e-12


def r9_rel_error(g: np.ndarray, o: np.ndarray, presum: np.ndarray) -> np.ndarray:
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    denom = np.maximum(np.abs(o), np.asarray(presum, dtype=np.float64))
    err = np.abs(g - o)
    out = np.zeros_like(err)
    nz = denom > 0
    out[nz] = err[nz] / denom[nz]
    out[~nz] = np.where(err[~nz] > 0, np.inf, 0.0)
    return out


def assert_fp64_parity(g, o, presum, what="ylt"):
    rel = r9_rel_error(g, o, presum)
    i = int(np.argmax(rel)) if rel.size else 0
    assert rel.size == 0 or rel[i] <= FP64_REL_TOL, (
        f"{what}: trial {i} gpu={g[i]!r} oracle={o[i]!r} presum={presum[i]!r} rel={rel[i]:.3e}")
    return float(rel.max()) if rel.size else 0.0


def load_workload(engine, w):
    """Load a Workload into an Engine; returns the layer handles."""
    engine.load_yet_from(w.yet)
    first = engine.load_pool(w.pool)
    return [engine.define_layer([first + j for j in L.elts], L.occ_ret, L.occ_lim, L.agg_ret,
                                L.agg_lim) for L in w.layers]
