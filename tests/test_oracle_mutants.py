"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a dropped
term, a wrong sign, a transposed operand, an off-by-one index), builds it on
the CPU and checks that the pin battery below rejects it.  The real oracle
must pass the same battery.
"""
import math
import os
import tempfile

import numpy as np
import pytest

import oracle
from test_oracle import GOLDEN, _dat_sum, _random_instance, hand_instance

SRC = os.path.join(os.path.dirname(oracle.__file__), "ara_oracle.c")

MUTANTS = {
    "drop_deductible": ("double v = loss - deductible;", "double v = loss;"),
    "drop_elt_limit": ("if (v > limit) v = limit;", ""),
    "drop_occ_limit": ("if (v > occ_lim) v = occ_lim;", ""),
    "occ_terms_swapped": ("double v = x - occ_ret;", "double v = x - occ_lim;"),
    "drop_agg_retention": ("double v = p - agg_ret;", "double v = p;"),
    "subtract_event": ("p = p + o;", "p = p - o;"),
    "first_elt_only": ("L->dats[(size_t)j * (size_t)L->catalog + (size_t)e]",
                       "L->dats[(size_t)0 * (size_t)L->catalog + (size_t)e]"),
    "drop_last_event": ("J->ylt[i] = trial_loss(J->L, J->ids + a, b - a, &s, NULL, NULL, NULL);",
                        "J->ylt[i] = trial_loss(J->L, J->ids + a, b - a - (b > a), &s, NULL, NULL, NULL);"),
    "yelt_inc_not_differenced": ("if (inc) inc[k] = a - prev;", "if (inc) inc[k] = a;"),
    "yelt_occ_max_first_event": ("if (inc[k] > m) m = inc[k];", "if (k == 0) m = inc[k];"),
    "pml_off_by_one": ("pml_out[r] = y[k - 1];", "pml_out[r] = y[k > 1 ? k - 2 : 0];"),
    "tvar_wrong_divisor": ("tvar_out[r] = s / (double)k;", "tvar_out[r] = s / (double)(k + 1);"),
    "clamp_occ_before_sum": ("x = x + ft1(l, L->ded[j], L->lim[j]);",
                             "x = x + ft2(ft1(l, L->ded[j], L->lim[j]), L->occ_ret, L->occ_lim);"),
}


def pin_battery(lib):
    """Return the list of pins that fail for this build of the oracle."""
    import json
    failed = []
    g, yet, pool, layer = hand_instance()
    ylt, pre = oracle.layer_ylt(yet, pool, layer, lib=lib)
    if ylt.tolist() != g["ylt"]:
        failed.append("hand_ylt")
    if oracle.event_table(3, pool, layer, lib=lib).tolist() != g["event_table"]:
        failed.append("hand_event_table")
    _, gy, gp, gl = hand_instance(neutral=True)
    if oracle.layer_ylt(gy, gp, gl, lib=lib)[0][0] != g["neutral_terms"]["ylt_trial0"]:
        failed.append("hand_neutral")
    p = json.load(open(GOLDEN))["pml_tvar"]
    pml, tvar = oracle.pml_tvar(np.array(p["ylt"]), p["return_periods"], lib=lib)
    if pml.tolist() != p["pml"] or tvar.tolist() != p["tvar"]:
        failed.append("hand_pml_tvar")
    y = g["yelt"]
    inc, out_off, occ_max, _, _ = oracle.layer_yelt(yet, pool, layer, lib=lib)
    if [inc[out_off[i]:out_off[i + 1]].tolist() for i in range(len(y["inc"]))] != y["inc"] or \
            occ_max.tolist() != y["occ_max"]:
        failed.append("hand_yelt")
    yet2, pool2, layer2 = _random_instance(1, neutral=True)
    raw = _dat_sum(pool2, layer2, yet2.catalog_size)
    trial_of = np.repeat(np.arange(yet2.n_trials), np.diff(yet2.offsets))
    ref = np.bincount(trial_of, weights=raw[yet2.ids], minlength=yet2.n_trials)
    got, _ = oracle.layer_ylt(yet2, pool2, layer2, lib=lib)
    if not np.allclose(got, ref, rtol=1e-13, atol=0):
        failed.append("segmented_sum")
    return failed


def test_real_oracle_passes_battery():
    assert pin_battery(oracle.load()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    msrc = tmp_path / "mutant.c"
    msrc.write_text(src.replace(old, new))
    lib = oracle.load(oracle.build(str(msrc), str(tmp_path / "libmutant.so"), force=True))
    assert pin_battery(lib), f"mutant {name} passed every pin"
