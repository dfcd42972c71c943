"""Pins of the cost model (Sec. 4.5, Eq. theoretical_speedup) against the
speedups the paper prints (tests/golden/paper_values.txt)."""
import os

import pytest

from oracle import cost

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def _golden():
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, value, tol = line.split()[:3]
            vals[name] = (float(value), float(tol))
    return vals


def test_speedups_printed_in_paper():
    g = _golden()
    s = cost.theoretical_speedup(Mf=2, Mc=1, N_ML=2, alpha=0.5, Rf=256, N_S=4)
    v, tol = g["speedup_mlsdc_3_2_2_half_vs_sdc_3_4"]
    assert abs(s - v) <= tol
    s = cost.theoretical_speedup(Mf=4, Mc=2, N_ML=4, alpha=0.5, Rf=256, N_S=8)
    v, tol = g["speedup_mlsdc_5_3_4_half_vs_sdc_5_8"]
    assert abs(s - v) <= tol
    s = cost.theoretical_speedup(Mf=2, Mc=1, N_ML=2, alpha=0.8, Rf=256, N_S=4)
    v, tol = g["speedup_theory_alpha_4_5"]
    assert abs(s - v) <= tol
    s = cost.theoretical_speedup(Mf=2, Mc=1, N_ML=2, alpha=0.5, Rf=256, N_S=4)
    v, tol = g["speedup_theory_alpha_1_2"]
    assert abs(s - v) <= tol
    v, tol = g["wallclock_reduction_mlsdc_3_2_2"]
    assert abs((1 - 1 / s) - v) <= tol


def test_cost_ratio_closed_form():
    # C_c/C_f = R_c (R_c + 1) / (R_f (R_f + 1)) when R_c = alpha R_f
    assert cost.coarse_cost_ratio(0.5, 256) == pytest.approx(128 * 129 / (256 * 257), rel=1e-15)
