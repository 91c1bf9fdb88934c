"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each case copies ``oracle/tcorr_oracle.c``, applies one plausible mistake (a
dropped term, a wrong sign or index, an off-by-one bound, a transposed
layout, a wrong normalisation), compiles the copy into a temporary library and
runs the pins against it.  The copy must fail at least one pin; a mistake that
no pin notices would mean the pins do not pin the oracle.
"""
import os

import pytest

import oracle
from tests import oracle_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "tcorr_oracle.c")

# (name, text to replace, replacement, which occurrence (0-based))
MUTANTS = [
    ("last_origin_dropped", "t0 + tau <= T - 1; t0 += s", "t0 + tau < T - 1; t0 += s", 0),
    ("stride_ignored", "t0 + tau <= T - 1; t0 += s", "t0 + tau <= T - 1; t0 += 1", 0),
    ("msd_sign", "double d = q[c] - p[c];", "double d = q[c] + p[c];", 0),
    ("acf_same_time", "term += p[c] * q[c];", "term += p[c] * p[c];", 0),
    ("component_dropped", "for (int c = 0; c < 3; ++c) {", "for (int c = 0; c < 2; ++c) {", 0),
    ("n_origins_off_by_one", "return (T - 1 - tau) / s + 1;", "return (T - tau) / s + 1;", 0),
    ("per_component_norm", "out[l] = total / ((double)N *", "out[l] = total / ((double)(3 * N) *", 0),
    ("origin_not_added", "const double *q = later + 3 * (t0 + tau);", "const double *q = later + 3 * tau;", 0),
    ("layout_transposed", "J->x[(t * N + i) * 3 + c]", "J->x[(i * T + t) * 3 + c]", 0),
    ("atom_sum_overwritten", "out[l] += acc;", "out[l] = acc;", 0),
    ("trapezoid_half_dropped", "I += dt * (c[k - 1] + c[k]) / 2.0;", "I += dt * (c[k - 1] + c[k]);", 0),
    ("trapezoid_right_point", "I += dt * (c[k - 1] + c[k]) / 2.0;", "I += dt * (c[k] + c[k]) / 2.0;", 0),
    ("einstein_no_2", "*D_slope = (sxy / sxx) / (2.0 * dim);", "*D_slope = (sxy / sxx) / (double)dim;", 0),
    ("einstein_time_axis", "const double dx = (double)k * dt - xbar;", "const double dx = (double)k - xbar;", 0),
    ("xcf_second_signal_ignored", "later[3 * t + c] = (double)J->y[", "later[3 * t + c] = (double)J->x[", 0),
    ("xcf_time_roles_swapped", "const double *p = traj + 3 * t0;\n                const double *q = later + 3 * (t0 + tau);",
     "const double *p = later + 3 * t0;\n                const double *q = traj + 3 * (t0 + tau);", 0),
    ("collective_ref_ignored", "if (ref >= 0) v -= (double)x[(ref * N + i) * 3 + c];", "", 0),
    ("collective_weight_ignored", "sum += (w ? (double)w[i] : 1.0) * v;", "sum += v;", 0),
    ("collective_ref_wrong_atom", "v -= (double)x[(ref * N + i) * 3 + c];", "v -= (double)x[(ref * N) * 3 + c];", 0),
    ("weight_ignored", "if (J->w) acc *= (double)J->w[i];", "", 0),
    ("weighted_norm_by_atoms", "if (w) out[l] = total / (wsum *", "if (w) out[l] = total / ((double)N *", 0),
    ("collective_component_fixed", "double v = (double)x[(t * N + i) * 3 + c];",
     "double v = (double)x[(t * N + i) * 3];", 0),
]


def _mutate(text, old, new, occurrence):
    pos = -1
    for _ in range(occurrence + 1):
        pos = text.find(old, pos + 1)
        assert pos >= 0, f"mutation anchor not found: {old!r}"
    return text[:pos] + new + text[pos + len(old):]


@pytest.mark.parametrize("name,old,new,occ", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, name, old, new, occ):
    with open(SRC) as f:
        text = f.read()
    mutated = _mutate(text, old, new, occ)
    assert mutated != text
    src = tmp_path / f"{name}.c"
    src.write_text(mutated)
    lib = oracle.load_library(oracle.compile_oracle(str(src), str(tmp_path / f"lib{name}.so")))
    caught = []
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(lib)
        except (AssertionError, ValueError):
            caught.append(pin.__name__)
            break
    assert caught, f"no pin caught the planted mistake {name}"
