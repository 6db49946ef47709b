"""Plants plausible mistakes in a copy of the oracle (CPU only) and checks that the pins in
test_oracle_pins.py catch every one of them: a wrong reversal index, a dropped or sign-flipped
coordinate term, a strict threshold, a non-strict update, min/max swaps, a lost bundle visit
order, gradient slips, and slips in the length term TN (Eq. 3), the polyline length and the
direction inference of Section 2.4."""
import ctypes
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "seg_oracle.c")

MUTANTS = {
    "reversal_index": ("static int rev(int i) { return NPTS - 1 - i; }",
                       "static int rev(int i) { return NPTS - i - (i > 0); }"),
    "drop_z_term": ("return sqrt(dx * dx + dy * dy + dz * dz);", "return sqrt(dx * dx + dy * dy);"),
    "sign_slip": ("double dx = p[0] - q[0]", "double dx = p[0] + q[0]"),
    "strict_threshold": ("if (d <= thr[bundle_of[c]] && d < r->dist)",
                         "if (d < thr[bundle_of[c]] && d < r->dist)"),
    "nonstrict_update": ("if (d <= thr[bundle_of[c]] && d < r->dist)",
                         "if (d <= thr[bundle_of[c]] && d <= r->dist)"),
    "max_becomes_min": ("if (e > md) md = e;", "if (e < md || i == 0) md = e;"),
    "orientation_max": ("double d = dd <= dr ? dd : dr;\n        if (d <= thr",
                        "double d = dd >= dr ? dd : dr;\n        if (d <= thr"),
    "no_bundle_order": ("for (int64_t c = 0; c < M; ++c) ord[cnt[bundle_of[c]]++] = c;",
                        "for (int64_t c = 0; c < M; ++c) ord[c] = c;"),
    "cascade_strict": ("if (x > th) alive_r = 0;", "if (x >= th) alive_r = 0;"),
    "grad_t_sign": ("g[9 + r] += u[r];", "g[9 + r] -= u[r];"),
    "grad_uses_moved_point": ("g[3 * r + c] += u[r] * x[3 * is + c];",
                              "g[3 * r + c] += u[r] * y[3 * is + c];"),
    "grad_centroid_index": ("int pi = o ? rev(is) : is;", "int pi = is;"),
    "tn_signed_difference": ("double r = fabs(ls - lc) / m;", "double r = (ls - lc) / m;"),
    "tn_squared_ratio": ("return (r + 1.0) * (r + 1.0) - 1.0;", "return r * r;"),
    "length_drops_a_segment": ("for (int i = 0; i + 1 < NPTS; ++i) l += d_E",
                               "for (int i = 1; i + 1 < NPTS; ++i) l += d_E"),
    "resample_by_index": ("const double sk = k * L / (NPTS - 1);",
                          "const double sk = c[(m - 1) * k / (NPTS - 1)];"),
    "resample_no_interpolation": ("o[3 * k + r] = q[3 * j + r] + w * (q[3 * (j + 1) + r] - q[3 * j + r]);",
                                  "o[3 * k + r] = q[3 * j + r];"),
    "multi_strict_threshold": ("if (best[b] <= 0.0) row[b >> 5] |= 1u << (b & 31);",
                               "if (best[b] < 0.0) row[b >> 5] |= 1u << (b & 31);"),
    "inference_takes_larger": ("int o = ed <= er ? 0 : 1; /* direction inference */",
                               "int o = ed <= er ? 1 : 0; /* direction inference */"),
    "inference_skipped": ("    m = o ? er : ed;\n    for (int q = 0; q < 4; ++q) { /* test3 */",
                          "    m = o ? er : ed;\n    if (0) { double dd, dr; dme_both(a, b, &dd, &dr);"
                          " return (dd <= dr ? dd : dr) + tn_term(ls, lc); }\n"
                          "    if (1) { double dd, dr; dme_both(a, b, &dd, &dr);"
                          " if ((dd <= dr ? dd : dr) > th) return INFINITY;"
                          " *orient = dd <= dr ? 0 : 1; return (dd <= dr ? dd : dr) + tn_term(ls, lc); }\n"
                          "    for (int q = 0; q < 4; ++q) { /* test3 */"),
}

PINS = [pins.test_worked_examples_dme, pins.test_worked_examples_labels,
        pins.test_parallel_offsets_closed_form, pins.test_single_point_changes_each_coordinate,
        pins.test_identities, pins.test_labels_vs_sorted_brute_force,
        pins.test_exact_ties_and_threshold_edges, pins.test_grad_translation_closed_form,
        pins.test_grad_reversed_orientation_closed_form,
        pins.test_grad_frozen_structure_fd, pins.test_lengths_closed_forms,
        pins.test_tn_worked_example,
        pins.test_direction_inference_can_miss_the_closer_orientation,
        pins.test_resample_closed_forms, pins.test_multi_label_hand_cases]


def _gold():
    import json
    with open(pins.GOLD) as fh:
        return json.load(fh)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path, monkeypatch):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new, 1))
    so = tmp_path / "mut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                    "-o", str(so), str(mut), "-lm"], check=True)
    monkeypatch.setattr(oracle, "_lib", oracle._bind(ctypes.CDLL(str(so))))
    gold = _gold()
    caught = []
    for pin in PINS:
        try:
            if pin.__code__.co_argcount == 1:
                pin(gold)
            else:
                pin()
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"no pin catches mutant {name}"
