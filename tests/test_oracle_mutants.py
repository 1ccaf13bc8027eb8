"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each mutant is a copy of ``oracle/xe_oracle.c`` with one plausible mistake written into it (a dropped
term, a wrong sign, a wrong index, a swapped nibble, ...). The mutant is compiled into a temporary
directory and every pin of test_oracle.py is run against it: at least one pin must fail. This shows
that the pins constrain each part of the oracle rather than only restating it.
"""
import os

import pytest

import oracle
from tests import test_oracle as T

SRC = os.path.join(os.path.dirname(oracle.__file__), "xe_oracle.c")

MUTANTS = {
    # conjugate taken on the wrong side: V = conj(x_i) x_j
    "conjugate_side": ("si += (int64_t)bi[t] * aj[t] - (int64_t)ai[t] * bj[t];",
                       "si += (int64_t)ai[t] * bj[t] - (int64_t)bi[t] * aj[t];"),
    # dropped imaginary-imaginary term of the real part
    "dropped_term": ("sr += (int64_t)ai[t] * aj[t] + (int64_t)bi[t] * bj[t];",
                     "sr += (int64_t)ai[t] * aj[t];"),
    # transposed operand in the imaginary part
    "transposed_operand": ("si += (int64_t)bi[t] * aj[t] - (int64_t)ai[t] * bj[t];",
                           "si += (int64_t)bj[t] * aj[t] - (int64_t)ai[t] * bi[t];"),
    # wrong packed-triangle row offset
    "triangle_index": ("return (int64_t)i * n - (int64_t)i * (i - 1) / 2 + (j - i);",
                       "return (int64_t)i * n - (int64_t)i * (i + 1) / 2 + (j - i);"),
    # nibbles swapped (low = real)
    "nibble_order": ("*re = hi >= 8 ? hi - 16 : hi;\n    *im = lo >= 8 ? lo - 16 : lo;",
                     "*re = lo >= 8 ? lo - 16 : lo;\n    *im = hi >= 8 ? hi - 16 : hi;"),
    # -8 read as +8 (sign extension off by one)
    "sign_extension": ("*re = hi >= 8 ? hi - 16 : hi;", "*re = hi > 8 ? hi - 16 : hi;"),
    # int32 overflow never reported
    "no_overflow_check": ("if (sr > INT32_MAX || sr < INT32_MIN || si > INT32_MAX || si < INT32_MIN) ovf = 1;",
                          "(void)0;"),
    # duplicates overwrite (last arrival wins)
    "last_duplicate_wins": ("if (filled[(size_t)slot * G + g]) { stats[1]++; continue; }",
                            "if (filled[(size_t)slot * G + g]) { stats[1]++; }"),
    # loss counted per packet instead of per sample
    "loss_per_packet": ("for (int ff = 0; ff < 8; ++ff) lost[8 * g + ff] += 4;",
                        "for (int ff = 0; ff < 8; ++ff) lost[8 * g + ff] += 1;"),
    # missing packets not zero-filled
    "no_zero_fill": ("memset(frame + ((size_t)(4 * slot + tt) * F + (8 * g + ff)) * N, 0, (size_t)N);",
                     "(void)tt;"),
    # late / early swapped
    "late_early_swapped": ("if (seq < seq0) { stats[2]++; continue; }", "if (seq < seq0) { stats[3]++; continue; }"),
    # intersection correction with the wrong sign
    "intersection_sign": ("- flag_pairs[(size_t)f * P + p];", "+ flag_pairs[(size_t)f * P + p];"),
    # flag pair intersections without the diagonal (i == j)
    "flag_pairs_no_diagonal": ("for (int j = i; j < N; ++j)\n                        if ((bits[j / 8] >> (j % 8)) & 1)",
                               "for (int j = i + 1; j < N; ++j)\n                        if ((bits[j / 8] >> (j % 8)) & 1)"),
    # flags of duplicate packets counted again
    "flags_of_duplicates": ("if (seen[(size_t)slot * G + g]) continue;", "(void)0;"),
    # footer bits read most significant first
    "flag_bit_order": ("if (!((bits[i / 8] >> (i % 8)) & 1)) continue;", "if (!((bits[i / 8] >> (7 - i % 8)) & 1)) continue;"),
    # time shift taken towards earlier samples
    "time_shift_direction": ("const int src = t - delays[n];", "const int src = t + delays[n] < T ? t + delays[n] : -1;"),
    # pairs of shifted inputs share the larger delay's leading samples
    "time_shift_counts_max": ("const int m = delays[i] < delays[j] ? delays[i] : delays[j];",
                              "const int m = delays[i] > delays[j] ? delays[i] : delays[j];"),
    # normalisation applied as a product instead of a quotient
    "normalize_product": ("out[2 * q] = (float)((double)vis[2 * q] / (double)n[q]);",
                          "out[2 * q] = (float)((double)vis[2 * q] * (double)n[q]);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    lib = oracle.compile_source(str(mut), str(tmp_path / "libmutant.so"))
    o = oracle.Oracle(lib)
    caught = []
    for pin in T.PINS:
        try:
            pin(o)
        except (AssertionError, ValueError):
            caught.append(pin.__name__)
    assert caught, f"no pin detects the planted mistake {name}"
