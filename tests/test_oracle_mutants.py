"""Planted mistakes: each plausible slip in the oracle must fail a pin.

Every case copies the oracle's C source, changes one expression (a dropped
term, a wrong sign or bound, a transposed bit order), compiles the copy on
the CPU and runs the independent pins of test_oracle_pins against it.  The
retyped threshold values are deliberately left out of the pins used here,
so the threshold mutants have to be caught by the brute-force and
construction pins.
"""
import os

import pytest

import oracle as oracle_pkg
import test_oracle_pins as pins
import test_oracle_seeds as seed_pins

MUTANTS = {
    "unpack_msb_first": ("codes[k] = (uint8_t)((byte >> (2 * (k % 4))) & 3);",
                         "codes[k] = (uint8_t)((byte >> (2 * (3 - k % 4))) & 3);"),
    "token_lsb_first": ("for (int k = 0; k < q - 1 - j; k++) weight *= 4;",
                        "for (int k = 0; k < j; k++) weight *= 4;"),
    "span_without_overlap": ("int64_t e = s + bin_len + overlap;", "int64_t e = s + bin_len;"),
    "span_drops_last_token": ("        for (int64_t i = s; i + q <= e; i++) {\n            int64_t t",
                              "        for (int64_t i = s; i + q < e; i++) {\n            int64_t t"),
    "threshold_q_minus_1": ("return n_tokens - (int64_t)q * E;", "return n_tokens - (int64_t)(q - 1) * E;"),
    "threshold_q_plus_1": ("return n_tokens - (int64_t)q * E;", "return n_tokens - (int64_t)(q + 1) * E;"),
    "token_count_off_by_one": ("int64_t n_tokens = L - q + 1;", "int64_t n_tokens = L - q;"),
    "strict_compare": ("pass[c] = (sum >= T) ? 1 : 0;", "pass[c] = (sum > T) ? 1 : 0;"),
    "read_drops_last_token": ("for (int64_t i = 0; i + q <= L; i++) {\n        int64_t t = oracle_token(read + i, q);",
                              "for (int64_t i = 0; i + q < L; i++) {\n        int64_t t = oracle_token(read + i, q);"),
    "no_multiplicity": ("sum += bank_row[t];",
                        "sum += bank_row[t] && (i == 0 || oracle_token(read + i - 1, q) != t);"),
    # seed locations and the Seed Location Checker
    "seeds_overlapping": ("for (int64_t o = 0; o + k <= L; o += k) seed_at[n_seeds++] = o;",
                          "for (int64_t o = 0; o + k <= L; o += 1) seed_at[n_seeds++] = o;"),
    "seed_vote_no_offset": ("int64_t start = where[j] - o;", "int64_t start = where[j];"),
    "seed_no_clamp_at_zero": ("if (start < 0) start = 0;", "if (start < 0) start = -start;"),
    "seed_ties_to_higher_bin": ("    return (x->bin > y->bin) - (x->bin < y->bin);\n}\n\nstatic int oracle_cmp_vote_bin",
                                "    return (x->bin < y->bin) - (x->bin > y->bin);\n}\n\nstatic int oracle_cmp_vote_bin"),
    "seed_keeps_fewest_votes": ("if (x->votes != y->votes) return x->votes > y->votes ? -1 : 1;",
                                "if (x->votes != y->votes) return x->votes < y->votes ? -1 : 1;"),
    "seed_misses_last_position": ("    for (int64_t p = 0; p + k <= len; p++) {\n        int64_t key = oracle_seed_key(ref + p, k);\n        int64_t i = key >= 0 ? oracle_find_key(keys, u, (uint64_t)key) : -1;\n        if (i >= 0) count[i + 1]++;",
                                  "    for (int64_t p = 0; p + k < len; p++) {\n        int64_t key = oracle_seed_key(ref + p, k);\n        int64_t i = key >= 0 ? oracle_find_key(keys, u, (uint64_t)key) : -1;\n        if (i >= 0) count[i + 1]++;"),
    "locate_segment_off_by_one": ("seg[m * seg_stride + j] = (begin + j < end) ? ref[begin + j] : 4;",
                                  "seg[m * seg_stride + j] = (begin + j <= end) ? ref[begin + j] : 4;"),
}


def _pin_suite(o):
    pins.test_unpack_bit_order(o)
    pins.test_token_values(o)
    pins.test_bins_closed_forms(o)
    for args in [(3, 32, 10, 500), (5, 100, 40, 1500), (4, 17, 0, 4)]:
        pins.test_bank_matches_substring_search(o, *args)
    pins.test_filter_matches_brute_force(o)
    pins.test_aaaaa_example(o)
    pins.test_fig5b_error_propagation(o)
    pins.test_exact_match_count(o)
    pins.test_threshold_is_worst_case_of_spaced_substitutions(o)
    pins.test_no_miss_within_edit_distance(o, 4, 4, 1)
    pins.test_invariants_sum_bound_monotone_scan(o)
    pins.test_short_reads(o)
    seed_pins.test_hand_example_votes_cap_and_ties(o)
    seed_pins.test_brute_force_string_search(o, 1)
    seed_pins.test_locate_hand_example(o)


def test_unmodified_oracle_passes_suite():
    _pin_suite(oracle_pkg.Oracle())


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(os.path.join(os.path.dirname(oracle_pkg.__file__), "grim_oracle.c")).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    path = tmp_path / f"mut_{name}.c"
    path.write_text(src.replace(old, new))
    so = oracle_pkg.build(force=True, src=str(path), out=str(tmp_path / f"lib_{name}.so"))
    mutant = oracle_pkg.Oracle(oracle_pkg.load(so))
    with pytest.raises((AssertionError, ValueError)):
        _pin_suite(mutant)
