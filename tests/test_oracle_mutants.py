"""Mutation tests for the oracle's pins (CPU only).

Each case copies ``oracle/sws_oracle.c``, plants one plausible mistake (a dropped addend, a
transposed operand, a wrong index or constant, a wrong tie-break ...), compiles the copy into
a temporary directory and runs pins against it.  The pins must reject every mutant; a mutant
that survives means the pins cannot tell a correct oracle from a broken one.
"""

import os

import pytest

import oracle
import pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "sws_oracle.c")

# (name, exact text in the oracle, replacement, pins expected to catch it)
MUTANTS = [
    ("eq2_drops_last_addend",
     "for (j = 1; j < w; ++j) acc = acc + v[p + j];",
     "for (j = 1; j < w - 1; ++j) acc = acc + v[p + j];",
     [pins.check_eq2_closed_forms]),
    ("eq2_window_count_short",
     "m = n - (uint64_t)w + 1;\n    for (p = 0; p < m; ++p)",
     "m = n - (uint64_t)w + 1;\n    for (p = 0; p + 1 < m; ++p)",
     [pins.check_eq2_vs_algorithms]),
    ("min_uses_wrong_comparison",
     "acc = v[p + j] < acc ? v[p + j] : acc;",
     "acc = v[p + j] > acc ? v[p + j] : acc;",
     [pins.check_eq2_closed_forms]),
    ("affine_operands_transposed",
     "uint32_t nB = a * B + b;",
     "uint32_t nB = A * b + B;",
     [pins.check_eq2_closed_forms, pins.check_eq2_vs_algorithms]),
    ("f32_window_offset",
     "for (j = 1; j < w; ++j) acc = acc + (double)v[p + j];",
     "for (j = 1; j < w; ++j) acc = acc + (double)v[p + j - 1];",
     [pins.check_eq2_closed_forms]),
    ("kmer_forward_reversed",
     "for (j = 0; j < k; ++j) v = v * 4 + (uint64_t)base_at(s, i + j);",
     "for (j = 0; j < k; ++j) v = v * 4 + (uint64_t)base_at(s, i + k - 1 - j);",
     [pins.check_kmers_exhaustive8]),
    ("revcomp_without_complement",
     "v = v * 4 + (uint64_t)(3 - base_at(s, i + j));",
     "v = v * 4 + (uint64_t)(base_at(s, i + j));",
     [pins.check_kmers_exhaustive8]),
    ("hash_wrong_shift",
     "key = key ^ (key >> 24);",
     "key = key ^ (key >> 23);",
     [pins.check_hash]),
    ("hash_mask_only_at_end",
     "key = (key + (key << 3) + (key << 8)) & m;",
     "key = (key + (key << 3) + (key << 8));",
     [pins.check_hash]),
    ("canonical_is_max",
     "c = f < r ? f : r;",
     "c = f > r ? f : r;",
     [pins.check_kmers_exhaustive8]),
    ("minimizer_rightmost_tie",
     "if (key[j] < key[best]) best = j; /* strict: the leftmost minimum wins */",
     "if (key[j] <= key[best]) best = j;",
     [pins.check_minimizers_bruteforce]),
    ("minimizer_no_dedup",
     "if (!have_last || best != last) sink_put(o, key[best], a + best - pos_base);",
     "sink_put(o, key[best], a + best - pos_base);",
     [pins.check_fig2_example, pins.check_minimizers_bruteforce]),
    ("minimizer_window_one_short",
     "for (j = p + 1; j < p + (uint64_t)w; ++j)\n            if (key[j] < key[best]) best = j; /* strict",
     "for (j = p + 1; j + 1 < p + (uint64_t)w; ++j)\n            if (key[j] < key[best]) best = j; /* strict",
     [pins.check_minimizers_bruteforce]),
    ("nblock_end_off_by_one",
     "for (t = lo; t < hi; ++t) isn[t] = 1;",
     "for (t = lo; t + 1 < hi; ++t) isn[t] = 1;",
     [pins.check_minimizers_bruteforce]),
    ("deque_pops_equal_keys",
     "while (tail > head && key[dq[tail - 1]] > key[j]) tail--;",
     "while (tail > head && key[dq[tail - 1]] >= key[j]) tail--;",
     [pins.check_minimizers_bruteforce]),
    ("keys_deque_pops_equal_keys",
     "while (back > front && key[q[back - 1]] > key[i]) back--;",
     "while (back > front && key[q[back - 1]] >= key[i]) back--;",
     [pins.check_batch_and_keys]),
    ("keys_deque_dedup_by_value",
     "if (!have_prev || q[front] != prev) sink_put(&o, key[q[front]], q[front]);",
     "if (!have_prev || key[q[front]] != key[prev]) sink_put(&o, key[q[front]], q[front]);",
     [pins.check_batch_and_keys]),
    ("table_offsets_unshifted",
     "offsets[(t[i].h >> shift) + 1]++;",
     "offsets[(t[i].h >> shift)]++;",
     [pins.check_table]),
    ("seed_filter_inclusive",
     "if (max_occ != 0 && a - lo > max_occ) continue;",
     "if (max_occ != 0 && a - lo >= max_occ) continue;",
     [pins.check_seed_hits]),
    ("seed_search_upper_bound",
     "if (t[mid].h < qh[i]) lo = mid + 1;",
     "if (t[mid].h <= qh[i]) lo = mid + 1;",
     [pins.check_seed_hits]),
    ("strand_forward_complement_order",
     "rc = rc + ((uint64_t)(3 - b) << (2 * j));  /* complement, read backwards */",
     "rc = rc * 4 + (uint64_t)(3 - b);",
     [pins.check_strands]),
    ("batch_positions_global",
     "run_minimizers_naive(s, (uint64_t)offs[r], (uint64_t)offs[r + 1], k, w, mode, (uint64_t)offs[r], &o);",
     "run_minimizers_naive(s, (uint64_t)offs[r], (uint64_t)offs[r + 1], k, w, mode, 0, &o);",
     [pins.check_batch_and_keys]),
]


@pytest.mark.parametrize("name,old,new,checks", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_mutant(tmp_path, name, old, new, checks):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    so = str(tmp_path / "libmutant.so")
    oracle.build(force=True, src=str(mut), out=so)
    lib = oracle.load(so)
    caught = []
    for check in checks:
        try:
            check(lib)
        except AssertionError:
            caught.append(check.__name__)
    assert caught, f"mutant {name} survived {[c.__name__ for c in checks]}"
