"""The oracle's pins catch plausible slips.  Each case copies the oracle's C
source, plants one mistake (a dropped term, a swapped operand, an off-by-one),
compiles it on the CPU and runs pins from test_oracle_pins.py against it; at
least one must fail.  Nothing here touches a GPU."""
import os
import subprocess

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "rmat_oracle.c")

MUTATIONS = [
    ("b and c swapped in the expansion", "child.p = e.p * P[s];\n            child.len = e.len + 1;",
     "child.p = e.p * P[s == 1 ? 2 : (s == 2 ? 1 : s)];\n            child.len = e.len + 1;",
     [lambda: pins.test_exact_distribution_equals_kronecker(*list(pins._distribution_cases())[5])]),
    ("row and column bits swapped", "                r = (r << 1) | (uint64_t)(s >> 1);\n                c = (c << 1) | (uint64_t)(s & 1);\n            }\n            filled += take;",
     "                r = (r << 1) | (uint64_t)(s & 1);\n                c = (c << 1) | (uint64_t)(s >> 1);\n            }\n            filled += take;",
     [lambda: pins.test_per_level_quadrant_frequencies("alias_variable")]),
    ("stop rule off by one", "heap.n + ndone + 3 < bound", "heap.n + ndone + 3 <= bound",
     [lambda: pins.test_table_sizes_fig1("variable", 12, 4093)]),
    ("Philox multiplier typo", "#define PHILOX_M0 0xD2511F53u", "#define PHILOX_M0 0xD2511F35u",
     [pins.test_philox_matches_independent_engine]),
    ("Philox output words rotated", "(uint32_t)e, (uint32_t)(e >> 32)};\n    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};\n    uint32_t out[4];\n    orc_philox4x32_10(ctr, key, out);\n    return out[n % 4];",
     "(uint32_t)e, (uint32_t)(e >> 32)};\n    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};\n    uint32_t out[4];\n    orc_philox4x32_10(ctr, key, out);\n    return out[(n + 1) % 4];",
     [pins.test_philox_matches_independent_engine]),
    ("Vose drops a term", "rest[l] -= C - rest[s];", "rest[l] -= C;",
     [lambda: pins.test_weights_and_alias_roundtrip(lambda: oracle.Table.fixed([pins.ASYM], 4))]),
    ("remainder to the smallest fractions", "if (a->frac != b->frac) return (a->frac < b->frac) - (a->frac > b->frac);",
     "if (a->frac != b->frac) return (a->frac > b->frac) - (a->frac < b->frac);",
     [lambda: pins.test_weights_and_alias_roundtrip(lambda: oracle.Table.variable(*pins.G500, 26, 4096))]),
    ("draw keeps the column on equality", "return r < t->thr[j] ? j : t->alias[j];", "return r <= t->thr[j] ? j : t->alias[j];",
     [pins.test_draw_keeps_column_with_probability_thr_over_C_exactly]),
    ("naive sampler uses a+c for the second threshold", "T[3 * lvl + 1] = naive_threshold(P[0] + P[1]);",
     "T[3 * lvl + 1] = naive_threshold(P[0] + P[2]);",
     [lambda: pins.test_per_level_quadrant_frequencies("naive")]),
    ("undirected keeps the larger index first", "            c = orc_scramble(c, k, consts);\n        }\n        if (undirected && r > c)",
     "            c = orc_scramble(c, k, consts);\n        }\n        if (undirected && r < c)",
     [pins.test_undirected_mirrors_lower_triangle]),
    ("scramble shift loses a bit", "int h = (k + 1) / 2;", "int h = k / 2;",
     [lambda: pins.test_scramble_is_a_bijection(1, 3)]),
    ("scramble multiplier may be even", "out[2 * i] = (splitmix64_next(&st) | 1ull) & mask;",
     "out[2 * i] = splitmix64_next(&st) & mask;",
     [lambda: pins.test_scramble_is_a_bijection(12, 7), lambda: pins.test_scramble_is_a_bijection(16, 123456789)]),
    ("split sends b's edges to c's quadrant", "    part_rec(x, depth + 1, 2 * R, 2 * C + 1, nb);      /* b: upper right */\n    part_rec(x, depth + 1, 2 * R + 1, 2 * C, nc);",
     "    part_rec(x, depth + 1, 2 * R, 2 * C + 1, nc);      /* b: upper right */\n    part_rec(x, depth + 1, 2 * R + 1, 2 * C, nb);",
     [pins.test_quadrant_split_is_multinomial]),
    ("b conditioned on b + c only", "const double den_b = (P[1] + P[2]) + P[3]", "const double den_b = (P[1] + P[2])",
     [pins.test_quadrant_split_is_multinomial]),
    ("inversion recurrence off by one", "f *= a / (double)x - sr;", "f *= a / (double)(x + 1) - sr;",
     [lambda: pins.test_binomial_matches_exact_pmf(7, 0.3), lambda: pins.test_binomial_matches_exact_pmf(40, 0.2)]),
    ("BTRS candidate shifted", "const double c = nd * p + 0.5;", "const double c = nd * p + 1.5;",
     [lambda: pins.test_binomial_matches_exact_pmf(60, 0.4), lambda: pins.test_binomial_matches_exact_pmf(100, 0.5)]),
    ("Kronecker row and column digits swapped", "r = r * n0 + (uint64_t)(s / t->n0);\n                c = c * n0 + (uint64_t)(s % t->n0);",
     "r = r * n0 + (uint64_t)(s % t->n0);\n                c = c * n0 + (uint64_t)(s / t->n0);",
     [pins.test_kron_generated_edges_follow_kronecker_power]),
    ("Kronecker stop rule keeps the 2 x 2 slack", "heap.n + ndone + (size_t)(S - 1) < bound", "heap.n + ndone + 3 < bound",
     [lambda: pins.test_kron_table_sizes_and_prefix_code(3, 104)]),
    ("tile prefix dropped", "        uint64_t r = pre_r, c = pre_c;", "        uint64_t r = pre_r, c = 0;",
     [pins.test_partitioned_graph_has_the_kronecker_distribution]),
    ("per-level groups drawn in reverse order", "const orc_table *t = tables[ngroups > 1 ? n : 0];",
     "const orc_table *t = tables[ngroups > 1 ? (uint64_t)ngroups - 1 - n : 0];",
     [lambda: pins.test_per_level_generation_follows_each_levels_parameters(2)]),
    ("Kronecker truncation keeps the bottom digits",
     "                int s = t->sym[(size_t)sel * KRON_MAX_DEPTH + lvl];\n                r = r * n0 + (uint64_t)(s / t->n0);",
     "                int s = t->sym[(size_t)sel * KRON_MAX_DEPTH + (L - take) + lvl];\n                r = r * n0 + (uint64_t)(s / t->n0);",
     [pins.test_kron_generated_edges_follow_kronecker_power]),
    ("edge numbering restarts in every tile", "x->first[x->n] = x->next;", "x->first[x->n] = 0;",
     [pins.test_tile_counts_expectation_and_numbering]),
]


def _build_mutant(tmp_path, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, old
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    hdr = os.path.join(os.path.dirname(SRC), "rmat_oracle.h")
    (tmp_path / "rmat_oracle.h").write_text(open(hdr).read())
    so = tmp_path / "mutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", str(so), str(path), "-lm"],
                   check=True)
    return oracle.load(str(so))


@pytest.mark.parametrize("name,old,new,checks", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new, checks):
    mutant = _build_mutant(tmp_path, old, new)
    saved = oracle._lib
    oracle._lib = mutant
    try:
        caught = False
        for check in checks:
            try:
                check()
            except (AssertionError, ValueError):
                caught = True
        assert caught, f"no pin caught: {name}"
    finally:
        oracle._lib = saved
