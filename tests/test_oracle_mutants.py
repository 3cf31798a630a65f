"""The pins catch plausible mistakes: each mutant of the oracle must fail at least one pin.

Each case copies the oracle's C source to a temporary directory, plants one mistake (a wrong
neighbour index, a dropped condition, swapped sublattice order, an off-by-one or reversed draw
order in the dyadic construction, a wrong Philox operand, a non-strict threshold, a wrong height
path, a wrong packed offset, a missing flip, a missing counter field, q replaced by p, and on X x Y
lattices a row count and a row length confused with each other, a wrong factor or sign in the
two-time correlation, the origin's height change counted at a neighbour or with the wrong sign; in the random-
sequential dynamics the site from the wrong bits, the wrong active words, too few attempts)
and runs
the oracle pin tests against the mutant.  CPU only; the GPU library is not involved.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "sx_plus_left": ("int64_t xr = (x + 1) % X;", "int64_t xr = (x + X - 1) % X;"),
    "drop_c_in_min": ("int is_min = (*a == 0 && *b == 0 && *c == 1 && *d == 1);",
                      "int is_min = (*a == 0 && *b == 0 && *d == 1);"),
    "odd_first": ("for (int s = 0; s <= 1; s++) {\n            #pragma omp parallel for schedule(static) reduction(+:org, tot)\n"
                  "            for (int64_t y = 0; y < Y; y++)",
                  "for (int s1 = 0; s1 <= 1; s1++) { int s = 1 - s1;\n"
                  "            #pragma omp parallel for schedule(static) reduction(+:org, tot)\n"
                  "            for (int64_t y = 0; y < Y; y++)"),
    "dyadic_off_by_one": ("return R >= ((uint64_t)1 << n) - P;", "return R > ((uint64_t)1 << n) - P;"),
    "dyadic_lsb_first": ("for (int i = 1; i <= n; i++) R = (R << 1) | draw_bits[i - 1];",
                         "for (int i = n; i >= 1; i--) R = (R << 1) | draw_bits[i - 1];"),
    "philox_wrong_key_word": ("uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c1 ^ k0;",
                              "uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c1 ^ k1;"),
    "uniform_non_strict": ("return (uint64_t)oracle_site_uniform(r->L, r->seed, t, s, x, y) < T;",
                           "return (uint64_t)oracle_site_uniform(r->L, r->seed, t, s, x, y) <= T;"),
    "height_column_uses_sx": ("if (y > 0) h0 += 2 * (int64_t)by[y * X + 0] - 1;\n        col0[y] = h0;",
                              "if (y > 0) h0 += 2 * (int64_t)bx[y * X + 0] - 1;\n        col0[y] = h0;"),
    "pack_swapped_s_d": ("uint64_t idx = ((uint64_t)(s * 2 + d) * (uint64_t)Y + (uint64_t)y) * W + (k >> 5);",
                         "uint64_t idx = ((uint64_t)(d * 2 + s) * (uint64_t)Y + (uint64_t)y) * W + (k >> 5);"),
    "flip_three_of_four": ("*a ^= 1; *b ^= 1; *c ^= 1; *d ^= 1;", "*a ^= 1; *b ^= 1; *c ^= 1;"),
    "tag_missing": ("ctr[3] = (uint32_t)tag | ((uint32_t)(g >> 32) << 1);",
                    "ctr[3] = ((uint32_t)(g >> 32) << 1);"),
    "removal_uses_p": ("uint64_t P = removal ? r->Pq : r->Pp;", "uint64_t P = r->Pp;"),
    "t_missing_from_counter": ("ctr[1] = (uint32_t)t;", "ctr[1] = 0;"),
    # X x Y lattices: a row count or row length used where the other belongs
    "rect_row_successor_mod_X": ("int dh = update_site(&r, bx, by, X, y, (y + 1) % Y, x, y, t, s);",
                                 "int dh = update_site(&r, bx, by, X, y, (y + 1) % X, x, y, t, s);"),
    "rect_pack_plane_of_X_rows": ("uint64_t idx = ((uint64_t)(s * 2 + d) * (uint64_t)Y + (uint64_t)y) * W + (k >> 5);",
                                  "uint64_t idx = ((uint64_t)(s * 2 + d) * (uint64_t)X + (uint64_t)y) * W + (k >> 5);"),
    "rect_N_is_X_squared": ("unsigned __int128 N = (unsigned __int128)((uint64_t)X * (uint64_t)Y);",
                            "unsigned __int128 N = (unsigned __int128)((uint64_t)X * (uint64_t)X);"),
    "rect_draws_keyed_by_row_count": (
        "if (X < 2 || (X & 1) || Y < 2 || (Y & 1)) return -1;\n    if (rule_make(&r, X, seed, p, q, mode))",
        "if (X < 2 || (X & 1) || Y < 2 || (Y & 1)) return -1;\n    if (rule_make(&r, Y, seed, p, q, mode))"),
    # origin height counter
    "origin_counts_a_neighbour": ("if (x == 0 && y == 0) org += dh;", "if (x == 1 && y == 0) org += dh;"),
    "height_change_sign_of_removal": ("return is_min ? 2 : -2;", "return 2;"),
    # random-sequential dynamics on the 4 x 4 words
    "rs_site_from_low_bits": ("const int i = (int)(out[0] >> 28);", "const int i = (int)(out[0] & 15);"),
    "rs_active_words_in_columns": ("if (((wx + wy) & 1) != ph) continue;", "if ((wx & 1) != ph) continue;"),
    "rs_eight_attempts": ("for (int a = 0; a < 16; a++) {", "for (int a = 0; a < 8; a++) {"),
    # two-time correlation
    "corr_product_uses_a_twice": ("Sab += (__int128)ha[i] * hb[i];", "Sab += (__int128)ha[i] * ha[i];"),
    "corr_numerator_sign": ("__int128 cnum = (__int128)n * Sab - Sa * Sb;",
                            "__int128 cnum = Sa * Sb - (__int128)n * Sab;"),
}
# mutants that only an X x Y lattice with X != Y can show run against those pins alone
RECT_ONLY = {"rect_row_successor_mod_X", "rect_pack_plane_of_X_rows", "rect_N_is_X_squared",
             "rect_draws_keyed_by_row_count"}

# fastest pins first: a mutant stops at its first failing pin (-x)
PIN_TESTS = ["tests/test_oracle_philox.py", "tests/test_oracle_decisions.py",
             "tests/test_oracle_rect.py", "tests/test_oracle_rules.py"]
RECT_PINS = ["tests/test_oracle_rect.py"]
CORR_ONLY = {"corr_product_uses_a_twice", "corr_numerator_sign"}
CORR_PINS = ["tests/test_oracle_corr.py"]
HEIGHT_ONLY = {"origin_counts_a_neighbour", "height_change_sign_of_removal"}
HEIGHT_PINS = ["tests/test_oracle_height.py"]
RS_ONLY = {"rs_site_from_low_bits", "rs_active_words_in_columns", "rs_eight_attempts"}
RS_PINS = ["tests/test_oracle_rs.py"]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    src = open(os.path.join(ROOT, "oracle", "sca_oracle.c")).read()
    before, after = MUTANTS[name]
    assert src.count(before) == 1, "mutation site moved: " + name
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "*.tmp*", "__pycache__"))
    (tmp_path / "oracle" / "sca_oracle.c").write_text(src.replace(before, after))
    shutil.copytree(os.path.join(ROOT, "tests"), tmp_path / "tests",
                    ignore=shutil.ignore_patterns("__pycache__", "test_oracle_mutants.py"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp_path / "pytest.ini")
    pins = (RECT_PINS if name in RECT_ONLY else CORR_PINS if name in CORR_ONLY else
            HEIGHT_PINS if name in HEIGHT_ONLY else RS_PINS if name in RS_ONLY else PIN_TESTS)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        *pins], cwd=str(tmp_path), capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 1, "mutant %s survived:\n%s" % (name, r.stdout[-2000:])
    assert "failed" in r.stdout
