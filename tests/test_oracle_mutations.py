"""Planted mistakes in the oracle must be caught by its pins.

Each case copies the oracle source, plants one plausible mistake (a dropped
Jacobian term, a wrong sign, a transposed operand, an off-by-one row, a
wrong tie-break), and runs the pin tests against the mutant in a child
process: at least one pin must fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "tpc_oracle.c")

MUTANTS = {
    "jacobian_y_q_dropped": ("  J[0][4] = -k->K * dx * dx / (2.0 * cm3);", "  J[0][4] = 0.0;"),
    "jacobian_s_q_sign": ("  J[2][4] = -k->K * dx;", "  J[2][4] = k->K * dx;"),
    "jacobian_z_s_dropped": ("  J[1][2] = t * dx * sm / cm3;", "  J[1][2] = 0.0;"),
    "propagation_dy_sign": ("  double dy = dx * (s1 + s2) / (c1 + c2);", "  double dy = -dx * (s1 + s2) / (c1 + c2);"),
    "covariance_not_transposed": ("      for (int m = 0; m < 5; m++) a += T[i][m] * J[j][m];",
                                  "      for (int m = 0; m < 5; m++) a += T[i][m] * J[m][j];"),
    "gain_uses_wrong_column": ("    G[i][1] = s->C[i][0] * I01 + s->C[i][1] * I11;",
                               "    G[i][1] = s->C[i][1] * I01 + s->C[i][0] * I11;"),
    "link_tiebreak_reversed": ("      int better = D < b->best || (D == b->best && (d < b->d || (d == b->d && u < b->u)));",
                               "      int better = D < b->best || (D == b->best && (d > b->d || (d == b->d && u > b->u)));"),
    "link_window_y_too_small": ("static float window_y_k(int k) { return (float)(k * 2.0 * ((245.8 - 85.2) / 158.0) + 0.5); }",
                                "static float window_y_k(int k) { return (float)(k * 1.0 * ((245.8 - 85.2) / 158.0) + 0.5); }"),
    "clean_one_sided": ("    R->up_m[c] = (u >= 0 && R->dn[u] == c) ? u : -1;", "    R->up_m[c] = u;"),
    "owner_prefers_higher_id": (
        "    uint64_t key = ((uint64_t)(uint32_t)R->f_n[t] << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)t);\n"
        "    const int32_t *h = R->f_hits + (int64_t)t * NROW;\n    for (int i = 0; i < R->f_n[t]; i++)\n"
        "      if (key > R->owner[h[i]]) R->owner[h[i]] = key;",
        "    uint64_t key = ((uint64_t)(uint32_t)R->f_n[t] << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)t);\n"
        "    const int32_t *h = R->f_hits + (int64_t)t * NROW;\n    for (int i = 0; i < R->f_n[t]; i++)\n"
        "      if (key >= R->owner[h[i]] || (R->owner[h[i]] >> 32) == (key >> 32)) R->owner[h[i]] = key;"),
    "bin_scan_off_by_one": ("      while (p < b && it[p].bin < k) p++;", "      while (p < b && it[p].bin <= k) p++;"),
    "chi2_cross_term_dropped": ("  s->chi2 += r0 * (I00 * r0 + I01 * r1) + r1 * (I01 * r0 + I11 * r1);",
                                "  s->chi2 += r0 * I00 * r0 + r1 * I11 * r1;"),
    "max_miss_off_by_one_outward": ("      misses = 0;\n    } else if (++misses >= cfg->max_miss) {",
                                    "      misses = 0;\n    } else if (++misses > cfg->max_miss) {"),
    "max_miss_off_by_one_inward": ("        misses = 0;\n      } else if (++misses >= cfg->max_miss) {",
                                   "        misses = 0;\n      } else if (misses++ >= cfg->max_miss) {"),
    "max_miss_one_short_outward": ("      misses = 0;\n    } else if (++misses >= cfg->max_miss) {",
                                   "      misses = 0;\n    } else if (++misses >= cfg->max_miss - 1) {"),
    "edge_margin_sign": ("  double lim = s->x * TAN10 + k->cfg->edge;", "  double lim = s->x * TAN10 - k->cfg->edge;"),
    "edge_margin_dropped": ("  double lim = s->x * TAN10 + k->cfg->edge;", "  double lim = s->x * TAN10;"),
    "edge_test_never_stops": ("  return fabs(s->p[0]) > lim;", "  return fabs(s->p[0]) > lim + 1e9;"),
    "link_skip_window_not_scaled": ("WY2 = window_y_k(2), WZ2 = window_z_k(2);", "WY2 = window_y_k(1), WZ2 = window_z_k(1);"),
    "link_skip_despite_adjacent_pair": (
        "    if (cfg->link_skip && !(b.d >= 0 && b.best <= cfg->d_max) && row >= 2 && row <= NROW - 3) {",
        "    if (cfg->link_skip && row >= 2 && row <= NROW - 3) {"),
    "link_skip_both_sides_not_last": ("          if (b.d >= 0 && b.best <= cfg->d_max) break;\n          b.best = b.second = INFINITY;",
                                      "          if (0) break;\n          b.best = b.second;"),
    "link_skip_adjacent_chord_fraction": (
        "        float fm = (X32[row] - X32[row + dr[m]]) / (X32[row + ur[m]] - X32[row + dr[m]]);",
        "        float fm = f;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    env = dict(os.environ, TPC_ORACLE_MUTANT_SRC=str(mutant))
    proc = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert proc.returncode != 0, f"mutant {name} survived the pins:\n{proc.stdout[-2000:]}"
