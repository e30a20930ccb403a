"""The oracle's pins catch plausible mistakes: each mutant below is a copy of
oracle/bbe_oracle.c with one deliberate error (in the oracle, on the CPU); the pin suites
(tests/test_oracle_rng.py, tests/test_oracle_race.py, tests/test_oracle_places.py,
tests/test_oracle_trajectory.py, tests/test_oracle_preference.py, tests/test_oracle_orders.py,
tests/test_oracle_time_law.py) must fail
against every mutant."""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "bbe_oracle.c")

MUTANTS = {
    "blocking_boundary_inclusive": ("blocked = !(Delta_c > race->theta[c]);", "blocked = !(Delta_c >= race->theta[c]);"),
    "delta_min_ignores_leader": ("prev[c] < prev[i_plus] ? prev[c] : prev[i_plus]", "prev[c]"),
    "finish_line_exclusive": ("if (dn[c] >= race->L) any_finished = 1;", "if (dn[c] > race->L) any_finished = 1;"),
    "winner_first_index": ("if (winner < 0 || tau < best_tau) {", "if (winner < 0) {"),
    "responsiveness_sign": ("kr[c] = BBE_ORACLE_KAPPA * ((2.0f * race->rho[c]) - 1.0f);",
                            "kr[c] = BBE_ORACLE_KAPPA * (1.0f - (2.0f * race->rho[c]));"),
    "preference_when_blocked": ("S_c = R_c * delta_min;", "S_c = (R_c * race->P[c]) * delta_min;"),
    "farthest_in_front": ("if (i_plus < 0 || d[i] < d[i_plus]) i_plus = i;", "if (i_plus < 0 || d[i] > d[i_plus]) i_plus = i;"),
    "philox_multiplier": ("const uint32_t M0 = 0xD2511F53u", "const uint32_t M0 = 0xD2511F55u"),
    "philox_key_bump_first": ("        if (round > 0) {\n            k0 += W0;", "        if (round >= 0) {\n            k0 += W0;"),
    "box_muller_pair_order": ("return (t & 1u) ? radius * sv : radius * cv;", "return (t & 1u) ? radius * cv : radius * sv;"),
    "log_coefficient": ("-0x1.000428p-2f", "-0x1.100428p-2f"),
    "sin_quadrant": ("case 1: *sin_out = cv;  *cos_out = -sv; break;", "case 1: *sin_out = cv;  *cos_out = sv; break;"),
    "uniform_scale": ("return 0x1.bb67aep+0f * ((2.0f * u) - 1.0f);", "return 0x1.bb67aep+0f * (u - 1.0f);"),
    "steps_exclude_finish": ("            ++t;\n            break;\n        }", "            break;\n        }"),
    "update_not_synchronous": ("        race_step(race, kr, invL, d, prev, seed, r, k, (uint32_t)t, S);",
                               "        race_step(race, kr, invL, d, prev, seed, r, k, (uint32_t)t, S);\n        for (int c = 0; c < race->n; ++c) if (c == 0) d[c] += S[c];"),
    "floor_dropped": ("if (S_c < BBE_ORACLE_S_FLOOR) S_c = BBE_ORACLE_S_FLOOR;", ";"),
    "counter_word_swap": ("uint32_t ctr[4] = { k, t >> 2, c, r };", "uint32_t ctr[4] = { k, t >> 2, r, c };"),
    "places_in_index_order": ("if (best < 0 || tau < best_tau) {", "if (best < 0) {"),
    "finished_competitors_stop": ("        if (placed >= places) break;\n        for (int c = 0; c < n; ++c) {\n",
                                  "        if (placed >= places) break;\n        for (int c = 0; c < n; ++c) {\n            if (finished[c]) continue;\n"),
    "places_short_of_n": ("int kk = places < n ? places : n;", "int kk = places < n ? places : n - 1;"),
    "trajectory_records_start": ("if (d_traj) memcpy(d_traj + t * n, dn,", "if (d_traj) memcpy(d_traj + t * n, d,"),
    "trajectory_ends_at_first_finisher": (
        "int all_in = 1;\n        for (int c = 0; c < n; ++c) {\n            dn[c] = d[c] + S[c];\n"
        "            if (!(dn[c] >= race->L)) all_in = 0;",
        "int all_in = 0;\n        for (int c = 0; c < n; ++c) {\n            dn[c] = d[c] + S[c];\n"
        "            if (dn[c] >= race->L) all_in = 1;"),
    "preference_unclamped": ("if (m > 1.0f) m = 1.0f;", ";"),
    "preference_additive": ("p = p * (1.0f - weights[i] * m);", "p = p - weights[i] * m;"),
    "time_law_sign": ("return fmaf(kr, u - 0.5f, 1.0f);", "return fmaf(kr, 0.5f - u, 1.0f);"),
    "time_law_uncapped": ("    if (u > 1.0f) u = 1.0f;\n    return fmaf(kr, u - 0.5f", "    return fmaf(kr, u - 0.5f"),
    "time_law_ignores_elapsed": ("float u = (t0 + (float)t) * invT;", "float u = (float)t * invT;"),
    "time_law_uses_position": ("? responsiveness_time(kr[c], race->t0, t, invT)", "? responsiveness(kr[c], d[c], invL)"),
    "order_tuple_reversed": ("for (int j = 0; j < kk; ++j) code = code * n + order[j];",
                             "for (int j = kk - 1; j >= 0; --j) code = code * n + order[j];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert old in src, f"mutation site of {name} not found"
    msrc = tmp_path / "bbe_oracle.c"
    msrc.write_text(src.replace(old, new, 1))
    so = oracle.compile_source(str(msrc), str(tmp_path / "libmutant.so"))
    env = dict(os.environ, BBE_ORACLE_LIB=so)
    # the quick suites first: -x stops at the first failing pin
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                          os.path.join(ROOT, "tests", "test_oracle_preference.py"),
                          os.path.join(ROOT, "tests", "test_oracle_time_law.py"),
                          os.path.join(ROOT, "tests", "test_oracle_trajectory.py"),
                          os.path.join(ROOT, "tests", "test_oracle_orders.py"),
                          os.path.join(ROOT, "tests", "test_oracle_race.py"),
                          os.path.join(ROOT, "tests", "test_oracle_places.py"),
                          os.path.join(ROOT, "tests", "test_oracle_rng.py")],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode != 0, f"mutant {name} passed every pin:\n{res.stdout[-2000:]}"
