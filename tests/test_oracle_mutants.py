"""Planted mistakes in the oracle must fail its pins (CPU only).

Each mutant below is a copy of oracle/oracle.cpp with one plausible mistake
planted in it: a wrong entry of the Pauli product table, a flipped sign, a
swapped cos/sin, a dropped term, a transposed index, an inverted inequality,
the wrong gate or digit order, damping at the wrong point, and so on.  Every
mutant is compiled on its own and the pins (tests/test_oracle_pins.py and
tests/test_oracle_groups.py, which compare the oracle with state vectors,
density matrices, closed forms, Burnside counts and brute force) are run
against it through the PP_ORACLE_SO override.  The test passes only if the
pins fail for every mutant.  The two stored-trajectory checks are left out:
their expected values were written by the oracle itself, so they would catch
a mutant without saying anything about the pins' strength.

Each substitution names the exact text it replaces and how often that text
occurs in oracle.cpp, so an edit of the oracle that moves the text makes this
test fail loudly instead of silently testing nothing.
"""
import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "oracle.cpp")
PINS = [os.path.join(HERE, "test_oracle_pins.py"), os.path.join(HERE, "test_oracle_groups.py")]
DESELECT = "not stored_ring_trajectories and not stored_heisenberg_trajectory"

# (name, [(text, replacement, occurrences of text in oracle.cpp, which one)])
MUTANTS = [
    # --- Pauli product and the branch rule (App. A, Prop. 1 proof)
    ("product_table_x_row_reversed",
     [("{{1, 0}, {0, 0}, {3, 1}, {2, 3}}", "{{1, 0}, {0, 0}, {3, 3}, {2, 1}}", 1, 0)]),
    ("product_table_wrong_letter",
     [("{{2, 0}, {3, 3}, {0, 0}, {1, 1}}", "{{2, 0}, {3, 3}, {0, 0}, {3, 1}}", 1, 0)]),
    ("identity_site_anticommutes",
     [("return a != 0 && b != 0 && a != b;", "return a != 0 && a != b;", 1, 0)]),
    ("anticommutes_if_any_site_does",
     [("if (anti % 2 == 0) {\n      next[Q] += d;", "if (anti == 0) {\n      next[Q] += d;", 1, 0)]),
    ("child_sign_flipped",
     [("int e = (phase + 1) % 4;", "int e = (phase + 3) % 4;", 1, 0)]),
    ("cos_and_sin_swapped",
     [("next[Q] += c * d;", "next[Q] += s * d;", 1, 0)]),
    ("child_term_dropped",
     [("next[R] += sign * (s * d);", "(void)sign;", 1, 0)]),
    ("half_angle_convention",
     [("const double c = std::cos(theta);\n  const double s = std::sin(theta);",
       "const double c = std::cos(theta / 2);\n  const double s = std::sin(theta / 2);", 1, 0)]),
    ("gates_applied_in_time_order",
     [("for (int g = n_gates - 1; g >= 0; --g) {", "for (int g = 0; g < n_gates; ++g) {", 2, 0)]),
    # --- encoding (Definition "Lowest integer representation")
    ("mask_letters_y_and_z_swapped",
     [("if (xb && zb) l = 2;\n    if (!xb && zb) l = 3;",
       "if (xb && zb) l = 3;\n    if (!xb && zb) l = 2;", 1, 0)]),
    ("export_x_and_z_swapped",
     [("x[i * st->W + w] = key[w];\n      z[i * st->W + w] = key[st->W + w];",
       "z[i * st->W + w] = key[w];\n      x[i * st->W + w] = key[st->W + w];", 1, 0)]),
    ("digit_order_reversed",
     [("for (int q = (int)a.size() - 1; q >= 0; --q) {",
       "for (int q = 0; q < (int)a.size(); ++q) {", 1, 0)]),
    # --- Algorithm 2 (Z_n), Algorithm 3 (S_n), other groups
    ("zn_misses_last_rotation",
     [("for (int j = 1; j < (int)s.size(); ++j) {",
       "for (int j = 1; j + 1 < (int)s.size(); ++j) {", 1, 0)]),
    ("sn_layout_x_first",
     [("for (int k = 0; k < nz; ++k) r[q++] = 3;", "for (int k = 0; k < nz; ++k) r[q++] = 1;", 1, 0),
      ("for (int k = 0; k < nx; ++k) r[q++] = 1;", "for (int k = 0; k < nx; ++k) r[q++] = 3;", 1, 0)]),
    ("sn_counts_x_as_y",
     [("if (ch == 2) ++ny;", "if (ch == 1) ++ny;", 1, 0)]),
    ("dihedral_without_reflections",
     [("      out.push_back(ref);\n", "", 1, 0)]),
    ("torus_wraps_rows_by_row_length",
     [("m[q] = (x + dx) % lx + lx * ((y + dy) % ly);", "m[q] = (x + dx) % lx + lx * ((y + dy) % lx);",
       1, 0)]),
    # --- merging (Eq. O-merging) and ingest (Algorithm 1 step 1)
    ("merge_overwrites_instead_of_accumulating",
     [("merged[canonical(kv.first, group)] += kv.second;",
       "merged[canonical(kv.first, group)] = kv.second;", 1, 0)]),
    ("ingest_overwrites_duplicates",
     [("st->terms[s] += coef[i];", "st->terms[s] = coef[i];", 1, 0)]),
    # --- truncation
    ("truncation_keeps_the_small_terms",
     [("!(std::fabs(c) >= eps)", "!(std::fabs(c) <= eps)", 1, 0)]),
    ("weight_limit_off_by_one",
     [("if (wmax >= 0 && weight(s) > wmax) return false;",
       "if (wmax >= 0 && weight(s) >= wmax) return false;", 2, 0)]),
    ("batched_weight_limit_off_by_one",
     [("if (wmax >= 0 && weight(s) > wmax) return false;",
       "if (wmax >= 0 && weight(s) >= wmax) return false;", 2, 1)]),
    # --- noise (per gate and per layer)
    ("gate_noise_counts_the_whole_support",
     [("for (int q : support) k += (Q[q] != 0);\n      if (k > 0) d = d * damp[k];",
       "for (int q : support) k += 1;\n      if (k > 0) d = d * damp[k];", 1, 0)]),
    ("gate_noise_factor_parameterised_wrongly",
     [("damp[k] = damp[k - 1] * (1.0 - p);", "damp[k] = damp[k - 1] * (1.0 - 4.0 * p / 3.0);", 2, 0)]),
    ("gate_noise_after_the_rotation",
     [("    if (noise_mode == 1) {\n      int k = 0;\n      for (int q : support) k += (Q[q] != 0);\n"
       "      if (k > 0) d = d * damp[k];\n    }\n",
       "    auto dmp = [&](const std::string& S) {\n      int k = 0;\n"
       "      if (noise_mode == 1)\n        for (int q : support) k += (S[q] != 0);\n"
       "      return damp[k];\n    };\n", 1, 0),
      ("next[Q] += d;\n      continue;", "next[Q] += d * dmp(Q);\n      continue;", 1, 0),
      ("next[Q] += c * d;", "next[Q] += c * d * dmp(Q);", 1, 0),
      ("next[R] += sign * (s * d);", "next[R] += sign * (s * d) * dmp(R);", 1, 0)]),
    ("layer_noise_ignores_weight",
     [("std::exp(-gamma * (double)weight(kv.first))", "std::exp(-gamma)", 1, 0)]),
    ("layer_noise_after_the_gates",
     [("  if (noise_mode == 2) orc_damp_layer(h, p, eps, wmax);\n", "", 1, 0),
      ("  if (group != 0) orc_symmetry_merge(h, group, eps, wmax);\n",
       "  if (noise_mode == 2) orc_damp_layer(h, p, eps, wmax);\n"
       "  if (group != 0) orc_symmetry_merge(h, group, eps, wmax);\n", 1, 0)]),
    # --- overlaps (Algorithm 1 step 3; the symmetrised overlap)
    ("bloch_components_transposed",
     [("return bloch[3 * q + (letter - 1)];", "return bloch[3 * q + (3 - letter)];", 1, 0)]),
    ("zn_overlap_not_averaged",
     [("return acc / (double)st->n;", "return acc;", 1, 0)]),
    ("sn_overlap_x_site_uses_y_component",
     [("(double)x * bloch_value(bloch, k, 1)", "(double)x * bloch_value(bloch, k, 2)", 1, 0)]),
    ("sn_overlap_wrong_divisor",
     [("cur[at(x, y, z)] = v / (double)left;", "cur[at(x, y, z)] = v / (double)n;", 1, 0)]),
    ("expectation_drops_the_coefficient",
     [("acc += kv.second * sym_overlap(st, kv.first, bloch, group);",
       "acc += sym_overlap(st, kv.first, bloch, group);", 1, 0)]),
    # --- live-term count (the gate-update metric)
    ("updates_count_the_children",
     [("st->updates += (double)st->terms.size();\n  std::unordered_map<std::string, double> next;",
       "std::unordered_map<std::string, double> next;", 1, 0),
      ("  st->terms.swap(next);\n  truncate_all(st, eps, wmax);",
       "  st->updates += (double)next.size();\n  st->terms.swap(next);\n  truncate_all(st, eps, wmax);",
       1, 0)]),
    # --- batched rows (one coefficient per angle set)
    ("batched_gates_applied_in_time_order",
     [("for (int g = n_gates - 1; g >= 0; --g) {", "for (int g = 0; g < n_gates; ++g) {", 2, 1)]),
    ("batched_child_sign_flipped",
     [("double sign = ((phase + 1) % 4 == 0) ? 1.0 : -1.0;",
       "double sign = ((phase + 3) % 4 == 0) ? 1.0 : -1.0;", 1, 0)]),
    ("batched_first_columns_angle_everywhere",
     [("c[b] = std::cos(theta[b]);", "c[b] = std::cos(theta[0]);", 1, 0)]),
    ("batched_angle_rows_transposed",
     [("theta + (size_t)g * st->B", "theta + (size_t)g", 1, 0)]),
    ("batched_noise_exponent_dropped",
     [("for (int b = 0; b < B; ++b) d[b] = d[b] * damp[k];",
       "for (int b = 0; b < B; ++b) d[b] = d[b] * damp[1];", 1, 0)]),
    ("batched_noise_on_first_column_only",
     [("for (int b = 0; b < B; ++b) d[b] = d[b] * damp[k];", "d[0] = d[0] * damp[k];", 1, 0)]),
    ("batched_noise_factor_parameterised_wrongly",
     [("damp[k] = damp[k - 1] * (1.0 - p);", "damp[k] = damp[k - 1] * (1.0 - 4.0 * p / 3.0);", 2, 1)]),
    ("batched_keep_needs_every_column",
     [("    if (std::fabs(v) >= eps) return true;\n  return false;",
       "    if (!(std::fabs(v) >= eps)) return false;\n  return true;", 1, 0)]),
    ("batched_ingest_overwrites_duplicates",
     [("for (int b = 0; b < B; ++b) r[b] += coef[i * B + b];",
       "for (int b = 0; b < B; ++b) r[b] = coef[i * B + b];", 1, 0)]),
    ("batched_updates_count_the_children",
     [("st->updates += (double)st->terms.size();\n  std::unordered_map<std::string, std::vector<double>> next;",
       "std::unordered_map<std::string, std::vector<double>> next;", 1, 0),
      ("  st->terms.swap(next);\n  btruncate(st, eps, wmax);",
       "  st->updates += (double)next.size();\n  st->terms.swap(next);\n  btruncate(st, eps, wmax);",
       1, 0)]),
    ("batched_merge_overwrites",
     [("for (int b = 0; b < st->B; ++b) row[b] += kv.second[b];",
       "for (int b = 0; b < st->B; ++b) row[b] = kv.second[b];", 1, 0)]),
    # --- further mistakes: argmax for argmin, truncation skipped after a merge,
    # the second mask word, single-site phases, other weights and lookups
    ("representative_is_the_largest",
     [("if (a[q] != b[q]) return (uint8_t)a[q] < (uint8_t)b[q];",
       "if (a[q] != b[q]) return (uint8_t)a[q] > (uint8_t)b[q];", 1, 0)]),
    ("merge_not_truncated",
     [("  symmetry_merge(st, group);\n  truncate_all(st, eps, wmax);\n  return 0;",
       "  symmetry_merge(st, group);\n  return 0;", 1, 0)]),
    ("ingest_not_truncated",
     [("  if (group != 0) symmetry_merge(st, group);\n  truncate_all(st, eps, wmax);\n  return st;",
       "  if (group != 0) symmetry_merge(st, group);\n  return st;", 1, 0)]),
    ("batched_merge_not_truncated",
     [("    bmerge(st, group);\n    btruncate(st, eps, wmax);\n  }",
       "    bmerge(st, group);\n  }", 1, 0)]),
    ("layer_noise_as_power_of_one_minus_gamma",
     [("std::exp(-gamma * (double)weight(kv.first))", "std::pow(1.0 - gamma, (double)weight(kv.first))", 1, 0)]),
    ("batched_expect_uses_first_column",
     [("out[b] += kv.second[b] * ov;", "out[b] += kv.second[0] * ov;", 1, 0)]),
    ("second_mask_word_ignored",
     [("int xb = (x[q / 64] >> (q % 64)) & 1;\n    int zb = (z[q / 64] >> (q % 64)) & 1;",
       "int xb = (x[0] >> (q % 64)) & 1;\n    int zb = (z[0] >> (q % 64)) & 1;", 1, 0)]),
    ("phase_from_last_site_only",
     [("      phase += pr.phase;\n    }\n    // P Q", "      phase = pr.phase;\n    }\n    // P Q", 1, 0)]),
    ("weight_counts_only_z",
     [("for (char ch : s) w += (ch != 0);", "for (char ch : s) w += (ch == 3);", 1, 0)]),
    ("sn_table_lookup_y_and_z_swapped",
     [("return st->sn_table[((size_t)nx * S + ny) * S + nz];",
       "return st->sn_table[((size_t)nx * S + nz) * S + ny];", 1, 0)]),
    ("element_overlap_divided_by_n",
     [("return acc / (double)els.size();", "return acc / (double)st->n;", 1, 0)]),
    ("zn_overlap_skips_identity_translation",
     [("for (int j = 0; j < st->n; ++j) acc += product_overlap(translate(s, j), bloch);",
       "for (int j = 1; j < st->n; ++j) acc += product_overlap(translate(s, j), bloch);", 1, 0)]),
    ("sn_overlap_drops_identity_sites",
     [("if (i > 0) v += (double)i * bloch_value(bloch, k, 0) * next[at(x, y, z)];\n", "", 1, 0)]),
    ("merge_always_by_translations",
     [("merged[canonical(kv.first, group)] += kv.second;", "merged[canonical(kv.first, 1)] += kv.second;", 1, 0)]),
    ("batched_merge_always_by_translations",
     [("auto& row = merged[canonical(kv.first, group)];", "auto& row = merged[canonical(kv.first, 1)];", 1, 0)]),
    ("letters_y_written_without_x",
     [("if (l == 1 || l == 2) x[q / 64]", "if (l == 1) x[q / 64]", 1, 0)]),
    ("batched_commuting_row_dropped",
     [("      for (int b = 0; b < B; ++b) r[b] += d[b];\n      continue;",
       "      continue;", 1, 0)]),
    ("batched_cos_on_child",
     [("for (int b = 0; b < B; ++b) rr[b] += sign * (s[b] * d[b]);",
       "for (int b = 0; b < B; ++b) rr[b] += sign * (c[b] * d[b]);", 1, 0)]),
    ("torus_rows_not_translated",
     [("for (int dy = 0; dy < ly; ++dy)", "for (int dy = 0; dy < 1; ++dy)", 1, 0)]),
    ("keep_ignores_eps_sign_of_negative",
     [("if (eps > 0.0 && !(std::fabs(c) >= eps)) return false;",
       "if (eps > 0.0 && !(c >= eps)) return false;", 1, 0)]),
    ("batched_keep_ignores_abs",
     [("    if (std::fabs(v) >= eps) return true;", "    if (v >= eps) return true;", 1, 0)]),
    ("export_second_word_into_the_first",
     [("if (l == 1 || l == 2) x[q / 64] |=", "if (l == 1 || l == 2) x[0] |=", 1, 0),
      ("if (l == 2 || l == 3) z[q / 64] |=", "if (l == 2 || l == 3) z[0] |=", 1, 0)]),
]


def _mutate(text, subs):
    for old, new, count, which in subs:
        assert text.count(old) == count, f"expected {count} occurrence(s) of {old!r}"
        at = -1
        for _ in range(which + 1):
            at = text.index(old, at + 1)
        text = text[:at] + new + text[at + len(old):]
    return text


def _run_mutant(name, subs, base, workdir):
    src = os.path.join(workdir, name + ".cpp")
    lib = os.path.join(workdir, name + ".so")
    with open(src, "w") as f:
        f.write(_mutate(base, subs))
    b = subprocess.run(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared",
                        src, "-o", lib], capture_output=True, text=True)
    if b.returncode != 0:
        return name, "build failed", b.stderr[-400:]
    env = dict(os.environ, PP_ORACLE_SO=lib)
    try:
        r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-p",
                            "no:cacheprovider", "-k", DESELECT, "-rf"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    except subprocess.TimeoutExpired:
        return name, "caught", "timed out"
    if r.returncode == 0:
        return name, "survived", r.stdout[-300:]
    failed = re.findall(r"^FAILED (\S+)", r.stdout, flags=re.M)
    return name, "caught", failed[0] if failed else r.stdout[-300:]


def test_mutant_list_applies_to_the_oracle():
    with open(SRC) as f:
        base = f.read()
    names = [m[0] for m in MUTANTS]
    assert len(names) == len(set(names))
    for name, subs in MUTANTS:
        assert _mutate(base, subs) != base, name


def test_every_planted_mistake_fails_a_pin(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    with open(SRC) as f:
        base = f.read()
    workers = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(lambda m: _run_mutant(m[0], m[1], base, str(tmp_path)), MUTANTS))
    bad = [(n, s, d) for n, s, d in results if s != "caught"]
    assert not bad, "mutants the pins did not catch:\n" + "\n".join(f"{n}: {s}: {d}" for n, s, d in bad)
