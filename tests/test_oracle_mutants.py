"""Planted mistakes in the oracle, on the CPU.

Each mutant is a copy of oracle/sp_oracle.c with one plausible mistake -- a
dropped term, a wrong bound, sign, shift or index, a transposed operand, a
reversed order -- compiled on its own and loaded in place of the oracle for
one test.  The pins of test_oracle_pins.py named beside it (closed forms,
published vectors, hand-worked examples, brute force, invariants) must reject
it.  A mutant that all of its pins accepted would be a mistake the pins
cannot tell from the paper's arithmetic."""
import inspect
import os

import pytest

import oracle as O
import test_oracle_pins as P

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "sp_oracle.c")

# (name, original text, mistaken text, pins that must reject it)
MUTANTS = [
    ("tau_bound", "((uint64_t)8 << t) < (uint64_t)theta", "((uint64_t)8 << t) <= (uint64_t)theta",
     ["test_tau_closed_form"]),
    ("lsb_index", "if ((x >> i) & 1u) return i;", "if ((x >> i) & 1u) return i + 1;",
     ["test_lsb_definition"]),
    ("splitmix64_shift", "z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;", "z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ull;",
     ["test_splitmix64_published_vector"]),
    ("mas_low_half", "return (uint32_t)(v >> 32);", "return (uint32_t)v;",
     ["test_mas_closed_forms"]),
    ("draw_order", "a[i] = or_splitmix64(&s);\n    b[i] = or_splitmix64(&s);",
     "b[i] = or_splitmix64(&s);\n    a[i] = or_splitmix64(&s);", ["test_hash_params_draw_order"]),
    ("h2_low_bits", "return h1 >> 29; }", "return h1 & 7u; }",
     ["test_no_false_negative_invariant", "test_single_window_finds_all_planted"]),
    ("idx_mod_32", "uint32_t bitpos = (p->isb[i] + j) % L;", "uint32_t bitpos = (p->isb[i] + j) % 32;",
     ["test_idx_hand_worked_examples"]),
    ("lp_shift", "lp |= ((ip >> j) & 1u) << (j - r);", "lp |= ((ip >> j) & 1u) << j;",
     ["test_rp_lp_split"]),
    ("no_cover_check", "if (!covered) return 5;", "if (0) return 5;", ["test_param_constraints"]),
    ("no_overlap_check", "if (!shared) return 6;", "if (0) return 6;", ["test_param_constraints"]),
    ("sample_strict", "if (or_lsb(h1) >= tau) {", "if (or_lsb(h1) > tau) {",
     ["test_sampling_boundary_is_inclusive"]),
    ("seav_row_offset", "rp * sea_bytes + or_row_offset(p, i) + or_idx(p, i, lp)", "rp * sea_bytes + or_idx(p, i, lp)",
     ["test_single_window_finds_all_planted"]),
    ("ldc_word_dropped", "* ldc_words + h3 / 32;", "* ldc_words;", ["test_ldc_zero_count_expectation"]),
    ("ldca_row_dropped", "uint64_t word = ((uint64_t)i * lc + col) * ldc_words",
     "uint64_t word = ((uint64_t)0 * lc + col) * ldc_words", ["test_lemma1_psu_monte_carlo"]),
    ("ldc_of_oip", "uint64_t col = or_lh(a, b, p->lc_log2, i, hip);", "uint64_t col = or_lh(a, b, p->lc_log2, i, oip);",
     ["test_ldc_zero_count_expectation", "test_single_window_finds_all_planted"]),
    ("merge_xor", "dst[i] |= src[i];", "dst[i] ^= src[i];", ["test_merge_equals_concatenation"]),
    ("est_sign", "return -k * log((double)z0 / k);", "return k * log((double)z0 / k);",
     ["test_est_formula_values"]),
    ("z_theta_off_by_one", "if (or_est(k_log2, z) >= (double)theta) return z;",
     "if (or_est(k_log2, z) >= (double)theta) return z - 1;", ["test_z_theta_closed_form"]),
    ("hse_weight", "if (or_popcount(row[c]) >= 3) hse[i][nhse[i]++] = c;",
     "if (or_popcount(row[c]) >= 4) hse[i][nhse[i]++] = c;", ["test_detect_matches_forward_brute_force"]),
    ("seu_weight", "if (or_popcount(seu) >= 3) {", "if (or_popcount(seu) >= 2) {",
     ["test_detect_matches_forward_brute_force"]),
    ("no_agreement", "if (assigned[bp] && value[bp] != v) { consistent = 0; break; }",
     "if (0) { consistent = 0; break; }", ["test_detect_matches_forward_brute_force"]),
    ("ip_transposed", "ip = (uint32_t)(((uint64_t)lp << p->r) | rp);", "ip = (uint32_t)(((uint64_t)rp << L) | lp);",
     ["test_detect_matches_forward_brute_force"]),
    ("lp_bit_order", "lp |= (uint32_t)value[j] << j;", "lp |= (uint32_t)value[j] << (L - 1 - j);",
     ["test_detect_matches_forward_brute_force"]),
    ("uldc_or", "u &= ldca[((uint64_t)i * lc + col) * ldc_words + w];",
     "u |= ldca[((uint64_t)i * lc + col) * ldc_words + w];", ["test_detect_matches_forward_brute_force"]),
    ("z0_strict", "if (zeros <= zt) {", "if (zeros < zt) {", ["test_threshold_boundary_is_inclusive"]),
    ("saturated_est", "cand.est = zeros == 0 ? (double)k * log((double)k) : or_est(p->k_log2, zeros);",
     "cand.est = zeros == 0 ? 0.0 : or_est(p->k_log2, zeros);", ["test_detect_reports_est_and_saturation"]),
    ("sort_descending", "return (u->ip > v->ip) - (u->ip < v->ip);", "return (u->ip < v->ip) - (u->ip > v->ip);",
     ["test_detect_matches_forward_brute_force"]),
    ("cap_flag", "return n_found > cap ? -1 : 0;", "return n_found >= cap ? -1 : 0;",
     ["test_detect_cap_truncates_and_flags"]),
    ("psu_columns", "double keep0 = pow(1.0 - 1.0 / k, n_pairs / lc);",
     "double keep0 = pow(1.0 - 1.0 / k, n_pairs * lc);", ["test_theorem1_is_the_argmin_of_lemma1"]),
    ("lr_star_log", "return -v_ldcs * log(2.0) / (n_pairs * log(1.0 - 1.0 / k));",
     "return -v_ldcs * log(3.0) / (n_pairs * log(1.0 - 1.0 / k));", ["test_theorem1_is_the_argmin_of_lemma1"]),
]


@pytest.fixture(scope="module")
def source():
    with open(SRC) as f:
        return f.read()


def _load_variant(text, name, tmp_path, monkeypatch):
    """Builds `text` as the oracle library and loads it in place of the
    oracle (the package builds and loads whatever _SRC / _LIB name; the
    original library comes back when monkeypatch undoes these).  A variant
    that does not compile fails here, not inside a pin."""
    src = tmp_path / f"sp_oracle_{name}.c"
    src.write_text(text)
    monkeypatch.setattr(O, "_SRC", str(src))
    monkeypatch.setattr(O, "_LIB", str(tmp_path / f"_sp_oracle_{name}.so"))
    monkeypatch.setattr(O, "_lib", None)
    O._load()


def _call(pin):
    fn = getattr(P, pin)
    fn(**({"seed": 21} if "seed" in inspect.signature(fn).parameters else {}))


def test_pins_accept_an_equivalent_copy(source, tmp_path, monkeypatch):
    """Control: a copy that differs only in a comment is built and swapped in
    the same way, and the pins the mutants use all pass on it."""
    _load_variant(source.replace("/* g = 8 */", "/* g = 8 (copy) */"), "copy", tmp_path, monkeypatch)
    assert O._LIB.endswith("_sp_oracle_copy.so")
    for pin in sorted({p for m in MUTANTS for p in m[3]}):
        _call(pin)


@pytest.mark.parametrize("name,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_a_planted_mistake(name, old, new, pins, source, tmp_path, monkeypatch):
    assert source.count(old) == 1, f"the site of mutant {name} is not found exactly once"
    _load_variant(source.replace(old, new), name, tmp_path, monkeypatch)
    rejected = []
    for pin in pins:
        try:
            _call(pin)
        except Exception:  # an assertion, or any error the mistake causes downstream
            rejected.append(pin)
    assert rejected, f"no pin rejects the planted mistake {name}"
