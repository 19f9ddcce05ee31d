"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in a temporary copy of the oracle's C source
(a dropped term, a flipped sign, a wrong rounding, a shifted index, a swapped
operand), builds it, and runs the pin suite against it: at least one pin must
fail.  The committed oracle is never modified.
"""
import os
import subprocess

import pytest

import oracle
import test_oracle_comb_pins as comb_pins
import test_oracle_mean_pins as mean_pins
import test_oracle_bs_pins as bs_pins
import test_oracle_refine_pins as refine_pins
import test_oracle_pe_pins as pe_pins
import test_oracle_pins as pins
import test_oracle_residual_pins as residual_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "sfft_oracle.c")

# (name, original text, mutated text)
MUTANTS = [
    ("phase sign", "unit_root(-(tau[l] * f), N)", "unit_root((tau[l] * f), N)"),
    ("gain dropped", "unit_root(-(tau[l] * f), N) / G;", "unit_root(-(tau[l] * f), N);"),
    ("hash floors", "int64_t hh = (p + half) / NB;", "int64_t hh = p / NB;"),
    ("dft sign", "double a = -2.0 * M_PI * (double)t / (double)B;",
     "double a = 2.0 * M_PI * (double)t / (double)B;"),
    ("sinc centre", "(m == 0) ? 1.0 / (double)B", "(m == 0) ? 1.0"),
    ("gaussian width", "(double)B * sqrt(log2((double)N))", "(double)B * log2((double)N)"),
    ("fold index", "int64_t j = mod_pos(m, B);", "int64_t j = mod_pos(q, B);"),
    ("gather shift sign", "mod_pos(sigma[l] * m + tau[l], N);\n            int64_t j",
     "mod_pos(sigma[l] * m - tau[l], N);\n            int64_t j"),
    ("vote without inverse", "int64_t f = mod_pos(sigma_inv[l] * p, N);", "int64_t f = p;"),
    ("even median", "return 0.5 * (v[n / 2 - 1] + v[n / 2]);", "return v[n / 2];"),
    ("tie order", "return (x->id > y->id) - (x->id < y->id);", "return (x->id < y->id) - (x->id > y->id);"),
    ("philox multiplier", "M1 = 0xCA5A826395121157ULL", "M1 = 0xCA5A826395121159ULL"),
    ("sigma parity", "int64_t s = 2 * (int64_t)(out[0] % (uint64_t)(N / 2)) + 1;",
     "int64_t s = (int64_t)(out[0] % (uint64_t)N) | 1;"),
    ("threshold off by one", "if (sc[f] >= T) cand[n++]", "if (sc[f] > T) cand[n++]"),
    # phase-encoding, iterative variant
    ("pe phase sign", "double phi = atan2(cimag(r), creal(r));", "double phi = -atan2(cimag(r), creal(r));"),
    ("pe backward shift", "t1 = mod_pos(tau[r] + 1, N);", "t1 = mod_pos(tau[r] - 1, N);"),
    ("pe subtraction turn", "unit_root(tau * f, N); /* x^_f", "unit_root(-tau * f, N); /* x^_f"),
    ("pe gain offset reversed", "int64_t nu = mod_pos(p - k * NB, N);", "int64_t nu = mod_pos(k * NB - p, N);"),
    ("pe no hash check", "if (h != k) continue; /* not a lone", "if (0) continue; /* not a lone"),
    ("pe estimate without gain", "unit_root(-tau * f, N) / G;", "unit_root(-tau * f, N);"),
    # spike-train pre-filter
    ("comb dft sign", "double a = -2.0 * M_PI * (double)((i * j) % Bc) / (double)Bc;",
     "double a = 2.0 * M_PI * (double)((i * j) % Bc) / (double)Bc;"),
    ("comb stride", "int64_t n = mod_pos(tau_c[c] + j * stride, N);", "int64_t n = mod_pos(tau_c[c] + j, N);"),
    ("comb filter off", "if (kept[mod_pos(cand[q], Bc)]) cand[ncand++] = cand[q];", "cand[ncand++] = cand[q];"),
    ("comb shifts from the voting loops", "tau + L, (int64_t)c * K", "tau, (int64_t)c * K"),
    # averaging estimator
    ("mean without 1/L", "est[2 * c] = sr / (double)L;", "est[2 * c] = sr;"),
    ("mean replaced by the median", "if (combine == ORACLE_MEAN) {", "if (0) {"),
    ("mean skips loop 0", "for (int l = 0; l < L; ++l) {\n                sr += re[l];",
     "for (int l = 1; l < L; ++l) {\n                sr += re[l];"),
    # iterative-framework refinement
    ("refine subtracts itself", "if (d == c) continue;", "if (0) continue;"),
    ("refine turn sign", "r -= v * unit_root(tau[l] * gq, N) * G;", "r -= v * unit_root(-(tau[l] * gq), N) * G;"),
    # (G~ is even up to the window's one unpaired edge tap, so a reversed offset
    # is nearly an equivalent mutant; the gain at the wrong coefficient's offset is not)
    ("refine gain at f's offset", "int64_t nu = mod_pos(sigma[l] * gq - h * NB, N);",
     "int64_t nu = mod_pos(o, N);"),
    ("refine uses the new values", "for (int64_t q = 0; q < 2 * n; ++q) cur[q] = val[q];",
     "for (int64_t q = 0; q < 0; ++q) cur[q] = val[q];"),
    # location by binary or multi-scale search
    ("bs digit sign", "double v = creal(rho_j * unit_root(-cand * (N >> m), N));",
     "double v = creal(rho_j * unit_root(cand * (N >> m), N));"),
    ("bs shift one scale coarser", "s[j + 1] = N >> m;", "s[j + 1] = N >> (m - 1);"),
    ("bs residue without sigma", "int64_t pr = mod_pos(sigma * r, W);", "int64_t pr = mod_pos(r, W);"),
    ("bs no hash-back", "if (h != k) continue; /* located in a neighbouring bucket: leakage */",
     "if (0) continue; /* located in a neighbouring bucket: leakage */"),
    ("bs no lone-coefficient test", "if (res > rho * (double)J * e0) continue;", "if (0) continue;"),
    ("bs window not centred", "int64_t lo_p = k * NB - W / 2;", "int64_t lo_p = k * NB;"),
    ("bs threshold without the noise floor", "if (kappa * emed > thr) thr = kappa * emed;", "(void)emed;"),
    # final residual-energy check
    ("residual without subtraction", "oracle_pe_subtract(N, B, sigma[l], tau[l], Gfull, n, idx, val, r);",
     "(void)val;"),
    ("residual of loop 0 only", "for (int l = 0; l < L; ++l) {\n        for (int64_t k = 0; k < 2 * B; ++k) r[k]",
     "for (int l = 0; l < 1; ++l) {\n        for (int64_t k = 0; k < 2 * B; ++k) r[k]"),
    ("residual energy without the imaginary part",
     "for (int64_t k = 0; k < B; ++k) er += r[2 * k] * r[2 * k] + r[2 * k + 1] * r[2 * k + 1];",
     "for (int64_t k = 0; k < B; ++k) er += r[2 * k] * r[2 * k];"),
]

PIN_CHECKS = [
    pins.test_philox_known_answer,
    lambda: pins.test_loop_params_stream_and_inverse(1 << 16),
    pins.test_flat_bucket_worked_example,
    pins.test_scaling_worked_example,
    pins.test_gaussian_width_example,
    lambda: pins.test_window_taps_shape(1 << 12, 16),
    lambda: pins.test_filter_gain_against_fft(1 << 12, 16),
    pins.test_hash_rounding_brute_force,
    lambda: pins.test_bucketize_closed_form(1 << 10, 16, 3),
    pins.test_select_brute_force_with_ties,
    lambda: pins.test_vote_brute_force(1 << 10, 16, 6, 5, 3),
    lambda: pins.test_estimate_exact_for_one_sparse(1 << 12, 16, 5),
    pins.test_median_combination,
    pins.test_topk_brute_force,
    pins.test_exact_recovery_noiseless,
    lambda: pe_pins.test_gain_full_against_numpy_fft(1 << 12, 16),
    lambda: pe_pins.test_unit_shift_turns_lone_coefficient(1 << 12, 32, 777),
    lambda: pe_pins.test_subtraction_removes_known_coefficients(1 << 12, 32, 6),
    pe_pins.test_locate_finds_lone_coefficients,
    lambda: pe_pins.test_exact_recovery_noiseless(1 << 12, 5, 32, range(6)),
    pe_pins.test_one_sparse_is_exact_and_stops,
    pe_pins.test_iterations_resolve_a_collision,
    lambda: comb_pins.test_comb_energy_closed_form(1 << 12, 64, 7),
    comb_pins.test_comb_keeps_largest_classes_with_ties,
    lambda: comb_pins.test_filtered_candidates_are_voting_candidates_in_kept_classes(0),
    lambda: comb_pins.test_exact_recovery_noiseless(1 << 16, 10, 64, 8, 256),
    lambda: mean_pins.test_mean_exact_on_one_sparse(1 << 12, 16, 5, 1234),
    mean_pins.test_mean_is_linear_and_median_is_not,
    mean_pins.test_two_coefficients_closed_form,
    lambda: refine_pins.test_one_pass_from_true_values_is_exact(oracle.MEDIAN),
    refine_pins.test_passes_remove_the_mean_bias,
    refine_pins.test_lone_coefficient_unchanged,
    lambda: bs_pins.test_shift_schedule(1 << 16, 64, 1, [0] + [(1 << 16) >> m for m in range(1, 12)]),
    lambda: bs_pins.test_lone_coefficient_located_exactly(1 << 12, 16, 1),
    bs_pins.test_matches_exhaustive_search_under_noise,
    bs_pins.test_shared_bucket_rejected,
    lambda: bs_pins.test_exact_recovery_noiseless(1 << 12, 5, 32, 1),
    bs_pins.test_pure_noise_stops_after_one_iteration,
    residual_pins.test_exact_recovery_leaves_nothing,
    lambda: residual_pins.test_planted_miss_closed_form(3),
    residual_pins.test_flipped_value_leaves_four_times_the_tone,
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name!r} not unique"
    mut = tmp_path / "sfft_oracle.c"
    mut.write_text(src.replace(old, new))
    hdr = os.path.join(os.path.dirname(SRC), "sfft_oracle.h")
    (tmp_path / "sfft_oracle.h").write_text(open(hdr).read())
    so = tmp_path / "liboracle_mutant.so"
    subprocess.check_call(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-o", str(so), str(mut), "-lm"])
    failed = []
    with oracle.use_library(str(so)):
        for check in PIN_CHECKS:
            try:
                check()
            except (AssertionError, ValueError, IndexError):
                failed.append(getattr(check, "__name__", "lambda"))
    assert failed, f"no pin caught the planted mistake {name!r}"
