"""Plant plausible mistakes in a copy of the oracle and check that the pins
of tests/test_oracle_pins.py catch every one (the oracle is only trusted if
its pins would notice a dropped term, a wrong sign or index, or a transposed
operand).  Each mutant is compiled from a patched copy of fg21_oracle.c in a
temporary directory; the real oracle is never modified."""
import os
import subprocess

import pytest

import oracle as O
from oracle import build as OB
import test_oracle_pins as pins

MUTANTS = {
    "beta_sign_fast": ("fg += A[((size_t)i * F + f) * T + t] * pow(nu[f] / nu0, -th[i]);",
                       "fg += A[((size_t)i * F + f) * T + t] * pow(nu[f] / nu0, th[i]);"),
    "drop_tcmb_in_sky": ("return (t230 - t_cmb) * pow(nu / nu0, -beta) + t_cmb;",
                         "return (t230 - t_cmb) * pow(nu / nu0, -beta);"),
    "drop_tcmb_B_term": ("M[((size_t)p * F + f) * T + t] = fg + t_cmb * B[(size_t)f * T + t] + s21;",
                         "M[((size_t)p * F + f) * T + t] = fg + s21;"),
    "beam_norm_factor": ("return 2.0 * (p + 1.0) * pow(c, p);", "return (p + 1.0) * pow(c, p);"),
    "beam_horizon": ("if (c <= 0.0) return 0.0;", "if (c <= -0.2) return 0.0; if (c < 0) c = -c;"),
    "A_transposed": ("fg += A[((size_t)i * F + f) * T + t] * pow(nu[f] / nu0, -th[i]);",
                     "fg += A[((size_t)i * T + t) * F + f] * pow(nu[f] / nu0, -th[i]);"),
    "drop_normalisation": ("sum += log(2.0 * 3.14159265358979323846 * sig * sig) + r * r / (sig * sig);",
                           "sum += r * r / (sig * sig);"),
    "sigma_not_squared": ("sum += log(2.0 * 3.14159265358979323846 * sig * sig) + r * r / (sig * sig);",
                          "sum += log(2.0 * 3.14159265358979323846 * sig * sig) + r * r / sig;"),
    "t21_width": ("return a21 * exp(-(d * d) / (2.0 * s21 * s21));", "return a21 * exp(-(d * d) / (s21 * s21));"),
    "recursive_split_point": ("double a = R[best].a, b = R[best].b, mid = 0.5 * (a + b);",
                              "double a = R[best].a, b = R[best].b, mid = (a + 2.0 * b) / 3.0;"),
    "recursive_min_mass": ("if (m[r] > m[best] || (m[r] == m[best] && R[r].a < R[best].a)) best = r;",
                           "if (m[r] < m[best] || (m[r] == m[best] && R[r].a < R[best].a)) best = r;"),
    "cinv_strict": ("if (cum[k] >= c) {", "if (cum[k] > c) {"),
    "hier_narrowest": ("if (wr > wb || (wr == wb && R[r].a < R[best].a)) best = r;",
                       "if (wr < wb || (wr == wb && R[r].a < R[best].a)) best = r;"),
    "weights_unnormalised": ("acc += d > 0.0 ? num / d : 0.0;", "acc += num;"),
    "weights_average_F_only": ("w_out[q] = acc / ((double)F * (double)T);", "w_out[q] = acc / (double)F;"),
    "label_boundary": ("if (beta[q] > edges[j]) lab = j;", "if (beta[q] >= edges[j]) lab = j;"),
    "precompute_npix": ("for (int i = 0; i < N; ++i) A[((size_t)i * F + f) * T + t] = acc[i] / (double)npix;",
                        "for (int i = 0; i < N; ++i) A[((size_t)i * F + f) * T + t] = acc[i] / (double)(npix - 1);"),
    "pixel_model_one_region": ("double tm = (t230[q] - t_cmb) * pow(nu[f] / nu0, -th[labels[q]]) + t_cmb;",
                               "double tm = (t230[q] - t_cmb) * pow(nu[f] / nu0, -th[0]) + t_cmb;"),
    "noise_unscaled": ("if (noise) v += sigma_noise * noise[ft];", "if (noise) v += noise[ft];"),
    "sky_weight_no_horizon": ("num = c > 0.0 ? orc_tsky(t230[q], beta[q], nu[f], nu0, t_cmb) : 0.0;",
                              "num = orc_tsky(t230[q], beta[q], nu[f], nu0, t_cmb);"),
    "ab_alpha_dropped": ("fg += th[Nb + i] * K[(((size_t)i * Nb + j) * F + f) * T + t] * pow(nu[f] / nu0, -th[j]);",
                         "fg += K[(((size_t)i * Nb + j) * F + f) * T + t] * pow(nu[f] / nu0, -th[j]);"),
    "ab_alpha_beta_swapped": ("fg += th[Nb + i] * K[(((size_t)i * Nb + j) * F + f) * T + t] * pow(nu[f] / nu0, -th[j]);",
                              "fg += th[Nb + j % Na] * K[(((size_t)i * Nb + j) * F + f) * T + t] * pow(nu[f] / nu0, -th[i % Nb]);"),
    "ab_K_transposed": ("fg += th[Nb + i] * K[(((size_t)i * Nb + j) * F + f) * T + t] * pow(nu[f] / nu0, -th[j]);",
                        "fg += th[Nb + i] * K[(((size_t)j * Na + i) * F + f) * T + t] * pow(nu[f] / nu0, -th[j]);"),
    "ab_alpha_mask_ignored": ("double ma = lab_a[q] == i ? 1.0 : 0.0;", "double ma = 1.0;"),
    "ab_pixel_alpha_label": ("double tm = th[Nb + lab_a[q]] * (t230[q] - t_cmb) * pow(nu[f] / nu0, -th[lab_b[q]]) + t_cmb;",
                             "double tm = th[Nb + lab_b[q] % Na] * (t230[q] - t_cmb) * pow(nu[f] / nu0, -th[lab_b[q]]) + t_cmb;"),
    "ab_sigma_index": ("double sig = th[NP + 3];\n        double sum = 0.0;\n        for (int f = 0; f < F; ++f) {\n            double s21 = orc_t21(nu[f], th[NP], th[NP + 1], th[NP + 2]);\n            for (int t = 0; t < T; ++t) {\n                double m = orc_fg_ab",
                       "double sig = th[NP + 2];\n        double sum = 0.0;\n        for (int f = 0; f < F; ++f) {\n            double s21 = orc_t21(nu[f], th[NP], th[NP + 1], th[NP + 2]);\n            for (int t = 0; t < T; ++t) {\n                double m = orc_fg_ab"),
    "ab_trough_params": ("M[((size_t)p * F + f) * T + t] =\n                    orc_fg_ab(Na, Nb, F, T, K, nu, nu0, th, f, t) + t_cmb * B[(size_t)f * T + t] + s21;",
                         "M[((size_t)p * F + f) * T + t] =\n                    orc_fg_ab(Na, Nb, F, T, K, nu, nu0, th, f, t) + t_cmb * B[(size_t)f * T + t];"),
    "noise_sigma_not_squared": ("sum += lnorm + res * res / (sigma_n * sigma_n);", "sum += lnorm + res * res / sigma_n;"),
    "boxmuller_radius": ("double r = sqrt(-2.0 * log(u1));", "double r = sqrt(-log(u1));"),
    "boxmuller_same_angle": ("if (2 * j + 1 < n_cells) z[2 * j + 1] = r * sin(two_pi * u2);",
                             "if (2 * j + 1 < n_cells) z[2 * j + 1] = r * cos(two_pi * u2);"),
    "philox_key_dropped": ("uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;", "uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1;"),
    "philox_two_rounds": ("for (int r = 0; r < 10; ++r) {", "for (int r = 0; r < 2; ++r) {"),
    "philox_low_half": ("uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;", "uint32_t n2 = (uint32_t)p0 ^ c3 ^ k1;"),
    "noise_q_strict": ("c += L_noise[k] <= L_bar[i];", "c += L_noise[k] < L_bar[i];"),
}

PINS = [
    pins.test_t21_special_values,
    lambda: pins.test_beam_is_a_directivity(1.2),
    pins.test_flat_beam_counts_pixels_above_horizon,
    lambda: pins.test_fast_model_equals_pixel_model("recursive", 5),
    pins.test_single_region_is_a_power_law,
    lambda: pins.test_equal_beta_collapse("hierarchical", 5),
    pins.test_constant_beta_sky_reproduces_simulated_data,
    pins.test_simulated_data_closed_form,
    pins.test_noiseless_identity,
    pins.test_loglike_is_a_sum_of_gaussian_logpdfs,
    pins.test_weights_special_cases,
    pins.test_beam_weighting_tracks_the_beam,
    lambda: [pins.test_partition_matches_brute_force(s, k) for s in ("recursive", "hierarchical")
             for k in range(6)],
    lambda: pins.test_partitions_are_nested("hierarchical", "beam"),
    lambda: pins.test_hierarchical_base_regions_have_equal_mass(4),
    pins.test_recursive_edges_are_dyadic_midpoints,
    lambda: pins.test_embedding_identity("recursive"),
    lambda: pins.test_ab_fast_model_equals_pixel_model("recursive", "hierarchical", 4, 3),
    pins.test_ab_unit_amplitudes_reduce_to_beta_model,
    pins.test_ab_scaled_template_reproduces_simulated_data,
    pins.test_ab_flat_beam_closed_form,
    pins.test_ab_noiseless_identity_and_gaussian_logpdf,
    lambda: pins.test_ab_amplitude_embedding_identity("hierarchical"),
    pins.test_noise_loglike_is_a_scaled_chi_square,
    pins.test_noise_draws_are_standard_normal_and_independent,
    pins.test_philox_mixing,
    lambda: pins.test_philox_matches_library_engine(__import__("pathlib").Path(__import__("tempfile").mkdtemp())),
    pins.test_noise_q_special_values,
]


def _caught(pin):
    try:
        pin()
    except Exception:       # assertion or numerical blow-up: the pin noticed
        return True
    return False


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(OB.SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = src.replace(old, new)
    c_path = os.path.join(tmp_path, "mut.c")
    so_path = os.path.join(tmp_path, "libmut.so")
    open(c_path, "w").write(mutated)
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                           "-o", so_path, c_path, "-lm"])
    prev = O.use_library(so_path)
    try:
        caught = [i for i, pin in enumerate(PINS) if _caught(pin)]
    finally:
        O.restore_library(prev)
    assert caught, f"no pin caught mutant {name}"


def test_unmutated_oracle_passes_every_pin():
    assert not [i for i, pin in enumerate(PINS) if _caught(pin)]
