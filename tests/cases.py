"""Shared parity cases: seeded inputs, oracle expectations and tolerances.

Every expected value comes from the FP64 oracle (oracle/); inputs come from
paper_2603_13196_gb300.inputs.  Nothing here calls the CUDA library.

Tolerances (derived from the arithmetic of each form):
  * logL, any point: |dlogL| <= 1e-2 + C u sum_{f,t} |r| (S + |r|) / sigma_n^2
    (logl_tolerance): each residual r is formed from terms of size S (the
    point's departure from the request reference, or the whole foreground for
    the plain form) with relative error ~u, and d(r^2 / 2 sigma^2) = r dr / sigma^2.
  * logL at near-posterior points (chi2 / (F T sigma^2) <= 10): |dlogL| <= 1e-2.
  * T_model per (p, f, t) at near-posterior points: |dT| <= 1e-3 K.
  * T_model per (p, f, t), any point: |dT| <= 1e-3 K + REL_T[prec] * scale, the
    scale being what the form's arithmetic carries (t_model_scale): the
    departure from the request reference plus |D - M| for the
    reference-subtracted forms, the whole foreground for the plain form.
"""
from __future__ import annotations

import functools
import math
import os

import numpy as np

import oracle as O
from paper_2603_13196_gb300 import inputs as I

# Unit roundoff of the operand representation of each form: split 16-bit
# (hi + mid) keeps 22 significand bits for FP16 (2 x 11) and 16 for BF16
# (2 x 8); the SIMT forms are FP32 (24 bits).
U = {"fp16x3": 2.0 ** -22, "bf16x3": 2.0 ** -16, "fp32_delta": 2.0 ** -24, "fp32_direct": 2.0 ** -24}
# Per-point logL tolerance (first order in the rounding of r):
#   |dlogL| <= 1e-2 + C u sum_{f,t} |r| (S + |r|) / sigma_n^2
# r = D - M (oracle), S the magnitude the form's arithmetic carries at each
# (f, t): the departure of the point from the request reference (sum_i |A_i|
# |w(beta_p,i) - w(bbar_i)|) for the reference-subtracted forms, the whole
# foreground for the plain form; dref is carried too (|dref| <= S + |r| +
# |T21|).  C = 16 covers the three split products (3u each operand pair) and
# the FP32 accumulation over K <= 100 terms with headroom.
C_TOL = 16.0
# T_model per (p,f,t), relative to the same magnitude (see t_model_scale).
REL_T = {k: C_TOL * v for k, v in U.items()}


@functools.lru_cache(maxsize=None)
def workload_case(k: int, P: int = None):
    """(wl, sky, obs, oracle model, data, params) of workload k (1..3)."""
    wl = I.workload(k)
    sky, obs = wl.sky(), wl.obs()
    m = O.build_model(sky, obs, wl.N, wl.scheme, wl.weighting)
    data = O.simulate_data(sky, obs, np.array(I.FIDUCIAL_T21), I.NOISE_K, wl.noise())
    params = wl.params(P)
    return wl, sky, obs, m, data, params


def small_case(npix=3072, N=5, F=31, T=7, window=4.0, seed=77, scheme="recursive", weighting="beam",
               lst0=3.0, achromatic_p=None):
    sky = I.make_sky(npix, seed)
    obs = I.make_obs(F, T, window, lst0, achromatic_p=achromatic_p)
    m = O.build_model(sky, obs, N, scheme, weighting)
    data = O.simulate_data(sky, obs, np.array(I.FIDUCIAL_T21), I.NOISE_K, I.noise_draws(F, T, seed))
    return sky, obs, m, data


def near_posterior(m, obs, dbeta: float, P: int, seed: int = 5, sigma=I.NOISE_K):
    """Data equal to the N-region model at a truth theta* plus 25 mK noise, and
    P points scattered uniformly by +-dbeta around theta* (sigma_n = 25 mK)."""
    N = m.A.shape[0]
    rng = I.rng(seed, I.SUB_PARAMS, 77)
    truth = np.concatenate([rng.uniform(2.5, 2.7, N), [0.155, 85.0, 15.0, sigma]])
    data = O.fast_model(m.A, m.B, obs, truth)[0] + sigma * I.noise_draws(obs.F, obs.T, seed, 3)
    pts = I.scatter_around(truth, P, dbeta, seed)
    return truth, data, pts


def expected(m, obs, data, params):
    """(logL, chi2/(2 sigma^2)) from the oracle."""
    L = O.loglike(m.A, m.B, data, obs, params)
    c2 = O.chi2(m.A, m.B, data, obs, params)
    sig = params[:, -1]
    return L, c2 / (2.0 * sig * sig)


def reference_beta(params, N):
    """The kernels' reference point: the midrange of beta_i over the request's
    valid points."""
    ok = np.all(np.isfinite(params), axis=1) & (params[:, N + 3] > 0) & (params[:, N + 2] != 0)
    if not ok.any():
        return np.zeros(N)
    v = params[ok, :N]
    return 0.5 * (v.min(axis=0) + v.max(axis=0))


def logl_tolerance(prec: str, m, obs, data, params) -> np.ndarray:
    """Per-point bound on |dlogL| for precision `prec` (see the module notes)."""
    N = m.A.shape[0]
    M = O.fast_model(m.A, m.B, obs, params)
    r = np.abs(data[None] - M)
    if prec == "fp32_direct":
        # the plain form rounds each of its N + 4 terms (A32, the FP32 power
        # law, the products, T_CMB B, the trough) at the size of the foreground
        S, C = np.abs(M), 4.0 * (N + 4)
    else:
        S, C = foreground_departure(m, obs, params, reference_beta(params, N)), C_TOL
    return 1e-2 + C * U[prec] * np.sum(r * (S + r), axis=(1, 2)) / params[:, N + 3] ** 2


def foreground_departure(m, obs, params, beta_ref):
    """S_abs[p,f,t] = sum_i |A_i| |w(beta_p,i) - w(beta_ref,i)| (K)."""
    N = m.A.shape[0]
    L = np.log(obs.nu / obs.nu0)
    w = np.exp(-params[:, :N, None] * L[None, None, :])          # [P,N,F]
    w0 = np.exp(-beta_ref[:, None] * L[None, :])                  # [N,F]
    d = np.abs(w - w0[None])
    return np.einsum("pif,ift->pft", d, np.abs(m.A))


def t_model_scale(prec, m, obs, data, params):
    """Magnitude carried by each form's arithmetic for T_model[p,f,t]: the
    departure from the request reference plus the residual |D - M| for the
    reference-subtracted forms; the foreground sum for the plain form."""
    if prec == "fp32_direct":
        return foreground_magnitude(m, obs, params)
    bbar = reference_beta(params, m.A.shape[0])
    r = np.abs(data[None] - O.fast_model(m.A, m.B, obs, params))
    return foreground_departure(m, obs, params, bbar) + r


def foreground_magnitude(m, obs, params):
    N = m.A.shape[0]
    L = np.log(obs.nu / obs.nu0)
    w = np.exp(-params[:, :N, None] * L[None, None, :])
    return np.einsum("pif,ift->pft", w, np.abs(m.A))


# Regression ceilings.  The derived bound above is the contract; each family of
# parity checks also keeps its worst err/tol below a ceiling of 4x the figure
# measured on a GB300 (kept beside it), so that an accuracy regression well
# inside the derived bound still fails.  FG21_CEILING_COLLECT=1 reports the
# ratios without applying the ceilings (to re-measure after a deliberate
# change of the arithmetic).
CEILING_FACTOR = 4.0
# worst err / tol of each family over its GPU tests (one GB300 run of the whole
# -m gpu suite with FG21_CEILING_COLLECT=1); 0 means the comparison was exact
MEASURED_ERR_OVER_TOL = {
    'T_model_near_bf16x3_1e-05': 1.734e-03,
    'T_model_near_bf16x3_1e-06': 1.895e-03,
    'T_model_near_fp16x3_1e-05': 4.270e-05,
    'T_model_near_fp16x3_1e-06': 4.810e-05,
    'T_model_near_fp32_delta_1e-05': 2.792e-05,
    'T_model_near_fp32_delta_1e-06': 1.752e-05,
    'T_model_prior_bf16x3': 3.500e-02,
    'T_model_prior_fp16x3': 5.606e-02,
    'T_model_prior_fp32_delta': 1.024e-01,
    'T_model_prior_fp32_direct': 4.321e-01,
    'ab_invalid_fp16x3': 1.380e-02,
    'ab_invalid_fp32_delta': 6.032e-02,
    'ab_invalid_fp32_direct': 6.738e-02,
    'ab_multi_fp16x3': 1.748e-02,
    'ab_near_abs_fp16x3_0.0001_0.001': 1.764e-01,
    'ab_near_abs_fp16x3_1e-05_0.0001': 3.310e-01,
    'ab_near_abs_fp16x3_1e-06_1e-06': 7.095e-03,
    'ab_near_abs_fp32_delta_0.0001_0.001': 6.025e-01,
    'ab_near_abs_fp32_delta_1e-05_0.0001': 3.744e-01,
    'ab_near_abs_fp32_delta_1e-06_1e-06': 2.094e-03,
    'ab_near_bf16x3_0.0001_0.001': 1.404e-03,
    'ab_near_bf16x3_1e-05_0.0001': 1.450e-03,
    'ab_near_bf16x3_1e-06_1e-06': 1.341e-03,
    'ab_near_fp16x3_0.0001_0.001': 2.154e-02,
    'ab_near_fp16x3_1e-05_0.0001': 1.507e-02,
    'ab_near_fp16x3_1e-06_1e-06': 4.036e-03,
    'ab_near_fp32_delta_0.0001_0.001': 9.020e-02,
    'ab_near_fp32_delta_1e-05_0.0001': 5.313e-02,
    'ab_near_fp32_delta_1e-06_1e-06': 1.700e-03,
    'ab_prior_bf16x3': 8.620e-03,
    'ab_prior_fp16x3': 4.736e-02,
    'ab_prior_fp32_delta': 9.645e-02,
    'ab_prior_fp32_direct': 1.538e-01,
    'ab_serve_noalloc_vs_direct': 0.000e+00,
    'after_timeout_fp16x3': 1.434e-02,
    'autotune_fp16x3': 1.282e-02,
    'graph_fp16x3': 9.261e-03,
    'graph_fp32_delta': 3.277e-02,
    'graph_multi_fp16x3': 1.822e-02,
    'host_call_fp16x3': 9.646e-03,
    'host_call_fp32_delta': 3.236e-02,
    'invalid_fp16x3': 1.039e-02,
    'invalid_fp32_delta': 3.236e-02,
    'invalid_fp32_direct': 1.450e-01,
    'limits_fp32_delta': 5.041e-02,
    'max_shape_bf16x3': 2.067e-03,
    'max_shape_fp16x3': 3.456e-02,
    'max_shape_fp32_delta': 5.763e-02,
    'max_shape_fp32_direct': 9.241e-03,
    'multi_fp16x3': 1.876e-02,
    'multi_fp32_delta': 2.970e-02,
    'multi_fp32_direct': 1.234e-02,
    'near_abs_fp16x3_0.0001': 2.489e-01,
    'near_abs_fp16x3_1e-05': 4.268e-02,
    'near_abs_fp16x3_1e-06': 1.052e-02,
    'near_abs_fp32_delta_0.0001': 6.929e-01,
    'near_abs_fp32_delta_1e-05': 5.839e-02,
    'near_abs_fp32_delta_1e-06': 4.844e-03,
    'near_bf16x3_0.0001': 3.213e-03,
    'near_bf16x3_1e-05': 2.011e-03,
    'near_bf16x3_1e-06': 9.085e-04,
    'near_fp16x3_0.0001': 4.325e-03,
    'near_fp16x3_1e-05': 3.881e-03,
    'near_fp16x3_1e-06': 4.448e-03,
    'near_fp32_delta_0.0001': 3.151e-02,
    'near_fp32_delta_1e-05': 1.571e-02,
    'near_fp32_delta_1e-06': 3.687e-03,
    'noalloc_fp16x3': 9.475e-03,
    'noise_1_500': 3.383e-01,
    'noise_2_500': 5.206e-02,
    'noise_30100_128': 2.880e-03,
    'noise_4097_64': 5.209e-04,
    'noise_51_2000': 3.886e-02,
    'noise_through_likelihood_fp16x3': 6.235e-04,
    'noise_through_likelihood_fp32_delta': 1.938e-04,
    'series_ab_degree3': 5.062e-02,
    'series_ab_degree5': 3.691e-02,
    'series_ab_degree8': 1.663e-02,
    'series_ab_squarings': 1.348e-02,
    'series_degree3_bf16x3': 1.131e-03,
    'series_degree3_fp16x3': 4.149e-02,
    'series_degree5_bf16x3': 1.429e-03,
    'series_degree5_fp16x3': 3.567e-02,
    'series_degree8_bf16x3': 1.669e-03,
    'series_degree8_fp16x3': 1.836e-02,
    'series_squarings_bf16x3': 2.396e-03,
    'series_squarings_fp16x3': 1.174e-02,
    'serve_mixed_fp16x3': 2.098e-02,
    'simt_chunks_fp32_delta': 7.330e-02,
    'simt_chunks_fp32_direct': 1.579e-01,
    'simt_remainder_fp32_delta': 7.865e-02,
    'simt_remainder_fp32_direct': 1.042e-01,
    'simt_small_fp32_delta': 3.475e-02,
    'simt_small_fp32_direct': 8.179e-02,
    'simt_w1_fp32_delta': 4.148e-02,
    'simt_w1_fp32_direct': 5.938e-02,
    'tc_prior_bf16x3': 8.163e-03,
    'tc_prior_fp16x3': 2.573e-02,
    'w1_bf16x3': 2.449e-03,
    'w1_fp16x3': 6.776e-03,
    'w1_fp32_delta': 4.148e-02,
    'w1_fp32_direct': 5.938e-02,
    'w2_fp16x3': 1.165e-02,
    'w2_fp32_direct': 3.936e-02,
    'w3_graph_fp16x3': 1.466e-02,
    'w3_near_0.0001': 3.439e-03,
    'w3_near_1e-05': 7.813e-03,
    'w3_near_1e-06': 6.956e-03,
    'w3_near_abs_1e-05': 3.493e-01,
    'w3_near_abs_1e-06': 9.393e-02,
    'w4_full_multi': 1.652e-02,
    'w5_served_mix': 1.541e-02,
}


def check_logl(family, got, want, tol, label=""):
    """Assert |got - want| <= tol element-wise and max(err / tol) under the
    family's regression ceiling; returns max(err / tol)."""
    from conftest import report
    got, want = np.asarray(got, dtype=np.float64), np.asarray(want, dtype=np.float64)
    err = np.abs(got - want)
    tol = np.broadcast_to(np.asarray(tol, dtype=np.float64), err.shape)
    ratio = float(np.max(err / tol)) if err.size else 0.0
    report("ceiling:" + family, max_err_over_tol=ratio, label=label, max_abs=float(err.max()) if err.size else 0.0)
    assert np.all(err <= tol), fmt_err(f"{family} {label}", got, want, tol)
    if os.environ.get("FG21_CEILING_COLLECT"):
        return ratio
    assert family in MEASURED_ERR_OVER_TOL, f"no regression ceiling recorded for {family}"
    measured = MEASURED_ERR_OVER_TOL[family]
    ceil = CEILING_FACTOR * measured
    assert ratio <= ceil, (f"{family} {label}: worst err/tol {ratio:.3e} above the regression ceiling {ceil:.3e} "
                           f"({CEILING_FACTOR:g} x the {measured:.3e} measured)")
    return ratio


def fmt_err(name, got, want, tol):
    err = np.abs(got - want)
    k = int(np.argmax(err / tol))
    return f"{name}: max|err|={err.max():.3e} worst err/tol={float((err / tol)[k]):.3f} at {k}"


def sigma_floor():
    return math.log(2 * math.pi * I.NOISE_K ** 2)


# ------------------------------------------------ amplitude / spectral-index
# Models with amplitude regions (oracle.OracleModelAB): K[Na, Nb, F, T],
# params [P, Nb+Na+4].  The kernels' reference point is the midrange of every
# foreground parameter (beta_j and alpha_i) over the request's valid points.

def small_case_ab(npix=2048, Nb=4, Na=3, F=21, T=5, window=4.0, seed=91, scheme="recursive",
                  scheme_a="hierarchical"):
    sky = I.make_sky(npix, seed)
    obs = I.make_obs(F, T, window, 3.0)
    m = O.build_model_ab(sky, obs, Nb, scheme, "beam", Na, I.amplitude_field(sky), scheme_a, "beam")
    data = O.simulate_data(sky, obs, np.array(I.FIDUCIAL_T21), I.NOISE_K, I.noise_draws(F, T, seed))
    return sky, obs, m, data


def expected_ab(m, obs, data, params):
    L = O.loglike_ab(m.K, m.B, data, obs, params)
    c2 = O.chi2_ab(m.K, m.B, data, obs, params)
    sig = params[:, -1]
    return L, c2 / (2.0 * sig * sig)


def valid_ab(params, Nb, Na):
    NP = Nb + Na
    return (np.all(np.isfinite(params), axis=1) & (params[:, NP + 3] > 0) & (params[:, NP + 2] != 0)
            & np.all(params[:, Nb:NP] > 0, axis=1))


def logl_tolerance_ab(prec: str, m, obs, data, params) -> np.ndarray:
    """logl_tolerance for the joint model: S = sum_ij |K_ij| |alpha_i w_j(beta_p)
    - abar_i w_j(bbar)| for the reference-subtracted forms (the departure from
    the reference point), the whole foreground for the plain form."""
    Na, Nb = m.K.shape[:2]
    NP = Nb + Na
    M = O.fast_model_ab(m.K, m.B, obs, params)
    r = np.abs(data[None] - M)
    L = np.log(obs.nu / obs.nu0)
    w = params[:, Nb:NP, None, None] * np.exp(-params[:, None, :Nb, None] * L)      # [P,Na,Nb,F]
    if prec == "fp32_direct":
        S = np.einsum("pijf,ijft->pft", np.abs(w), np.abs(m.K))
        C = 4.0 * (Na * Nb + 4)
    else:
        ok = valid_ab(params, Nb, Na)
        v = params[ok, :NP]
        ref = 0.5 * (v.min(axis=0) + v.max(axis=0))
        w0 = ref[Nb:NP, None, None] * np.exp(-ref[None, :Nb, None] * L)           # [Na,Nb,F]
        S = np.einsum("pijf,ijft->pft", np.abs(w - w0[None]), np.abs(m.K))
        C = C_TOL
    return 1e-2 + C * U[prec] * np.sum(r * (S + r), axis=(1, 2)) / params[:, NP + 3] ** 2


def near_posterior_ab(m, obs, dbeta: float, dalpha: float, P: int, seed: int = 6, sigma=I.NOISE_K):
    """Data = the joint model at a truth (beta in [2.5, 2.7], alpha in
    [0.95, 1.05]) plus 25 mK noise; P points moved by U(+-dbeta) in beta and
    by relative U(+-dalpha) in alpha."""
    Na, Nb = m.K.shape[:2]
    rng = I.rng(seed, I.SUB_PARAMS, 78)
    truth = np.concatenate([rng.uniform(2.5, 2.7, Nb), rng.uniform(0.95, 1.05, Na), [0.155, 85.0, 15.0, sigma]])
    data = O.fast_model_ab(m.K, m.B, obs, truth)[0] + sigma * I.noise_draws(obs.F, obs.T, seed, 4)
    g = I.rng(seed, I.SUB_PARAMS, 79)
    pts = np.repeat(truth[None], P, axis=0)
    pts[:, :Nb] += g.uniform(-dbeta, dbeta, size=(P, Nb))
    pts[:, Nb:Nb + Na] *= 1.0 + g.uniform(-dalpha, dalpha, size=(P, Na))
    return truth, data, pts


# ------------------------------------------------ nested sampling, serving size
# A run of the serving workload's size (N = 9 regions, F = 151, T = 10 LST bins
# over 6 h, 3072-pixel sky, n_live = 500, 128 deletions per iteration, 5 D inner
# slice steps): data from the 9-region model at the regions' mean spectral
# indices plus 25 mK noise.  The prior on beta is [2.35, 2.75]: the sky's two
# lowest regions have mean indices of 2.418 and 2.438, below the workloads'
# prior bound of 2.45, where no sampler could reach the likelihood's peak.
NS_SERVING = dict(npix=3072, sky_seed=41, N=9, F=151, T=10, window_h=6.0, lst0_h=5.0, noise_seed=41,
                  n_live=500, num_delete=128, beta_prior=(2.35, 2.75))


def ns_serving_problem():
    """(sky, obs, oracle model, data, truth, prior) of the serving-size run."""
    from paper_2603_13196_gb300 import ns
    c = NS_SERVING
    sky = I.make_sky(c["npix"], c["sky_seed"])
    obs = I.make_obs(c["F"], c["T"], c["window_h"], lst0_h=c["lst0_h"])
    m = O.build_model(sky, obs, c["N"], "recursive")
    truth = np.concatenate([O.region_truth(sky, m.labels, c["N"], m.w), [0.155, 85.0, 15.0, I.NOISE_K]])
    data = O.fast_model(m.A, m.B, obs, truth)[0] + I.NOISE_K * I.noise_draws(obs.F, obs.T, c["noise_seed"])
    prior = ns.region_model_prior(c["N"], beta=c["beta_prior"])
    return sky, obs, m, data, truth, prior
