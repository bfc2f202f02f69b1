"""GPU parity of the tensor-core (tcgen05) path against the FP64 oracle,
through the C ABI: prior draws at several shapes (ragged tiles, t-chunks,
K = 16 / 32 / 64), near-posterior sets with the absolute 1e-2 nats bound,
per-channel model temperatures, invalid points, BF16 operands."""
import numpy as np
import pytest

import cases
import oracle as O
from conftest import report

pytestmark = pytest.mark.gpu

SHAPES = [
    # (npix, N, F, T, P)
    (1024, 3, 9, 1, 1),        # one point, one LST bin, K = 16
    (2048, 5, 31, 7, 129),     # ragged tile tail
    (2048, 14, 17, 20, 300),   # K = 16 exactly
    (2048, 30, 11, 40, 257),   # K = 32
    (3072, 40, 9, 9, 140),     # K = 64
    (1024, 4, 5, 300, 130),    # two t-chunks (T > 256)
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "npix%d_N%d_F%d_T%d_P%d" % s)
@pytest.mark.parametrize("prec", ["fp16x3", "bf16x3"])
def test_tc_prior_draws(fg21lib, shape, prec):
    npix, N, F, T, P = shape
    sky, obs, m, data = cases.small_case(npix=npix, N=N, F=F, T=T, window=3.0)
    model = fg21lib.fg21_build_regions(sky, obs, N)
    assert np.array_equal(model.labels, m.labels)
    fg21lib.fg21_model_set_data(model, data)
    params = cases.I.prior_draws(P, N, seed=N * 7 + T)
    got = fg21lib.fg21_loglike_batch(model, params, prec)
    want, dterm = cases.expected(m, obs, data, params)
    tol = cases.logl_tolerance(prec, m, obs, data, params)
    report(f"tc_prior_{prec}_{shape}", max_abs=np.max(np.abs(got - want)),
           max_rel_dterm=np.max(np.abs(got - want) / np.abs(dterm)))
    cases.check_logl(f"tc_prior_{prec}", got, want, tol, str(shape))


@pytest.mark.parametrize("prec", ["fp16x3", "fp32_delta", "fp32_direct", "bf16x3"])
@pytest.mark.parametrize("dbeta", [1e-6, 1e-5, 1e-4])
def test_near_posterior(fg21lib, prec, dbeta):
    """Points within the posterior bulk of an N-region truth: the absolute
    1e-2 nats bound for the reference-subtracted forms; the plain FP32 form's
    error is recorded (it is the comparator and is expected to miss it)."""
    sky, obs, m, _ = cases.small_case(npix=3072, N=9, F=151, T=20, window=6.0)
    truth, data, pts = cases.near_posterior(m, obs, dbeta, 512)
    model = fg21lib.fg21_build_regions(sky, obs, 9)
    fg21lib.fg21_model_set_data(model, data)
    got = fg21lib.fg21_loglike_batch(model, pts, prec)
    want, dterm = cases.expected(m, obs, data, pts)
    err = np.abs(got - want)
    red = 2 * dterm / (obs.F * obs.T)
    report(f"near_post_{prec}_{dbeta}", max_abs=err.max(), max_chi2_red=red.max(), min_chi2_red=red.min())
    if prec in ("fp16x3", "fp32_delta"):
        near = red <= 10
        cases.check_logl(f"near_abs_{prec}_{dbeta}", got[near], want[near], 1e-2)
    tol = cases.logl_tolerance(prec, m, obs, data, pts)
    if prec != "fp32_direct":
        cases.check_logl(f"near_{prec}_{dbeta}", got, want, tol)


@pytest.mark.parametrize("prec", ["fp16x3", "bf16x3", "fp32_delta", "fp32_direct"])
def test_model_temperature_prior_draws(fg21lib, prec):
    """T_model[p,f,t] of the kernel's own arithmetic against eq. fast_forward_model,
    relative to the magnitude the form carries (prior draws, far from the data)."""
    sky, obs, m, data = cases.small_case(npix=2048, N=6, F=41, T=5)
    model = fg21lib.fg21_build_regions(sky, obs, 6)
    fg21lib.fg21_model_set_data(model, data)
    params = cases.I.prior_draws(40, 6, seed=9)
    got = fg21lib.fg21_model_eval(model, params, prec)
    want = O.fast_model(m.A, m.B, obs, params)
    scale = cases.t_model_scale(prec, m, obs, data, params)
    tol = 1e-3 + cases.REL_T[prec] * scale
    err = np.abs(got - want)
    report(f"T_model_prior_{prec}", max_abs=err.max(), max_rel_scale=np.max(err / scale))
    cases.check_logl(f"T_model_prior_{prec}", got, want, tol)


@pytest.mark.parametrize("prec", ["fp16x3", "fp32_delta", "fp32_direct", "bf16x3"])
@pytest.mark.parametrize("dbeta", [1e-6, 1e-5])
def test_model_temperature_near_posterior(fg21lib, prec, dbeta):
    """|dT_model| <= 1e-3 K per (p, f, t) at points within the posterior bulk
    (data = N-region truth + 25 mK noise) for the reference-subtracted forms;
    the plain FP32 form's error (one FP32 ulp of a 1e4 K foreground is ~1e-3 K)
    is recorded."""
    sky, obs, m, _ = cases.small_case(npix=3072, N=9, F=151, T=4, window=2.0)
    truth, data, pts = cases.near_posterior(m, obs, dbeta, 64)
    model = fg21lib.fg21_build_regions(sky, obs, 9)
    fg21lib.fg21_model_set_data(model, data)
    got = fg21lib.fg21_model_eval(model, pts, prec)
    want = O.fast_model(m.A, m.B, obs, pts)
    err = np.abs(got - want)
    report(f"T_model_near_{prec}_{dbeta}", max_abs=err.max())
    if prec != "fp32_direct":
        cases.check_logl(f"T_model_near_{prec}_{dbeta}", got, want, 1e-3)


def test_invalid_points(fg21lib):
    sky, obs, m, data = cases.small_case(npix=1024, N=3, F=9, T=2)
    model = fg21lib.fg21_build_regions(sky, obs, 3)
    fg21lib.fg21_model_set_data(model, data)
    params = cases.I.prior_draws(10, 3, seed=1)
    params[1, 0] = np.nan
    params[3, -1] = 0.0          # sigma_n = 0
    params[5, -1] = -1.0         # sigma_n < 0
    params[7, 5] = 0.0           # sigma21 = 0
    params[8, 4] = np.inf
    for prec in ("fp16x3", "fp32_delta", "fp32_direct"):
        got = fg21lib.fg21_loglike_batch(model, params, prec)
        bad = [1, 3, 5, 7, 8]
        assert np.all(np.isneginf(got[bad]))
        assert fg21lib.fg21_last_invalid_count() == 5
        good = [0, 2, 4, 6, 9]
        want, dterm = cases.expected(m, obs, data, params[good])
        cases.check_logl(f"invalid_{prec}", got[good], want, cases.logl_tolerance(prec, m, obs, data, params[good]))


def test_empty_batch_and_errors(fg21lib):
    sky, obs, m, data = cases.small_case(npix=512, N=2, F=5, T=1)
    model = fg21lib.fg21_build_regions(sky, obs, 2)
    assert fg21lib.fg21_loglike_batch(model, np.empty((0, 6))).shape == (0,)
    with pytest.raises(fg21lib.Fg21Error) as e:
        fg21lib.fg21_loglike_batch(model, np.zeros((3, 6)), precision=7)
    assert e.value.code == fg21lib.FG21_E_ARG


def test_workload1_all_precisions(fg21lib):
    wl, sky, obs, m, data, params = cases.workload_case(1)
    model = fg21lib.fg21_build_regions(sky, obs, wl.N, wl.scheme)
    assert np.array_equal(model.labels, m.labels)
    np.testing.assert_array_equal(model.edges, m.edges)
    A, B = fg21lib.fg21_model_get_arrays(model)
    np.testing.assert_allclose(A, m.A, rtol=1e-12, atol=1e-12 * np.abs(m.A).max())
    np.testing.assert_allclose(B, m.B, rtol=1e-12)
    fg21lib.fg21_model_set_data(model, data)
    want, dterm = cases.expected(m, obs, data, params)
    for prec in ("fp16x3", "bf16x3", "fp32_delta", "fp32_direct"):
        got = fg21lib.fg21_loglike_batch(model, params, prec)
        tol = cases.logl_tolerance(prec, m, obs, data, params)
        report(f"w1_{prec}", max_abs=np.max(np.abs(got - want)),
               max_rel_dterm=np.max(np.abs(got - want) / np.abs(dterm)))
        cases.check_logl(f"w1_{prec}", got, want, tol)


def test_workload2_full(fg21lib):
    wl, sky, obs, m, data, params = cases.workload_case(2)
    model = fg21lib.fg21_build_regions(sky, obs, wl.N, wl.scheme)
    assert np.array_equal(model.labels, m.labels)
    fg21lib.fg21_model_set_data(model, data)
    want, dterm = cases.expected(m, obs, data, params)
    for prec in ("fp16x3", "fp32_direct"):
        got = fg21lib.fg21_loglike_batch(model, params, prec)
        tol = cases.logl_tolerance(prec, m, obs, data, params)
        report(f"w2_{prec}", max_abs=np.max(np.abs(got - want)),
               max_rel_dterm=np.max(np.abs(got - want) / np.abs(dterm)))
        cases.check_logl(f"w2_{prec}", got, want, tol)


def test_workload3_benchmark_configuration_sampled(fg21lib):
    """The benchmark's own workload and launch configuration (49152-pixel sky,
    N = 24, F = 301, T = 100, 16384 prior draws; the work split fg21_autotune
    picks; the step replayed from a CUDA graph): labels equal the oracle's, and
    every 64th logL (256 points the oracle evaluates one by one) is within the
    derived tolerance."""
    torch = pytest.importorskip("torch")
    wl, sky, obs, m, data, params = cases.workload_case(3)      # the oracle's model, built once per session
    model = fg21lib.fg21_build_regions(sky, obs, wl.N, wl.scheme, wl.weighting)
    assert np.array_equal(model.labels, m.labels)
    fg21lib.fg21_model_set_data(model, data)
    P = params.shape[0]
    d_p = torch.from_numpy(params).cuda()
    d_l = torch.empty(P, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    fg21lib.fg21_autotune(model, d_p.data_ptr(), P, d_l.data_ptr(), "fp16x3", s)
    g = fg21lib.fg21_graph_create(model, d_p.data_ptr(), P, d_l.data_ptr(), "fp16x3")
    g.launch(s)
    assert g.sync_status(s) == 0
    got = d_l.cpu().numpy()
    g.close()
    idx = np.arange(0, P, 64)
    want, dterm = cases.expected(m, obs, data, params[idx])
    tol = cases.logl_tolerance("fp16x3", m, obs, data, params[idx])
    err = np.abs(got[idx] - want)
    report("w3_graph_sampled", max_abs=err.max(), max_rel_dterm=np.max(err / np.abs(dterm)),
           max_err_over_tol=np.max(err / tol))
    cases.check_logl("w3_graph_fp16x3", got[idx], want, tol)
    assert np.all(np.isfinite(got))


# the largest shapes each path takes: N = 62 fills K = 64 on the tensor path,
# T = 192 is one full-width t-chunk (the ring drops to its minimum of two stage
# slots), T = 193 splits into two chunks; N = 126 is the SIMT and build limit
MAX_SHAPES = [
    # (npix, N, F, T, P, precisions)
    (4096, 62, 7, 192, 300, ("fp16x3", "bf16x3")),
    (4096, 62, 5, 193, 131, ("fp16x3",)),
    (4096, 126, 5, 3, 200, ("fp32_delta", "fp32_direct")),
]


@pytest.mark.parametrize("shape", MAX_SHAPES, ids=lambda s: "N%d_F%d_T%d_P%d" % s[1:5])
def test_maximum_shapes(fg21lib, shape):
    npix, N, F, T, P, precs = shape
    sky, obs, m, data = cases.small_case(npix=npix, N=N, F=F, T=T, window=12.0)
    model = fg21lib.fg21_build_regions(sky, obs, N)
    assert np.array_equal(model.labels, m.labels)
    fg21lib.fg21_model_set_data(model, data)
    params = cases.I.prior_draws(P, N, seed=N + T)
    want, dterm = cases.expected(m, obs, data, params)
    for prec in precs:
        got = fg21lib.fg21_loglike_batch(model, params, prec)
        tol = cases.logl_tolerance(prec, m, obs, data, params)
        report(f"max_shape_{prec}_N{N}_T{T}", max_err_over_tol=np.max(np.abs(got - want) / tol))
        cases.check_logl(f"max_shape_{prec}", got, want, tol, f"N{N}_T{T}")
    model.close()


def test_limits_refused(fg21lib):
    """One past each limit is refused with its documented code, not evaluated."""
    sky, obs, m, data = cases.small_case(npix=2048, N=63, F=5, T=2)
    model = fg21lib.fg21_build_regions(sky, obs, 63)
    fg21lib.fg21_model_set_data(model, data)
    params = cases.I.prior_draws(10, 63, seed=2)
    with pytest.raises(fg21lib.Fg21Error) as e:
        fg21lib.fg21_loglike_batch(model, params, "fp16x3")
    assert e.value.code == fg21lib.FG21_E_RANGE
    # the SIMT forms take N = 63
    got = fg21lib.fg21_loglike_batch(model, params, "fp32_delta")
    want, _ = cases.expected(m, obs, data, params)
    cases.check_logl("limits_fp32_delta", got, want, cases.logl_tolerance("fp32_delta", m, obs, data, params))
    model.close()
    with pytest.raises(fg21lib.Fg21Error) as e:
        fg21lib.fg21_build_regions(sky, obs, 127)
    assert e.value.code == fg21lib.FG21_E_ARG


_W3_NEAR = {}


def _w3_near(fg21lib, dbeta):
    """The benchmark's sky, model and launch configuration (graph replay of
    16384 points) in the nested-sampling regime: data from the 24-region model
    at a truth plus 25 mK noise, points within dbeta in beta of it; every 64th
    logL (256 points the oracle evaluates one by one) with the oracle's value,
    chi2 / (F T) and the derived tolerance.  Computed once per dbeta."""
    if dbeta in _W3_NEAR:
        return _W3_NEAR[dbeta]
    torch = pytest.importorskip("torch")
    wl, sky, obs, m, _, _ = cases.workload_case(3)
    truth, data, pts = cases.near_posterior(m, obs, dbeta, wl.P)
    model = fg21lib.fg21_build_regions(sky, obs, wl.N, wl.scheme, wl.weighting)
    fg21lib.fg21_model_set_data(model, data)
    d_p = torch.from_numpy(pts).cuda()
    d_l = torch.empty(wl.P, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    g = fg21lib.fg21_graph_create(model, d_p.data_ptr(), wl.P, d_l.data_ptr(), "fp16x3")
    g.launch(s)
    assert g.sync_status(s) == 0
    got = d_l.cpu().numpy()
    g.close()
    model.close()
    idx = np.arange(0, wl.P, 64)
    want, dterm = cases.expected(m, obs, data, pts[idx])
    red = 2 * dterm / (obs.F * obs.T)
    tol = cases.logl_tolerance("fp16x3", m, obs, data, pts[idx])
    _W3_NEAR[dbeta] = (got[idx], want, red, tol)
    return _W3_NEAR[dbeta]


@pytest.mark.parametrize("dbeta", [1e-6, 1e-5, 1e-4])
def test_workload3_near_posterior_sampled(fg21lib, dbeta):
    """At the benchmark size, near the posterior: the derived tolerance at
    every sampled point, and the absolute 1e-2 nats bound wherever chi2 / (F T)
    <= 10 for dbeta = 1e-6 (chi2 / (F T) about 1.06) and 1e-5 (up to 7)."""
    got, want, red, tol = _w3_near(fg21lib, dbeta)
    err = np.abs(got - want)
    near = red <= 10
    report(f"w3_near_posterior_sampled_{dbeta}", max_abs=err.max(), max_chi2_red=red.max(),
           min_chi2_red=red.min(), n_near=near.sum(), max_abs_near=err[near].max() if near.any() else 0.0,
           max_err_over_tol=np.max(err / tol))
    cases.check_logl(f"w3_near_{dbeta}", got, want, tol)
    assert near.any()
    if dbeta <= 1e-5:
        cases.check_logl(f"w3_near_abs_{dbeta}", got[near], want[near], 1e-2)


@pytest.mark.xfail(strict=True, reason="known gap: at dbeta = 1e-4 the 80 of 256 sampled points whose departures "
                                       "cancel to chi2/(F T) <= 10 reach |dlogL| = 1.8e-2 (GB300): the FP32 weights "
                                       "and the accumulator's rounding toward zero of departure-sized partial sums")
def test_workload3_near_posterior_absolute_bound_dbeta_1e_4(fg21lib):
    """The absolute 1e-2 nats bound at dbeta = 1e-4 wherever chi2 / (F T) <=
    10.  Expected to fail (strict: a pass means the gap closed and the mark must
    go).  There the points' departures from the batch reference are ~10 times
    their residuals and cancel across the 24 regions; FP32 weights alone
    (rounded once per point, region and channel, and so coherent over the 100
    LST bins) leave ~1.1e-2, and the FP32 accumulator's rounding toward zero of
    departure-sized partial sums adds the rest.  The regression ceiling of this
    case is held by test_workload3_near_posterior_sampled[0.0001]."""
    got, want, red, tol = _w3_near(fg21lib, 1e-4)
    near = red <= 10
    assert near.any()
    assert np.all(np.abs(got[near] - want[near]) <= 1e-2)


def test_workload3_near_posterior_dbeta_1e_4_recorded(fg21lib):
    """The absolute error at dbeta = 1e-4 where chi2 / (F T) <= 10 stays below
    3e-2 nats: a regression ceiling of 1.7x the 1.8e-2 measured on a GB300."""
    got, want, red, tol = _w3_near(fg21lib, 1e-4)
    near = red <= 10
    err = np.abs(got[near] - want[near])
    report("w3_near_abs_1e-4_recorded", max_abs_near=err.max(), n_near=near.sum())
    assert err.max() <= 3e-2, f"max |dlogL| {err.max():.3e} at dbeta = 1e-4, chi2/(F T) <= 10"


# Batch spreads that select each form of the weight series (the kernel derives
# it from the spread: max |beta - bbar| * max |ln(nu/nu0)|, about 1.53 here):
# degree 3 (spread 1e-3), degree 5 (3e-2), degree 8 (the prior box, 0.35) and
# degree 8 after two halvings undone by squarings (beta in [1.8, 3.6]).
SERIES_CASES = [("degree3", 1e-3), ("degree5", 3e-2), ("degree8", None), ("squarings", (1.8, 3.6))]


@pytest.mark.parametrize("case,spread", SERIES_CASES, ids=[c[0] for c in SERIES_CASES])
@pytest.mark.parametrize("prec", ["fp16x3", "bf16x3"])
def test_weight_series_forms(fg21lib, case, spread, prec):
    """Every form of the weights' expm1 series (degree 3, 5, 8 and squarings)
    against eq. fast_forward_model / eq. likelihood in the oracle, through the
    lean kernel (spectral-index regions, K = 32)."""
    sky, obs, m, data = cases.small_case(npix=2048, N=24, F=41, T=12, window=4.0)
    model = fg21lib.fg21_build_regions(sky, obs, 24)
    fg21lib.fg21_model_set_data(model, data)
    g = np.random.default_rng(17)
    P = 300
    if spread is None:
        params = cases.I.prior_draws(P, 24, seed=23)
    elif isinstance(spread, tuple):
        params = cases.I.prior_draws(P, 24, seed=23)
        params[:, :24] = g.uniform(spread[0], spread[1], size=(P, 24))
    else:
        centre = cases.I.prior_draws(1, 24, seed=24)[0]
        params = cases.I.scatter_around(centre, P, spread, 25)
    got = fg21lib.fg21_loglike_batch(model, params, prec)
    want, _ = cases.expected(m, obs, data, params)
    tol = cases.logl_tolerance(prec, m, obs, data, params)
    cases.check_logl(f"series_{case}_{prec}", got, want, tol)
    model.close()


@pytest.mark.parametrize("case,spread", SERIES_CASES, ids=[c[0] for c in SERIES_CASES])
def test_weight_series_forms_amplitude_regions(fg21lib, case, spread):
    """The same series forms through the generic kernel (amplitude regions:
    the series runs in y = d nL + ln(alpha / abar), degree chosen at run time)."""
    Nb, Na = 6, 3
    sky, obs, m, data = cases.small_case_ab(npix=2048, Nb=Nb, Na=Na, F=31, T=8)
    model = fg21lib.fg21_build_regions_ab(sky, obs, Nb, "recursive", "beam", Na, cases.I.amplitude_field(sky),
                                          "hierarchical", "beam")
    fg21lib.fg21_model_set_data(model, data)
    g = np.random.default_rng(19)
    P = 200
    params = cases.I.prior_draws_ab(P, Nb, Na, seed=29)
    if isinstance(spread, tuple):
        params[:, :Nb] = g.uniform(spread[0], spread[1], size=(P, Nb))
    elif spread is not None:
        centre = params[0].copy()
        params = np.repeat(centre[None], P, axis=0)
        params[:, :Nb] += g.uniform(-spread, spread, size=(P, Nb))
        params[:, Nb:Nb + Na] *= 1.0 + g.uniform(-spread, spread, size=(P, Na))
    got = fg21lib.fg21_loglike_batch(model, params, "fp16x3")
    want, _ = cases.expected_ab(m, obs, data, params)
    tol = cases.logl_tolerance_ab("fp16x3", m, obs, data, params)
    cases.check_logl(f"series_ab_{case}", got, want, tol)
    model.close()
