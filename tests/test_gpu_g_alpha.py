"""GPU parity of the joint amplitude / spectral-index model (N_alpha > 1;
Sec. 2.2 eqs. forward_model, chromatic_function, fast_forward_model) against
the FP64 oracle, through the C ABI: every precision on prior draws at several
shapes (K = 16 / 32 / 64, ragged tiles, two t-chunks, one free global gain),
near-posterior sets with the absolute 1e-2 nats bound, model temperatures,
invalid scale factors, and the batched / graph paths mixing joint and
spectral-index-only models."""
import numpy as np
import pytest

import cases
import oracle as O
from conftest import report
from paper_2603_13196_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SHAPES = [
    # (npix, Nb, Na, F, T, P)
    (1024, 3, 2, 9, 1, 1),        # one point, one LST bin, K = 16
    (2048, 3, 4, 21, 5, 129),     # ragged tile tail, K = 16
    (2048, 5, 4, 17, 20, 300),    # K = 32
    (3072, 12, 5, 9, 9, 140),     # K = 64 (60 components)
    (1024, 2, 3, 5, 300, 130),    # two t-chunks (T > 192)
    (1024, 6, 1, 13, 4, 200),     # one amplitude region: a free global gain
]


def _model(fg21lib, sky, obs, m):
    Na, Nb = m.K.shape[:2]
    model = fg21lib.fg21_build_regions_ab(sky, obs, Nb, "recursive", "beam", Na, I.amplitude_field(sky),
                                          "hierarchical", "beam")
    assert np.array_equal(model.labels, m.labels_b) and np.array_equal(model.labels_alpha, m.labels_a)
    assert fg21lib.fg21_model_shape(model) == dict(n_beta=Nb, n_alpha=Na, n_params=Nb + Na + 4)
    A, _ = fg21lib.fg21_model_get_arrays(model)
    np.testing.assert_allclose(A, m.K.reshape(Na * Nb, obs.F, obs.T), rtol=1e-12,
                               atol=1e-13 * np.abs(m.K).max())
    return model


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "npix%d_Nb%d_Na%d_F%d_T%d_P%d" % s)
@pytest.mark.parametrize("prec", ["fp16x3", "bf16x3", "fp32_delta", "fp32_direct"])
def test_ab_prior_draws(fg21lib, shape, prec):
    npix, Nb, Na, F, T, P = shape
    sky, obs, m, data = cases.small_case_ab(npix=npix, Nb=Nb, Na=Na, F=F, T=T, window=3.0)
    model = _model(fg21lib, sky, obs, m)
    fg21lib.fg21_model_set_data(model, data)
    params = I.prior_draws_ab(P, Nb, Na, seed=Nb * 7 + Na)
    got = fg21lib.fg21_loglike_batch(model, params, prec)
    want, dterm = cases.expected_ab(m, obs, data, params)
    tol = cases.logl_tolerance_ab(prec, m, obs, data, params)
    report(f"ab_prior_{prec}_{shape}", max_abs=np.max(np.abs(got - want)),
           max_rel_dterm=np.max(np.abs(got - want) / np.abs(dterm)))
    cases.check_logl(f"ab_prior_{prec}", got, want, tol, str(shape))


@pytest.mark.parametrize("prec", ["fp16x3", "fp32_delta", "bf16x3"])
@pytest.mark.parametrize("dbeta,dalpha", [(1e-6, 1e-6), (1e-5, 1e-4), (1e-4, 1e-3)])
def test_ab_near_posterior(fg21lib, prec, dbeta, dalpha):
    """Points in the posterior bulk of a joint-model truth: the absolute 1e-2
    nats bound wherever chi2 / (F T) <= 10 for the FP16 split and FP32 delta
    forms, the derived tolerance everywhere."""
    sky, obs, m, _ = cases.small_case_ab(npix=3072, Nb=6, Na=3, F=151, T=10, window=6.0)
    truth, data, pts = cases.near_posterior_ab(m, obs, dbeta, dalpha, 384)
    model = _model(fg21lib, sky, obs, m)
    fg21lib.fg21_model_set_data(model, data)
    got = fg21lib.fg21_loglike_batch(model, pts, prec)
    want, dterm = cases.expected_ab(m, obs, data, pts)
    err = np.abs(got - want)
    red = 2 * dterm / (obs.F * obs.T)
    report(f"ab_near_post_{prec}_{dbeta}_{dalpha}", max_abs=err.max(), max_chi2_red=red.max())
    if prec in ("fp16x3", "fp32_delta"):
        near = red <= 10
        assert near.any()
        cases.check_logl(f"ab_near_abs_{prec}_{dbeta}_{dalpha}", got[near], want[near], 1e-2)
    tol = cases.logl_tolerance_ab(prec, m, obs, data, pts)
    cases.check_logl(f"ab_near_{prec}_{dbeta}_{dalpha}", got, want, tol)


@pytest.mark.parametrize("prec", ["fp16x3", "fp32_delta"])
def test_ab_model_temperatures(fg21lib, prec):
    """T_model[p, f, t] of the joint model within 1e-3 K of the oracle at
    near-posterior points."""
    sky, obs, m, _ = cases.small_case_ab(npix=2048, Nb=4, Na=2, F=41, T=6, window=4.0)
    truth, data, pts = cases.near_posterior_ab(m, obs, 1e-5, 1e-4, 64)
    model = _model(fg21lib, sky, obs, m)
    fg21lib.fg21_model_set_data(model, data)
    got = fg21lib.fg21_model_eval(model, pts, prec)
    want = O.fast_model_ab(m.K, m.B, obs, pts)
    err = np.abs(got - want)
    report(f"ab_tmodel_{prec}", max_abs=err.max())
    assert err.max() <= 1e-3


def test_ab_invalid_points(fg21lib):
    """alpha_i <= 0, a non-finite alpha, sigma_n <= 0: logL = -inf and
    counted; the other points match the oracle."""
    sky, obs, m, data = cases.small_case_ab(npix=1024, Nb=3, Na=2, F=11, T=3)
    model = _model(fg21lib, sky, obs, m)
    fg21lib.fg21_model_set_data(model, data)
    params = I.prior_draws_ab(40, 3, 2, seed=3)
    params[1, 3] = 0.0
    params[5, 4] = -0.5
    params[9, 3] = np.nan
    params[17, -1] = -0.01
    bad = [1, 5, 9, 17]
    ok = np.setdiff1d(np.arange(40), bad)
    for prec in ("fp16x3", "fp32_delta", "fp32_direct"):
        got = fg21lib.fg21_loglike_batch(model, params, prec)
        assert fg21lib.fg21_last_invalid_count() == 4
        assert np.all(np.isneginf(got[bad]))
        want, _ = cases.expected_ab(m, obs, data, params[ok])
        cases.check_logl(f"ab_invalid_{prec}", got[ok], want, cases.logl_tolerance_ab(prec, m, obs, data, params[ok]))


def test_ab_multi_and_graph_mixed_with_beta_only(fg21lib):
    """One persistent launch over joint and spectral-index-only models: each
    request equals its single evaluation bit for bit and the oracle; a CUDA
    graph of the same batch repeats it exactly."""
    torch = pytest.importorskip("torch")
    sky_a, obs_a, m_a, data_a = cases.small_case_ab(npix=2048, Nb=5, Na=3, F=31, T=8)
    sky_b, obs_b, m_b, data_b = cases.small_case(npix=2048, N=7, F=23, T=5)
    mod_a = _model(fg21lib, sky_a, obs_a, m_a)
    fg21lib.fg21_model_set_data(mod_a, data_a)
    mod_b = fg21lib.fg21_build_regions(sky_b, obs_b, 7)
    fg21lib.fg21_model_set_data(mod_b, data_b)
    pa = I.prior_draws_ab(300, 5, 3, seed=11)
    pb = I.prior_draws(200, 7, seed=12)
    got = fg21lib.fg21_loglike_multi([mod_a, mod_b], [pa, pb], "fp16x3")
    assert np.array_equal(got[0], fg21lib.fg21_loglike_batch(mod_a, pa, "fp16x3"))
    assert np.array_equal(got[1], fg21lib.fg21_loglike_batch(mod_b, pb, "fp16x3"))
    want_a, _ = cases.expected_ab(m_a, obs_a, data_a, pa)
    cases.check_logl("ab_multi_fp16x3", got[0], want_a, cases.logl_tolerance_ab("fp16x3", m_a, obs_a, data_a, pa))
    want_b, _ = cases.expected(m_b, obs_b, data_b, pb)
    cases.check_logl("ab_multi_fp16x3", got[1], want_b, cases.logl_tolerance("fp16x3", m_b, obs_b, data_b, pb),
                     "beta-only")
    dev = torch.device("cuda:0")
    dpa, dpb = torch.from_numpy(pa).to(dev), torch.from_numpy(pb).to(dev)
    la = torch.empty(300, dtype=torch.float64, device=dev)
    lb = torch.empty(200, dtype=torch.float64, device=dev)
    g = fg21lib.fg21_graph_create_multi([mod_a, mod_b], [dpa.data_ptr(), dpb.data_ptr()], [300, 200],
                                        [la.data_ptr(), lb.data_ptr()], "fp16x3")
    s = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        fg21lib.fg21_graph_launch(g, s)
        assert fg21lib.fg21_graph_sync_status(g, s) == 0
        assert np.array_equal(la.cpu().numpy(), got[0]) and np.array_equal(lb.cpu().numpy(), got[1])
    g.close()


def test_ab_served_and_allocation_free(fg21lib):
    """The serving loop (bit for bit the direct call's results) and the
    allocation-free device call (within tolerance of them) run amplitude-mask
    models."""
    import ctypes as C
    torch = pytest.importorskip("torch")
    sky, obs, m, data = cases.small_case_ab(npix=2048, Nb=5, Na=3, F=31, T=8)
    model = _model(fg21lib, sky, obs, m)
    fg21lib.fg21_model_set_data(model, data)
    params = I.prior_draws_ab(500, 5, 3, seed=21)
    direct = fg21lib.fg21_loglike_batch(model, params, "fp16x3")
    srv = fg21lib.Server(mem_budget_bytes=1 << 30, max_batch_points=4096, max_wait_us=100, max_inflight=2)
    rid, admitted = fg21lib.fg21_serve_register_run(srv, model)
    assert admitted
    t, out = fg21lib.fg21_serve_submit(srv, rid, params)
    assert fg21lib.fg21_serve_wait(srv, t, 60000) == 0
    srv.close()
    np.testing.assert_array_equal(out, direct)
    d_p = torch.from_numpy(params).cuda()
    d_na = torch.full((500,), float("nan"), dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    rc = fg21lib.lib().fg21_loglike_batch_device_noalloc(model.handle, C.c_void_p(d_p.data_ptr()), 500,
                                                          C.c_void_p(d_na.data_ptr()), 0, C.c_void_p(s))
    assert rc == 0, fg21lib.lib().fg21_last_error()
    torch.cuda.synchronize()
    tol = cases.logl_tolerance_ab("fp16x3", m, obs, data, params)
    cases.check_logl("ab_serve_noalloc_vs_direct", d_na.cpu().numpy(), direct, tol)
