"""GPU tests of the CUDA-graph evaluation (fg21_graph_*): a replay gives the
direct device call's logL bit for bit, follows new parameter values written
into the same buffers, repeats exactly, and an uneven multi-model graph
equals fg21_loglike_multi and the oracle within tolerance."""
import numpy as np
import pytest

import cases
from paper_2603_13196_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp16x3", "fp32_delta"])
def test_graph_matches_device_call_and_follows_params(fg21lib, prec):
    import torch
    sky, obs, m, data = cases.small_case(npix=2048, N=9, F=61, T=12, window=4.0)
    model = fg21lib.fg21_build_regions(sky, obs, 9)
    fg21lib.fg21_model_set_data(model, data)
    stream = torch.cuda.current_stream().cuda_stream
    P = 700
    p1, p2 = I.prior_draws(P, 9, seed=11), I.prior_draws(P, 9, seed=12)
    d_p = torch.from_numpy(p1).cuda()
    d_g = torch.full((P,), float("nan"), dtype=torch.float64, device="cuda")
    d_ref = torch.empty(P, dtype=torch.float64, device="cuda")
    g = fg21lib.fg21_graph_create(model, d_p.data_ptr(), P, d_g.data_ptr(), prec)
    for params in (p1, p2):
        d_p.copy_(torch.from_numpy(params))
        g.launch(stream)
        assert g.sync_status(stream) == 0
        fg21lib.fg21_loglike_batch_device(model, d_p.data_ptr(), P, d_ref.data_ptr(), prec, stream)
        fg21lib.fg21_model_sync_status(model, stream)
        got, ref = d_g.cpu().numpy(), d_ref.cpu().numpy()
        assert np.array_equal(got, ref)
        want, _ = cases.expected(m, obs, data, params)
        cases.check_logl(f"graph_{prec}", got, want, cases.logl_tolerance(prec, m, obs, data, params))
    # repeated replays are exact
    first = d_g.clone()
    for _ in range(5):
        g.launch(stream)
    g.sync_status(stream)
    assert torch.equal(first, d_g)
    g.close()


def test_graph_multi_matches_multi_and_oracle(fg21lib):
    import torch
    wls = I.uneven_batch(4, P_range=(100, 600))
    mods, params, dps, dls = [], [], [], []
    for wl in wls:
        sky, obs = wl.sky(), wl.obs()
        om = cases.O.build_model(sky, obs, wl.N, wl.scheme, wl.weighting)
        data = cases.O.simulate_data(sky, obs, np.array(I.FIDUCIAL_T21), I.NOISE_K, wl.noise())
        m = fg21lib.fg21_build_regions(sky, obs, wl.N, wl.scheme, wl.weighting)
        fg21lib.fg21_model_set_data(m, data)
        p = wl.params()
        mods.append((wl, obs, om, data, m))
        params.append(p)
        dps.append(torch.from_numpy(p).cuda())
        dls.append(torch.full((p.shape[0],), float("nan"), dtype=torch.float64, device="cuda"))
    stream = torch.cuda.current_stream().cuda_stream
    g = fg21lib.fg21_graph_create_multi([x[4] for x in mods], [t.data_ptr() for t in dps],
                                        [p.shape[0] for p in params], [t.data_ptr() for t in dls], "fp16x3")
    g.launch(stream)
    assert g.sync_status(stream) == 0
    ref = fg21lib.fg21_loglike_multi([x[4] for x in mods], params, "fp16x3")
    for (wl, obs, om, data, m), p, d, r in zip(mods, params, dls, ref):
        got = d.cpu().numpy()
        assert np.array_equal(got, r), wl.name
        want, _ = cases.expected(om, obs, data, p)
        cases.check_logl("graph_multi_fp16x3", got, want, cases.logl_tolerance("fp16x3", om, obs, data, p), wl.name)
    g.close()


@pytest.mark.parametrize("prec", ["fp16x3", "fp32_delta"])
def test_host_call_pinned_buffers_and_its_cached_graph(fg21lib, prec):
    """The host-buffer call replays a graph it keeps per (size, precision, work
    split): page-locked and pageable buffers give the same logL, which equals the
    direct device call bit for bit; a new size, a new tuned split and invalid
    points all go through it correctly."""
    import torch
    sky, obs, m, data = cases.small_case(npix=2048, N=7, F=41, T=9, window=4.0)
    model = fg21lib.fg21_build_regions(sky, obs, 7)
    fg21lib.fg21_model_set_data(model, data)
    stream = torch.cuda.current_stream().cuda_stream

    def device_call(params):
        d_p = torch.from_numpy(params).cuda()
        d_l = torch.empty(params.shape[0], dtype=torch.float64, device="cuda")
        fg21lib.fg21_loglike_batch_device(model, d_p.data_ptr(), params.shape[0], d_l.data_ptr(), prec, stream)
        assert fg21lib.fg21_model_sync_status(model, stream) == 0
        return d_l.cpu().numpy()

    p1, p2 = I.prior_draws(300, 7, seed=3), I.prior_draws(129, 7, seed=4)
    a = fg21lib.fg21_loglike_batch(model, p1, prec)              # pageable: staged; captures the graph
    hp = torch.empty(p1.shape, dtype=torch.float64, pin_memory=True).numpy()
    hp[:] = p1
    ho = torch.empty(p1.shape[0], dtype=torch.float64, pin_memory=True).numpy()
    b = fg21lib.fg21_loglike_batch(model, hp, prec, out=ho)     # page-locked: direct DMA, replay
    assert b is ho and np.array_equal(a, b)
    assert np.array_equal(a, device_call(p1))
    c = fg21lib.fg21_loglike_batch(model, p2, prec)              # another size: a new graph
    assert np.array_equal(c, device_call(p2))
    assert np.array_equal(fg21lib.fg21_loglike_batch(model, p1, prec), a)
    want, _ = cases.expected(m, obs, data, p1)
    cases.check_logl(f"host_call_{prec}", a, want, cases.logl_tolerance(prec, m, obs, data, p1))
    # a tuned work split for this size replaces the kept graph
    d_p = torch.from_numpy(p1).cuda()
    d_l = torch.empty(300, dtype=torch.float64, device="cuda")
    fg21lib.fg21_autotune(model, d_p.data_ptr(), 300, d_l.data_ptr(), prec, stream)
    t = fg21lib.fg21_loglike_batch(model, p1, prec)
    assert np.array_equal(t, device_call(p1))
    cases.check_logl(f"host_call_{prec}", t, want, cases.logl_tolerance(prec, m, obs, data, p1), "timed")
    # invalid points: -inf and counted through the replayed graph
    p3 = p1.copy()
    p3[5, -1] = -1.0
    p3[7, 0] = np.nan
    r = fg21lib.fg21_loglike_batch(model, p3, prec)
    assert np.isneginf(r[5]) and np.isneginf(r[7]) and np.all(np.isfinite(np.delete(r, [5, 7])))
    assert fg21lib.fg21_last_invalid_count() == 2
    model.close()
