"""GPU tests of the measured work-split autotuner (fg21_autotune): it returns a
valid split with a time, the split is used by later plans of that model and
size, and the results under it match the oracle within tolerance and are the
same through the host and the device calls."""
import numpy as np
import pytest

import cases
from paper_2603_13196_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_autotune_split_is_valid_and_results_hold(fg21lib):
    import torch
    sky, obs, m, data = cases.small_case(npix=2048, N=9, F=61, T=12, window=4.0)
    model = fg21lib.fg21_build_regions(sky, obs, 9)
    fg21lib.fg21_model_set_data(model, data)
    stream = torch.cuda.current_stream().cuda_stream
    P = 1500
    params = I.prior_draws(P, 9, seed=21)
    d_p = torch.from_numpy(params).cuda()
    d_l = torch.empty(P, dtype=torch.float64, device="cuda")
    cpg, ms = fg21lib.fg21_autotune(model, d_p.data_ptr(), P, d_l.data_ptr(), "fp16x3", stream)
    assert 1 <= cpg <= obs.F and ms > 0
    fg21lib.fg21_loglike_batch_device(model, d_p.data_ptr(), P, d_l.data_ptr(), "fp16x3", stream)
    fg21lib.fg21_model_sync_status(model, stream)
    dev = d_l.cpu().numpy()
    host = fg21lib.fg21_loglike_batch(model, params, "fp16x3")
    assert np.array_equal(dev, host)
    want, _ = cases.expected(m, obs, data, params)
    cases.check_logl("autotune_fp16x3", host, want, cases.logl_tolerance("fp16x3", m, obs, data, params))
    # a request of another size keeps the planner's split and still matches
    p2 = I.prior_draws(300, 9, seed=22)
    got2 = fg21lib.fg21_loglike_batch(model, p2, "fp16x3")
    want2, _ = cases.expected(m, obs, data, p2)
    cases.check_logl("autotune_fp16x3", got2, want2, cases.logl_tolerance("fp16x3", m, obs, data, p2), "P=300")
