"""The allocation-free device call (for callers that cannot allocate GPU
memory during a call) gives the regular device call's results, on two calls in
a row, within the tolerance the parity tests use.  Collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import cases
from paper_2603_13196_gb300 import fg21, inputs as I

pytestmark = pytest.mark.gpu


def test_noalloc_matches_device_call_twice(fg21lib):
    import torch
    sky, obs, m, data = cases.small_case(npix=2048, N=9, F=61, T=12, window=4.0)
    model = fg21lib.fg21_build_regions(sky, obs, 9)
    fg21lib.fg21_model_set_data(model, data)
    stream = torch.cuda.current_stream().cuda_stream
    for call, (P, seed) in enumerate([(700, 1), (333, 2)]):
        params = I.prior_draws(P, 9, seed=seed)
        d_p = torch.from_numpy(params).cuda()
        d_ref = torch.empty(P, dtype=torch.float64, device="cuda")
        d_na = torch.full((P,), float("nan"), dtype=torch.float64, device="cuda")
        fg21lib.fg21_loglike_batch_device(model, d_p.data_ptr(), P, d_ref.data_ptr(), "fp16x3", stream)
        fg21lib.fg21_model_sync_status(model, stream)
        rc = fg21lib.lib().fg21_loglike_batch_device_noalloc(model.handle, C.c_void_p(d_p.data_ptr()), P,
                                                              C.c_void_p(d_na.data_ptr()), 0, C.c_void_p(stream))
        assert rc == 0, fg21lib.lib().fg21_last_error()
        torch.cuda.synchronize()
        ref, got = d_ref.cpu().numpy(), d_na.cpu().numpy()
        tol = cases.logl_tolerance("fp16x3", m, obs, data, params)
        assert np.all(np.abs(got - ref) <= tol), call
        want, _ = cases.expected(m, obs, data, params)
        cases.check_logl("noalloc_fp16x3", got, want, tol, f"call {call}")


def test_noalloc_rejects_oversized_request(fg21lib):
    """A request above the scratch limit is refused before any launch.  The
    parameter and logL buffers are real device buffers of the request's full
    size, so a regressed size check would evaluate them instead of touching
    memory the call was not given."""
    import torch
    sky, obs, m, data = cases.small_case(npix=1024, N=30, F=301, T=100, window=4.0)
    model = fg21lib.fg21_build_regions(sky, obs, 30)
    fg21lib.fg21_model_set_data(model, data)
    P = 400000
    d_p = torch.zeros((P, 34), dtype=torch.float64, device="cuda")
    d_l = torch.zeros(P, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = fg21lib.lib().fg21_loglike_batch_device_noalloc(model.handle, C.c_void_p(d_p.data_ptr()), P,
                                                          C.c_void_p(d_l.data_ptr()), 0, C.c_void_p(stream))
    assert rc == fg21lib.FG21_E_RANGE
    assert "scratch" in fg21lib.lib().fg21_last_error().decode()
    torch.cuda.synchronize()
    assert not torch.any(d_l != 0)         # nothing was launched
    model.close()
