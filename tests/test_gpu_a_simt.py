"""GPU parity of the SIMT forms (plain FP32 and FP32 reference-subtracted)
against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import cases
from conftest import report

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32_delta", "fp32_direct"])
@pytest.mark.parametrize("P", [1, 129])
def test_simt_small(fg21lib, prec, P):
    sky, obs, m, data = cases.small_case()
    model = fg21lib.fg21_build_regions(sky, obs, 5)
    assert np.array_equal(model.labels, m.labels)
    fg21lib.fg21_model_set_data(model, data)
    params = cases.I.prior_draws(P, 5, seed=3)
    got = fg21lib.fg21_loglike_batch(model, params, prec)
    want, dterm = cases.expected(m, obs, data, params)
    tol = cases.logl_tolerance(prec, m, obs, data, params)
    report(f"simt_small_{prec}_{P}", max_abs=np.max(np.abs(got - want)),
           max_rel_dterm=np.max(np.abs(got - want) / np.abs(dterm)))
    cases.check_logl(f"simt_small_{prec}", got, want, tol, f"P={P}")


@pytest.mark.parametrize("prec", ["fp32_delta", "fp32_direct"])
def test_simt_workload1(fg21lib, prec):
    wl, sky, obs, m, data, params = cases.workload_case(1)
    model = fg21lib.fg21_build_regions(sky, obs, wl.N, wl.scheme)
    assert np.array_equal(model.labels, m.labels)
    fg21lib.fg21_model_set_data(model, data)
    got = fg21lib.fg21_loglike_batch(model, params, prec)
    want, dterm = cases.expected(m, obs, data, params)
    tol = cases.logl_tolerance(prec, m, obs, data, params)
    report(f"simt_w1_{prec}", max_abs=np.max(np.abs(got - want)),
           max_rel_dterm=np.max(np.abs(got - want) / np.abs(dterm)))
    cases.check_logl(f"simt_w1_{prec}", got, want, tol)


# t-chunks: T = 300 is three rounds of 128 staged columns; N = 120 stages 64
# columns per round (two 128-column slabs of 121 rows would not fit shared
# memory; the threshold is N = 110), so T = 150 is three rounds of 64.
SIMT_CHUNK_SHAPES = [(1024, 4, 5, 300, 130), (4096, 120, 5, 150, 129)]


@pytest.mark.parametrize("shape", SIMT_CHUNK_SHAPES, ids=lambda s: "npix%d_N%d_F%d_T%d_P%d" % s)
@pytest.mark.parametrize("prec", ["fp32_delta", "fp32_direct"])
def test_simt_t_chunks(fg21lib, shape, prec):
    npix, N, F, T, P = shape
    sky, obs, m, data = cases.small_case(npix=npix, N=N, F=F, T=T, window=8.0)
    model = fg21lib.fg21_build_regions(sky, obs, N)
    fg21lib.fg21_model_set_data(model, data)
    params = cases.I.prior_draws(P, N, seed=N + T)
    got = fg21lib.fg21_loglike_batch(model, params, prec)
    want, _ = cases.expected(m, obs, data, params)
    tol = cases.logl_tolerance(prec, m, obs, data, params)
    cases.check_logl(f"simt_chunks_{prec}", got, want, tol, f"N{N}_T{T}")
    model.close()
