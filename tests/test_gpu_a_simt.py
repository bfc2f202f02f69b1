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


# t-chunks: T = 300 is three rounds of 128 staged columns (128, 128, 44), and
# N = 120, T = 150 two rounds (128, 22) of 121-row slabs, near the largest
# block the region cap (N <= 126) allows.
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


# Past the first round, the column blocks of 8 that do not fill a round of the
# four column slots go one point per thread: T sets how many are left
# (ceil(T / 8) mod 4) and whether the last block is partial.  T = 5, 8, 17:
# fewer blocks than slots, whole tiles in one round (17: the third block
# partial); 32: one full round, no leftover; 40, 48, 56: one round and 1, 2, 3
# leftovers; 100: three rounds and one partial leftover (the benchmark's T).
SIMT_REMAINDER_T = [5, 8, 17, 32, 40, 48, 56, 100]


@pytest.mark.parametrize("T", SIMT_REMAINDER_T)
@pytest.mark.parametrize("prec", ["fp32_delta", "fp32_direct"])
def test_simt_column_remainders(fg21lib, prec, T):
    sky, obs, m, data = cases.small_case(npix=1024, N=6, F=7, T=T, window=8.0, seed=T)
    model = fg21lib.fg21_build_regions(sky, obs, 6)
    assert np.array_equal(model.labels, m.labels)
    fg21lib.fg21_model_set_data(model, data)
    params = cases.I.prior_draws(133, 6, seed=200 + T)
    got = fg21lib.fg21_loglike_batch(model, params, prec)
    want, _ = cases.expected(m, obs, data, params)
    tol = cases.logl_tolerance(prec, m, obs, data, params)
    cases.check_logl(f"simt_remainder_{prec}", got, want, tol, f"T{T}")
    model.close()
