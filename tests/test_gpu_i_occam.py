"""The maximum-likelihood side of the Occam experiment (Sec. 4.1, Sec. 6.1) on
the GPU: log L_max(N) of nested schemes never decreases with N (the embedding
identity plus a warm start), every reported maximum is the oracle's
likelihood at the returned point, and the curves of the non-nested splits are
recorded beside them."""
import numpy as np
import pytest

import oracle as O
from conftest import report
from paper_2603_13196_gb300 import inputs as I, occam

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def problem(fg21lib):
    sky = I.make_sky(3072, 61)
    obs = I.make_obs(51, 8, 6.0, lst0_h=20.0)
    data = O.simulate_data(sky, obs, np.array(I.FIDUCIAL_T21), I.NOISE_K, I.noise_draws(obs.F, obs.T, 61))
    return sky, obs, data


@pytest.mark.parametrize("scheme", ["recursive", "hierarchical", "linear", "percentile"])
def test_logl_max_curve(fg21lib, problem, scheme):
    sky, obs, data = problem
    Ns = list(range(1, 11))
    curve = occam.logl_max_curve(sky, obs, data, scheme, Ns, I.FIDUCIAL_T21, rounds=30, batch=2048, seed=5)
    L = np.array([c.logL_max for c in curve])
    report(f"occam_{scheme}", **{f"N{c.N}": c.logL_max for c in curve}, n_evals=sum(c.n_evals for c in curve))
    # each maximum is the oracle's (sigma-profiled) likelihood of the returned point
    for c in curve:
        m = O.build_model(sky, obs, c.N, scheme)
        np.testing.assert_array_equal(m.edges, c.edges)
        th = np.concatenate([c.beta, I.FIDUCIAL_T21, [1.0]])[None, :]
        c2 = O.chi2(m.A, m.B, data, obs, th)[0]
        assert abs(occam.profiled_logL(c2, obs.F * obs.T) - c.logL_max) < 1e-6 * abs(c.logL_max) + 1e-2
    if scheme in ("recursive", "hierarchical"):
        # nested: non-decreasing up to the rounding of the GPU form (FP32 delta)
        assert np.all(np.diff(L) >= -1e-2), L
    # more regions than one always fit better than a single region
    assert L.max() > L[0]
