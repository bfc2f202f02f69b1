"""Host logic of the Occam experiment (paper_2603_13196_gb300.occam), on the
CPU against the oracle: the embedding of a nested level-N point into level
N+1 reproduces the forward model exactly, and the sigma_n-profiled
likelihood is the maximum of eq. likelihood over sigma_n."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2603_13196_gb300 import fg21, inputs as I, occam


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("scheme", ["recursive", "hierarchical"])
def test_embed_reproduces_the_model(scheme):
    sky = I.make_sky(2048, 41)
    obs = I.make_obs(9, 3, 4.0, lst0_h=2.0)
    for N in (1, 2, 5, 8):
        _, e0, _, _ = fg21.fg21_build_regions_host(sky, obs, N, scheme)
        _, e1, _, _ = fg21.fg21_build_regions_host(sky, obs, N + 1, scheme)
        m0 = O.build_model(sky, obs, N, scheme)
        m1 = O.build_model(sky, obs, N + 1, scheme)
        beta = I.prior_draws(1, N, seed=N)[0, :N]
        th0 = np.concatenate([beta, [0.155, 85.0, 15.0, 0.025]])
        th1 = np.concatenate([occam.embed(beta, e0, e1), [0.155, 85.0, 15.0, 0.025]])
        np.testing.assert_allclose(O.fast_model(m1.A, m1.B, obs, th1), O.fast_model(m0.A, m0.B, obs, th0),
                                   rtol=1e-12)


def test_profiled_logl_is_the_maximum_over_sigma():
    sky = I.make_sky(1024, 43)
    obs = I.make_obs(21, 2, 2.0)
    m = O.build_model(sky, obs, 3, "recursive")
    data = O.simulate_data(sky, obs, np.array(I.FIDUCIAL_T21), 0.025, I.noise_draws(21, 2, 1))
    th = np.concatenate([O.region_truth(sky, m.labels, 3), [0.155, 85.0, 15.0, 1.0]])[None, :]
    c2 = O.chi2(m.A, m.B, data, obs, th)[0]
    lp = occam.profiled_logL(c2, obs.F * obs.T)
    s_hat = math.sqrt(c2 / (obs.F * obs.T))
    grid = s_hat * np.exp(np.linspace(-0.5, 0.5, 201))
    ths = np.repeat(th, len(grid), axis=0)
    ths[:, -1] = grid
    L = O.loglike(m.A, m.B, data, obs, ths)
    assert abs(lp - L.max()) <= 1e-9 * abs(lp) + 1e-6
    assert np.argmax(L) == 100        # at s_hat
