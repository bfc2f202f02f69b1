"""The batched nested slice sampler on problems with known evidence (CPU)."""
import math

import numpy as np
import pytest
import scipy.special

from paper_2603_13196_gb300 import ns


def gaussian_problem(d=3, sig=0.05, mu=None):
    mu = np.full(d, 0.5) if mu is None else np.asarray(mu)
    prior = ns.Prior(["uniform"] * d, np.zeros(d), np.ones(d))

    def ll(th):
        r = (th - mu) / sig
        return -0.5 * np.sum(r * r, axis=1) - d * math.log(sig * math.sqrt(2 * math.pi))
    return prior, ll


def test_batched_deletion_shrinkage():
    """eq. log_xgpu: E[log X] after deleting b of n is -sum_{i<b} 1/(n-i), close to
    ln((n-b)/n); equals the digamma difference psi(n-b+1) - psi(n+1) exactly."""
    for n, b in [(500, 100), (200, 40), (50, 1)]:
        e = ns.expected_log_shrinkage(n, b)
        assert abs(e - (scipy.special.digamma(n - b + 1) - scipy.special.digamma(n + 1))) < 1e-12
        assert abs(e - math.log((n - b) / n)) < 1.0 / (n - b)
    assert ns.expected_log_shrinkage(10, 1) == -0.1


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gaussian_in_unit_box_evidence(seed):
    """A normalised Gaussian well inside the unit box has Z = 1 (log Z = 0)."""
    prior, ll = gaussian_problem(d=3, sig=0.05, mu=[0.4, 0.55, 0.6])
    res = ns.NestedSlice(prior, ll, n_live=200, num_delete=40, seed=seed).run()
    assert abs(res.logZ) < 3.5 * res.logZ_err + 0.05, (res.logZ, res.logZ_err)
    # information of a narrow Gaussian posterior against the unit box
    H_true = 3 * (math.log(1 / (0.05 * math.sqrt(2 * math.pi))) - 0.5)
    assert abs(res.H - H_true) < 0.5
    # quadrature weights cover the unit prior volume
    assert abs(np.sum(np.exp(res.dead_logw)) - 1.0) < 1e-9


def test_posterior_mean_recovered():
    prior, ll = gaussian_problem(d=2, sig=0.03, mu=[0.3, 0.7])
    res = ns.NestedSlice(prior, ll, n_live=150, num_delete=30, seed=4).run()
    w = np.exp(res.dead_logL + res.dead_logw - res.logZ)
    mean = (w[:, None] * res.dead_theta).sum(axis=0) / w.sum()
    np.testing.assert_allclose(mean, [0.3, 0.7], atol=0.01)


def test_region_prior_transform():
    pr = ns.region_model_prior(3)
    u = np.array([[0.0, 0.5, 1.0, 0.0, 0.5, 1.0, 0.5]])
    th = pr.transform(u)[0]
    np.testing.assert_allclose(th[:3], [2.45, 2.8, 3.15])
    np.testing.assert_allclose(th[3:6], [0.0, 125.0, 40.0])
    np.testing.assert_allclose(th[6], math.sqrt(1e-3 * 0.1))     # log-uniform midpoint


def test_checkpoint_resume_is_exact():
    """A run stopped after a few iterations, checkpointed (through pickle, as a
    file would hold it) and resumed by a fresh sampler ends exactly where the
    uninterrupted run ends: same evidence, same dead points, same counters."""
    import pickle
    prior, ll = gaussian_problem(d=3, sig=0.1)
    kw = dict(n_live=100, num_delete=20, num_inner_steps=6)
    full = ns.NestedSlice(prior, ll, seed=5, **kw).run()
    first = ns.NestedSlice(prior, ll, seed=5, **kw)
    assert first.run(stop_after=7) is None
    state = pickle.loads(pickle.dumps(first.state_dict()))
    assert state["it"] == 7
    resumed = ns.NestedSlice(prior, ll, seed=999, **kw).run(resume=state)   # the checkpoint's generator takes over
    assert resumed.logZ == full.logZ and resumed.H == full.H
    assert resumed.n_like == full.n_like and resumed.n_rounds == full.n_rounds
    assert resumed.iterations == full.iterations
    assert np.array_equal(resumed.dead_logL, full.dead_logL)
    assert np.array_equal(resumed.dead_theta, full.dead_theta)
    with pytest.raises(ValueError):
        ns.NestedSlice(prior, ll, seed=5, n_live=50, num_delete=20, num_inner_steps=6).run(resume=state)
