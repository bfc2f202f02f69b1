"""End to end: batched nested slice sampling fed by libfg21's serving loop
reaches the log-evidence of the same sampler fed by the FP64 oracle, within
sampling error (independent seeds)."""
import math

import numpy as np
import pytest

import oracle as O
from conftest import report
from paper_2603_13196_gb300 import inputs as I, ns

pytestmark = pytest.mark.gpu


def problem():
    sky = I.make_sky(1024, 31)
    obs = I.make_obs(51, 1, 0.0, lst0_h=5.0)
    N = 3
    om = O.build_model(sky, obs, N, "hierarchical")
    truth = np.concatenate([O.region_truth(sky, om.labels, N, om.w), [0.155, 85.0, 15.0, 0.025]])
    data = O.fast_model(om.A, om.B, obs, truth)[0] + 0.025 * I.noise_draws(obs.F, obs.T, 31)
    return sky, obs, N, om, data, truth


def test_evidence_gpu_serve_vs_oracle(fg21lib):
    sky, obs, N, om, data, truth = problem()
    prior = ns.region_model_prior(N)
    model = fg21lib.fg21_build_regions(sky, obs, N, "hierarchical")
    fg21lib.fg21_model_set_data(model, data)
    srv = fg21lib.Server(mem_budget_bytes=1 << 30, max_batch_points=8192, max_wait_us=0, max_inflight=2)
    like = ns.ServeLikelihood(fg21lib, srv, model)
    kw = dict(n_live=200, num_delete=40, num_inner_steps=5 * prior.dim)
    gpu = ns.NestedSlice(prior, like, seed=11, **kw).run()
    like.close()
    st = fg21lib.fg21_serve_stats(srv)
    srv.close()
    orc = ns.NestedSlice(prior, lambda th: O.loglike(om.A, om.B, data, obs, th), seed=12, **kw).run()
    err = math.sqrt(gpu.logZ_err ** 2 + orc.logZ_err ** 2)
    report("ns_evidence", logZ_gpu=gpu.logZ, logZ_oracle=orc.logZ, err=err, H=gpu.H, n_like=gpu.n_like,
           rounds=gpu.n_rounds, p50_ms=st["p50_ms"], p99_ms=st["p99_ms"], logLmax_gpu=gpu.logL_max,
           logLmax_oracle=orc.logL_max)
    assert abs(gpu.logZ - orc.logZ) < 3.0 * err, (gpu.logZ, orc.logZ, err)
    # the best-fit likelihood is the noise floor of the exact model: chi2 ~ F T
    floor = -0.5 * obs.F * obs.T * math.log(2 * math.pi * 0.025 ** 2) - 0.5 * obs.F * obs.T
    assert abs(gpu.logL_max - floor) < 4 * math.sqrt(obs.F * obs.T)


def test_evidence_serving_size(fg21lib):
    """A run of the serving workload's size (9 regions, F = 151, T = 10, n_live
    500, 128 deletions per iteration, 5 D inner steps) fed by the serving loop
    reaches the log-evidence of the same sampler fed by the FP64 oracle
    (tests/golden/ns_serving_reference.json, written by
    make_ns_serving_reference.py, an independent seed) within twice their
    combined sampling error sqrt(H / n_live); its best likelihood is near the
    likelihood of the truth."""
    import json
    import os
    import cases
    ref = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                      "ns_serving_reference.json")))
    sky, obs, om, data, truth, prior = cases.ns_serving_problem()
    c = cases.NS_SERVING
    model = fg21lib.fg21_build_regions(sky, obs, c["N"], "recursive")
    assert np.array_equal(model.labels, om.labels)
    fg21lib.fg21_model_set_data(model, data)
    srv = fg21lib.Server(mem_budget_bytes=1 << 30, max_batch_points=8192, max_wait_us=0, max_inflight=2)
    like = ns.ServeLikelihood(fg21lib, srv, model)
    r = ns.NestedSlice(prior, like, n_live=c["n_live"], num_delete=c["num_delete"],
                       num_inner_steps=5 * prior.dim, seed=2002).run()
    like.close()
    st = fg21lib.fg21_serve_stats(srv)
    srv.close()
    err = math.sqrt(r.logZ_err ** 2 + ref["logZ_err"] ** 2)
    report("ns_evidence_serving_size", logZ_gpu=r.logZ, logZ_oracle=ref["logZ"], err=err, H=r.H,
           n_like=r.n_like, rounds=r.n_rounds, p50_ms=st["p50_ms"], p99_ms=st["p99_ms"], logLmax_gpu=r.logL_max,
           logL_truth=ref["logL_truth"])
    assert abs(r.logZ - ref["logZ"]) < 2.0 * err, (r.logZ, ref["logZ"], err)
    assert r.logL_max > ref["logL_truth"] - 3.0 * prior.dim, (r.logL_max, ref["logL_truth"])
