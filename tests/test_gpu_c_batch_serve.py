"""GPU tests of the uneven multi-model launch and of the continuous-batching
server: every request's result equals the oracle within tolerance and is
bit-identical alone and in the mix; admission by memory budget; cancellation;
unregistering a run with queued requests."""
import threading

import numpy as np
import pytest

import cases
import oracle as O
from conftest import report
from paper_2603_13196_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _models(fg21lib, wls):
    out = []
    for wl in wls:
        sky, obs = wl.sky(), wl.obs()
        om = O.build_model(sky, obs, wl.N, wl.scheme, wl.weighting)
        data = O.simulate_data(sky, obs, np.array(I.FIDUCIAL_T21), I.NOISE_K, wl.noise())
        m = fg21lib.fg21_build_regions(sky, obs, wl.N, wl.scheme, wl.weighting)
        assert np.array_equal(m.labels, om.labels)
        fg21lib.fg21_model_set_data(m, data)
        out.append((wl, obs, om, data, m))
    return out


@pytest.fixture(scope="module")
def uneven(fg21lib):
    wls = I.uneven_batch(8, P_range=(100, 700))
    return _models(fg21lib, wls)


def test_multi_matches_oracle_and_single(fg21lib, uneven):
    params = [wl.params() for wl, *_ in uneven]
    got = fg21lib.fg21_loglike_multi([m for *_, m in uneven], params, "fp16x3")
    for (wl, obs, om, data, m), p, g in zip(uneven, params, got):
        want, dterm = cases.expected(om, obs, data, p)
        tol = cases.logl_tolerance("fp16x3", om, obs, data, p)
        report(f"multi_{wl.name}", max_abs=np.max(np.abs(g - want)))
        cases.check_logl("multi_fp16x3", g, want, tol, wl.name)
        single = fg21lib.fg21_loglike_batch(m, p, "fp16x3")
        assert np.array_equal(single, g), wl.name       # same work split alone and batched


def test_multi_simt_precisions(fg21lib, uneven):
    sub = uneven[:3]
    params = [wl.params() for wl, *_ in sub]
    for prec in ("fp32_delta", "fp32_direct"):
        got = fg21lib.fg21_loglike_multi([m for *_, m in sub], params, prec)
        for (wl, obs, om, data, m), p, g in zip(sub, params, got):
            want, dterm = cases.expected(om, obs, data, p)
            cases.check_logl(f"multi_{prec}", g, want, cases.logl_tolerance(prec, om, obs, data, p), wl.name)


def test_serve_alone_equals_mixed(fg21lib, uneven):
    srv = fg21lib.Server(mem_budget_bytes=1 << 34, max_batch_points=4096, max_wait_us=2000, max_inflight=2)
    runs = []
    for wl, obs, om, data, m in uneven:
        rid, admitted = fg21lib.fg21_serve_register_run(srv, m)
        assert admitted
        runs.append(rid)
    reqs = []
    rng = I.rng(3, I.SUB_ARRIVALS)
    for j in range(24):
        k = int(rng.integers(0, len(uneven)))
        wl = uneven[k][0]
        P = int(rng.integers(1, 400))
        reqs.append((k, I.prior_draws(P, wl.N, seed=j, extra=k)))
    # mixed: submitted from several threads at once
    results = [None] * len(reqs)

    def client(idx):
        for j in idx:
            k, p = reqs[j]
            t, out = fg21lib.fg21_serve_submit(srv, runs[k], p)
            assert fg21lib.fg21_serve_wait(srv, t, 60000) == 0
            results[j] = out.copy()

    ths = [threading.Thread(target=client, args=(list(range(c, len(reqs), 4)),)) for c in range(4)]
    [t.start() for t in ths]
    [t.join() for t in ths]
    st = fg21lib.fg21_serve_stats(srv)
    report("serve_mixed", p50_ms=st["p50_ms"], p99_ms=st["p99_ms"], launches=st["launches"],
           requests=st["requests_done"])
    assert st["requests_done"] == len(reqs)
    assert st["launches"] <= len(reqs)
    for j, (k, p) in enumerate(reqs):
        wl, obs, om, data, m = uneven[k]
        alone = fg21lib.fg21_loglike_batch(m, p, "fp16x3")
        assert np.array_equal(alone, results[j]), j
        want, dterm = cases.expected(om, obs, data, p)
        cases.check_logl("serve_mixed_fp16x3", results[j], want, cases.logl_tolerance("fp16x3", om, obs, data, p),
                         str(j))
    srv.close()


def test_serve_admission_cancel_unregister(fg21lib):
    # three runs of one shape (equal resident bytes), a budget that holds one
    wls = [I.Workload(f"adm{k}", 1024, 6, 41, 5, 3.0, 64, seed=900 + k) for k in range(3)]
    mods = _models(fg21lib, wls)
    size = fg21lib.fg21_model_info(mods[0][4])["device_bytes"]
    assert all(fg21lib.fg21_model_info(x[4])["device_bytes"] == size for x in mods)
    srv = fg21lib.Server(mem_budget_bytes=int(1.5 * size), max_batch_points=4096, max_wait_us=100,
                         max_inflight=1)
    r0, a0 = fg21lib.fg21_serve_register_run(srv, mods[0][4])
    r1, a1 = fg21lib.fg21_serve_register_run(srv, mods[1][4])
    assert a0 and not a1
    st = fg21lib.fg21_serve_stats(srv)
    assert st["runs_admitted"] == 1 and st["runs_waiting"] == 1
    p1 = wls[1].params(50)
    t1, out1 = fg21lib.fg21_serve_submit(srv, r1, p1)
    assert fg21lib.fg21_serve_wait(srv, t1, 200) == fg21lib.FG21_E_TIMEOUT    # waiting for admission
    t_c, _ = fg21lib.fg21_serve_submit(srv, r1, p1)
    assert fg21lib.fg21_serve_cancel(srv, t_c) == 0
    assert fg21lib.fg21_serve_wait(srv, t_c, 1000) == fg21lib.FG21_E_CANCELLED
    fg21lib.fg21_serve_unregister_run(srv, r0)          # frees budget -> r1 admitted
    assert fg21lib.fg21_serve_wait(srv, t1, 60000) == 0
    assert np.array_equal(out1, fg21lib.fg21_loglike_batch(mods[1][4], p1, "fp16x3"))
    # a queued request of a run that goes away completes as cancelled
    r2, a2 = fg21lib.fg21_serve_register_run(srv, mods[2][4])
    assert not a2
    t2, _ = fg21lib.fg21_serve_submit(srv, r2, wls[2].params(10))
    fg21lib.fg21_serve_unregister_run(srv, r2)
    assert fg21lib.fg21_serve_wait(srv, t2, 1000) == fg21lib.FG21_E_CANCELLED
    # a run larger than the whole budget is refused
    big = I.Workload("big", 1024, 12, 41, 9, 3.0, 64, seed=990)
    bm = _models(fg21lib, [big])[0][4]
    with pytest.raises(fg21lib.Fg21Error) as e:
        fg21lib.fg21_serve_register_run(srv, bm)
    assert e.value.code == fg21lib.FG21_E_RANGE
    srv.close()
