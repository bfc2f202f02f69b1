"""The two mixed workloads at their full sizes, in the launch configurations the
library runs them in, checked on sampled outputs the oracle evaluates one by one:

- workload 4: 32 instances (N 4..30, T 1..60, P 256..8192 prior draws, each with
  its own sky window and partition) in one persistent launch (fg21_loglike_multi)
  and in a captured multi-model graph, which must equal the launch bit for bit;
- workload 5: the serving mix, 64 runs (N in {5,9,14,20,30}, T in {1,10,50}) and
  its 256 requests of 128..4096 points (550,000 points in all) submitted from
  several threads at once; each sampled request equals the same points evaluated
  alone bit for bit."""
import threading

import numpy as np
import pytest

import cases
import oracle as O
from conftest import report
from paper_2603_13196_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _sample(P, n, seed):
    """n sorted indices in [0, P) that always include the first and last point."""
    g = np.random.default_rng(seed)
    idx = set(g.choice(P, size=min(P, n - 2), replace=False).tolist()) | {0, P - 1}
    return np.array(sorted(idx))


def _check(family, name, om, obs, data, params, got, idx):
    want, dterm = cases.expected(om, obs, data, params[idx])
    tol = cases.logl_tolerance("fp16x3", om, obs, data, params[idx])
    assert np.all(np.isfinite(got))
    return cases.check_logl(family, got[idx], want, tol, name)


def test_workload4_full_size_multi_and_graph(fg21lib):
    torch = pytest.importorskip("torch")
    wls = I.uneven_batch()
    assert len(wls) == 32
    mods = []
    for wl in wls:
        sky, obs = wl.sky(), wl.obs()
        om = O.build_model(sky, obs, wl.N, wl.scheme, wl.weighting)
        data = O.simulate_data(sky, obs, np.array(I.FIDUCIAL_T21), I.NOISE_K, wl.noise())
        m = fg21lib.fg21_build_regions(sky, obs, wl.N, wl.scheme, wl.weighting)
        assert np.array_equal(m.labels, om.labels), wl.name
        fg21lib.fg21_model_set_data(m, data)
        mods.append((wl, obs, om, data, m))
    params = [wl.params() for wl in wls]
    got = fg21lib.fg21_loglike_multi([x[4] for x in mods], params, "fp16x3")
    worst = 0.0
    for k, ((wl, obs, om, data, m), p, g) in enumerate(zip(mods, params, got)):
        worst = max(worst, _check("w4_full_multi", wl.name, om, obs, data, p, g, _sample(p.shape[0], 12, k)))

    # the same batch captured as one graph on device buffers
    dps = [torch.from_numpy(p).cuda() for p in params]
    dls = [torch.empty(p.shape[0], dtype=torch.float64, device="cuda") for p in params]
    s = torch.cuda.current_stream().cuda_stream
    g = fg21lib.fg21_graph_create_multi([x[4] for x in mods], [t.data_ptr() for t in dps],
                                        [p.shape[0] for p in params], [t.data_ptr() for t in dls], "fp16x3")
    g.launch(s)
    assert g.sync_status(s) == 0
    for k, (t, ref) in enumerate(zip(dls, got)):
        assert np.array_equal(t.cpu().numpy(), ref), wls[k].name
    g.close()
    report("w4_full_multi", models=len(wls), points=int(sum(p.shape[0] for p in params)), max_err_over_tol=worst)
    for x in mods:
        x[4].close()


def test_workload5_full_size_served_mix(fg21lib):
    runs, reqs = I.serving_mix()
    assert len(runs) == 64 and len(reqs) == 256
    srv = fg21lib.Server(mem_budget_bytes=60 << 30, max_batch_points=65536, max_wait_us=200, max_inflight=2)
    models, datas, rids = [], [], []
    for run in runs:
        sky, obs = run.sky(), run.obs()
        data = O.simulate_data(sky, obs, np.array(I.FIDUCIAL_T21), I.NOISE_K, run.noise())
        m = fg21lib.fg21_build_regions(sky, obs, run.N, "recursive")
        fg21lib.fg21_model_set_data(m, data)
        rid, admitted = fg21lib.fg21_serve_register_run(srv, m)
        assert admitted
        models.append(m)
        datas.append(data)
        rids.append(rid)
    results = [None] * len(reqs)
    codes = [None] * len(reqs)

    def client(idx):
        for j in idx:
            k, p = reqs[j]
            t, out = fg21lib.fg21_serve_submit(srv, rids[k], p)
            codes[j] = fg21lib.fg21_serve_wait(srv, t, 120000)
            results[j] = out.copy()

    ths = [threading.Thread(target=client, args=(list(range(c, len(reqs), 8)),)) for c in range(8)]
    [t.start() for t in ths]
    [t.join() for t in ths]
    st = fg21lib.fg21_serve_stats(srv)
    assert all(c == 0 for c in codes)
    assert st["requests_done"] == len(reqs)
    # every 8th request: alone = mixed bit for bit, and 12 sampled points against the oracle
    oracle_models = {}
    worst = 0.0
    for j in range(0, len(reqs), 8):
        k, p = reqs[j]
        run = runs[k]
        assert np.array_equal(fg21lib.fg21_loglike_batch(models[k], p, "fp16x3"), results[j]), j
        if k not in oracle_models:
            oracle_models[k] = O.build_model(run.sky(), run.obs(), run.N, "recursive")
            assert np.array_equal(models[k].labels, oracle_models[k].labels), k
        worst = max(worst, _check("w5_served_mix", f"req{j}_run{k}", oracle_models[k], run.obs(), datas[k], p, results[j],
                                  _sample(p.shape[0], 12, j)))
    report("w5_full_served", requests=len(reqs), points=int(sum(p.shape[0] for _, p in reqs)),
           launches=st["launches"], p50_ms=st["p50_ms"], p99_ms=st["p99_ms"], max_err_over_tol=worst)
    srv.close()
    for m in models:
        m.close()
