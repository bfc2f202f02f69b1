"""The seeded input generator (shared by the oracle and the library tests): each
workload constructor is reproducible and draws within its stated ranges."""
import numpy as np

from paper_2603_13196_gb300 import inputs as I


def test_workloads_1_to_3():
    sizes = {1: (3072, 3, 151, 1, 64), 2: (12288, 9, 151, 20, 4096), 3: (49152, 24, 301, 100, 16384)}
    for k, (npix, N, F, T, P) in sizes.items():
        wl = I.workload(k)
        assert (wl.npix, wl.N, wl.F, wl.T, wl.P) == (npix, N, F, T, P)
        p1, p2 = wl.params(P=32), wl.params(P=32)
        assert np.array_equal(p1, p2) and p1.shape == (32, N + 4)
        assert np.all((p1[:, :N] >= 2.45) & (p1[:, :N] <= 3.15))
        assert np.all((p1[:, -1] >= 1e-3) & (p1[:, -1] <= 0.1))        # sigma_n, log-uniform range
        assert not np.array_equal(wl.params(P=32, extra=1), p1)        # replicas draw other batches


def test_uneven_batch_ranges_and_reproducibility():
    a, b = I.uneven_batch(), I.uneven_batch()
    assert len(a) == 32
    assert [(w.N, w.T, w.P, w.lst0_h) for w in a] == [(w.N, w.T, w.P, w.lst0_h) for w in b]
    assert all(4 <= w.N <= 30 and 1 <= w.T <= 60 and 256 <= w.P <= 8192 for w in a)
    assert all((w.window_h == 0.0) == (w.T == 1) for w in a)
    assert len({w.N for w in a}) > 5 and len({w.T for w in a}) > 5      # a real mix


def test_serving_mix():
    runs, reqs = I.serving_mix()
    runs2, reqs2 = I.serving_mix()
    assert len(runs) == 64 and len(reqs) == 256
    assert [(r.N, r.T) for r in runs[:15]] == [(n, t) for t in (1, 10, 50) for n in (5, 9, 14, 20, 30)]
    assert all((r.window_h == 0.0) == (r.T == 1) for r in runs)
    assert all(0 <= k < 64 and 128 <= p.shape[0] <= 4096 and p.shape[1] == runs[k].N + 4 for k, p in reqs)
    assert all(k == k2 and np.array_equal(p, p2) for (k, p), (k2, p2) in zip(reqs, reqs2))
    assert runs[3].obs().T == runs[3].T and runs[3].sky().npix == 3072
