"""GPU parity of the accuracy-criterion workload (Sec. 5.2.2) against the FP64
oracle: the noise-only likelihood distribution L_noise over Philox4x32-10 /
Box-Muller realisations (odd and even cell counts, the benchmark's F*T, noise
and likelihood widths that differ), bit-for-bit reproducibility, the device
q count, and the same numbers through the main likelihood kernel on data
that the model describes up to the drawn noise."""
import math

import numpy as np
import pytest

import cases
import oracle as O
from conftest import report
from paper_2603_13196_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _gpu_noise(fg21lib, n, s_noise, s_n, K, seed):
    d = torch.empty(K, dtype=torch.float64, device="cuda:0")
    fg21lib.fg21_noise_loglike(n, s_noise, s_n, K, seed, d.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return d


def _tolerance(L, n, s_noise, s_n):
    """FP32 logarithm of u = (x + 1) / 2^32: |d r^2| <= 2^-22 (1 + r^2 / 2) per
    pair, so |dL| <= 1/2 (s_noise/s_n)^2 2^-22 (n + S) with S = sum z^2; x4
    headroom, plus FP64 rounding of the sums."""
    ratio2 = (s_noise / s_n) ** 2
    S = (-2.0 * L - n * math.log(2 * math.pi * s_n * s_n)) / max(ratio2, 1e-300)
    return 4.0 * 0.5 * ratio2 * 2.0 ** -22 * (n + S) + 1e-10 * np.abs(L)


@pytest.mark.parametrize("n,s_noise,s_n,K", [(30100, 0.025, 0.025, 128), (51, 0.025, 0.025, 2000),
                                             (1, 0.02, 0.01, 500), (2, 0.025, 0.03, 500), (4097, 0.0, 0.025, 64)])
def test_noise_loglike_matches_oracle(fg21lib, n, s_noise, s_n, K):
    seed = 2603131960 + n
    got = _gpu_noise(fg21lib, n, s_noise, s_n, K, seed).cpu().numpy()
    want = O.noise_loglike(n, s_noise, s_n, K, seed)
    tol = _tolerance(want, n, s_noise, s_n)
    report(f"noise_{n}_{K}", max_abs=np.max(np.abs(got - want)), max_err_over_tol=np.max(np.abs(got - want) / tol))
    cases.check_logl(f"noise_{n}_{K}", got, want, tol)


def test_noise_reproducible_and_seeded(fg21lib):
    a = _gpu_noise(fg21lib, 30100, 0.025, 0.025, 300, 11)
    b = _gpu_noise(fg21lib, 30100, 0.025, 0.025, 300, 11)
    c = _gpu_noise(fg21lib, 30100, 0.025, 0.025, 300, 12)
    assert torch.equal(a, b)
    assert not torch.equal(a, c)
    # realisation k does not depend on K (counter-based draws)
    d = _gpu_noise(fg21lib, 30100, 0.025, 0.025, 100, 11)
    assert torch.equal(a[:100], d)


def test_noise_q_device_count(fg21lib):
    """q on the device equals the oracle's count over the same values, and is
    near the analytic lower-tail probability of the scaled chi-square law."""
    n, s, K = 30100, 0.025, 4096
    d = _gpu_noise(fg21lib, n, s, s, K, 5)
    L = d.cpu().numpy()
    L_bar = np.concatenate([np.quantile(L, [0.0, 0.01, 0.37, 0.5, 1.0]), [L.min() - 1.0, L.max() + 1.0], L[:5]])
    q = fg21lib.fg21_noise_q(d.data_ptr(), K, L_bar)
    np.testing.assert_array_equal(q, O.noise_q(L, L_bar))
    import scipy.stats
    for p in (0.01, 0.1, 0.5):
        c = scipy.stats.chi2(df=n).ppf(1.0 - p)
        Lp = -0.5 * (n * math.log(2 * math.pi * s * s) + c)
        qp = fg21lib.fg21_noise_q(d.data_ptr(), K, [Lp])[0]
        assert abs(qp - p) < 4 * math.sqrt(p * (1 - p) / K) + 1e-3, (p, qp)


def test_noise_loglike_through_the_likelihood_kernel(fg21lib):
    """L_noise[k] is the likelihood of theta against data = M(theta) + the
    realisation's noise: the same numbers from fg21_loglike_batch (FP32 delta and
    FP16 split forms) on those data vectors, within their tolerances."""
    sky, obs, m, _ = cases.small_case(npix=2048, N=5, F=31, T=7, window=4.0)
    model = fg21lib.fg21_build_regions(sky, obs, 5)
    n, s, K, seed = obs.F * obs.T, I.NOISE_K, 6, 77
    theta = np.concatenate([O.region_truth(sky, m.labels, 5), [0.155, 85.0, 15.0, s]])
    M = O.fast_model(m.A, m.B, obs, theta)[0]
    z = O.noise_draws(n, K, seed).reshape(K, obs.F, obs.T)
    L_gpu = _gpu_noise(fg21lib, n, s, s, K, seed).cpu().numpy()
    for k in range(K):
        data = M + s * z[k]
        fg21lib.fg21_model_set_data(model, data)
        pts = np.repeat(theta[None], 3, axis=0)
        for prec in ("fp32_delta", "fp16x3"):
            got = fg21lib.fg21_loglike_batch(model, pts, prec)
            tol = cases.logl_tolerance(prec, m, obs, data, pts)
            cases.check_logl(f"noise_through_likelihood_{prec}", got, np.full(3, L_gpu[k]),
                             tol + _tolerance(L_gpu[k:k + 1], n, s, s), str(k))


def test_noise_argument_errors(fg21lib):
    d = torch.empty(4, dtype=torch.float64, device="cuda:0")
    for args in ((0, 0.025, 0.025, 4), (10, 0.025, 0.0, 4), (10, -1.0, 0.025, 4), (10, 0.025, 0.025, -1)):
        with pytest.raises(fg21lib.Fg21Error) as e:
            fg21lib.fg21_noise_loglike(*args, 1, d.data_ptr())
        assert e.value.code == fg21lib.FG21_E_ARG
    fg21lib.fg21_noise_loglike(10, 0.025, 0.025, 0, 1, d.data_ptr())      # K = 0: nothing to do
