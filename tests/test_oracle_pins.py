"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's formula: each checks a closed form, an
invariant, a library routine, a second independent route, or brute force
from the definitions on tiny inputs, so that a dropped term, a wrong sign or
index, or a transposed operand in oracle/fg21_oracle.c fails at least one of
them (tests/test_oracle_mutations.py plants such mistakes and checks that).
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.stats

import oracle as O
from paper_2603_13196_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def small_case(npix=3072, F=21, T=3, window=6.0, seed=11, **kw):
    sky = I.make_sky(npix, seed, **{k: v for k, v in kw.items() if k in ("beta_const", "t230_const")})
    obs = I.make_obs(F, T, window, lst0_h=kw.get("lst0_h", 17.0), achromatic_p=kw.get("achromatic_p"),
                     lo=kw.get("lo", 50.0), hi=kw.get("hi", 200.0))
    return sky, obs


# ----------------------------------------------------------------- constants

def test_paper_constants_fixture_matches_inputs():
    g = json.load(open(GOLDEN))
    assert I.FIDUCIAL_T21 == (g["t21_fiducial"]["A21_K"], g["t21_fiducial"]["nu21_MHz"],
                              g["t21_fiducial"]["sigma21_MHz"])
    assert I.NOISE_K == g["noise_K"]["value"]
    assert I.NU0_MHZ == g["nu0_MHz"]["value"]


def test_t21_special_values():
    """eq. t21model at the fiducial trough: peak A21 at nu21, e^-1/2 one width
    away, e^-2 two widths away, symmetric about nu21."""
    g = json.load(open(GOLDEN))["t21_fiducial"]
    a, c, s = g["A21_K"], g["nu21_MHz"], g["sigma21_MHz"]
    v = O.t21([c, c + s, c - s, c + 2 * s, c - 2 * s], a, c, s)
    np.testing.assert_allclose(v, [a, a * math.exp(-0.5), a * math.exp(-0.5), a * math.exp(-2),
                                   a * math.exp(-2)], rtol=1e-15)
    # a negative width is the same trough; zero amplitude is flat zero
    np.testing.assert_allclose(O.t21([70.0], a, c, -s), O.t21([70.0], a, c, s), rtol=0)
    assert O.t21([70.0], 0.0, c, s)[0] == 0.0


# ---------------------------------------------------------------------- beam

@pytest.mark.parametrize("p", [0.0, 1.2, 1.8])
def test_beam_is_a_directivity(p):
    """(1/4pi) integral D dOmega = 1 for D = 2(p+1)cos^p above the horizon
    (hemisphere integral of cos^p is 2pi/(p+1)); on the Fibonacci sphere the
    discrete B[f,t] converges to 1 as Npix grows."""
    errs = []
    for npix in (768, 3072, 12288):
        sky, obs = small_case(npix=npix, F=3, T=4, achromatic_p=p)
        labels = np.zeros(npix, dtype=np.int32)
        _, B = O.precompute(sky, obs, labels, 1)
        errs.append(np.max(np.abs(B - 1.0)))
    # the flat beam (p = 0) has a step at the horizon, so pixel counting converges slowly
    assert errs[1] < (1e-2 if p == 0.0 else 1e-4)
    assert errs[2] < errs[0]


def test_flat_beam_counts_pixels_above_horizon():
    """p = 0: D = 2 on the visible hemisphere, so A = (T0 - T_CMB) * 2 n_up / Npix and
    B = 2 n_up / Npix for a constant sky, n_up = pixels with z.v > 0."""
    T0 = 500.0
    sky, obs = small_case(npix=3072, F=4, T=3, achromatic_p=0.0, t230_const=T0)
    labels = np.zeros(sky.npix, dtype=np.int32)
    A, B = O.precompute(sky, obs, labels, 1)
    for t in range(obs.T):
        n_up = int(np.sum(sky.dirs @ obs.zenith[t] > 0))
        np.testing.assert_allclose(B[:, t], 2.0 * n_up / sky.npix, rtol=1e-13)
        np.testing.assert_allclose(A[0, :, t], (T0 - I.T_CMB) * 2.0 * n_up / sky.npix, rtol=1e-13)


# ----------------------------------------------------- forward model routes

@pytest.mark.parametrize("scheme,N", [("recursive", 5), ("hierarchical", 6), ("linear", 4)])
def test_fast_model_equals_pixel_model(scheme, N):
    """eq. fast_forward_model with precomputed A equals eq. forward_model integrated
    per pixel (linearity of the beam integral), for arbitrary per-region beta."""
    sky, obs = small_case(npix=1536, F=9, T=3)
    m = O.build_model(sky, obs, N, scheme)
    th = I.prior_draws(4, N, seed=5)
    M1 = O.fast_model(m.A, m.B, obs, th)
    M2 = O.pixel_model(sky, obs, m.labels, N, th)
    np.testing.assert_allclose(M1, M2, rtol=1e-11)


def test_single_region_is_a_power_law():
    """N = 1, achromatic beam, T = 1: M - T_CMB B - T21 = S (nu/nu0)^-beta, so
    ln of it is linear in ln nu with slope -beta and equals S at nu = nu0,
    where S is the beam-weighted template; with a flat beam (p = 0) and a
    constant template T0, S = (T0 - T_CMB) 2 n_up / Npix."""
    T0 = 700.0
    sky, obs = small_case(npix=3072, F=16, T=1, achromatic_p=0.0, t230_const=T0, lo=50.0, hi=230.0)
    m = O.build_model(sky, obs, 1, "recursive")
    beta = 2.71
    th = np.array([[beta, 0.0, 100.0, 10.0, 0.01]])
    M = O.fast_model(m.A, m.B, obs, th)[0, :, 0]
    y = np.log(M - I.T_CMB * m.B[:, 0])
    slope, icpt = np.polyfit(np.log(obs.nu), y, 1)
    assert abs(slope + beta) < 1e-11
    n_up = int(np.sum(sky.dirs @ obs.zenith[0] > 0))
    S = (T0 - I.T_CMB) * 2.0 * n_up / sky.npix
    assert obs.nu[-1] == 230.0
    np.testing.assert_allclose(M[-1] - I.T_CMB * m.B[-1, 0], S, rtol=1e-12)


@pytest.mark.parametrize("scheme,N", [("recursive", 7), ("hierarchical", 5), ("linear", 4),
                                      ("percentile", 3)])
def test_equal_beta_collapse(scheme, N):
    """All beta_i equal: sum_i A_i (nu/nu0)^-beta collapses to one power law of the
    summed beam-weighted sky, independent of the partition (the A_i partition
    the template)."""
    sky, obs = small_case(npix=2048, F=7, T=2)
    ref = O.build_model(sky, obs, 1, "recursive")
    m = O.build_model(sky, obs, N, scheme)
    np.testing.assert_allclose(m.A.sum(axis=0), ref.A[0], rtol=1e-12)
    th1 = np.array([[2.6, 0.1, 80.0, 12.0, 0.02]])
    thN = np.concatenate([[2.6] * N, [0.1, 80.0, 12.0, 0.02]])[None, :]
    np.testing.assert_allclose(O.fast_model(m.A, m.B, obs, thN), O.fast_model(ref.A, ref.B, obs, th1),
                               rtol=1e-12)


def test_constant_beta_sky_reproduces_simulated_data():
    """A sky with one spectral index everywhere is exactly an N-region model at
    beta_i = beta0: eq. simantenna (noise-free) equals eq. fast_forward_model + T21."""
    beta0 = 2.63
    sky, obs = small_case(npix=2048, F=11, T=3, beta_const=beta0)
    m = O.build_model(sky, obs, 3, "percentile")
    t21p = np.array(I.FIDUCIAL_T21)
    data = O.simulate_data(sky, obs, t21p)
    th = np.concatenate([[beta0] * 3, t21p, [0.025]])[None, :]
    np.testing.assert_allclose(O.fast_model(m.A, m.B, obs, th)[0], data, rtol=1e-12)


def test_simulated_data_closed_form():
    """Flat beam, constant template T0, constant beta: the antenna temperature is
    (2 n_up/Npix) [(T0 - T_CMB)(nu/nu0)^-beta + T_CMB] + T21 + sigma * noise."""
    T0, beta0 = 400.0, 2.5
    sky, obs = small_case(npix=1024, F=6, T=2, achromatic_p=0.0, t230_const=T0, beta_const=beta0)
    t21p = np.array([0.2, 120.0, 20.0])
    noise = I.noise_draws(obs.F, obs.T, 3)
    data = O.simulate_data(sky, obs, t21p, 0.025, noise)
    for t in range(obs.T):
        frac = 2.0 * np.sum(sky.dirs @ obs.zenith[t] > 0) / sky.npix
        sky_t = frac * ((T0 - I.T_CMB) * (obs.nu / I.NU0_MHZ) ** (-beta0) + I.T_CMB)
        trough = 0.2 * np.exp(-0.5 * ((obs.nu - 120.0) / 20.0) ** 2)
        np.testing.assert_allclose(data[:, t], sky_t + trough + 0.025 * noise[:, t], rtol=1e-12)


# ----------------------------------------------------------------- likelihood

def test_noiseless_identity():
    """Data equal to the model at theta*: lnL(theta*) = -1/2 F T ln(2 pi sigma^2)."""
    sky, obs = small_case(npix=1024, F=13, T=4)
    m = O.build_model(sky, obs, 4, "recursive")
    th = np.concatenate([O.region_truth(sky, m.labels, 4), [0.155, 85.0, 15.0, 0.025]])[None, :]
    data = O.fast_model(m.A, m.B, obs, th)[0]
    L = O.loglike(m.A, m.B, data, obs, th)[0]
    expect = -0.5 * obs.F * obs.T * math.log(2 * math.pi * 0.025 ** 2)
    assert abs(L - expect) <= 1e-12 * abs(expect)


def test_loglike_is_a_sum_of_gaussian_logpdfs():
    """eq. likelihood equals the sum of scipy's normal log-densities of the data
    about the model with scale sigma_n."""
    sky, obs = small_case(npix=512, F=5, T=2)
    m = O.build_model(sky, obs, 2, "recursive")
    data = O.simulate_data(sky, obs, np.array(I.FIDUCIAL_T21), 0.025, I.noise_draws(5, 2, 1))
    th = I.prior_draws(5, 2, seed=3)
    th[:, :2] = O.region_truth(sky, m.labels, 2) + 1e-4
    L = O.loglike(m.A, m.B, data, obs, th)
    M = O.fast_model(m.A, m.B, obs, th)
    for p in range(5):
        ref = scipy.stats.norm.logpdf(data, loc=M[p], scale=th[p, -1]).sum()
        assert abs(L[p] - ref) <= 1e-10 * abs(ref)
    c2 = O.chi2(m.A, m.B, data, obs, th)
    np.testing.assert_allclose(c2, ((data[None] - M) ** 2).sum(axis=(1, 2)), rtol=1e-12)


# ------------------------------------------------------------------ weighting

def test_weights_special_cases():
    """Each importance map reduces to the simpler one when its extra factor is
    constant: uniform = 1/Npix; horizon with T = 1 = H / n_up; sky weighting of a
    constant sky = horizon weighting; beam weighting with a flat beam (p = 0) =
    sky weighting.  All sum to one."""
    sky, obs = small_case(npix=1024, F=5, T=1)
    w_u = O.weights(sky, obs, "uniform")
    np.testing.assert_allclose(w_u, 1.0 / sky.npix, rtol=1e-14)
    up = (sky.dirs @ obs.zenith[0] > 0)
    w_h = O.weights(sky, obs, "horizon")
    np.testing.assert_allclose(w_h, up / up.sum(), rtol=1e-14, atol=0)
    csky, cobs = small_case(npix=1024, F=5, T=3, t230_const=300.0, beta_const=2.6)
    np.testing.assert_allclose(O.weights(csky, cobs, "sky"), O.weights(csky, cobs, "horizon"),
                               rtol=1e-12)
    fsky, fobs = small_case(npix=1024, F=5, T=3, achromatic_p=0.0)
    np.testing.assert_allclose(O.weights(fsky, fobs, "beam"), O.weights(fsky, fobs, "sky"),
                               rtol=1e-12)
    for wt in ("beam", "sky", "horizon", "uniform"):
        assert abs(O.weights(sky, obs, wt).sum() - 1.0) < 1e-12


def test_beam_weighting_tracks_the_beam():
    """With a constant sky the beam weight of a pixel at time t is proportional to
    D(pix); with T = 1 this is cos^p of the zenith angle, normalised."""
    sky, obs = small_case(npix=1024, F=1, T=1, t230_const=300.0, beta_const=2.6, achromatic_p=1.5,
                          lo=100.0, hi=100.0)
    w = O.weights(sky, obs, "beam")
    c = np.maximum(sky.dirs @ obs.zenith[0], 0.0) ** 1.5
    np.testing.assert_allclose(w, c / c.sum(), rtol=1e-12, atol=1e-300)


# ------------------------------------------------------------------ partition

def _brute_cdf(beta, w, x):
    return sum(wi for bi, wi in zip(beta, w) if bi <= x)


def _brute_cinv(beta, w, c):
    cands = [b for b in sorted(set(beta)) if _brute_cdf(beta, w, b) >= c]
    return cands[0] if cands else max(beta)


def _brute_partition(beta, w, N, scheme):
    """Algorithms 1 and 2 and the Sec. 4.1 splits, straight from the definitions
    (Algorithm 1 refines only base regions, the nested reading):
    C(beta') = sum of w over pixels with beta <= beta' (eq. weighted_cdf), region
    mass = C(b) - C(a) (lowest region: C(b)), intervals kept as python lists."""
    bmin, bmax = min(beta), max(beta)
    if scheme == "recursive":
        R = [(bmin, bmax, True)]
        while len(R) < N:
            def mass(r):
                a, b, low = r
                return _brute_cdf(beta, w, b) - (0.0 if low else _brute_cdf(beta, w, a))
            best = max(range(len(R)), key=lambda k: (mass(R[k]), -R[k][0]))
            a, b, low = R.pop(best)
            mid = 0.5 * (a + b)
            R += [(a, mid, low), (mid, b, False)]
        edges = [bmin] + sorted(r[1] for r in R)
    elif scheme == "hierarchical":
        nb = 2 ** int(math.floor(math.log2(N)))
        cs = [j / nb for j in range(nb + 1)]
        bs = [bmin] + [_brute_cinv(beta, w, c) for c in cs[1:-1]] + [bmax]
        R = [(bs[j], bs[j + 1], cs[j], cs[j + 1], True) for j in range(nb)]
        while len(R) < N:
            cand = [k for k in range(len(R)) if R[k][4]]
            best = max(cand, key=lambda k: (R[k][1] - R[k][0], -R[k][0]))
            a, b, ca, cb, _ = R.pop(best)
            cm = 0.5 * (ca + cb)
            bm = _brute_cinv(beta, w, cm)
            R += [(a, bm, ca, cm, False), (bm, b, cm, cb, False)]
        edges = [bmin] + sorted(r[1] for r in R)
    elif scheme == "linear":
        edges = [bmin] + [bmin + (bmax - bmin) * j / N for j in range(1, N)] + [bmax]
    else:
        sb = sorted(beta)
        n = len(beta)
        edges = [bmin] + [sb[math.ceil(j * n / N) - 1] for j in range(1, N)] + [bmax]
    labels = [sum(1 for e in edges[1:-1] if b > e) for b in beta]
    return edges, labels


@pytest.mark.parametrize("scheme", ["recursive", "hierarchical", "linear", "percentile"])
@pytest.mark.parametrize("seed", range(6))
def test_partition_matches_brute_force(scheme, seed):
    """Tiny maps (<= 16 pixels, tied betas, zero weights, dyadic weights so every
    sum is exact): the sorted-prefix oracle equals the definitions label for label."""
    g = np.random.default_rng(100 + seed)
    npix = int(g.integers(5, 17))
    beta = np.round(g.uniform(2.4, 3.2, npix), 2)            # ties likely
    w = g.integers(0, 9, npix).astype(np.float64)
    w[0] = max(w[0], 1.0)
    w = w / 2.0 ** math.ceil(math.log2(w.sum()))                # dyadic, sum <= 1
    w[np.argmax(w)] += 1.0 - w.sum()                            # exact sum 1
    for N in range(1, 9):
        e_o, l_o, _ = O.partition(beta, w, N, scheme)
        e_b, l_b = _brute_partition(list(beta), list(w), N, scheme)
        assert list(l_o) == l_b, (N, e_o, e_b)
        np.testing.assert_array_equal(e_o, e_b)


@pytest.mark.parametrize("scheme", ["recursive", "hierarchical"])
@pytest.mark.parametrize("weighting", ["beam", "sky", "horizon"])
def test_partitions_are_nested(scheme, weighting):
    """Sec. 4.3: every region at level N is a union of regions at level N+1
    (edge sets grow by inclusion, labels at N are a function of labels at N+1)."""
    sky, obs = small_case(npix=3072, F=9, T=3)
    w = O.weights(sky, obs, weighting)
    prev = None
    for N in range(1, 18):
        edges, labels, _ = O.partition(sky.beta, w, N, scheme)
        assert np.all(np.diff(edges) >= 0)
        if prev is not None:
            pe, pl = prev
            assert set(pe.tolist()) <= set(edges.tolist())
            for j in range(N):
                sel = labels == j
                if sel.any():
                    assert len(np.unique(pl[sel])) == 1
        prev = (edges, labels)


def test_linear_split_is_not_nested():
    """Sec. 4.1: equal-width splits redefine all boundaries (3 -> 4 regions)."""
    sky, obs = small_case(npix=3072, F=3, T=1)
    w = O.weights(sky, obs, "uniform")
    e3, _, _ = O.partition(sky.beta, w, 3, "linear")
    e4, _, _ = O.partition(sky.beta, w, 4, "linear")
    assert not set(e3.tolist()) <= set(e4.tolist())


@pytest.mark.parametrize("N", [2, 4, 8, 16])
def test_hierarchical_base_regions_have_equal_mass(N):
    """Sec. 4.3.1: the N_base regions each hold 1/N_base of the importance, to
    within the largest single pixel weight."""
    sky, obs = small_case(npix=3072, F=9, T=3)
    w = O.weights(sky, obs, "beam")
    _, labels, _ = O.partition(sky.beta, w, N, "hierarchical")
    mass = np.bincount(labels, weights=w, minlength=N)
    assert np.all(np.abs(mass - 1.0 / N) <= w.max() + 1e-15)


def test_recursive_edges_are_dyadic_midpoints():
    """Alg. 2 bisects at beta midpoints: every edge is beta_min + k (beta_max - beta_min)/2^j."""
    sky, obs = small_case(npix=3072, F=9, T=3)
    w = O.weights(sky, obs, "beam")
    edges, _, _ = O.partition(sky.beta, w, 12, "recursive")
    lo, hi = sky.beta.min(), sky.beta.max()
    x = (edges - lo) / (hi - lo) * 2 ** 12
    np.testing.assert_allclose(x, np.round(x), atol=1e-6)


@pytest.mark.parametrize("scheme", ["recursive", "hierarchical"])
def test_embedding_identity(scheme):
    """Nesting makes level N a special case of level N+1: giving both children of
    the split region the parent's beta reproduces T_model and lnL exactly, so
    L_max can only grow with N (Sec. 4.1 and Sec. 6.1)."""
    sky, obs = small_case(npix=2048, F=9, T=3)
    t21p = np.array(I.FIDUCIAL_T21)
    data = O.simulate_data(sky, obs, t21p, 0.025, I.noise_draws(obs.F, obs.T, 9))
    for N in (3, 6, 9):
        mN = O.build_model(sky, obs, N, scheme)
        mN1 = O.build_model(sky, obs, N + 1, scheme)
        thN = I.prior_draws(6, N, seed=N)
        # region j at N+1 is (e'_j, e'_{j+1}]; its parent is the level-N region holding e'_{j+1}
        parent_of = np.array([int(np.sum(mN.edges[1:-1] < mN1.edges[j + 1])) for j in range(N + 1)])
        thN1 = np.concatenate([thN[:, parent_of], thN[:, N:]], axis=1)
        np.testing.assert_allclose(O.fast_model(mN1.A, mN1.B, obs, thN1), O.fast_model(mN.A, mN.B, obs, thN),
                                   rtol=1e-12)
        np.testing.assert_allclose(O.loglike(mN1.A, mN1.B, data, obs, thN1),
                                   O.loglike(mN.A, mN.B, data, obs, thN), rtol=1e-12)


def test_partition_margin_reported():
    """The oracle reports how close its deciding comparisons came to a tie; on
    the synthetic workloads it stays far above FP64 rounding."""
    wl = I.workload(1)
    m = O.build_model(wl.sky(), wl.obs(), wl.N, wl.scheme)
    assert 1e-9 < m.margin <= 1.0


# ------------------------------------------------------------ amplitude masks
# The joint model of eqs. forward_model / chromatic_function /
# fast_forward_model with N_alpha amplitude regions (partitioning a per-pixel
# field, here ln T230 or a direction coordinate) besides the N_beta
# spectral-index regions.

def _ab_model(sky, obs, Nb, Na, scheme="recursive", scheme_a="hierarchical", field=None):
    field = I.amplitude_field(sky) if field is None else field
    return O.build_model_ab(sky, obs, Nb, scheme, "beam", Na, field, scheme_a, "beam")


@pytest.mark.parametrize("scheme,scheme_a,Nb,Na", [("recursive", "hierarchical", 4, 3),
                                                  ("hierarchical", "recursive", 3, 5),
                                                  ("linear", "percentile", 2, 2)])
def test_ab_fast_model_equals_pixel_model(scheme, scheme_a, Nb, Na):
    """eq. fast_forward_model over K (both masks) equals eq. forward_model
    integrated per pixel, for arbitrary alpha and beta."""
    sky, obs = small_case(npix=1024, F=7, T=3)
    m = _ab_model(sky, obs, Nb, Na, scheme, scheme_a)
    th = I.prior_draws_ab(4, Nb, Na, seed=7)
    th[1, Nb:Nb + Na] = [3.0 if i == 1 else 0.0 for i in range(Na)]     # one amplitude region alone
    np.testing.assert_allclose(O.fast_model_ab(m.K, m.B, obs, th),
                               O.pixel_model_ab(sky, obs, m.labels_a, Na, m.labels_b, Nb, th), rtol=1e-11)


def test_ab_unit_amplitudes_reduce_to_beta_model():
    """The amplitude masks partition the template, so sum_i K_ij = A_j of the
    spectral-index model with the same beta regions, and alpha = 1 gives its
    forward model and likelihood."""
    sky, obs = small_case(npix=1536, F=9, T=2)
    m = _ab_model(sky, obs, 5, 3)
    mb = O.build_model(sky, obs, 5, "recursive")
    np.testing.assert_array_equal(m.labels_b, mb.labels)
    np.testing.assert_allclose(m.K.sum(axis=0), mb.A, rtol=1e-12, atol=1e-12 * np.abs(mb.A).max())
    thb = I.prior_draws(3, 5, seed=2)
    thab = np.concatenate([thb[:, :5], np.ones((3, 3)), thb[:, 5:]], axis=1)
    np.testing.assert_allclose(O.fast_model_ab(m.K, m.B, obs, thab), O.fast_model(mb.A, mb.B, obs, thb),
                               rtol=1e-12)
    data = O.simulate_data(sky, obs, np.array(I.FIDUCIAL_T21), 0.025, I.noise_draws(obs.F, obs.T, 4))
    np.testing.assert_allclose(O.loglike_ab(m.K, m.B, data, obs, thab), O.loglike(mb.A, mb.B, data, obs, thb),
                               rtol=1e-12)


def test_ab_scaled_template_reproduces_simulated_data():
    """A constant-beta sky whose template is scaled by a_i on amplitude region i
    (T230' - T_CMB = a_i (T230 - T_CMB)) is exactly the joint model at
    alpha = a, beta_j = beta0: eq. simantenna on the scaled sky (noise-free)
    equals eq. fast_forward_model over the unscaled K."""
    beta0 = 2.58
    sky, obs = small_case(npix=2048, F=9, T=3, beta_const=beta0)
    Na, Nb = 4, 2
    m = _ab_model(sky, obs, Nb, Na, scheme="percentile", scheme_a="recursive", field=sky.dirs[:, 0].copy())
    a = np.array([0.8, 1.25, 1.0, 0.5])
    scaled = I.Sky(dirs=sky.dirs, t230=I.T_CMB + a[m.labels_a] * (sky.t230 - I.T_CMB), beta=sky.beta)
    t21p = np.array(I.FIDUCIAL_T21)
    data = O.simulate_data(scaled, obs, t21p)
    th = np.concatenate([[beta0] * Nb, a, t21p, [0.025]])[None, :]
    np.testing.assert_allclose(O.fast_model_ab(m.K, m.B, obs, th)[0], data, rtol=1e-12)


def test_ab_flat_beam_closed_form():
    """Flat beam (p = 0), constant template T0, T = 1: K[i,j] = (T0 - T_CMB)
    2 n_ij / Npix with n_ij the visible pixels of both regions, so the
    foreground is (T0 - T_CMB)(2/Npix) sum_ij alpha_i n_ij (nu/nu0)^-beta_j."""
    T0 = 600.0
    sky, obs = small_case(npix=1024, F=5, T=1, achromatic_p=0.0, t230_const=T0)
    Na, Nb = 3, 2
    m = _ab_model(sky, obs, Nb, Na, scheme="percentile", scheme_a="linear", field=sky.dirs[:, 1].copy())
    up = sky.dirs @ obs.zenith[0] > 0
    th = np.array([[2.5, 2.9, 0.7, 1.1, 1.4, 0.0, 100.0, 10.0, 0.01]])
    fg = np.zeros(obs.F)
    for i in range(Na):
        for j in range(Nb):
            n_ij = int(np.sum(up & (m.labels_a == i) & (m.labels_b == j)))
            fg += th[0, Nb + i] * (T0 - I.T_CMB) * 2.0 * n_ij / sky.npix * (obs.nu / I.NU0_MHZ) ** (-th[0, j])
    M = O.fast_model_ab(m.K, m.B, obs, th)[0, :, 0]
    np.testing.assert_allclose(M - I.T_CMB * m.B[:, 0], fg, rtol=1e-12)


def test_ab_noiseless_identity_and_gaussian_logpdf():
    """Data = the joint model at theta*: lnL(theta*) = -1/2 F T ln(2 pi sigma^2);
    elsewhere lnL is scipy's sum of normal log-densities about the model."""
    sky, obs = small_case(npix=1024, F=11, T=3)
    Nb, Na = 3, 2
    m = _ab_model(sky, obs, Nb, Na)
    th = np.concatenate([O.region_truth(sky, m.labels_b, Nb), [1.02, 0.97], [0.155, 85.0, 15.0, 0.025]])[None, :]
    data = O.fast_model_ab(m.K, m.B, obs, th)[0]
    L = O.loglike_ab(m.K, m.B, data, obs, th)[0]
    expect = -0.5 * obs.F * obs.T * math.log(2 * math.pi * 0.025 ** 2)
    assert abs(L - expect) <= 1e-12 * abs(expect)
    ths = I.prior_draws_ab(4, Nb, Na, seed=8)
    ths[:, :Nb] = th[0, :Nb] + 1e-4
    Ls = O.loglike_ab(m.K, m.B, data, obs, ths)
    Ms = O.fast_model_ab(m.K, m.B, obs, ths)
    for p in range(4):
        ref = scipy.stats.norm.logpdf(data, loc=Ms[p], scale=ths[p, -1]).sum()
        assert abs(Ls[p] - ref) <= 1e-10 * abs(ref)
    np.testing.assert_allclose(O.chi2_ab(m.K, m.B, data, obs, ths), ((data[None] - Ms) ** 2).sum(axis=(1, 2)),
                               rtol=1e-12)


@pytest.mark.parametrize("scheme_a", ["recursive", "hierarchical"])
def test_ab_amplitude_embedding_identity(scheme_a):
    """Nested amplitude regions: giving both children of the split amplitude
    region the parent's alpha reproduces T_model and lnL at N_alpha + 1."""
    sky, obs = small_case(npix=2048, F=7, T=2)
    data = O.simulate_data(sky, obs, np.array(I.FIDUCIAL_T21), 0.025, I.noise_draws(obs.F, obs.T, 5))
    Nb = 3
    for Na in (2, 3, 5):
        m = _ab_model(sky, obs, Nb, Na, scheme_a=scheme_a)
        m1 = _ab_model(sky, obs, Nb, Na + 1, scheme_a=scheme_a)
        th = I.prior_draws_ab(5, Nb, Na, seed=Na)
        parent_of = np.array([int(np.sum(m.edges_a[1:-1] < m1.edges_a[i + 1])) for i in range(Na + 1)])
        th1 = np.concatenate([th[:, :Nb], th[:, Nb + parent_of], th[:, Nb + Na:]], axis=1)
        np.testing.assert_allclose(O.fast_model_ab(m1.K, m1.B, obs, th1), O.fast_model_ab(m.K, m.B, obs, th),
                                   rtol=1e-12)
        np.testing.assert_allclose(O.loglike_ab(m1.K, m1.B, data, obs, th1),
                                   O.loglike_ab(m.K, m.B, data, obs, th), rtol=1e-12)


def test_ab_amplitude_partition_nested_on_log_template():
    """The partition Algorithms applied to the amplitude field stay nested."""
    sky, obs = small_case(npix=3072, F=5, T=2)
    w = O.weights(sky, obs, "beam")
    field = I.amplitude_field(sky)
    for scheme in ("recursive", "hierarchical"):
        prev = None
        for N in range(1, 10):
            edges, labels, _ = O.partition(field, w, N, scheme)
            if prev is not None:
                assert set(prev[0].tolist()) <= set(edges.tolist())
                for j in range(N):
                    sel = labels == j
                    if sel.any():
                        assert len(np.unique(prev[1][sel])) == 1
            prev = (edges, labels)


# ------------------------------------------------- noise-only likelihood (q_i)
# Sec. 5.2.2: L_noise is the likelihood of data the model describes up to
# Gaussian noise; -2 L_noise - n ln(2 pi sigma_n^2) = (sigma_noise / sigma_n)^2
# chi^2_n exactly, whatever the model.

def test_noise_loglike_is_a_scaled_chi_square():
    """KS test of the oracle's L_noise against the chi-square law (n cells, odd
    and even counts, sigma_noise != sigma_n)."""
    for n, s_noise, s_n in ((51, 0.025, 0.025), (200, 0.025, 0.03), (1, 0.02, 0.01)):
        L = O.noise_loglike(n, s_noise, s_n, 3000, seed=12345 + n)
        x = (-2.0 * L - n * math.log(2 * math.pi * s_n ** 2)) * (s_n / s_noise) ** 2
        p = scipy.stats.kstest(x, scipy.stats.chi2(df=n).cdf).pvalue
        assert p > 1e-3, (n, p)


def test_noise_draws_are_standard_normal_and_independent():
    """Both members of each Box-Muller pair are N(0, 1) (KS), uncorrelated with
    each other and across realisations and cells."""
    z = O.noise_draws(64, 400, seed=7)
    for part in (z[:, 0::2].ravel(), z[:, 1::2].ravel()):
        assert scipy.stats.kstest(part, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(z[:, 0::2].ravel(), z[:, 1::2].ravel())[0, 1]) < 0.02
    assert abs(np.corrcoef(z[:-1].ravel(), z[1:].ravel())[0, 1]) < 0.02
    assert abs(np.corrcoef(z[:, :-1].ravel(), z[:, 1:].ravel())[0, 1]) < 0.02
    # different seeds give different streams; the same seed the same stream
    assert not np.array_equal(O.noise_draws(8, 2, seed=1), O.noise_draws(8, 2, seed=2))
    np.testing.assert_array_equal(O.noise_draws(8, 2, seed=3), O.noise_draws(8, 2, seed=3))


_PHILOX_SHIM = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdint>
extern "C" void ref_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
    const uint64_t seed = (uint64_t)key[0] | ((uint64_t)key[1] << 32);
    const uint64_t offset = (uint64_t)ctr[0] | ((uint64_t)ctr[1] << 32);
    const uint64_t subseq = (uint64_t)ctr[2] | ((uint64_t)ctr[3] << 32);
    at::Philox4_32 e(seed, subseq, offset);
    for (int i = 0; i < 4; ++i) out[i] = e();
}
"""


def test_philox_matches_library_engine(tmp_path):
    """The oracle's Philox4x32-10 equals PyTorch's independent header-only
    engine (at::Philox4_32: key = seed, counter = (offset, subsequence)) word
    for word, on random and extreme counters and keys."""
    import ctypes
    import subprocess
    torch_ext = pytest.importorskip("torch.utils.cpp_extension")
    src = tmp_path / "ref.cpp"
    so = tmp_path / "libref.so"
    src.write_text(_PHILOX_SHIM)
    inc = [f"-I{p}" for p in torch_ext.include_paths()]
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", *inc, str(src), "-o", str(so)])
    ref = ctypes.CDLL(str(so))
    U = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
    ref.ref_philox.argtypes = [U, U, U]
    ref.ref_philox.restype = None
    g = np.random.default_rng(17)
    cases = [(np.zeros(4), np.zeros(2)), (np.full(4, 2 ** 32 - 1), np.full(2, 2 ** 32 - 1))]
    cases += [(g.integers(0, 2 ** 32, 4, dtype=np.uint64), g.integers(0, 2 ** 32, 2, dtype=np.uint64))
              for _ in range(300)]
    for ctr, key in cases:
        ctr = np.asarray(ctr, dtype=np.uint64).astype(np.uint32)
        key = np.asarray(key, dtype=np.uint64).astype(np.uint32)
        want = np.empty(4, dtype=np.uint32)
        ref.ref_philox(ctr, key, want)
        np.testing.assert_array_equal(O.philox4x32_10(ctr, key), want)


def test_philox_mixing():
    """Philox4x32-10 avalanche: flipping any single bit of the counter or key
    flips about half of the 128 output bits (a dropped key injection, a
    missing round or a wrong product half would not), and the outputs of
    consecutive counters are uniform (KS on their 32-bit words)."""
    g = np.random.default_rng(3)
    flips = []
    for trial in range(60):
        ctr = g.integers(0, 2 ** 32, 4, dtype=np.uint64).astype(np.uint32)
        key = g.integers(0, 2 ** 32, 2, dtype=np.uint64).astype(np.uint32)
        base = O.philox4x32_10(ctr, key)
        for word, bit in ((trial % 4, trial % 32), (None, trial % 32)):
            c2, k2 = ctr.copy(), key.copy()
            if word is None:
                k2[trial % 2] ^= np.uint32(1 << bit)
            else:
                c2[word] ^= np.uint32(1 << bit)
            out = O.philox4x32_10(c2, k2)
            flips.append(sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(base, out)))
    flips = np.array(flips)
    assert abs(flips.mean() - 64) < 3 and flips.min() > 30
    words = np.concatenate([O.philox4x32_10(np.array([j, 0, 0, 0]), np.array([9, 0])) for j in range(2000)])
    assert scipy.stats.kstest(words / 2.0 ** 32, "uniform").pvalue > 1e-3


def test_noise_q_special_values():
    """q is a lower-tail fraction: 0 below every realisation, 1 above all, and
    at the analytic p-quantile of the scaled chi-square law it is p within
    binomial error."""
    n, s = 101, 0.025
    L = O.noise_loglike(n, s, s, 4000, seed=99)
    assert O.noise_q(L, [L.min() - 1.0])[0] == 0.0 and O.noise_q(L, [L.max()])[0] == 1.0
    for p in (0.01, 0.1, 0.5):
        # L <= L_bar  <=>  chi2 >= c:  P = 1 - F(c) = p
        c = scipy.stats.chi2(df=n).ppf(1.0 - p)
        L_bar = -0.5 * (n * math.log(2 * math.pi * s * s) + c)
        q = O.noise_q(L, [L_bar])[0]
        assert abs(q - p) < 4 * math.sqrt(p * (1 - p) / 4000) + 1e-3, (p, q)
