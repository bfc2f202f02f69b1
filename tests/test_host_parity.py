"""Host half of the library (region building, precompute, data simulation)
against the oracle, on the CPU: labels and edges bit-exact, A / B / data to
FP64 summation-order rounding."""
import numpy as np
import pytest

import oracle as O
from paper_2603_13196_gb300 import fg21, inputs as I


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _compare(sky, obs, N, scheme, weighting):
    lab, edges, A, B = fg21.fg21_build_regions_host(sky, obs, N, scheme, weighting)
    m = O.build_model(sky, obs, N, scheme, weighting)
    if m.margin <= 1e-12:
        # a deciding comparison is a tie to FP64 rounding (e.g. equal pixel
        # weights whose running sum lands on a target mass): either neighbour
        # of the tie is a correct answer, so each edge may move by one sorted
        # pixel; the region arrays then differ, so stop here
        sb = np.sort(sky.beta)
        pos_l = np.searchsorted(sb, edges)
        pos_o = np.searchsorted(sb, m.edges)
        assert np.all(np.abs(pos_l - pos_o) <= 1)
        return
    assert np.array_equal(lab, m.labels)
    assert np.array_equal(edges, m.edges)
    np.testing.assert_allclose(A, m.A, rtol=1e-12, atol=1e-13 * np.abs(m.A).max())
    np.testing.assert_allclose(B, m.B, rtol=1e-12)


@pytest.mark.parametrize("k", [1, 2])
def test_workloads(k):
    wl = I.workload(k)
    _compare(wl.sky(), wl.obs(), wl.N, wl.scheme, wl.weighting)


@pytest.mark.parametrize("scheme", ["recursive", "hierarchical", "linear", "percentile"])
@pytest.mark.parametrize("weighting", ["beam", "sky", "horizon", "uniform"])
def test_schemes_and_weightings(scheme, weighting):
    sky = I.make_sky(3072, 21)
    obs = I.make_obs(21, 5, 4.0, lst0_h=18.0)
    for N in (1, 2, 7, 12):
        _compare(sky, obs, N, scheme, weighting)


def test_uneven_batch_models():
    for wl in I.uneven_batch(6):
        _compare(wl.sky(), wl.obs(), wl.N, wl.scheme, wl.weighting)


@pytest.mark.parametrize("T", [1, 9])
def test_simulated_data(T):
    sky = I.make_sky(2048, 5)
    obs = I.make_obs(41, T, 6.0, lst0_h=1.0)
    noise = I.noise_draws(41, T, 2)
    for t21, sig, nz in (((0.155, 85.0, 15.0), 0.025, noise), ((0.0, 100.0, 10.0), 0.0, None)):
        got = fg21.fg21_simulate_data(sky, obs, t21, sig, nz)
        want = O.simulate_data(sky, obs, np.array(t21), sig, nz)
        np.testing.assert_allclose(got, want, rtol=1e-12)


def test_empty_regions_are_allowed():
    """A partition finer than the distinct beta values leaves empty regions with
    zero A rows (recursive bisection of a map with only three spectral indices)."""
    sky = I.make_sky(512, 3)
    sky = I.Sky(dirs=sky.dirs, t230=sky.t230, beta=np.choose(np.arange(512) % 3, [2.5, 2.6, 2.9]))
    obs = I.make_obs(7, 2, 2.0)
    lab, edges, A, B = fg21.fg21_build_regions_host(sky, obs, 8, "recursive")
    counts = np.bincount(lab, minlength=8)
    assert (counts == 0).any()
    assert np.all(A[counts == 0] == 0.0)
    _compare(sky, obs, 8, "recursive", "beam")


# ------------------------------------------------ amplitude / spectral-index
def _compare_ab(sky, obs, Nb, scheme, weighting, Na, field, scheme_a, weighting_a):
    lab, edges, lab_a, edges_a, K, B = fg21.fg21_build_regions_ab_host(sky, obs, Nb, scheme, weighting, Na, field,
                                                                       scheme_a, weighting_a)
    m = O.build_model_ab(sky, obs, Nb, scheme, weighting, Na, field, scheme_a, weighting_a)
    assert m.margin > 1e-12, "degenerate seed: a deciding comparison is a near-tie"
    assert np.array_equal(lab, m.labels_b) and np.array_equal(edges, m.edges_b)
    assert np.array_equal(lab_a, m.labels_a) and np.array_equal(edges_a, m.edges_a)
    np.testing.assert_allclose(K, m.K, rtol=1e-12, atol=1e-13 * np.abs(m.K).max())
    np.testing.assert_allclose(B, m.B, rtol=1e-12)


@pytest.mark.parametrize("scheme,scheme_a", [("recursive", "hierarchical"), ("hierarchical", "recursive"),
                                             ("percentile", "linear")])
@pytest.mark.parametrize("weighting_a", ["beam", "sky"])
def test_amplitude_regions(scheme, scheme_a, weighting_a):
    """Spectral-index and amplitude labels bit-exact, K over the intersections
    to summation-order rounding (the library builds K as one set of
    combined-label sums, the oracle from the two masks)."""
    sky = I.make_sky(1536, 31)
    obs = I.make_obs(13, 3, 4.0, lst0_h=5.0)
    field = I.amplitude_field(sky)
    for Nb, Na in ((3, 2), (5, 4), (1, 3), (6, 1)):
        _compare_ab(sky, obs, Nb, scheme, "beam", Na, field, scheme_a, weighting_a)


def test_amplitude_regions_errors():
    sky = I.make_sky(256, 2)
    obs = I.make_obs(5, 2, 1.0)
    field = I.amplitude_field(sky)
    with pytest.raises(fg21.Fg21Error) as e:
        fg21.fg21_build_regions_ab_host(sky, obs, 3, "recursive", "beam", 0, field)
    assert e.value.code == fg21.FG21_E_ARG
    with pytest.raises(fg21.Fg21Error):
        fg21.fg21_build_regions_ab_host(sky, obs, 12, "recursive", "beam", 11, field)     # 132 components
    bad = field.copy()
    bad[7] = np.inf
    with pytest.raises(fg21.Fg21Error):
        fg21.fg21_build_regions_ab_host(sky, obs, 3, "recursive", "beam", 2, bad)


@pytest.mark.parametrize("scheme", ["recursive", "hierarchical"])
def test_partition_ties_randomized(scheme):
    """The library's partition (a priority queue for Algorithm 2, one sort of the
    base regions for Algorithm 1) against the oracle's direct loops on small
    maps built for ties: spectral indices quantised to a few values (equal
    masses, zero-width regions, repeated edges) and uniform weights.  Both sides
    sum a region's mass over its pixels in sorted order, so regions holding the
    same number of equally weighted pixels tie exactly on both, and the tie
    rules (lowest lower edge, then the earlier region) alone decide: the
    comparison is exact, with no skip for small decision margins."""
    import dataclasses
    rng = np.random.default_rng(4242)
    obs = I.make_obs(5, 2, 2.0, lst0_h=6.0)
    checked = 0
    for case in range(60):
        npix = int(rng.integers(8, 160))
        sky = I.make_sky(npix, 300 + case)
        levels = int(rng.integers(2, 9))
        beta = 2.45 + 0.1 * rng.integers(0, levels, npix)
        sky = dataclasses.replace(sky, beta=beta)
        for N in (1, 2, 3, 5, 8, 13):
            if N > npix:
                continue
            lab, edges, _, _ = fg21.fg21_build_regions_host(sky, obs, N, scheme, "uniform")
            m = O.build_model(sky, obs, N, scheme, "uniform")
            assert np.array_equal(edges, m.edges), (case, N)
            assert np.array_equal(lab, m.labels), (case, N)
            checked += 1
    assert checked >= 100, checked
