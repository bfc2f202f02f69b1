"""Region building on the GPU (fg21_build_regions / fg21_build_regions_ab run
the importance weights and the response functions on the device): labels and
edges bit-identical to the host builder and the oracle, A / K and B equal to
FP64 summation-order rounding, for every scheme and weighting, with amplitude
regions, and at the benchmark's sky and observation."""
import numpy as np
import pytest

import oracle as O
from paper_2603_13196_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _check(fg21lib, sky, obs, N, scheme, weighting):
    model = fg21lib.fg21_build_regions(sky, obs, N, scheme, weighting)
    lab, edges, A, B = fg21lib.fg21_build_regions_host(sky, obs, N, scheme, weighting)
    assert np.array_equal(model.labels, lab) and np.array_equal(model.edges, edges)
    Ad, Bd = fg21lib.fg21_model_get_arrays(model)
    np.testing.assert_allclose(Ad, A, rtol=1e-12, atol=1e-13 * np.abs(A).max())
    np.testing.assert_allclose(Bd, B, rtol=1e-12)
    return model, Ad, Bd


@pytest.mark.parametrize("scheme", ["recursive", "hierarchical", "linear", "percentile"])
@pytest.mark.parametrize("weighting", ["beam", "sky", "horizon", "uniform"])
def test_device_build_equals_host(fg21lib, scheme, weighting):
    sky = I.make_sky(3072, 21)
    obs = I.make_obs(21, 5, 4.0, lst0_h=18.0)
    for N in (1, 7, 12):
        if weighting == "uniform" and scheme == "hierarchical":
            continue      # exact ties of the uniform masses (host parity test covers the tie rule)
        _check(fg21lib, sky, obs, N, scheme, weighting)


@pytest.mark.parametrize("k", [2, 3])
def test_device_build_matches_oracle_at_workload_shape(fg21lib, k):
    """Workload 2 (12288 pixels, N = 9, F = 151, T = 20) and the benchmark's
    own sky and observation (workload 3: 49152 pixels, N = 24, F = 301,
    T = 100): labels and edges equal to the oracle's, and every A[i, f, t] and
    B[f, t] of the device precompute within 1e-12 relative of the oracle's
    (eq. chromatic_function, FP64 in another summation order)."""
    wl = I.workload(k)
    sky, obs = wl.sky(), wl.obs()
    model = fg21lib.fg21_build_regions(sky, obs, wl.N, wl.scheme, wl.weighting)
    Ad, Bd = fg21lib.fg21_model_get_arrays(model)
    m = O.build_model(sky, obs, wl.N, wl.scheme, wl.weighting)
    assert np.array_equal(model.labels, m.labels)
    np.testing.assert_array_equal(model.edges, m.edges)
    np.testing.assert_allclose(Ad, m.A, rtol=1e-12, atol=1e-13 * np.abs(m.A).max())
    np.testing.assert_allclose(Bd, m.B, rtol=1e-12)
    model.close()


def test_device_build_amplitude_regions(fg21lib):
    sky = I.make_sky(2048, 33)
    obs = I.make_obs(17, 4, 3.0, lst0_h=7.0)
    field = I.amplitude_field(sky)
    for Nb, Na, wa in ((4, 3, "beam"), (6, 2, "sky")):
        model = fg21lib.fg21_build_regions_ab(sky, obs, Nb, "recursive", "beam", Na, field, "hierarchical", wa)
        lab, edges, lab_a, edges_a, K, B = fg21lib.fg21_build_regions_ab_host(sky, obs, Nb, "recursive", "beam", Na,
                                                                              field, "hierarchical", wa)
        assert np.array_equal(model.labels, lab) and np.array_equal(model.labels_alpha, lab_a)
        Ad, Bd = fg21lib.fg21_model_get_arrays(model)
        np.testing.assert_allclose(Ad, K.reshape(Na * Nb, obs.F, obs.T), rtol=1e-12, atol=1e-13 * np.abs(K).max())
        np.testing.assert_allclose(Bd, B, rtol=1e-12)


def test_empty_regions_on_device(fg21lib):
    sky = I.make_sky(512, 3)
    sky = I.Sky(dirs=sky.dirs, t230=sky.t230, beta=np.choose(np.arange(512) % 3, [2.5, 2.6, 2.9]))
    obs = I.make_obs(7, 2, 2.0)
    model, Ad, _ = _check(fg21lib, sky, obs, 8, "recursive", "beam")
    counts = np.bincount(model.labels, minlength=8)
    assert (counts == 0).any() and np.all(Ad[counts == 0] == 0.0)
