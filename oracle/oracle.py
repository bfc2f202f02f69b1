"""ctypes front end of the FP64 oracle (test infrastructure only).

Each function names the definition of arXiv 2603.13196 it evaluates; the C
code in fg21_oracle.c carries the arithmetic.  Arrays are float64, C order:
A[N, F, T], B[F, T], data[F, T], params[P, N+4] = [beta_1..beta_N, A21, nu21,
sigma21, sigma_n], model[P, F, T].
"""
from __future__ import annotations

import ctypes as C
import dataclasses

import numpy as np

from . import build as _build

SCHEMES = {"recursive": 0, "hierarchical": 1, "linear": 2, "percentile": 3}
WEIGHTINGS = {"beam": 0, "sky": 1, "horizon": 2, "uniform": 3}

_lib = None
_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_I32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_I64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        L.orc_t21.restype = C.c_double
        L.orc_t21.argtypes = [C.c_double] * 4
        L.orc_weights.restype = C.c_int
        L.orc_weights.argtypes = [C.c_int64, _D, _D, _D, C.c_int, _D, C.c_double, C.c_int, _D, _D,
                                  C.c_double, C.c_int, _D]
        L.orc_sorted_order.restype = None
        L.orc_sorted_order.argtypes = [C.c_int64, _D, _I64]
        L.orc_partition.restype = C.c_int
        L.orc_partition.argtypes = [C.c_int64, _D, _D, C.c_int, C.c_int, _D, _I32,
                                    C.POINTER(C.c_double)]
        L.orc_precompute.restype = C.c_int
        L.orc_precompute.argtypes = [C.c_int64, _D, _D, _I32, C.c_int, C.c_int, C.c_int, _D, _D,
                                     C.c_double, _D, _D]
        L.orc_fast_model.restype = None
        L.orc_fast_model.argtypes = [C.c_int, C.c_int, C.c_int, _D, _D, _D, C.c_double, C.c_double,
                                     _D, C.c_int64, _D]
        L.orc_pixel_model.restype = None
        L.orc_pixel_model.argtypes = [C.c_int64, _D, _D, _I32, C.c_int, C.c_int, _D, C.c_double,
                                      C.c_int, _D, _D, C.c_double, _D, C.c_int64, _D]
        L.orc_simulate_data.restype = None
        L.orc_simulate_data.argtypes = [C.c_int64, _D, _D, _D, C.c_int, _D, C.c_double, C.c_int,
                                        _D, _D, C.c_double, _D, C.c_double, C.c_void_p, _D]
        L.orc_precompute_ab.restype = C.c_int
        L.orc_precompute_ab.argtypes = [C.c_int64, _D, _D, _I32, C.c_int, _I32, C.c_int, C.c_int, C.c_int,
                                        _D, _D, C.c_double, _D, _D]
        L.orc_fast_model_ab.restype = None
        L.orc_fast_model_ab.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _D, _D, _D, C.c_double,
                                        C.c_double, _D, C.c_int64, _D]
        L.orc_pixel_model_ab.restype = None
        L.orc_pixel_model_ab.argtypes = [C.c_int64, _D, _D, _I32, C.c_int, _I32, C.c_int, C.c_int, _D,
                                         C.c_double, C.c_int, _D, _D, C.c_double, _D, C.c_int64, _D]
        for name in ("orc_loglike_ab", "orc_chi2_ab"):
            fn = getattr(L, name)
            fn.restype = None
            fn.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _D, _D, _D, _D, C.c_double, C.c_double,
                           _D, C.c_int64, _D]
        _U32 = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
        L.orc_philox4x32_10.restype = None
        L.orc_philox4x32_10.argtypes = [_U32, _U32, _U32]
        L.orc_noise_draws.restype = None
        L.orc_noise_draws.argtypes = [C.c_int64, C.c_int64, C.c_uint64, _D]
        L.orc_noise_loglike.restype = None
        L.orc_noise_loglike.argtypes = [C.c_int64, C.c_double, C.c_double, C.c_int64, C.c_uint64, _D]
        L.orc_noise_q.restype = None
        L.orc_noise_q.argtypes = [_D, C.c_int64, _D, C.c_int64, _D]
        for name in ("orc_loglike", "orc_chi2"):
            fn = getattr(L, name)
            fn.restype = None
            fn.argtypes = [C.c_int, C.c_int, C.c_int, _D, _D, _D, _D, C.c_double, C.c_double, _D,
                           C.c_int64, _D]
        _lib = L
    return _lib


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def t21(nu, a21, nu21, s21):
    """Gaussian trough, Sec. 2.1 eq. t21model."""
    L = lib()
    return np.array([L.orc_t21(float(x), a21, nu21, s21) for x in np.atleast_1d(nu)])


def weights(sky, obs, weighting="beam"):
    """Band- and LST-averaged pixel importance w[pix] (Sec. 4.2; sums to 1)."""
    w = np.empty(sky.npix)
    rc = lib().orc_weights(sky.npix, _c(sky.dirs), _c(sky.t230), _c(sky.beta), obs.F, _c(obs.nu),
                           obs.nu0, obs.T, _c(obs.zenith), _c(obs.beam_p), obs.t_cmb,
                           WEIGHTINGS[weighting], w)
    assert rc == 0
    return w


def sorted_order(beta):
    beta = _c(beta)
    out = np.empty(beta.shape[0], dtype=np.int64)
    lib().orc_sorted_order(beta.shape[0], beta, out)
    return out


def partition(beta, w, N, scheme="recursive"):
    """Algorithm 2 (recursive), Algorithm 1 (hierarchical), or the linear /
    percentile splits of Sec. 4.1.  Returns (edges[N+1], labels[Npix], margin)."""
    beta = _c(beta)
    edges = np.empty(N + 1)
    labels = np.empty(beta.shape[0], dtype=np.int32)
    margin = C.c_double(0.0)
    rc = lib().orc_partition(beta.shape[0], beta, _c(w), N, SCHEMES[scheme], edges, labels,
                             C.byref(margin))
    assert rc == 0, rc
    return edges, labels, margin.value


def precompute(sky, obs, labels, N):
    """A[i,f,t] (Sec. 2.2 eq. chromatic_function) and B[f,t] (beam normalisation)."""
    A = np.empty((N, obs.F, obs.T))
    B = np.empty((obs.F, obs.T))
    rc = lib().orc_precompute(sky.npix, _c(sky.dirs), _c(sky.t230), _c(labels, np.int32), N,
                              obs.F, obs.T, _c(obs.zenith), _c(obs.beam_p), obs.t_cmb, A, B)
    assert rc == 0
    return A, B


def fast_model(A, B, obs, params):
    """Sec. 2.2 eq. fast_forward_model + T21 -> M[P, F, T]."""
    params = _c(np.atleast_2d(params))
    N, F, T = A.shape
    P = params.shape[0]
    M = np.empty((P, F, T))
    lib().orc_fast_model(N, F, T, _c(A), _c(B), _c(obs.nu), obs.nu0, obs.t_cmb, params, P, M)
    return M


def pixel_model(sky, obs, labels, N, params):
    """Sec. 2.2 eq. forward_model integrated against the beam, per pixel -> M[P, F, T]."""
    params = _c(np.atleast_2d(params))
    P = params.shape[0]
    M = np.empty((P, obs.F, obs.T))
    lib().orc_pixel_model(sky.npix, _c(sky.dirs), _c(sky.t230), _c(labels, np.int32), N, obs.F,
                          _c(obs.nu), obs.nu0, obs.T, _c(obs.zenith), _c(obs.beam_p), obs.t_cmb,
                          params, P, M)
    return M


def simulate_data(sky, obs, t21p, sigma_noise=0.0, noise=None):
    """Sec. 2.1 eq. simantenna with the per-pixel beta of the sky -> data[F, T]."""
    data = np.empty((obs.F, obs.T))
    nz = None
    if noise is not None:
        noise = _c(noise)
        assert noise.shape == (obs.F, obs.T)
        nz = noise.ctypes.data_as(C.c_void_p)
    lib().orc_simulate_data(sky.npix, _c(sky.dirs), _c(sky.t230), _c(sky.beta), obs.F, _c(obs.nu),
                            obs.nu0, obs.T, _c(obs.zenith), _c(obs.beam_p), obs.t_cmb,
                            _c(t21p), float(sigma_noise), nz, data)
    return data


def loglike(A, B, data, obs, params):
    """Sec. 2.3.1 eq. likelihood -> logL[P]."""
    params = _c(np.atleast_2d(params))
    N, F, T = A.shape
    P = params.shape[0]
    out = np.empty(P)
    lib().orc_loglike(N, F, T, _c(A), _c(B), _c(data), _c(obs.nu), obs.nu0, obs.t_cmb, params,
                      P, out)
    return out


def chi2(A, B, data, obs, params):
    """sum_{f,t} (D - M)^2 per point (the data term of eq. likelihood, in K^2)."""
    params = _c(np.atleast_2d(params))
    N, F, T = A.shape
    P = params.shape[0]
    out = np.empty(P)
    lib().orc_chi2(N, F, T, _c(A), _c(B), _c(data), _c(obs.nu), obs.nu0, obs.t_cmb, params, P,
                   out)
    return out


# ------------------------------------------------------ amplitude masks
# Models with N_alpha amplitude regions as well (eqs. forward_model,
# chromatic_function, fast_forward_model of Sec. 2.2).  K[Na, Nb, F, T];
# params[P, Nb+Na+4] = [beta_1..beta_Nb, alpha_1..alpha_Na, A21, nu21,
# sigma21, sigma_n].

def precompute_ab(sky, obs, labels_a, Na, labels_b, Nb):
    """K[i,j,f,t] over the intersections of amplitude region i and
    spectral-index region j (eq. chromatic_function), and B[f,t]."""
    K = np.empty((Na, Nb, obs.F, obs.T))
    B = np.empty((obs.F, obs.T))
    rc = lib().orc_precompute_ab(sky.npix, _c(sky.dirs), _c(sky.t230), _c(labels_a, np.int32), Na,
                                 _c(labels_b, np.int32), Nb, obs.F, obs.T, _c(obs.zenith),
                                 _c(obs.beam_p), obs.t_cmb, K, B)
    assert rc == 0
    return K, B


def fast_model_ab(K, B, obs, params):
    """eq. fast_forward_model with amplitude masks + T21 -> M[P, F, T]."""
    params = _c(np.atleast_2d(params))
    Na, Nb, F, T = K.shape
    P = params.shape[0]
    assert params.shape[1] == Nb + Na + 4
    M = np.empty((P, F, T))
    lib().orc_fast_model_ab(Na, Nb, F, T, _c(K), _c(B), _c(obs.nu), obs.nu0, obs.t_cmb, params, P, M)
    return M


def pixel_model_ab(sky, obs, labels_a, Na, labels_b, Nb, params):
    """eq. forward_model with amplitude masks, integrated per pixel -> M[P, F, T]."""
    params = _c(np.atleast_2d(params))
    P = params.shape[0]
    assert params.shape[1] == Nb + Na + 4
    M = np.empty((P, obs.F, obs.T))
    lib().orc_pixel_model_ab(sky.npix, _c(sky.dirs), _c(sky.t230), _c(labels_a, np.int32), Na,
                             _c(labels_b, np.int32), Nb, obs.F, _c(obs.nu), obs.nu0, obs.T,
                             _c(obs.zenith), _c(obs.beam_p), obs.t_cmb, params, P, M)
    return M


def loglike_ab(K, B, data, obs, params):
    """Sec. 2.3.1 eq. likelihood over the amplitude-mask model -> logL[P]."""
    params = _c(np.atleast_2d(params))
    Na, Nb, F, T = K.shape
    P = params.shape[0]
    assert params.shape[1] == Nb + Na + 4
    out = np.empty(P)
    lib().orc_loglike_ab(Na, Nb, F, T, _c(K), _c(B), _c(data), _c(obs.nu), obs.nu0, obs.t_cmb, params,
                         P, out)
    return out


def chi2_ab(K, B, data, obs, params):
    params = _c(np.atleast_2d(params))
    Na, Nb, F, T = K.shape
    P = params.shape[0]
    out = np.empty(P)
    lib().orc_chi2_ab(Na, Nb, F, T, _c(K), _c(B), _c(data), _c(obs.nu), obs.nu0, obs.t_cmb, params, P,
                      out)
    return out


@dataclasses.dataclass
class OracleModelAB:
    Nb: int
    Na: int
    w_b: np.ndarray
    w_a: np.ndarray
    edges_b: np.ndarray
    labels_b: np.ndarray
    edges_a: np.ndarray
    labels_a: np.ndarray
    margin: float
    K: np.ndarray          # [Na, Nb, F, T]
    B: np.ndarray

    @property
    def N(self) -> int:    # components (rows of the flattened K)
        return self.Na * self.Nb


def build_model_ab(sky, obs, Nb, scheme, weighting, Na, field_a, scheme_a, weighting_a):
    """The oracle's fg21_build_regions_ab: spectral-index regions partition
    beta, amplitude regions partition the per-pixel `field_a`, each with its
    own scheme and importance weighting; then K over the intersections."""
    w_b = weights(sky, obs, weighting)
    edges_b, labels_b, m_b = partition(sky.beta, w_b, Nb, scheme)
    w_a = w_b if weighting_a == weighting else weights(sky, obs, weighting_a)
    edges_a, labels_a, m_a = partition(field_a, w_a, Na, scheme_a)
    K, B = precompute_ab(sky, obs, labels_a, Na, labels_b, Nb)
    return OracleModelAB(Nb, Na, w_b, w_a, edges_b, labels_b, edges_a, labels_a, min(m_b, m_a), K, B)


# ------------------------------------------- noise-only likelihood (q_i)
# The accuracy criterion of Sec. 5.2.2: the likelihood distribution of data
# that the model describes up to Gaussian noise, and the lower-tail
# probability q of a fitted likelihood under it.

def philox4x32_10(ctr, key):
    """Philox4x32-10 (Salmon et al. 2011) of one 128-bit counter and 64-bit key."""
    out = np.empty(4, dtype=np.uint32)
    lib().orc_philox4x32_10(np.ascontiguousarray(ctr, dtype=np.uint32), np.ascontiguousarray(key, dtype=np.uint32),
                            out)
    return out


def noise_draws(n_cells, K, seed):
    """Standard-normal draws [K, n_cells] of the noise realisations (Philox + Box-Muller)."""
    out = np.empty((K, n_cells))
    lib().orc_noise_draws(n_cells, K, seed, out)
    return out


def noise_loglike(n_cells, sigma_noise, sigma_n, K, seed):
    """L_noise[k] = -1/2 sum_cells [ln(2 pi sigma_n^2) + (sigma_noise z_k)^2 / sigma_n^2]."""
    out = np.empty(K)
    lib().orc_noise_loglike(n_cells, sigma_noise, sigma_n, K, seed, out)
    return out


def noise_q(L_noise, L_bar):
    """q_i = P(L_noise <= L_bar_i) for each L_bar_i."""
    L_bar = np.atleast_1d(np.asarray(L_bar, dtype=np.float64))
    q = np.empty(L_bar.shape[0])
    lib().orc_noise_q(_c(L_noise), len(L_noise), _c(L_bar), L_bar.shape[0], q)
    return q


@dataclasses.dataclass
class OracleModel:
    N: int
    w: np.ndarray
    edges: np.ndarray
    labels: np.ndarray
    margin: float
    A: np.ndarray
    B: np.ndarray


def build_model(sky, obs, N, scheme="recursive", weighting="beam"):
    """Weights -> CDF partition -> precompute, the oracle's fg21_build_regions."""
    w = weights(sky, obs, weighting)
    edges, labels, margin = partition(sky.beta, w, N, scheme)
    A, B = precompute(sky, obs, labels, N)
    return OracleModel(N, w, edges, labels, margin, A, B)


def region_truth(sky, labels, N, w=None):
    """Per-region mean spectral index (importance weighted if w is given); a
    natural 'true' point of the N-region model for data generation."""
    out = np.empty(N)
    for i in range(N):
        m = labels == i
        if not m.any():
            out[i] = 2.8
        elif w is None or w[m].sum() <= 0:
            out[i] = sky.beta[m].mean()
        else:
            out[i] = np.sum(sky.beta[m] * w[m]) / np.sum(w[m])
    return out


def use_library(path):
    """Load the oracle from another build of fg21_oracle.c (the mutation tests
    compile deliberately broken copies); returns the previous handle."""
    global _lib
    prev = _lib
    _lib = None
    _build_path = path

    def _fake_build():
        return _build_path
    orig = _build.build
    _build.build = _fake_build
    try:
        lib()
    finally:
        _build.build = orig
    return prev


def restore_library(prev):
    global _lib
    _lib = prev
