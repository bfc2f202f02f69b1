"""Python binding of libfg21 (include/fg21.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of its own; all likelihood work runs in the library's CUDA kernels.
If the compiled library is missing, loading fails loudly (run
`__graft_entry__.build()` or `python paper_2603_13196_gb300/build.py`); there is
no Python or CPU fallback.

Device buffers are passed as raw pointers (int), e.g. `tensor.data_ptr()` of a
torch CUDA tensor, and streams as raw `cudaStream_t` values
(`torch.cuda.current_stream().cuda_stream`).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

FG21_OK = 0
ERRORS = {-1: "FG21_E_ARG", -2: "FG21_E_NOMEM", -3: "FG21_E_CUDA", -4: "FG21_E_TIMEOUT", -5: "FG21_E_BUSY",
          -6: "FG21_E_STATE", -7: "FG21_E_NOTFOUND", -8: "FG21_E_CANCELLED", -9: "FG21_E_DEVICE",
          -10: "FG21_E_RANGE"}
FG21_E_ARG, FG21_E_NOMEM, FG21_E_CUDA, FG21_E_TIMEOUT, FG21_E_BUSY = -1, -2, -3, -4, -5
FG21_E_STATE, FG21_E_NOTFOUND, FG21_E_CANCELLED, FG21_E_DEVICE, FG21_E_RANGE = -6, -7, -8, -9, -10
SCHEMES = {"recursive": 0, "hierarchical": 1, "linear": 2, "percentile": 3}
WEIGHTINGS = {"beam": 0, "sky": 1, "horizon": 2, "uniform": 3}
PRECISIONS = {"fp16x3": 0, "bf16x3": 1, "fp32_delta": 2, "fp32_direct": 3}
MAX_REGIONS_TC = 62
MAX_REGIONS = 126


class Fg21Error(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {ERRORS.get(code, code)}: {msg}")
        self.code = code


class fg21_sky(C.Structure):
    _fields_ = [("npix", C.c_int64), ("dirs", C.c_void_p), ("t230", C.c_void_p), ("beta", C.c_void_p)]


class fg21_obs(C.Structure):
    _fields_ = [("F", C.c_int32), ("nu", C.c_void_p), ("nu0", C.c_double), ("T", C.c_int32),
                ("zenith", C.c_void_p), ("beam_p", C.c_void_p), ("t_cmb", C.c_double)]


class fg21_partition_opts(C.Structure):
    _fields_ = [("n_regions", C.c_int32), ("scheme", C.c_int32), ("weighting", C.c_int32)]


class fg21_amplitude_opts(C.Structure):
    _fields_ = [("n_regions", C.c_int32), ("scheme", C.c_int32), ("weighting", C.c_int32), ("field", C.c_void_p)]


class fg21_serve_opts(C.Structure):
    _fields_ = [("mem_budget_bytes", C.c_size_t), ("max_batch_points", C.c_int64), ("max_wait_us", C.c_int32),
                ("max_inflight", C.c_int32), ("precision", C.c_int32), ("device", C.c_int32)]


class fg21_stats(C.Structure):
    _fields_ = [("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double),
                ("evals_per_s", C.c_double), ("macs_per_s", C.c_double), ("requests_done", C.c_int64),
                ("points_done", C.c_int64), ("launches", C.c_int64), ("queue_depth", C.c_int64),
                ("admitted_bytes", C.c_size_t), ("runs_admitted", C.c_int32), ("runs_waiting", C.c_int32)]


_lib = None
_P = C.c_void_p
_SIGS = {
    "fg21_last_error": (C.c_char_p, []),
    "fg21_last_invalid_count": (C.c_int64, []),
    "fg21_version": (C.c_char_p, []),
    "fg21_device_count": (C.c_int, []),
    "fg21_build_regions": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "fg21_build_regions_host": (C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "fg21_build_regions_ab": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "fg21_build_regions_ab_host": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "fg21_model_shape": (C.c_int, [_P, _P, _P, _P]),
    "fg21_model_destroy": (C.c_int, [_P]),
    "fg21_model_set_data": (C.c_int, [_P, _P]),
    "fg21_model_get_arrays": (C.c_int, [_P, _P, _P]),
    "fg21_model_info": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "fg21_simulate_data": (C.c_int, [_P, _P, _P, C.c_double, _P, _P]),
    "fg21_loglike_batch": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int, _P]),
    "fg21_loglike_batch_device": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int, _P]),
    "fg21_loglike_batch_device_noalloc": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int, _P]),
    "fg21_model_sync_status": (C.c_int, [_P, _P, _P]),
    "fg21_selftest_bounded_wait": (C.c_int, [_P, _P, _P]),
    "fg21_selftest_mma_rounding": (C.c_int, [_P, _P, _P, _P, _P]),
    "fg21_autotune": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int, _P, _P, _P]),
    "fg21_model_eval": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int, _P]),
    "fg21_model_timing": (C.c_int, [_P, C.c_int]),
    "fg21_model_timing_totals": (C.c_int, [_P, _P, _P, _P, _P]),
    "fg21_loglike_multi": (C.c_int, [_P, _P, _P, _P, C.c_int, C.c_int, _P]),
    "fg21_graph_create": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int, _P]),
    "fg21_graph_create_multi": (C.c_int, [_P, _P, _P, _P, C.c_int, C.c_int, _P]),
    "fg21_graph_launch": (C.c_int, [_P, _P]),
    "fg21_graph_sync_status": (C.c_int, [_P, _P, _P]),
    "fg21_graph_destroy": (C.c_int, [_P]),
    "fg21_noise_loglike": (C.c_int, [C.c_int64, C.c_double, C.c_double, C.c_int64, C.c_uint64, _P, _P]),
    "fg21_noise_q": (C.c_int, [_P, C.c_int64, _P, C.c_int64, _P, _P]),
    "fg21_serve_create": (C.c_int, [_P, _P]),
    "fg21_serve_destroy": (C.c_int, [_P]),
    "fg21_serve_register_run": (C.c_int, [_P, _P, _P]),
    "fg21_serve_unregister_run": (C.c_int, [_P, C.c_int32]),
    "fg21_serve_submit": (C.c_int, [_P, C.c_int32, _P, C.c_int64, _P, _P]),
    "fg21_serve_wait": (C.c_int, [_P, C.c_int64, C.c_int32]),
    "fg21_serve_poll": (C.c_int, [_P, C.c_int64]),
    "fg21_serve_cancel": (C.c_int, [_P, C.c_int64]),
    "fg21_serve_stats": (C.c_int, [_P, _P]),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded libfg21 (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libfg21 is not built ({path} missing); run __graft_entry__.build()")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != FG21_OK:
        raise Fg21Error(rc, where, lib().fg21_last_error().decode())


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _prec(p) -> int:
    return PRECISIONS[p] if isinstance(p, str) else int(p)


class _Keep:
    """fg21_sky / fg21_obs structs plus the arrays they point into."""

    def __init__(self, sky, obs):
        self.dirs, self.t230, self.beta = _f64(sky.dirs), _f64(sky.t230), _f64(sky.beta)
        self.nu, self.zen, self.bp = _f64(obs.nu), _f64(obs.zenith), _f64(obs.beam_p)
        self.sky = fg21_sky(int(self.t230.shape[0]), _ptr(self.dirs), _ptr(self.t230), _ptr(self.beta))
        self.obs = fg21_obs(int(self.nu.shape[0]), _ptr(self.nu), float(obs.nu0), int(self.zen.shape[0]),
                            _ptr(self.zen), _ptr(self.bp), float(obs.t_cmb))


def fg21_version() -> str:
    return lib().fg21_version().decode()


def fg21_device_count() -> int:
    return int(lib().fg21_device_count())


def fg21_last_invalid_count() -> int:
    return int(lib().fg21_last_invalid_count())


def fg21_build_regions_host(sky, obs, n_regions: int, scheme="recursive", weighting="beam"):
    """-> (labels[npix] int32, edges[N+1], A[N,F,T], B[F,T])"""
    k = _Keep(sky, obs)
    opt = fg21_partition_opts(n_regions, SCHEMES[scheme], WEIGHTINGS[weighting])
    lab = np.empty(k.sky.npix, dtype=np.int32)
    edges = np.empty(n_regions + 1)
    A = np.empty((n_regions, k.obs.F, k.obs.T))
    B = np.empty((k.obs.F, k.obs.T))
    _check(lib().fg21_build_regions_host(C.byref(k.sky), C.byref(k.obs), C.byref(opt), _ptr(lab), _ptr(edges),
                                         _ptr(A), _ptr(B)), "fg21_build_regions_host")
    return lab, edges, A, B


def fg21_simulate_data(sky, obs, t21: Sequence[float], sigma_noise: float = 0.0,
                       noise: Optional[np.ndarray] = None) -> np.ndarray:
    k = _Keep(sky, obs)
    t = _f64(t21)
    out = np.empty((k.obs.F, k.obs.T))
    nz = None
    if noise is not None:
        nz = _f64(noise)
        assert nz.shape == out.shape
    _check(lib().fg21_simulate_data(C.byref(k.sky), C.byref(k.obs), _ptr(t), float(sigma_noise),
                                    _ptr(nz) if nz is not None else None, _ptr(out)), "fg21_simulate_data")
    return out


class Model:
    """Owner of an fg21_model handle (fg21_model_destroy on close / GC).  N is
    the number of components (rows of A); parameter rows have n_params values
    ([beta_1..beta_Nb, alpha_1..alpha_Na, A21, nu21, sigma21, sigma_n], Na = 0
    for spectral-index-only models)."""

    def __init__(self, handle: int, N: int, F: int, T: int, labels, edges, Nb: Optional[int] = None,
                 Na: int = 0, labels_alpha=None, edges_alpha=None):
        self.handle = C.c_void_p(handle)
        self.N, self.F, self.T = N, F, T
        self.Nb = N if Nb is None else Nb
        self.Na = Na
        self.n_params = self.Nb + self.Na + 4
        self.labels, self.edges = labels, edges
        self.labels_alpha, self.edges_alpha = labels_alpha, edges_alpha

    def close(self):
        if self.handle:
            lib().fg21_model_destroy(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fg21_build_regions(sky, obs, n_regions: int, scheme="recursive", weighting="beam") -> Model:
    k = _Keep(sky, obs)
    opt = fg21_partition_opts(n_regions, SCHEMES[scheme], WEIGHTINGS[weighting])
    out = C.c_void_p()
    lab = np.empty(k.sky.npix, dtype=np.int32)
    edges = np.empty(n_regions + 1)
    _check(lib().fg21_build_regions(C.byref(k.sky), C.byref(k.obs), C.byref(opt), C.byref(out), _ptr(lab),
                                    _ptr(edges)), "fg21_build_regions")
    return Model(out.value, n_regions, k.obs.F, k.obs.T, lab, edges)


def _amp_opts(n_alpha, scheme_a, weighting_a, field):
    f = _f64(field)
    return fg21_amplitude_opts(int(n_alpha), SCHEMES[scheme_a], WEIGHTINGS[weighting_a], _ptr(f)), f


def fg21_build_regions_ab(sky, obs, n_beta: int, scheme, weighting, n_alpha: int, field, scheme_a="hierarchical",
                          weighting_a="beam") -> Model:
    """Joint amplitude / spectral-index model: spectral-index regions by
    (scheme, weighting), amplitude regions partitioning `field` [npix] by
    (scheme_a, weighting_a); components i * n_beta + j."""
    k = _Keep(sky, obs)
    opt = fg21_partition_opts(n_beta, SCHEMES[scheme], WEIGHTINGS[weighting])
    aopt, keep = _amp_opts(n_alpha, scheme_a, weighting_a, field)
    assert keep.shape == (k.sky.npix,)
    out = C.c_void_p()
    lab = np.empty(k.sky.npix, dtype=np.int32)
    edges = np.empty(n_beta + 1)
    lab_a = np.empty(k.sky.npix, dtype=np.int32)
    edges_a = np.empty(n_alpha + 1)
    _check(lib().fg21_build_regions_ab(C.byref(k.sky), C.byref(k.obs), C.byref(opt), C.byref(aopt), C.byref(out),
                                       _ptr(lab), _ptr(edges), _ptr(lab_a), _ptr(edges_a)), "fg21_build_regions_ab")
    return Model(out.value, n_alpha * n_beta, k.obs.F, k.obs.T, lab, edges, Nb=n_beta, Na=n_alpha,
                 labels_alpha=lab_a, edges_alpha=edges_a)


def fg21_build_regions_ab_host(sky, obs, n_beta: int, scheme, weighting, n_alpha: int, field,
                               scheme_a="hierarchical", weighting_a="beam"):
    """-> (labels_beta, edges_beta, labels_alpha, edges_alpha, K[Na,Nb,F,T], B[F,T])"""
    k = _Keep(sky, obs)
    opt = fg21_partition_opts(n_beta, SCHEMES[scheme], WEIGHTINGS[weighting])
    aopt, keep = _amp_opts(n_alpha, scheme_a, weighting_a, field)
    lab = np.empty(k.sky.npix, dtype=np.int32)
    edges = np.empty(n_beta + 1)
    lab_a = np.empty(k.sky.npix, dtype=np.int32)
    edges_a = np.empty(n_alpha + 1)
    K = np.empty((n_alpha, n_beta, k.obs.F, k.obs.T))
    B = np.empty((k.obs.F, k.obs.T))
    _check(lib().fg21_build_regions_ab_host(C.byref(k.sky), C.byref(k.obs), C.byref(opt), C.byref(aopt), _ptr(lab),
                                            _ptr(edges), _ptr(lab_a), _ptr(edges_a), _ptr(K), _ptr(B)),
           "fg21_build_regions_ab_host")
    return lab, edges, lab_a, edges_a, K, B


def fg21_model_shape(m: Model) -> dict:
    nb, na, npar = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().fg21_model_shape(m.handle, C.byref(nb), C.byref(na), C.byref(npar)), "fg21_model_shape")
    return dict(n_beta=nb.value, n_alpha=na.value, n_params=npar.value)


def fg21_model_set_data(m: Model, data: np.ndarray):
    d = _f64(data)
    assert d.shape == (m.F, m.T)
    _check(lib().fg21_model_set_data(m.handle, _ptr(d)), "fg21_model_set_data")


def fg21_model_get_arrays(m: Model):
    A = np.empty((m.N, m.F, m.T))
    B = np.empty((m.F, m.T))
    _check(lib().fg21_model_get_arrays(m.handle, _ptr(A), _ptr(B)), "fg21_model_get_arrays")
    return A, B


def fg21_model_info(m: Model) -> dict:
    N, F, T, ne = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    nb = C.c_size_t()
    _check(lib().fg21_model_info(m.handle, C.byref(N), C.byref(F), C.byref(T), C.byref(ne), C.byref(nb)),
           "fg21_model_info")
    return dict(N=N.value, F=F.value, T=T.value, n_empty=ne.value, device_bytes=nb.value)


def fg21_loglike_batch(m: Model, params: np.ndarray, precision="fp16x3", stream: int = 0,
                       out: Optional[np.ndarray] = None) -> np.ndarray:
    """logL of every row of params (host arrays).  `out` (float64 [P], contiguous)
    receives the result when given; page-locked params / out are copied by DMA
    directly, without the library's staging copy."""
    p = _f64(params)
    assert p.ndim == 2 and p.shape[1] == m.n_params, p.shape
    if out is None:
        out = np.empty(p.shape[0])
    assert out.dtype == np.float64 and out.shape == (p.shape[0],) and out.flags.c_contiguous
    _check(lib().fg21_loglike_batch(m.handle, _ptr(p), p.shape[0], _ptr(out), _prec(precision), stream or None),
           "fg21_loglike_batch")
    return out


def fg21_loglike_batch_device(m: Model, d_params: int, P: int, d_logL: int, precision="fp16x3",
                              stream: int = 0):
    _check(lib().fg21_loglike_batch_device(m.handle, d_params, int(P), d_logL, _prec(precision), stream or None),
           "fg21_loglike_batch_device")


def fg21_loglike_batch_device_noalloc(m: Model, d_params: int, P: int, d_logL: int, precision="fp16x3",
                                      stream: int = 0):
    """The device call that allocates nothing (scratch in a static device array)."""
    _check(lib().fg21_loglike_batch_device_noalloc(m.handle, d_params, int(P), d_logL, _prec(precision),
                                                   stream or None), "fg21_loglike_batch_device_noalloc")


def fg21_model_sync_status(m: Model, stream: int = 0) -> int:
    n = C.c_int64()
    _check(lib().fg21_model_sync_status(m.handle, stream or None, C.byref(n)), "fg21_model_sync_status")
    return n.value


def fg21_selftest_mma_rounding(a16: np.ndarray, b16: np.ndarray, c: np.ndarray, stream: int = 0) -> np.ndarray:
    """d = c + a b by one tcgen05.mma (a [128,16], b [16 n, 16 k] float16; c [128,16] float32)."""
    a = np.ascontiguousarray(a16, dtype=np.float16)
    b = np.ascontiguousarray(b16, dtype=np.float16)
    cc = np.ascontiguousarray(c, dtype=np.float32)
    if a.shape != (128, 16) or b.shape != (16, 16) or cc.shape != (128, 16):
        raise ValueError("shapes: a [128, 16], b [16, 16], c [128, 16]")
    d = np.empty((128, 16), dtype=np.float32)
    _check(lib().fg21_selftest_mma_rounding(a.ctypes.data, b.ctypes.data, cc.ctypes.data, d.ctypes.data,
                                            stream or None), "fg21_selftest_mma_rounding")
    return d


def fg21_selftest_bounded_wait(stream: int = 0):
    """-> (return code, device status word, seconds each of the 4 warps waited).
    The expected outcome is FG21_E_DEVICE with bit 0 set: the code is returned,
    not raised."""
    st = C.c_uint32(0)
    el = (C.c_double * 4)()
    rc = lib().fg21_selftest_bounded_wait(C.byref(st), el, stream or None)
    if rc not in (FG21_OK, FG21_E_DEVICE):
        _check(rc, "fg21_selftest_bounded_wait")
    return rc, st.value, list(el)


def fg21_model_timing(m: Model, enable: bool = True):
    _check(lib().fg21_model_timing(m.handle, int(bool(enable))), "fg21_model_timing")


def fg21_model_timing_totals(m: Model):
    """-> (calls, prep_ms, main_ms, reduce_ms) summed over the calls recorded since
    fg21_model_timing(m, True)."""
    n = C.c_int64()
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    _check(lib().fg21_model_timing_totals(m.handle, C.byref(n), C.byref(a), C.byref(b), C.byref(c)),
           "fg21_model_timing_totals")
    return n.value, a.value, b.value, c.value


def fg21_model_eval(m: Model, params: np.ndarray, precision="fp16x3", stream: int = 0) -> np.ndarray:
    p = _f64(params)
    out = np.empty((p.shape[0], m.F, m.T))
    _check(lib().fg21_model_eval(m.handle, _ptr(p), p.shape[0], _ptr(out), _prec(precision), stream or None),
           "fg21_model_eval")
    return out


def fg21_loglike_multi(models: Sequence[Model], params: Sequence[np.ndarray], precision="fp16x3",
                       stream: int = 0):
    n = len(models)
    ps = [_f64(p) for p in params]
    outs = [np.empty(p.shape[0]) for p in ps]
    H = (C.c_void_p * n)(*[m.handle.value for m in models])
    PP = (C.c_void_p * n)(*[_ptr(p) for p in ps])
    NP = (C.c_int64 * n)(*[p.shape[0] for p in ps])
    LL = (C.c_void_p * n)(*[_ptr(o) for o in outs])
    _check(lib().fg21_loglike_multi(H, PP, NP, LL, n, _prec(precision), stream or None), "fg21_loglike_multi")
    return outs


def fg21_autotune(m: Model, d_params: int, P: int, d_logL: int, precision="fp16x3", stream: int = 0):
    """Measured work split for (m, precision, P); returns (channels per item, ms)."""
    cpg, ms = C.c_int32(0), C.c_double(0.0)
    _check(lib().fg21_autotune(m.handle, d_params, int(P), d_logL, _prec(precision), stream or None,
                               C.byref(cpg), C.byref(ms)), "fg21_autotune")
    return cpg.value, ms.value


# ------------------------------------------------------------ CUDA graphs
class Graph:
    """A captured likelihood evaluation of a fixed batch on fixed device buffers
    (fg21_graph_*); `launch` replays it.  The models and buffers must outlive it."""

    def __init__(self, handle: int, models, buffers):
        self.handle = C.c_void_p(handle)
        self._keep = (list(models), list(buffers))

    def launch(self, stream: int = 0):
        fg21_graph_launch(self, stream)

    def sync_status(self, stream: int = 0) -> int:
        return fg21_graph_sync_status(self, stream)

    def close(self):
        if self.handle.value:
            lib().fg21_graph_destroy(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fg21_graph_create(m: Model, d_params: int, P: int, d_logL: int, precision="fp16x3") -> Graph:
    """Device buffers given as integer addresses (e.g. torch tensor data_ptr())."""
    out = C.c_void_p()
    _check(lib().fg21_graph_create(m.handle, d_params, int(P), d_logL, _prec(precision), C.byref(out)),
           "fg21_graph_create")
    return Graph(out.value, [m], [])


def fg21_graph_create_multi(models: Sequence[Model], d_params: Sequence[int], P: Sequence[int],
                            d_logL: Sequence[int], precision="fp16x3") -> Graph:
    n = len(models)
    H = (C.c_void_p * n)(*[m.handle.value for m in models])
    PP = (C.c_void_p * n)(*[int(x) for x in d_params])
    NP = (C.c_int64 * n)(*[int(x) for x in P])
    LL = (C.c_void_p * n)(*[int(x) for x in d_logL])
    out = C.c_void_p()
    _check(lib().fg21_graph_create_multi(H, PP, NP, LL, n, _prec(precision), C.byref(out)),
           "fg21_graph_create_multi")
    return Graph(out.value, models, [])


def fg21_graph_launch(g: Graph, stream: int = 0):
    _check(lib().fg21_graph_launch(g.handle, stream or None), "fg21_graph_launch")


def fg21_graph_sync_status(g: Graph, stream: int = 0) -> int:
    inv = C.c_int64(0)
    _check(lib().fg21_graph_sync_status(g.handle, stream or None, C.byref(inv)), "fg21_graph_sync_status")
    return inv.value


def fg21_graph_destroy(g: Graph):
    g.close()


# ------------------------------------------------------------------ serving
def fg21_noise_loglike(n_cells: int, sigma_noise: float, sigma_n: float, K: int, seed: int, d_L_noise: int,
                       stream: int = 0):
    """L_noise of the accuracy criterion into the DEVICE buffer d_L_noise [K] (asynchronous)."""
    _check(lib().fg21_noise_loglike(int(n_cells), float(sigma_noise), float(sigma_n), int(K), int(seed), d_L_noise,
                                    stream or None), "fg21_noise_loglike")


def fg21_noise_q(d_L_noise: int, K: int, L_bar, stream: int = 0) -> np.ndarray:
    """q_i = P(L_noise <= L_bar_i) for each L_bar_i (waits for the stream)."""
    b = _f64(np.atleast_1d(L_bar))
    q = np.empty(b.shape[0])
    _check(lib().fg21_noise_q(d_L_noise, int(K), _ptr(b), b.shape[0], _ptr(q), stream or None), "fg21_noise_q")
    return q


class Server:
    """Owner of an fg21_server handle."""

    def __init__(self, mem_budget_bytes=60 << 30, max_batch_points=65536, max_wait_us=200, max_inflight=2,
                 precision="fp16x3", device=0):
        o = fg21_serve_opts(int(mem_budget_bytes), int(max_batch_points), int(max_wait_us), int(max_inflight),
                            _prec(precision), int(device))
        h = C.c_void_p()
        _check(lib().fg21_serve_create(C.byref(o), C.byref(h)), "fg21_serve_create")
        self.handle = h
        self._pending = {}

    def close(self):
        if self.handle:
            lib().fg21_serve_destroy(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fg21_serve_register_run(s: Server, m: Model):
    """-> (run_id, admitted: bool)"""
    rid = C.c_int32()
    rc = lib().fg21_serve_register_run(s.handle, m.handle, C.byref(rid))
    if rc not in (FG21_OK, FG21_E_BUSY):
        _check(rc, "fg21_serve_register_run")
    return rid.value, rc == FG21_OK


def fg21_serve_unregister_run(s: Server, run_id: int):
    _check(lib().fg21_serve_unregister_run(s.handle, int(run_id)), "fg21_serve_unregister_run")


def fg21_serve_submit(s: Server, run_id: int, params: np.ndarray):
    """-> (ticket, logL output array filled when the ticket completes)"""
    p = _f64(params)
    out = np.empty(p.shape[0])
    t = C.c_int64()
    _check(lib().fg21_serve_submit(s.handle, int(run_id), _ptr(p), p.shape[0], _ptr(out), C.byref(t)),
           "fg21_serve_submit")
    s._pending[t.value] = out
    return t.value, out


def fg21_serve_wait(s: Server, ticket: int, timeout_ms: int = -1) -> int:
    rc = lib().fg21_serve_wait(s.handle, int(ticket), int(timeout_ms))
    if rc != FG21_E_TIMEOUT:
        s._pending.pop(ticket, None)
    return rc


def fg21_serve_poll(s: Server, ticket: int) -> int:
    rc = lib().fg21_serve_poll(s.handle, int(ticket))
    if rc != FG21_E_BUSY:
        s._pending.pop(ticket, None)
    return rc


def fg21_serve_cancel(s: Server, ticket: int) -> int:
    return lib().fg21_serve_cancel(s.handle, int(ticket))


def fg21_serve_stats(s: Server) -> dict:
    st = fg21_stats()
    _check(lib().fg21_serve_stats(s.handle, C.byref(st)), "fg21_serve_stats")
    return {k: getattr(st, k) for k, _ in fg21_stats._fields_}
