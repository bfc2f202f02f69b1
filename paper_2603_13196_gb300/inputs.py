"""Seeded synthetic inputs for the region-partitioned global-21cm likelihood.

This module is the single fixture writer shared by the CUDA library's callers
(tests, bench, smoke) and the FP64 oracle.  It holds none of the method's
arithmetic: no beam, no weighting, no partition, no forward model and no
likelihood.  It only draws the raw inputs the method consumes:

* a pixelised sky (unit direction vectors in Galactic coordinates, the
  230 MHz template T230 and a per-pixel spectral index beta);
* the observation (channel frequencies, the beam's chromatic exponent p(nu),
  the zenith direction for each LST bin);
* parameter vectors theta_p = [beta_1..beta_N, A21, nu21, sigma21, sigma_n]
  (with amplitude scale factors alpha_1..alpha_Na after the betas for the
  joint amplitude / spectral-index model) drawn from the prior, or scattered
  around a chosen point;
* the per-pixel field the amplitude regions partition (ln T230);
* standard-normal noise draws.

The paper's own inputs (the 2008 Global Sky Model at N_side = 512, an
EM-simulated conical log-spiral beam and real observing dates, Sec. 2.1 and
the observing-window table) are not available; the recipe below stands in for
them with the same shapes and value structure: a bright Galactic plane
(T230 = 150 + 3000 exp(-|b|/8 deg) K times lognormal scatter), spectral
indices around 2.55 with a smooth longitude pattern, a broad cos^p beam whose
exponent oscillates with frequency (beam chromaticity), and a southern site
(latitude -30.7 deg) observing for a window of LST.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

BASE_SEED = 2603131960
# sub-stream ids of the seed tree: sky lognormal, beta noise, data noise,
# parameters, request arrivals / run mix
SUB_SKY, SUB_BETA, SUB_NOISE, SUB_PARAMS, SUB_ARRIVALS = 1, 2, 3, 4, 5

T_CMB = 2.725          # K; the paper never prints T_CMB, this is the standard value
NU0_MHZ = 230.0        # reference frequency of the template map (Sec. 2.1)
SITE_LAT_DEG = -30.7   # synthetic southern site
FIDUCIAL_T21 = (0.155, 85.0, 15.0)   # A21 [K], nu21 [MHz], sigma21 [MHz] (Sec. 2.1)
NOISE_K = 0.025        # 25 mK Gaussian noise (Sec. 2.1)

# IAU 1958 / J2000 rotation from equatorial (ICRS) to Galactic unit vectors.
_EQ_TO_GAL = np.array([
    [-0.0548755604162154, -0.8734370902348850, -0.4838350155487132],
    [+0.4941094278755837, -0.4448296299600112, +0.7469822444972189],
    [-0.8676661490190047, -0.1980763734312015, +0.4559837761750669],
])

# Prior ranges of the synthetic workloads (config ranges; the paper's table of
# priors uses sigma21 in [10, 20] and sigma_n in [1e-4, 1e-1]).
PRIOR = dict(beta=(2.45, 3.15), A21=(0.0, 0.25), nu21=(50.0, 200.0),
             sigma21=(5.0, 40.0), sigma_n=(1e-3, 0.1))


def rng(seed: int, sub: int, extra: int = 0) -> np.random.Generator:
    """Counter-free, reproducible stream `sub` of workload seed `seed`."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, sub, extra])))


@dataclasses.dataclass
class Sky:
    dirs: np.ndarray     # [Npix, 3] unit vectors, Galactic frame
    t230: np.ndarray     # [Npix] K
    beta: np.ndarray     # [Npix]

    @property
    def npix(self) -> int:
        return int(self.t230.shape[0])


@dataclasses.dataclass
class Obs:
    nu: np.ndarray       # [F] MHz
    zenith: np.ndarray   # [T, 3] unit vectors, Galactic frame
    beam_p: np.ndarray   # [F] exponent of the cos^p beam
    nu0: float = NU0_MHZ
    t_cmb: float = T_CMB

    @property
    def F(self) -> int:
        return int(self.nu.shape[0])

    @property
    def T(self) -> int:
        return int(self.zenith.shape[0])


def fibonacci_sphere(npix: int) -> np.ndarray:
    """Near-equal-area points: z = 1 - 2(k+1/2)/Npix, phi = pi(1+sqrt5)(k+1/2)."""
    k = np.arange(npix, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * k / npix
    phi = math.pi * (1.0 + math.sqrt(5.0)) * k
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def make_sky(npix: int, seed: int, beta_const: Optional[float] = None,
             t230_const: Optional[float] = None) -> Sky:
    dirs = fibonacci_sphere(npix)
    b = np.arcsin(np.clip(dirs[:, 2], -1.0, 1.0))
    l = np.arctan2(dirs[:, 1], dirs[:, 0])
    if t230_const is None:
        scatter = np.exp(0.3 * rng(seed, SUB_SKY).standard_normal(npix))
        t230 = (150.0 + 3000.0 * np.exp(-np.abs(b) / math.radians(8.0))) * scatter
    else:
        t230 = np.full(npix, float(t230_const))
    if beta_const is None:
        beta = 2.55 + 0.1 * np.sin(l) + 0.02 * rng(seed, SUB_BETA).standard_normal(npix)
    else:
        beta = np.full(npix, float(beta_const))
    return Sky(dirs=np.ascontiguousarray(dirs), t230=t230, beta=beta)


def channels(F: int, lo: float = 50.0, hi: float = 200.0) -> np.ndarray:
    return np.linspace(lo, hi, F)


def beam_exponent(nu: np.ndarray, achromatic: Optional[float] = None) -> np.ndarray:
    if achromatic is not None:
        return np.full_like(nu, float(achromatic))
    return 1.5 + 0.3 * np.sin(2.0 * math.pi * nu / 40.0)


def zenith_track(T: int, window_h: float, lst0_h: float = 0.0,
                 lat_deg: float = SITE_LAT_DEG) -> np.ndarray:
    """Zenith unit vectors (Galactic) at LST_k = LST0 + (k+1/2) window / T."""
    lst_h = lst0_h + (np.arange(T) + 0.5) * (window_h / T)
    ang = lst_h * (2.0 * math.pi / 24.0)
    lat = math.radians(lat_deg)
    eq = np.stack([math.cos(lat) * np.cos(ang), math.cos(lat) * np.sin(ang),
                   np.full(T, math.sin(lat))], axis=1)
    gal = eq @ _EQ_TO_GAL.T
    return gal / np.linalg.norm(gal, axis=1, keepdims=True)


def make_obs(F: int, T: int, window_h: float, lst0_h: float = 0.0,
             achromatic_p: Optional[float] = None, lo: float = 50.0,
             hi: float = 200.0) -> Obs:
    nu = channels(F, lo, hi)
    return Obs(nu=nu, zenith=zenith_track(T, window_h, lst0_h), beam_p=beam_exponent(nu, achromatic_p))


def prior_draws(P: int, N: int, seed: int, extra: int = 0, prior: dict = PRIOR) -> np.ndarray:
    """[P, N+4] rows [beta_1..beta_N, A21, nu21, sigma21, sigma_n]; sigma_n log-uniform."""
    g = rng(seed, SUB_PARAMS, extra)
    out = np.empty((P, N + 4))
    out[:, :N] = g.uniform(*prior["beta"], size=(P, N))
    out[:, N] = g.uniform(*prior["A21"], size=P)
    out[:, N + 1] = g.uniform(*prior["nu21"], size=P)
    out[:, N + 2] = g.uniform(*prior["sigma21"], size=P)
    lo, hi = prior["sigma_n"]
    out[:, N + 3] = np.exp(g.uniform(math.log(lo), math.log(hi), size=P))
    return out


# Amplitude scale factors alpha_i of the joint amplitude / spectral-index model
# (a gain correction of the template; the paper gives no prior for them).
PRIOR_ALPHA = (0.9, 1.1)


def amplitude_field(sky: Sky) -> np.ndarray:
    """The per-pixel value the amplitude regions partition: ln T230 (regions of
    similar template brightness share one scale factor)."""
    return np.log(sky.t230)


def prior_draws_ab(P: int, Nb: int, Na: int, seed: int, extra: int = 0, prior: dict = PRIOR,
                   alpha: tuple = PRIOR_ALPHA) -> np.ndarray:
    """[P, Nb+Na+4] rows [beta_1..beta_Nb, alpha_1..alpha_Na, A21, nu21, sigma21,
    sigma_n]; alpha uniform in `alpha`, the rest as prior_draws."""
    base = prior_draws(P, Nb, seed, extra, prior)
    a = rng(seed, SUB_PARAMS, 500 + extra).uniform(*alpha, size=(P, Na))
    return np.concatenate([base[:, :Nb], a, base[:, Nb:]], axis=1)


def scatter_around(theta: np.ndarray, P: int, dbeta: float, seed: int, extra: int = 0,
                   d21: float = 0.0) -> np.ndarray:
    """P copies of theta with beta_i moved by U(-dbeta, dbeta) (and, if d21 > 0,
    A21/nu21/sigma21 moved by relative U(-d21, d21)); sigma_n is kept."""
    theta = np.asarray(theta, dtype=np.float64)
    N = theta.shape[0] - 4
    g = rng(seed, SUB_PARAMS, 1000 + extra)
    out = np.repeat(theta[None, :], P, axis=0)
    out[:, :N] += g.uniform(-dbeta, dbeta, size=(P, N))
    if d21 > 0:
        out[:, N:N + 3] *= 1.0 + g.uniform(-d21, d21, size=(P, 3))
    return out


def noise_draws(F: int, T: int, seed: int, extra: int = 0) -> np.ndarray:
    return rng(seed, SUB_NOISE, extra).standard_normal((F, T))


@dataclasses.dataclass
class Workload:
    """One synthetic workload of the likelihood path."""
    name: str
    npix: int
    N: int
    F: int
    T: int
    window_h: float
    P: int
    scheme: str = "recursive"      # recursive | hierarchical | linear | percentile
    weighting: str = "beam"        # beam | sky | horizon | uniform
    seed: int = BASE_SEED
    lst0_h: float = 0.0

    def sky(self) -> Sky:
        return make_sky(self.npix, self.seed)

    def obs(self) -> Obs:
        return make_obs(self.F, self.T, self.window_h, self.lst0_h)

    def params(self, P: Optional[int] = None, extra: int = 0) -> np.ndarray:
        return prior_draws(self.P if P is None else P, self.N, self.seed, extra)

    def noise(self) -> np.ndarray:
        return noise_draws(self.F, self.T, self.seed)


def workload(k: int) -> Workload:
    """Workloads 1-3 of the likelihood path (4 and 5 are built from `uneven_batch`
    and the serving mix)."""
    if k == 1:
        return Workload("c1_npix3072_N3_F151_T1_P64", 3072, 3, 151, 1, 0.0, 64,
                        scheme="hierarchical", seed=BASE_SEED + 1)
    if k == 2:
        return Workload("c2_npix12288_N9_F151_T20_P4096", 12288, 9, 151, 20, 6.0, 4096,
                        seed=BASE_SEED + 2)
    if k == 3:
        return Workload("c3_npix49152_N24_F301_T100_P16384", 49152, 24, 301, 100, 12.0, 16384,
                        seed=BASE_SEED + 3)
    raise ValueError(k)


def uneven_batch(n_models: int = 32, seed: int = BASE_SEED + 4, npix: int = 3072,
                 F: int = 151, N_range=(4, 30), T_range=(1, 60), P_range=(256, 8192)):
    """Workload 4: n_models instances with N ~ U{4..30}, T ~ U{1..60},
    P ~ U{256..8192}; each with its own LST start (and so its own partition)."""
    g = rng(seed, SUB_ARRIVALS)
    out = []
    for m in range(n_models):
        N = int(g.integers(N_range[0], N_range[1] + 1))
        T = int(g.integers(T_range[0], T_range[1] + 1))
        P = int(g.integers(P_range[0], P_range[1] + 1))
        lst0 = float(g.uniform(0.0, 24.0))
        window = 0.0 if T == 1 else float(g.choice([1.0, 4.0, 6.0, 12.0]))
        out.append(Workload(f"m{m}_N{N}_T{T}_P{P}", npix, N, F, T, window, P,
                            seed=seed * 100 + m, lst0_h=lst0))
    return out


@dataclasses.dataclass
class ServingRun:
    """One nested-sampling run of the serving workload: its own 3072-pixel sky,
    F = 151 channels, N regions, T LST bins over its own window."""
    N: int
    T: int
    window_h: float
    lst0_h: float
    sky_seed: int
    noise_seed: int
    npix: int = 3072
    F: int = 151

    def sky(self) -> Sky:
        return make_sky(self.npix, self.sky_seed)

    def obs(self) -> Obs:
        return make_obs(self.F, self.T, self.window_h, lst0_h=self.lst0_h)

    def noise(self) -> np.ndarray:
        return noise_draws(self.F, self.T, self.noise_seed)


def serving_mix(n_runs: int = 64, n_requests: int = 256):
    """Workload 5: n_runs runs (N cycling through 5, 9, 14, 20, 30; T through 1,
    10, 50, each with its own window and LST start) and a pool of n_requests
    requests (run index, prior draws of 128..4096 points) to uniformly chosen
    runs.  -> (runs, [(run index, params)])."""
    g = rng(BASE_SEED + 5, SUB_ARRIVALS)
    Ns, Ts = [5, 9, 14, 20, 30], [1, 10, 50]
    runs = []
    for k in range(n_runs):
        N, T = Ns[k % 5], Ts[(k // 5) % 3]
        window = 0.0 if T == 1 else float(g.choice([2.0, 6.0, 12.0]))
        lst0 = float(g.uniform(0, 24))
        runs.append(ServingRun(N, T, window, lst0, BASE_SEED + 500 + k, k))
    reqs = []
    for j in range(n_requests):
        k = int(g.integers(0, n_runs))
        P = int(g.integers(128, 4097))
        reqs.append((k, prior_draws(P, runs[k].N, seed=j, extra=k)))
    return runs, reqs

