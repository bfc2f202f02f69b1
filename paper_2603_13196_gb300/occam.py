"""The maximum-likelihood side of the Occam experiment (Sec. 4.1 and Sec. 6.1
of arXiv 2603.13196): log L_max as a function of the number of regions N for
nested partition schemes (Algorithms 1 and 2) and for the observation-
independent linear and percentile splits.

Nested schemes make level N a special case of level N+1: the optimum at N,
with the split parent's spectral index given to both children, is a point of
the (N+1)-region model with the same forward model and likelihood (the
embedding identity).  A maximiser that starts level N+1 from that embedded
point and never discards its best candidate therefore returns a log L_max
that cannot decrease with N.  Linear and percentile splits redefine every
boundary at each N, so no such start exists and log L_max(N) may fall, which
is the inconsistency Sec. 4.1 describes.

Search: a batched cross-entropy maximiser over the spectral indices with the
21-cm trough held at given values and sigma_n profiled out analytically
(sigma^2 = chi^2 / (F T) maximises eq. likelihood, so log L_max =
-F T (ln(2 pi chi^2 / (F T)) + 1) / 2).  Every round evaluates one batch of
candidates with fg21_loglike_batch_device on the GPU (at sigma_n = 1 K, where
chi^2 = -2 log L - F T ln 2 pi), keeps the best point seen so far, and refits
the sampling distribution to the elite candidates.  This host-side driver
only proposes points; every likelihood runs in the library's kernels.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

from . import fg21


@dataclasses.dataclass
class LmaxResult:
    N: int
    scheme: str
    logL_max: float          # profiled over sigma_n
    chi2: float
    beta: np.ndarray         # the maximiser's spectral indices
    edges: np.ndarray
    n_evals: int


def profiled_logL(chi2: np.ndarray, n_cells: int) -> np.ndarray:
    """log L maximised over sigma_n for a given chi^2 (eq. likelihood)."""
    return -0.5 * n_cells * (np.log(2.0 * math.pi * np.asarray(chi2) / n_cells) + 1.0)


class Maximiser:
    """Batched cross-entropy search over beta on one model, on the GPU."""

    def __init__(self, model: "fg21.Model", trough: Sequence[float], precision: str = "fp32_delta",
                 batch: int = 4096, n_elite: int = 64, seed: int = 0):
        import torch
        self.torch = torch
        self.model = model
        self.trough = np.asarray(trough, dtype=np.float64)
        self.precision = precision
        self.batch = batch
        self.n_elite = n_elite
        self.rng = np.random.default_rng(seed)
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.d_params = torch.empty((batch, model.N + 4), dtype=torch.float64, device=self.dev)
        self.d_logL = torch.empty(batch, dtype=torch.float64, device=self.dev)
        self.n_evals = 0

    def chi2(self, beta: np.ndarray) -> np.ndarray:
        """chi^2 of each row of beta [B, N] (B <= batch) from one GPU call."""
        B = beta.shape[0]
        th = np.empty((B, self.model.N + 4))
        th[:, :self.model.N] = beta
        th[:, self.model.N:self.model.N + 3] = self.trough
        th[:, -1] = 1.0
        self.d_params[:B].copy_(self.torch.from_numpy(th))
        s = self.torch.cuda.current_stream().cuda_stream
        fg21.fg21_loglike_batch_device(self.model, self.d_params.data_ptr(), B, self.d_logL.data_ptr(),
                                       self.precision, s)
        fg21.fg21_model_sync_status(self.model, s)
        L = self.d_logL[:B].cpu().numpy()
        self.n_evals += B
        n = self.model.F * self.model.T
        return -2.0 * L - n * math.log(2.0 * math.pi)

    def run(self, start: np.ndarray, width: float, rounds: int = 40, bounds=(1.5, 4.5)):
        """Maximise from `start` (always one of the candidates); returns
        (best beta, its chi^2)."""
        N = self.model.N
        best = np.asarray(start, dtype=np.float64).copy()
        best_c2 = float(self.chi2(best[None])[0])
        mean, std = best.copy(), np.full(N, float(width))
        for _ in range(rounds):
            cand = mean[None] + std[None] * self.rng.standard_normal((self.batch - 1, N))
            cand = np.clip(np.concatenate([best[None], cand]), *bounds)
            c2 = self.chi2(cand)
            order = np.argsort(c2)
            if c2[order[0]] < best_c2:
                best, best_c2 = cand[order[0]].copy(), float(c2[order[0]])
            elite = cand[order[:self.n_elite]]
            mean = elite.mean(axis=0)
            std = np.maximum(elite.std(axis=0), 1e-7)
        return best, best_c2


def region_mean_beta(sky, labels: np.ndarray, N: int, w: Optional[np.ndarray] = None) -> np.ndarray:
    """A starting point: each region's (importance-weighted) mean spectral
    index; regions without pixels start at the mean of all pixels."""
    out = np.full(N, float(np.mean(sky.beta)))
    for i in range(N):
        m = labels == i
        if m.any():
            ww = np.ones(int(m.sum())) if w is None else w[m]
            out[i] = float(np.sum(sky.beta[m] * ww) / max(np.sum(ww), 1e-300)) if ww.sum() > 0 else sky.beta[m].mean()
    return out


def embed(beta_prev: np.ndarray, edges_prev: np.ndarray, edges_next: np.ndarray) -> np.ndarray:
    """The (N+1)-region point equal to an N-region point of a nested scheme:
    region j of level N+1 (the interval ending at edges_next[j+1]) inherits the
    spectral index of the level-N region that contains it."""
    N1 = len(edges_next) - 1
    parent = np.array([int(np.sum(edges_prev[1:-1] < edges_next[j + 1])) for j in range(N1)])
    return beta_prev[parent]


def logl_max_curve(sky, obs, data, scheme: str, N_values: Sequence[int], trough: Sequence[float],
                   weighting: str = "beam", rounds: int = 40, batch: int = 4096, seed: int = 0,
                   precision: str = "fp32_delta"):
    """log L_max(N) for one scheme.  Nested schemes (recursive, hierarchical)
    start each level from the embedded optimum of the previous one (after an
    independent start at the first N); linear and percentile splits start every
    level afresh from the region means."""
    nested = scheme in ("recursive", "hierarchical")
    out = []
    prev = None
    for N in N_values:
        model = fg21.fg21_build_regions(sky, obs, N, scheme, weighting)
        fg21.fg21_model_set_data(model, data)
        mx = Maximiser(model, trough, precision=precision, batch=batch, seed=seed + N)
        if nested and prev is not None:
            start, width = embed(prev.beta, prev.edges, model.edges), 0.01
        else:
            start, width = region_mean_beta(sky, model.labels, N), 0.05
        beta, c2 = mx.run(start, width, rounds=rounds)
        res = LmaxResult(N, scheme, float(profiled_logL(c2, obs.F * obs.T)), c2, beta, model.edges.copy(),
                         mx.n_evals)
        out.append(res)
        prev = res
        model.close()
    return out
