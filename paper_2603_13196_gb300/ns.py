"""Minimal batched nested slice sampling (Sec. 3 of arXiv 2603.13196).

Nested sampling (Sec. 3.1.2, eq. evidence_sum) with batched deletion: each
iteration removes the `num_delete` lowest-likelihood live points at once and
replaces them by as many independent slice-sampling chains, each constrained
to L > L_min,b (the largest likelihood of the deleted batch).  The i-th
deleted point of a batch (i = 0..b-1, ascending L) dies while n - i points are
live, so its expected log prior-volume shrinkage is 1/(n - i) (eq. log_xgpu);
its quadrature weight is X_before - X_after.

Replacement chains (Sec. 3.1.3): each starts from a randomly chosen surviving
live point and takes `num_inner_steps` hit-and-run slice steps in the unit
hypercube of the prior, along directions drawn in the geometry whitened by the
live points' covariance (a Cholesky factor of it), with a unit initial
bracket in whitened coordinates, stepping out and shrinkage (Neal's slice
sampler).  All chains advance in lock-step: every round gathers one candidate
per active chain and evaluates them as one batch, which is what makes the
likelihood a batched, GPU-friendly workload.

`loglike` is any callable mapping params [P, D] to logL [P] (the serving loop
of libfg21 through ServeLikelihood, or the FP64 oracle for a reference run).
The termination rule (not stated in the paper) is the usual one: stop when the
live points' remaining evidence, X * mean(L_live), is below exp(-3) of Z.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional

import numpy as np


@dataclasses.dataclass
class Prior:
    """Independent priors per parameter: 'uniform' on [lo, hi] or 'loguniform'."""
    kinds: list
    lo: np.ndarray
    hi: np.ndarray

    def transform(self, u: np.ndarray) -> np.ndarray:
        u = np.atleast_2d(u)
        out = np.empty_like(u)
        for j, k in enumerate(self.kinds):
            if k == "uniform":
                out[:, j] = self.lo[j] + (self.hi[j] - self.lo[j]) * u[:, j]
            else:
                a, b = math.log(self.lo[j]), math.log(self.hi[j])
                out[:, j] = np.exp(a + (b - a) * u[:, j])
        return out

    @property
    def dim(self) -> int:
        return len(self.kinds)


def region_model_prior(N: int, beta=(2.45, 3.15), a21=(0.0, 0.25), nu21=(50.0, 200.0), s21=(5.0, 40.0),
                       sigma=(1e-3, 0.1)) -> Prior:
    """Priors of the foreground + trough model (table of priors, Sec. 2.3.2, with
    the workload ranges): uniform beta_i, A21, nu21, sigma21; log-uniform sigma_n."""
    kinds = ["uniform"] * (N + 3) + ["loguniform"]
    lo = np.array([beta[0]] * N + [a21[0], nu21[0], s21[0], sigma[0]], dtype=float)
    hi = np.array([beta[1]] * N + [a21[1], nu21[1], s21[1], sigma[1]], dtype=float)
    return Prior(kinds, lo, hi)


@dataclasses.dataclass
class NSResult:
    logZ: float
    logZ_err: float            # sqrt(H / n_live)
    H: float                   # information (KL of posterior from prior)
    n_like: int                # likelihood evaluations
    n_rounds: int              # batched likelihood calls
    iterations: int
    logL_max: float
    dead_logL: np.ndarray
    dead_logw: np.ndarray      # log prior-volume weights of the dead points
    dead_theta: np.ndarray


def _logsumexp(a):
    a = np.asarray(a, dtype=float)
    m = np.max(a)
    if not np.isfinite(m):
        return m
    return m + math.log(np.sum(np.exp(a - m)))


class NestedSlice:
    """Batched nested slice sampler in the unit hypercube of `prior`."""

    def __init__(self, prior: Prior, loglike: Callable[[np.ndarray], np.ndarray], n_live: int = 500,
                 num_delete: Optional[int] = None, num_inner_steps: Optional[int] = None, seed: int = 0,
                 step_width: float = 1.0, max_step_out: int = 8, max_shrink: int = 60):
        self.prior = prior
        self.loglike = loglike
        self.D = prior.dim
        self.n = n_live
        self.b = num_delete if num_delete is not None else max(1, int(0.2 * n_live))
        self.steps = num_inner_steps if num_inner_steps is not None else 5 * self.D
        self.rng = np.random.default_rng(seed)
        self.w = step_width
        self.max_out = max_step_out
        self.max_shrink = max_shrink
        self.n_like = 0
        self.n_rounds = 0

    def _eval(self, u: np.ndarray) -> np.ndarray:
        self.n_like += u.shape[0]
        self.n_rounds += 1
        out = np.asarray(self.loglike(self.prior.transform(u)), dtype=float)
        return np.where(np.isnan(out), -np.inf, out)

    def _eval_cube(self, u: np.ndarray) -> np.ndarray:
        """logL for points in the cube, -inf outside (the prior's support)."""
        inside = np.all((u > 0.0) & (u < 1.0), axis=1)
        out = np.full(u.shape[0], -np.inf)
        if inside.any():
            out[inside] = self._eval(u[inside])
        return out

    def _directions(self, live_u: np.ndarray, k: int) -> np.ndarray:
        cov = np.cov(live_u.T) + 1e-12 * np.eye(self.D)
        Lc = np.linalg.cholesky(cov)
        g = self.rng.standard_normal((k, self.D))
        g /= np.linalg.norm(g, axis=1, keepdims=True)
        return g @ Lc.T                     # unit whitened step mapped to the cube

    def _slice_step(self, x: np.ndarray, lx: np.ndarray, Lmin: float, d: np.ndarray):
        """One hit-and-run slice step for every chain (rows of x), in lock-step rounds."""
        k = x.shape[0]
        r = self.rng.uniform(size=k)
        lo = -r * self.w
        hi = (1.0 - r) * self.w
        # stepping out, both ends, batched over the chains still expanding
        exp_lo = np.ones(k, bool)
        exp_hi = np.ones(k, bool)
        for _ in range(self.max_out):
            il, ih = np.nonzero(exp_lo)[0], np.nonzero(exp_hi)[0]
            if il.size + ih.size == 0:
                break
            cand = np.concatenate([x[il] + lo[il, None] * d[il], x[ih] + hi[ih, None] * d[ih]])
            lc = self._eval_cube(cand)
            out_lo = lc[:il.size] > Lmin
            out_hi = lc[il.size:] > Lmin
            lo[il[out_lo]] -= self.w
            hi[ih[out_hi]] += self.w
            exp_lo[il[~out_lo]] = False
            exp_hi[ih[~out_hi]] = False
        # shrinkage until a point inside the slice is found
        new_x = x.copy()
        new_l = lx.copy()
        active = np.ones(k, bool)
        for _ in range(self.max_shrink):
            idx = np.nonzero(active)[0]
            if idx.size == 0:
                break
            t = self.rng.uniform(lo[idx], hi[idx])
            cand = x[idx] + t[:, None] * d[idx]
            lc = self._eval_cube(cand)
            ok = lc > Lmin
            acc = idx[ok]
            new_x[acc] = cand[ok]
            new_l[acc] = lc[ok]
            active[acc] = False
            rej = idx[~ok]
            tr = t[~ok]
            lo[rej] = np.where(tr < 0, tr, lo[rej])
            hi[rej] = np.where(tr >= 0, tr, hi[rej])
        return new_x, new_l

    # ------------------------------------------------------------ state
    def _start(self):
        u = self.rng.uniform(size=(self.n, self.D))
        self._st = dict(u=u, lu=self._eval(u), logX=0.0, logZ=-np.inf, it=0, dead_l=[], dead_w=[], dead_t=[])

    def state_dict(self) -> dict:
        """A checkpoint of the run: live points, their likelihoods, the prior
        volume, the evidence so far, the dead points, the counters and the
        random generator's state.  `load_state` on a sampler built with the same
        prior, likelihood and settings continues the run exactly."""
        st = self._st
        return {"u": st["u"].copy(), "lu": st["lu"].copy(), "logX": st["logX"], "logZ": float(st["logZ"]),
                "it": st["it"], "dead_l": list(st["dead_l"]), "dead_w": list(st["dead_w"]),
                "dead_t": [t.copy() for t in st["dead_t"]], "n_like": self.n_like, "n_rounds": self.n_rounds,
                "rng": self.rng.bit_generator.state, "settings": (self.n, self.b, self.steps, self.D)}

    def load_state(self, state: dict):
        if tuple(state["settings"]) != (self.n, self.b, self.steps, self.D):
            raise ValueError("checkpoint of a run with other settings")
        self._st = {"u": state["u"].copy(), "lu": state["lu"].copy(), "logX": state["logX"],
                    "logZ": state["logZ"], "it": state["it"], "dead_l": list(state["dead_l"]),
                    "dead_w": list(state["dead_w"]), "dead_t": [t.copy() for t in state["dead_t"]]}
        self.n_like = state["n_like"]
        self.n_rounds = state["n_rounds"]
        self.rng.bit_generator.state = state["rng"]

    def _iterate(self, tol_logz: float) -> bool:
        """One batched deletion and replacement; True when the run has converged."""
        st = self._st
        u, lu = st["u"], st["lu"]
        st["it"] += 1
        order = np.argsort(lu, kind="stable")
        kill = order[:self.b]
        keep = order[self.b:]
        Lmin = lu[kill[-1]]
        logX, logZ = st["logX"], st["logZ"]
        for i, j in enumerate(kill):
            logX_new = logX - 1.0 / (self.n - i)
            logw = logX + math.log1p(-math.exp(logX_new - logX))
            st["dead_l"].append(lu[j])
            st["dead_w"].append(logw)
            st["dead_t"].append(u[j].copy())
            logZ = np.logaddexp(logZ, lu[j] + logw)
            logX = logX_new
        st["logX"], st["logZ"] = logX, logZ
        # replacements: chains from random survivors, whitened directions
        start = keep[self.rng.integers(0, keep.size, size=self.b)]
        x = u[start].copy()
        lx = lu[start].copy()
        for _ in range(self.steps):
            d = self._directions(u[keep], self.b)
            x, lx = self._slice_step(x, lx, Lmin, d)
        u[kill] = x
        lu[kill] = lx
        live_logZ = logX + _logsumexp(lu) - math.log(self.n)
        return live_logZ - logZ < tol_logz

    def _finish(self) -> NSResult:
        st = self._st
        u, lu, logX, logZ = st["u"], st["lu"], st["logX"], st["logZ"]
        dead_l, dead_w, dead_t = list(st["dead_l"]), list(st["dead_w"]), list(st["dead_t"])
        # remaining live points share the final volume equally
        for j in np.argsort(lu):
            logw = logX - math.log(self.n)
            dead_l.append(lu[j])
            dead_w.append(logw)
            dead_t.append(u[j].copy())
            logZ = np.logaddexp(logZ, lu[j] + logw)
        dl, dw = np.array(dead_l), np.array(dead_w)
        post = np.exp(dl + dw - logZ)
        H = float(np.sum(post * (dl - logZ)))
        return NSResult(logZ=float(logZ), logZ_err=math.sqrt(max(H, 0.0) / self.n), H=H, n_like=self.n_like,
                        n_rounds=self.n_rounds, iterations=st["it"], logL_max=float(np.max(dl)), dead_logL=dl,
                        dead_logw=dw, dead_theta=self.prior.transform(np.array(dead_t)))

    def run(self, max_iter: int = 100000, tol_logz: float = -3.0, stop_after: Optional[int] = None,
            resume: Optional[dict] = None) -> Optional[NSResult]:
        """Run to convergence (or max_iter iterations).  resume: a state_dict to
        continue from.  stop_after: return None after that many more iterations
        without finishing (take state_dict() then, to checkpoint)."""
        if resume is not None:
            self.load_state(resume)
        else:
            self._start()
        done = 0
        while self._st["it"] < max_iter:
            if stop_after is not None and done >= stop_after:
                return None
            done += 1
            if self._iterate(tol_logz):
                break
        return self._finish()


def expected_log_shrinkage(n: int, b: int) -> float:
    """E[log X] after one batched deletion of b points from n (eq. log_xgpu)."""
    return -sum(1.0 / (n - i) for i in range(b))


class ServeLikelihood:
    """Batched likelihood through libfg21's serving loop: each call is one
    request of a registered run (the run shares the GPU with other runs)."""

    def __init__(self, fg21, server, model, timeout_ms: int = 120000):
        self.fg21 = fg21
        self.server = server
        self.run_id, _ = fg21.fg21_serve_register_run(server, model)
        self.timeout = timeout_ms

    def __call__(self, params: np.ndarray) -> np.ndarray:
        t, out = self.fg21.fg21_serve_submit(self.server, self.run_id, params)
        rc = self.fg21.fg21_serve_wait(self.server, t, self.timeout)
        if rc != 0:
            raise RuntimeError(f"serve request failed with status {rc}")
        return out

    def close(self):
        self.fg21.fg21_serve_unregister_run(self.server, self.run_id)
