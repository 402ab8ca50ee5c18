"""Bayesian training of the sparse nonstationary GP by Markov chain Monte Carlo (App. C).

Per iteration, in this order:
  1. the mean coefficients beta;
  2. the core variance, the noise variance tau^2 and the Wendland s0 and r0;
  3. the bump positions h_ij and radii r_ij.
Each of these three blocks is an adaptive block Metropolis-Hastings random walk: Haario, Saksman and Tamminen
(2001), with the log-adaptive scaling of Shaby and Wells (2010).
  4. All amplitudes a_ij at once, binary, proposed from their prior Bernoulli(pi_ij^curr). The proposal equals the
     prior, so the acceptance ratio is the likelihood ratio alone.
  5. Closed-form Gibbs draws pi_ij ~ Beta(1 + a_ij, 2 - a_ij). That is the full conditional of pi_ij under its
     uniform prior and the Bernoulli amplitude.

B chains advance in lockstep, so every block update evaluates B proposals in one batched factorization.
Block 1 leaves C_z alone and only needs the solves with new residuals r = z - W beta.

Priors (App. C asks for proper, noninformative ones and leaves the choice open):
  - beta ~ N(0, k I) with k = 100^2 (Sec. 2.3);
  - every other continuous parameter uniform on a bounded interval the caller states;
  - pi_ij ~ U(0, 1) and a_ij | pi_ij ~ Bernoulli(pi_ij) (App. C).
The random walks move in unconstrained coordinates: logit of the position inside each interval. The target
there carries the transform's Jacobian, so the chain samples the stated prior times the likelihood.

Random numbers come from one seeded numpy Generator on the host. The log-likelihoods come from an evaluator, a
callable (thetas, resid, refactor) -> B log-likelihoods; GpEvaluator below runs the library on the GPU.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np

PRIOR_BETA_VAR = 100.0 ** 2


@dataclasses.dataclass
class Bounds:
    """Uniform prior intervals (lo, hi) of the continuous hyperparameters. Arrays are per coordinate or per bump;
    scalars apply to all."""
    core_var: tuple = (1e-3, 1e3)
    noise_var: tuple = (1e-6, 1e2)
    s0: tuple = (1e-3, 1e3)
    r0: tuple = (1e-4, 1.0)       # per coordinate (the core's support fixes the pattern whatever r0 is)
    h: tuple = (0.0, 1.0)         # bump centres, in the bump coordinates
    r: tuple = (1e-3, 1.0)        # bump radii


def _logit(x, lo, hi):
    t = (np.asarray(x, dtype=np.float64) - lo) / (hi - lo)
    return np.log(t) - np.log1p(-t)


def _expit(u, lo, hi):
    u = np.asarray(u, dtype=np.float64)
    t = np.where(u >= 0, 1.0 / (1.0 + np.exp(-np.abs(u))), np.exp(-np.abs(u)) / (1.0 + np.exp(-np.abs(u))))
    return lo + (hi - lo) * t


def _log_jacobian(u, lo, hi):
    """log |dx/du| of x = lo + (hi - lo) expit(u), summed: log(hi - lo) + log t + log(1 - t)."""
    u = np.asarray(u, dtype=np.float64)
    return float(np.sum(np.log(hi - lo) - np.logaddexp(0.0, -u) - np.logaddexp(0.0, u)))


class Block:
    """One adaptive random-walk block: its unconstrained coordinates, their uniform-prior intervals and the
    proposal state of each chain (covariance Sigma, log scale), adapted every `every` iterations. The
    adaptation step gamma_m = c0 / m^c1 decays, so the adaptation diminishes (Shaby and Wells 2010, Sec. 3)."""

    def __init__(self, name: str, lo: np.ndarray, hi: np.ndarray, nchains: int, init_sd: float = 0.1,
                 every: int = 20, c0: float = 1.0, c1: float = 0.8, gaussian: bool = False):
        self.name, self.lo, self.hi, self.gaussian = name, lo, hi, gaussian
        self.dim = lo.shape[0]
        self.target = 0.44 if self.dim == 1 else 0.234
        self.every, self.c0, self.c1 = every, c0, c1
        self.cov = np.repeat(np.eye(self.dim)[None] * init_sd ** 2, nchains, axis=0)
        self.log_scale = np.zeros(nchains)
        self.window: List[np.ndarray] = []
        self.accepts = np.zeros(nchains)
        self.rounds = 0
        self.tried = 0

    def to_u(self, x: np.ndarray) -> np.ndarray:
        return x.copy() if self.gaussian else _logit(x, self.lo, self.hi)

    def to_x(self, u: np.ndarray) -> np.ndarray:
        return u.copy() if self.gaussian else _expit(u, self.lo, self.hi)

    def log_prior(self, u: np.ndarray) -> float:
        """Prior density of x at u, in u (uniform prior: the Jacobian; beta: the normal prior)."""
        if self.gaussian:
            return float(-0.5 * np.sum(u * u) / PRIOR_BETA_VAR)
        return _log_jacobian(u, self.lo, self.hi)

    def propose(self, rng: np.random.Generator, u: np.ndarray) -> np.ndarray:
        """u* = u + N(0, exp(log_scale) Sigma), per chain; u is nchains x dim."""
        out = np.empty_like(u)
        for c in range(u.shape[0]):
            L = np.linalg.cholesky(self.cov[c] + 1e-12 * np.eye(self.dim))
            out[c] = u[c] + math.exp(0.5 * self.log_scale[c]) * (L @ rng.standard_normal(self.dim))
        return out

    def record(self, u: np.ndarray, accepted: np.ndarray) -> None:
        self.window.append(u.copy())
        self.accepts += accepted
        self.tried += 1
        if self.tried % self.every:
            return
        self.rounds += 1
        gamma = self.c0 / self.rounds ** self.c1
        rate = self.accepts / self.every
        self.log_scale += gamma * (rate - self.target)
        w = np.stack(self.window, axis=1)   # chains x every x dim
        for c in range(w.shape[0]):
            d = w[c] - w[c].mean(axis=0)
            sample_cov = d.T @ d / max(w.shape[1] - 1, 1)
            self.cov[c] += gamma * (sample_cov - self.cov[c])
        self.window.clear()
        self.accepts[:] = 0


@dataclasses.dataclass
class ChainState:
    theta: list          # per chain: a hyperparameter setting (an object with the fields of gp_hyper)
    beta: np.ndarray     # chains x p
    pi: np.ndarray       # chains x n1 n2
    loglik: np.ndarray   # chains: log-likelihood of the current state


class BlockMCMC:
    """B lockstep chains of the App. C sampler for data z with mean W beta (W: n x p, default a constant)."""

    def __init__(self, evaluator: Callable, z: np.ndarray, theta0, nchains: int, seed: int,
                 W: Optional[np.ndarray] = None, beta0: Optional[np.ndarray] = None, bounds: Optional[Bounds] = None,
                 init_sd: float = 0.1, every: int = 20, update_pi: bool = True,
                 blocks: Sequence[str] = ("mean", "core", "bumps", "amplitudes")):
        self.eval = evaluator
        self.z = np.asarray(z, dtype=np.float64)
        n = self.z.shape[0]
        self.W = np.ones((n, 1)) if W is None else np.asarray(W, dtype=np.float64)
        p = self.W.shape[1]
        self.rng = np.random.default_rng(seed)
        self.B = nchains
        bounds = Bounds() if bounds is None else bounds
        self.bounds = bounds
        self.update_pi = update_pi
        self.blocks_on = set(blocks)
        t0 = theta0
        self.nb = t0.n1 * t0.n2
        self.bd = t0.bump_dims
        d = t0.d
        self.core_lo = np.array([bounds.core_var[0], bounds.noise_var[0], bounds.s0[0]] + [bounds.r0[0]] * d)
        self.core_hi = np.array([bounds.core_var[1], bounds.noise_var[1], bounds.s0[1]] + [bounds.r0[1]] * d)
        self.bump_lo = np.array([bounds.h[0]] * (self.nb * self.bd) + [bounds.r[0]] * self.nb)
        self.bump_hi = np.array([bounds.h[1]] * (self.nb * self.bd) + [bounds.r[1]] * self.nb)
        self.blocks: Dict[str, Block] = {
            "mean": Block("mean", np.zeros(p), np.zeros(p), nchains, init_sd, every, gaussian=True),
            "core": Block("core", self.core_lo, self.core_hi, nchains, init_sd, every),
            "bumps": Block("bumps", self.bump_lo, self.bump_hi, nchains, init_sd, every),
        }
        for name, x, lo, hi in (("core", self._core_x(t0), self.core_lo, self.core_hi),
                                ("bumps", self._bump_x(t0), self.bump_lo, self.bump_hi)):
            if name in self.blocks_on and not np.all((x > lo) & (x < hi)):
                raise ValueError(f"the initial {name} parameters must lie strictly inside their prior bounds")
        theta = [t0.copy() for _ in range(nchains)]
        for t in theta:   # amplitudes start binary: a_ij = 1 where the initial amplitude is positive
            t.a = (np.asarray(t.a) > 0).astype(np.float64)
        beta = np.repeat((np.zeros(p) if beta0 is None else np.asarray(beta0, np.float64))[None], nchains, axis=0)
        pi = np.full((nchains, self.nb), 0.5)
        ll = np.asarray(self.eval(theta, self._resid(beta), True), dtype=np.float64)
        self.state = ChainState(theta=theta, beta=beta, pi=pi, loglik=ll)
        self.factor_holds_current = True
        self.accept_counts = {k: 0 for k in ("mean", "core", "bumps", "amplitudes")}
        self.iterations = 0

    # ---------------------------------------------------------------- parameter vectors of the blocks
    def _resid(self, beta: np.ndarray) -> np.ndarray:
        return self.z[None, :] - beta @ self.W.T

    def _core_x(self, t) -> np.ndarray:
        return np.concatenate([[t.core_var, t.noise_var, t.s0], np.asarray(t.r0, np.float64)])

    def _set_core(self, t, x: np.ndarray):
        t.core_var, t.noise_var, t.s0 = float(x[0]), float(x[1]), float(x[2])
        t.r0 = np.array(x[3:], dtype=np.float64)

    def _bump_x(self, t) -> np.ndarray:
        return np.concatenate([np.asarray(t.h, np.float64), np.asarray(t.r, np.float64)])

    def _set_bumps(self, t, x: np.ndarray):
        k = self.nb * self.bd
        t.h = np.array(x[:k], dtype=np.float64)
        t.r = np.array(x[k:], dtype=np.float64)

    # ---------------------------------------------------------------- the updates
    def _mh(self, name: str, get, put, refactor: bool) -> np.ndarray:
        blk = self.blocks[name]
        st = self.state
        u = np.stack([blk.to_u(get(c)) for c in range(self.B)])
        up = blk.propose(self.rng, u)
        prop_theta, prop_beta = st.theta, st.beta
        if name == "mean":
            prop_beta = up.copy()
        else:
            prop_theta = [t.copy() for t in st.theta]
            for c in range(self.B):
                put(prop_theta[c], blk.to_x(up[c]))
        need_factor = refactor or not self.factor_holds_current
        ll = np.asarray(self.eval(prop_theta, self._resid(prop_beta), need_factor), dtype=np.float64)
        log_u = np.log(self.rng.uniform(size=self.B))
        acc = np.zeros(self.B, dtype=bool)
        for c in range(self.B):
            ratio = (ll[c] + blk.log_prior(up[c])) - (st.loglik[c] + blk.log_prior(u[c]))
            acc[c] = bool(np.isfinite(ll[c]) and log_u[c] < ratio)
        for c in range(self.B):
            if acc[c]:
                st.loglik[c] = ll[c]
                if name == "mean":
                    st.beta[c] = prop_beta[c]
                else:
                    st.theta[c] = prop_theta[c]
        blk.record(np.where(acc[:, None], up, u), acc.astype(np.float64))
        if need_factor:   # the factor now holds the proposals: current only where every chain accepted
            self.factor_holds_current = bool(acc.all()) or name == "mean"
        return acc

    def _amplitudes(self) -> np.ndarray:
        st = self.state
        prop = [t.copy() for t in st.theta]
        draws = self.rng.uniform(size=(self.B, self.nb)) < st.pi
        for c in range(self.B):
            prop[c].a = draws[c].astype(np.float64)
        ll = np.asarray(self.eval(prop, self._resid(st.beta), True), dtype=np.float64)
        log_u = np.log(self.rng.uniform(size=self.B))
        acc = np.isfinite(ll) & (log_u < ll - st.loglik)   # the prior and the proposal cancel
        for c in range(self.B):
            if acc[c]:
                st.theta[c] = prop[c]
                st.loglik[c] = ll[c]
        self.factor_holds_current = bool(acc.all())
        return acc

    def _gibbs_pi(self) -> None:
        a = np.stack([np.asarray(t.a) > 0 for t in self.state.theta]).astype(np.float64)
        self.state.pi = self.rng.beta(1.0 + a, 2.0 - a)

    def step(self) -> Dict[str, np.ndarray]:
        """One iteration over the blocks in App. C's order; returns each block's acceptance per chain."""
        st = self.state
        out = {}
        if "mean" in self.blocks_on:
            out["mean"] = self._mh("mean", lambda c: st.beta[c], None, False)
        if "core" in self.blocks_on:
            out["core"] = self._mh("core", lambda c: self._core_x(st.theta[c]), self._set_core, True)
        if "bumps" in self.blocks_on:
            out["bumps"] = self._mh("bumps", lambda c: self._bump_x(st.theta[c]), self._set_bumps, True)
        if "amplitudes" in self.blocks_on:
            out["amplitudes"] = self._amplitudes()
        if self.update_pi:
            self._gibbs_pi()
        for k, v in out.items():
            self.accept_counts[k] += int(np.sum(v))
        self.iterations += 1
        return out

    def run(self, iters: int, callback: Optional[Callable] = None) -> None:
        for _ in range(iters):
            acc = self.step()
            if callback is not None:
                callback(self, acc)


class GpEvaluator:
    """Log-likelihoods of B settings through the library: one batched factorization (when the settings changed)
    and one batched solve per call. The point set is assembled once; its pattern is fixed by the core radii."""

    def __init__(self, ctx, pointset, nchains: int, precision: int):
        self.ctx, self.ps, self.B, self.precision = ctx, pointset, nchains, precision
        self.f = None
        self.calls = 0
        self.factorizations = 0

    def __call__(self, thetas: list, resid: np.ndarray, refactor: bool) -> np.ndarray:
        import torch
        if self.f is None:
            self.f = self.ctx.factor(self.ps, thetas, self.precision)
            self.factorizations += 1
        elif refactor:
            self.f.update(thetas)
            self.factorizations += 1
        r = torch.as_tensor(np.ascontiguousarray(resid), dtype=torch.float64, device=f"cuda:{self.ctx.device}")
        ll = self.f.loglik(r)
        self.calls += 1
        return ll.cpu().numpy().copy()

    def free(self) -> None:
        if self.f is not None:
            self.f.free()
            self.f = None
