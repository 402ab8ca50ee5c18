"""The App. C sampler (paper_2411_05869_gb300.mcmc), pinned on the CPU against exact answers:

  - Gibbs draws of pi_ij against the Beta(1 + a, 2 - a) moments.
  - The amplitude block against the exact posterior, enumerated over every binary amplitude vector.
  - The adaptive random walk against a Gaussian posterior in closed form.
  - The logit transforms' Jacobians, through a flat likelihood that must give back the uniform prior.
  - Bookkeeping against the oracle's log-likelihood on a small GP.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2411_05869_gb300 import mcmc, synth


def _theta(nb_dims=(1, 2), bump_dims=2, d=2):
    n1, n2 = nb_dims
    nb = n1 * n2
    rad = np.full(d, 0.2)
    return synth.Hyper(d=d, n1=n1, n2=n2, bump_dims=bump_dims, core_var=1.0, core_radius=rad, s0=1.0,
                       r0=rad.copy(), h=np.full(nb * bump_dims, 0.5), a=np.ones(nb), b=np.ones(nb),
                       r=np.full(nb, 0.3), noise_var=0.1)


def _flat(thetas, resid, refactor):
    return np.zeros(len(thetas))


def test_gibbs_pi_matches_beta_moments():
    B = 4000
    s = mcmc.BlockMCMC(_flat, np.zeros(5), _theta(), B, seed=1, blocks=())
    for t in s.state.theta:
        t.a = np.array([1.0, 0.0])
    s.step()
    pi = s.state.pi
    se = math.sqrt(2.0 / 36.0 / B)   # Beta(2, 1) and Beta(1, 2): variance 2 / (3^2 * 4)
    assert abs(pi[:, 0].mean() - 2.0 / 3.0) < 5 * se
    assert abs(pi[:, 1].mean() - 1.0 / 3.0) < 5 * se
    assert abs(pi[:, 0].var() - 2.0 / 36.0) < 0.01 and abs(pi[:, 1].var() - 2.0 / 36.0) < 0.01


def test_amplitude_block_samples_the_exact_posterior():
    table = {k: v for k, v in zip(itertools.product([0, 1], repeat=3), [0.0, 1.2, -0.7, 0.4, 2.0, -1.5, 0.9, 0.3])}
    pi = np.array([0.3, 0.6, 0.5])

    def ev(thetas, resid, refactor):
        return np.array([table[tuple(int(x) for x in t.a)] for t in thetas])

    B = 2000
    s = mcmc.BlockMCMC(ev, np.zeros(4), _theta(nb_dims=(1, 3)), B, seed=2, blocks=("amplitudes",),
                       update_pi=False)
    s.state.pi[:] = pi
    counts = {k: 0 for k in table}
    for it in range(60):
        s.step()
        if it >= 20:
            for t in s.state.theta:
                counts[tuple(int(x) for x in t.a)] += 1
    post = {k: math.exp(v) * np.prod([p if a else 1 - p for a, p in zip(k, pi)]) for k, v in table.items()}
    z = sum(post.values())
    total = sum(counts.values())
    for k in table:
        assert abs(counts[k] / total - post[k] / z) < 0.015, (k, counts[k] / total, post[k] / z)


def test_adaptive_walk_samples_a_gaussian_posterior():
    m = np.array([1.5, -0.5])
    P = np.array([[4.0, 1.5], [1.5, 2.0]])

    def ev(thetas, resid, refactor):   # z = 0 and W = I, so beta = -resid
        d = -resid - m[None, :]
        return -0.5 * np.einsum("bi,ij,bj->b", d, P, d)

    B, iters = 100, 1200
    s = mcmc.BlockMCMC(ev, np.zeros(2), _theta(), B, seed=3, W=np.eye(2), blocks=("mean",), update_pi=False,
                       init_sd=0.5)
    draws = []
    for it in range(iters):
        s.step()
        if it >= iters // 2:
            draws.append(s.state.beta.copy())
    x = np.concatenate(draws)
    Pp = P + np.eye(2) / mcmc.PRIOR_BETA_VAR
    mean = np.linalg.solve(Pp, P @ m)
    cov = np.linalg.inv(Pp)
    assert np.allclose(x.mean(axis=0), mean, atol=0.03)
    assert np.allclose(np.cov(x.T), cov, atol=0.04)
    rate = s.accept_counts["mean"] / (B * iters)
    assert 0.15 < rate < 0.45


def test_uniform_prior_is_recovered_through_the_transform():
    bounds = mcmc.Bounds(core_var=(1.0, 3.0), noise_var=(0.01, 0.5), s0=(0.5, 2.0), r0=(0.05, 0.2))
    B, iters = 100, 800
    t0 = _theta()
    t0.core_var, t0.r0 = 2.0, np.full(2, 0.1)
    with pytest.raises(ValueError):   # a start on an interval's end
        mcmc.BlockMCMC(_flat, np.zeros(3), _theta(), B, seed=4, bounds=bounds, blocks=("core",))
    s = mcmc.BlockMCMC(_flat, np.zeros(3), t0, B, seed=4, bounds=bounds, blocks=("core",), update_pi=False)
    cv, nv = [], []
    for it in range(iters):
        s.step()
        if it >= iters // 2:
            cv += [t.core_var for t in s.state.theta]
            nv += [t.noise_var for t in s.state.theta]
    cv, nv = np.array(cv), np.array(nv)
    assert abs(cv.mean() - 2.0) < 0.05 and abs(cv.var() - 4.0 / 12.0) < 0.03
    assert abs(nv.mean() - 0.255) < 0.01 and abs(nv.var() - 0.49 ** 2 / 12.0) < 0.004
    assert cv.min() > 1.0 and cv.max() < 3.0


def _oracle_evaluator(X, rp, col, perm):
    def ev(thetas, resid, refactor):
        return np.array([oracle.sparse_loglik(t, X, rp, col, perm, resid[k])["loglik"]
                         for k, t in enumerate(thetas)])
    return ev


def test_chain_bookkeeping_against_the_oracle_and_determinism():
    w = synth.spatial_2d(n=300, m=10, seed=synth.SEED_BASE + 40)
    hp = w.hyper
    rp, col = oracle.pattern(w.X, hp.core_radius)
    perm = oracle.fill_order(w.X, hp.core_radius, rp, col)
    z = np.random.default_rng(5).standard_normal(300) + 0.3
    ev = _oracle_evaluator(w.X, rp, col, perm)
    bounds = mcmc.Bounds(r0=(0.01, 2.0 * float(hp.core_radius[0])), r=(0.05, 0.5))

    def run():
        s = mcmc.BlockMCMC(ev, z, hp, 3, seed=6, bounds=bounds)
        s.run(3)
        return s

    s1, s2 = run(), run()
    for c in range(3):
        t = s1.state.theta[c]
        ref = oracle.sparse_loglik(t, w.X, rp, col, perm, z - s1.state.beta[c] @ s1.W.T)["loglik"]
        assert s1.state.loglik[c] == pytest.approx(ref, rel=1e-12, abs=1e-9)
        assert np.array_equal(s1.state.beta[c], s2.state.beta[c])
        assert s1.state.loglik[c] == s2.state.loglik[c]
        assert set(np.unique(t.a)) <= {0.0, 1.0}
    assert s1.accept_counts == s2.accept_counts
