"""Pins of the oracle's predictive variance diag(C_{y|z}) (Sec. 3.2), against facts the mathematics fixes:

- Far from every training input, the cross-covariance vanishes, and the variance is the prior one, in closed
  form from Eq. C_sparse and Eq. compSupp.
- At a training input the latent variance is positive and at most tau^2 (z_j alone already brings it below tau^2).
- Conditioning on more data never raises it.
- It equals 1 / (J^{-1})_{nn} for the joint covariance J of the training data and the test input: the Schur
  complement by a matrix inverse, a route independent of the oracle's triangular solves.
"""
import numpy as np
import pytest

import oracle
from paper_2411_05869_gb300 import synth


def _w(n=400, seed=31):
    return synth.spatial_2d(n=n, m=0, seed=synth.SEED_BASE + seed)


def test_far_from_the_data_the_variance_is_the_prior_variance():
    w = _w()
    hp = w.hyper
    xs = np.array([[3.0, 3.0], [-2.0, 0.5]])   # no training point within the core radius
    var = oracle.predictive_variance(hp, w.X, xs)
    for k, x in enumerate(xs):
        f = oracle.features(hp, x[None, :])[0]
        prior = hp.core_var * oracle.wendland(0.0) * (hp.s0 * oracle.wendland(0.0) + float(np.sum(f * f)))
        assert var[k] == pytest.approx(prior, rel=1e-14, abs=1e-15)
        assert var[k] == pytest.approx(oracle.cy(hp, x, x), rel=1e-14)


def test_at_training_inputs_the_variance_lies_in_zero_tau2():
    w = _w()
    hp = w.hyper
    var = oracle.predictive_variance(hp, w.X, w.X[:40])
    assert np.all(var > 0.0) and np.all(var <= hp.noise_var * (1 + 1e-9))


def test_more_data_never_raises_the_variance():
    w = _w(n=500)
    hp = w.hyper
    xs = np.random.default_rng(3).uniform(0, 1, (60, 2))
    v_all = oracle.predictive_variance(hp, w.X, xs)
    v_half = oracle.predictive_variance(hp, w.X[:250], xs)
    assert np.all(v_all <= v_half + 1e-12)
    assert np.any(v_all < v_half - 1e-6)


def test_variance_equals_the_inverse_of_the_joint_precision():
    w = _w(n=300)
    hp = w.hyper
    xs = np.random.default_rng(4).uniform(0, 1, (8, 2))
    var = oracle.predictive_variance(hp, w.X, xs)
    n = w.X.shape[0]
    for k, x in enumerate(xs):
        Z = np.vstack([w.X, x[None, :]])
        J = oracle.dense_cov(hp, Z, noise=False)
        J[np.arange(n), np.arange(n)] += hp.noise_var   # noise on the training inputs only
        assert var[k] == pytest.approx(1.0 / np.linalg.inv(J)[n, n], rel=1e-8)
