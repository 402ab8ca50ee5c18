"""Pins of the oracle's likelihood and prediction (Sec. 3.2, Sec. 3.3).

Dense log-likelihood against LAPACK (numpy slogdet/solve, run as a library), a tridiagonal case against the
continuant recurrence for its determinant, the sparse factor against the dense one and against the matrix
it factors, and the predictive mean against the dense kriging formula and the interpolation limit.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2411_05869_gb300 import synth


def _numpy_loglik(C, r):
    sign, ld = np.linalg.slogdet(C)
    assert sign > 0
    a = np.linalg.solve(C, r)
    return -0.5 * ld - 0.5 * r @ a - 0.5 * len(r) * math.log(2 * math.pi), ld, a


@pytest.fixture(scope="module")
def cfg1_small():
    w = synth.spatial_2d(n=900, m=60, seed=21)
    hp = w.hyper
    y = oracle.sample_dense(hp, w.X, w.normals)
    z = y + math.sqrt(hp.noise_var) * w.noise
    rp, col = oracle.pattern(w.X, hp.core_radius)
    perm = oracle.nd_order(w.X, hp.core_radius, rp, col)
    return w, z, rp, col, perm


def test_dense_loglik_against_lapack(cfg1_small):
    w, z, *_ = cfg1_small
    res = oracle.dense_loglik(w.hyper, w.X, z, want_alpha=True)
    C = oracle.dense_cov(w.hyper, w.X)
    ll, ld, a = _numpy_loglik(C, z)
    assert res["loglik"] == pytest.approx(ll, rel=1e-12)
    assert res["logdet"] == pytest.approx(ld, rel=1e-12)
    assert np.allclose(res["alpha"], a, rtol=1e-10, atol=1e-10 * np.abs(a).max())


def test_sparse_matches_dense(cfg1_small):
    w, z, rp, col, perm = cfg1_small
    d = oracle.dense_loglik(w.hyper, w.X, z, want_alpha=True)
    s = oracle.sparse_loglik(w.hyper, w.X, rp, col, perm, z, want_alpha=True)
    assert s["loglik"] == pytest.approx(d["loglik"], rel=1e-12)
    assert s["logdet"] == pytest.approx(d["logdet"], rel=1e-12)
    assert np.abs(s["alpha"] - d["alpha"]).max() <= 1e-10 * np.abs(d["alpha"]).max()


def test_sparse_factor_reconstructs_matrix():
    """|| P C P^T - L L^T ||_F / || C ||_F <= 1e-14 on the sparse structure."""
    w = synth.spatial_2d(n=350, m=1, seed=22, rho=0.12)
    rp, col = oracle.pattern(w.X, w.hyper.core_radius)
    perm = oracle.nd_order(w.X, w.hyper.core_radius, rp, col)
    L = oracle.sparse_factor_dense(w.hyper, w.X, rp, col, perm)
    C = oracle.dense_cov(w.hyper, w.X)
    Cp = C[np.ix_(perm, perm)]
    assert np.linalg.norm(Cp - L @ L.T) / np.linalg.norm(C) <= 1e-14
    assert np.allclose(np.triu(L, 1), 0.0)


def test_tridiagonal_continuant():
    """Points on a line with spacing 1 and support radius 1.5: C_z is tridiagonal; det by the continuant
    recurrence f_k = a_k f_{k-1} - b_{k-1}^2 f_{k-2} (tracked as ratios to stay in range)."""
    n = 400
    X = np.arange(n, dtype=float)[:, None]
    rng = np.random.default_rng(5)
    hp = synth.Hyper(d=1, n1=1, n2=2, bump_dims=1, core_var=1.3, core_radius=np.array([1.5]), s0=0.8,
                     r0=np.array([1.5]), h=np.array([100.0, 300.0]), a=np.array([1.0, 0.6]), b=np.ones(2),
                     r=np.array([40.0, 25.0]), noise_var=0.05)
    C = oracle.dense_cov(hp, X)
    assert np.all(np.triu(C, 2) == 0.0)
    a = np.diag(C)
    b = np.diag(C, 1)
    logdet = math.log(a[0])
    ratio = a[0]                   # f_k / f_{k-1}
    for k in range(1, n):
        ratio = a[k] - b[k - 1] ** 2 / ratio
        logdet += math.log(ratio)
    r = rng.standard_normal(n)
    rp, col = oracle.pattern(X, hp.core_radius)
    perm = oracle.nd_order(X, hp.core_radius, rp, col)
    s = oracle.sparse_loglik(hp, X, rp, col, perm, r)
    d = oracle.dense_loglik(hp, X, r)
    assert s["logdet"] == pytest.approx(logdet, rel=1e-12)
    assert d["logdet"] == pytest.approx(logdet, rel=1e-12)


def test_not_positive_definite_is_reported():
    w = synth.spatial_2d(n=200, m=1, seed=23)
    hp = w.hyper.copy()
    hp.noise_var = -50.0
    rp, col = oracle.pattern(w.X, hp.core_radius)
    perm = oracle.nd_order(w.X, hp.core_radius, rp, col)
    with pytest.raises(np.linalg.LinAlgError):
        oracle.sparse_loglik(hp, w.X, rp, col, perm, np.ones(200))
    with pytest.raises(np.linalg.LinAlgError):
        oracle.dense_loglik(hp, w.X, np.ones(200))


def test_predict_against_dense_kriging(cfg1_small):
    w, z, rp, col, perm = cfg1_small
    s = oracle.sparse_loglik(w.hyper, w.X, rp, col, perm, z, want_alpha=True)
    mu = np.linspace(-1, 1, w.Xtest.shape[0])
    m = oracle.predict(w.hyper, w.X, s["alpha"], w.Xtest, mu)
    # dense kriging: C_{y,z} from the joint C_y over (train + test) points; solve with LAPACK
    Xa = np.concatenate([w.X, w.Xtest])
    Cya = oracle.dense_cov(w.hyper, Xa, noise=False)
    n = w.X.shape[0]
    Kst = Cya[n:, :n]
    C = oracle.dense_cov(w.hyper, w.X)
    ref = mu + Kst @ np.linalg.solve(C, z)
    assert np.abs(m - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max())


def test_predict_interpolates_with_vanishing_noise():
    """tau^2 -> 0: m* at a training input equals the observation there (C_y = C_z on the training set)."""
    w = synth.spatial_2d(n=400, m=1, seed=24, noise_var=1e-10, rho=0.08)
    z = np.random.default_rng(3).standard_normal(400)
    rp, col = oracle.pattern(w.X, w.hyper.core_radius)
    perm = oracle.nd_order(w.X, w.hyper.core_radius, rp, col)
    s = oracle.sparse_loglik(w.hyper, w.X, rp, col, perm, z, want_alpha=True)
    m = oracle.predict(w.hyper, w.X, s["alpha"], w.X[:50])
    assert np.abs(m - z[:50]).max() < 1e-6
