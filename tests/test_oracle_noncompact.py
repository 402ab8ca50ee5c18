"""Pins of the oracle's non-compact core (App. B, Eq. PScov: the parametric nonstationary Matern core, smoothness 3/2,
with log-linear sigma(x) and Sigma(x)) and of the pattern it implies (the support of C_sparse, Eq. C_sparse), against
closed forms, a numpy restatement of the support rule, positive definiteness and the dense computation.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2411_05869_gb300 import synth


def _nc_hyper(d=2, n1=2, n2=2, seed=0, phi=0.0, r0=0.05, rbump=(0.05, 0.12), a=None, noise=1e-2):
    rng = np.random.default_rng(seed)
    nb = n1 * n2
    return synth.Hyper(d=d, n1=n1, n2=n2, bump_dims=d, core_var=1.0, core_radius=np.full(d, 1.0), s0=0.8,
                       r0=np.full(d, r0), h=rng.uniform(0, 1, nb * d),
                       a=rng.uniform(0.5, 2, nb) if a is None else np.full(nb, a), b=np.ones(nb),
                       r=rng.uniform(*rbump, nb), noise_var=noise, core_kind=1, sigma0=1.3, Sigma0=0.02,
                       phi_sigma=np.full(d, 0.7 * phi), phi_Sigma=np.full(d, -1.1 * phi))


def _matern32(t):
    return (1.0 + math.sqrt(3.0) * t) * math.exp(-math.sqrt(3.0) * t)


def test_stationary_limit_is_the_matern_core():
    """phi = 0, no bumps, r0 -> infinity: C_y = s0 sigma0^2 M(|x - x'| / sqrt(Sigma0)) (Sec. 2.3 special case 2)."""
    hp = _nc_hyper(phi=0.0, a=0.0)
    hp.r0 = np.full(2, 1e150)
    rng = np.random.default_rng(1)
    for _ in range(50):
        x, y = rng.uniform(0, 1, 2), rng.uniform(0, 1, 2)
        t = float(np.linalg.norm(x - y)) / math.sqrt(hp.Sigma0)
        assert oracle.cy(hp, x, y) == pytest.approx(hp.s0 * hp.sigma0 ** 2 * _matern32(t), rel=1e-13)


def test_paciorek_prefactor_and_diagonal_by_hand():
    """sigma(x) sigma(x') sqrt(Sigma(x) Sigma(x')) / ((Sigma(x) + Sigma(x')) / 2) M(sqrt(Q)) in 2-D, and
    C_core(x, x) = sigma(x)^2."""
    hp = _nc_hyper(phi=1.0, a=0.0)
    hp.r0 = np.full(2, 1e150)
    s0 = hp.s0
    rng = np.random.default_rng(2)
    for _ in range(50):
        x, y = rng.uniform(0, 1, 2), rng.uniform(0, 1, 2)
        sx = hp.sigma0 * math.exp(hp.phi_sigma @ x)
        sy = hp.sigma0 * math.exp(hp.phi_sigma @ y)
        Sx = hp.Sigma0 * math.exp(hp.phi_Sigma @ x)
        Sy = hp.Sigma0 * math.exp(hp.phi_Sigma @ y)
        avg = 0.5 * (Sx + Sy)
        ref = sx * sy * math.sqrt(Sx * Sy) / avg * _matern32(math.sqrt(float((x - y) @ (x - y)) / avg))
        assert oracle.cy(hp, x, y) == pytest.approx(s0 * ref, rel=1e-12)
        assert oracle.cy(hp, x, x) == pytest.approx(s0 * sx * sx, rel=1e-13)


def _support_numpy(hp, X):
    """The support rule restated with numpy arrays (same operation order, no fused operations)."""
    U = X / hp.r0
    n = X.shape[0]
    q2 = np.zeros((n, n))
    for k in range(X.shape[1]):
        dk = U[:, None, k] - U[None, :, k]
        q2 = q2 + dk * dk
    S = q2 < 1.0
    nb = hp.n1 * hp.n2
    H = hp.h.reshape(nb, hp.bump_dims)
    inside = np.zeros((n, nb), bool)
    for j in range(nb):
        s = np.zeros(n)
        for k in range(hp.bump_dims):
            dk = X[:, k] - H[j, k]
            s = s + dk * dk
        inside[:, j] = s < hp.r[j] * hp.r[j]
    fam = inside.reshape(n, hp.n1, hp.n2).any(axis=2)
    for i in range(hp.n1):
        S |= fam[:, i][:, None] & fam[:, i][None, :]
    return S


def test_pattern_is_the_support_of_csparse():
    hp = _nc_hyper(phi=0.5, seed=3)
    X = np.random.default_rng(3).uniform(0, 1, (500, 2))
    rp, col = oracle.pattern_sparse(hp, X)
    S = _support_numpy(hp, X)
    M = np.zeros_like(S)
    for i in range(500):
        M[i, col[rp[i]:rp[i + 1]]] = True
    assert np.array_equal(M, S)
    assert np.array_equal(M, M.T)
    # far pairs join only through a shared family; the dense C_y is zero exactly outside the pattern
    C = oracle.dense_cov(hp, X, noise=False)
    assert np.all(C[~S] == 0.0)
    dist = np.sqrt(((X[:, None] - X[None]) ** 2).sum(-1))
    assert np.any(S & (dist > 0.3)), "some pairs far apart share a bump family"


@pytest.mark.parametrize("seed", [4, 5])
def test_noncompact_cz_positive_definite(seed):
    """Prop. 1 with a PD core: C_y is PD (Schur product), so lambda_min(C_z) >= tau^2."""
    hp = _nc_hyper(phi=1.0, seed=seed, rbump=(0.1, 0.3))
    X = np.random.default_rng(seed).uniform(0, 1, (300, 2))
    C = oracle.dense_cov(hp, X)
    lam = np.linalg.eigvalsh(C)
    assert lam[0] >= hp.noise_var - 1e-12 * abs(lam[-1])


def test_sparse_loglik_on_the_support_equals_the_dense_loglik():
    """The left-looking sparse Cholesky on the support pattern gives the dense log-likelihood: the pattern holds
    every nonzero of C_z."""
    hp = _nc_hyper(phi=0.8, seed=6)
    X = np.random.default_rng(6).uniform(0, 1, (600, 2))
    r = np.random.default_rng(7).standard_normal(600)
    rp, col = oracle.pattern_sparse(hp, X)
    perm = oracle.fill_order(X, hp.r0, rp, col)
    sp = oracle.sparse_loglik(hp, X, rp, col, perm, r)
    de = oracle.dense_loglik(hp, X, r)
    assert sp["loglik"] == pytest.approx(de["loglik"], rel=1e-12)
