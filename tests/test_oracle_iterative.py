"""Pins of the oracle's iterative path (Sec. 3.3: stochastic Lanczos log-determinant, MINRES solve) against facts the
mathematics fixes, none of them a restatement of the oracle's recurrences:

- k Lanczos steps give a Gauss quadrature exact for polynomials of degree 2k - 1, so with k = n (a full Krylov space)
  v^T log(C) v is exact; unit vectors as probes then sum to tr log C = log det C (LAPACK slogdet).
- On a diagonal matrix with Rademacher probes, v^T log(D) v = tr log D for every probe, and k at least the number of
  distinct eigenvalues makes each quadrature exact.
- With random probes the estimate is unbiased: it lies within a few standard errors of the exact log-determinant.
- MINRES reaches numpy.linalg.solve's solution to its tolerance times the condition number; its residual estimate
  is non-increasing and equals the true residual; on a matrix with three distinct eigenvalues it ends in at most
  three steps; started at the solution it takes none.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import iterative as it
from paper_2411_05869_gb300 import synth


def _cz(n=300, seed=41):
    w = synth.spatial_2d(n=n, m=0, seed=synth.SEED_BASE + seed, rho=0.12)
    rp, col = oracle.pattern(w.X, w.hyper.core_radius)
    val = oracle.csr_values(w.hyper, w.X, rp, col)
    C = np.zeros((n, n))
    for i in range(n):
        C[i, col[rp[i]:rp[i + 1]]] = val[rp[i]:rp[i + 1]]
    return w, rp, col, val, C


def test_slq_with_a_full_krylov_space_is_exact():
    n = 14
    _, rp, col, val, C = _cz(n=n, seed=42)
    mv = it.csr_matvec(rp, col, val)
    est, gam = it.slq_logdet(mv, np.eye(n), k=n)
    sign, ref = np.linalg.slogdet(C)
    assert sign > 0
    assert est * n == pytest.approx(ref, rel=1e-10)   # mean over n unit probes = tr log C / n


def test_slq_on_a_diagonal_matrix_with_rademacher_probes():
    rng = np.random.default_rng(3)
    d = rng.choice([0.5, 2.0, 7.0, 11.0], size=200)
    mv = lambda x: (d * x.T).T if x.ndim == 1 else d[:, None] * x
    probes = rng.choice([-1.0, 1.0], size=(200, 6))
    est, gam = it.slq_logdet(mv, probes, k=6)
    assert est == pytest.approx(float(np.log(d).sum()), rel=1e-12)
    assert np.allclose(gam, np.log(d).sum(), rtol=1e-12)


def test_slq_estimate_is_unbiased():
    n = 400
    _, rp, col, val, C = _cz(n=n, seed=43)
    mv = it.csr_matvec(rp, col, val)
    rng = np.random.default_rng(7)
    probes = rng.choice([-1.0, 1.0], size=(n, 64))
    est, gam = it.slq_logdet(mv, probes, k=30)
    ref = np.linalg.slogdet(C)[1]
    se = gam.std(ddof=1) / math.sqrt(gam.shape[0])
    assert abs(est - ref) <= 4 * se + 1e-9 * abs(ref)


def test_minres_solution_monotone_residual_and_termination():
    n = 400
    _, rp, col, val, C = _cz(n=n, seed=44)
    mv = it.csr_matvec(rp, col, val)
    rng = np.random.default_rng(8)
    b = rng.standard_normal(n)
    x0 = rng.standard_normal(n)
    x, its, hist = it.minres(mv, b, x0, 1e-10, 5000)
    ref = np.linalg.solve(C, b)
    cond = np.linalg.cond(C)
    assert np.linalg.norm(x - ref) <= 1e-10 * cond * np.linalg.norm(ref) * 10
    assert all(h2 <= h1 * (1 + 1e-12) for h1, h2 in zip(hist, hist[1:])), "MINRES residuals never increase"
    assert np.linalg.norm(b - C @ x) == pytest.approx(hist[-1], rel=1e-6, abs=1e-12 * np.linalg.norm(b))
    # three distinct eigenvalues: the Krylov space is exhausted after three steps
    Q, _ = np.linalg.qr(rng.standard_normal((50, 50)))
    lam = np.repeat([1.0, 4.0, 9.0], [20, 20, 10])
    A = (Q * lam) @ Q.T
    x3, its3, _ = it.minres(lambda v: A @ v, b[:50], np.zeros(50), 1e-12, 100)
    assert its3 <= 3 and np.allclose(x3, np.linalg.solve(A, b[:50]), atol=1e-10)
    # started at the solution: no step
    _, its0, _ = it.minres(mv, C @ ref, ref, 1e-8, 100)
    assert its0 == 0


def test_iterative_loglik_against_the_dense_loglik():
    """The iterative estimate lies within the SLQ standard error of the exact log-likelihood (Sec. 3.3)."""
    w, rp, col, val, C = _cz(n=400, seed=45)
    rng = np.random.default_rng(9)
    r = rng.standard_normal(400)
    probes = rng.choice([-1.0, 1.0], size=(400, 64))
    out = it.iterative_loglik(rp, col, val, r, probes, 30, rng.standard_normal(400), tol=1e-10)
    ref = oracle.dense_loglik(w.hyper, w.X, r)
    se = out["gam"].std(ddof=1) / math.sqrt(64)
    assert out["quad"] == pytest.approx(ref["quad"], rel=1e-8)
    assert abs(out["logdet"] - ref["logdet"]) <= 4 * se
    assert abs(out["loglik"] - ref["loglik"]) <= 2 * se + 1e-8 * abs(ref["loglik"])
