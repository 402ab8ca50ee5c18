"""The oracle of the paper's iterative path (Sec. 3.3): the stochastic Lanczos quadrature estimate of log det C_z and
the MINRES solve of C_z alpha = r. TEST INFRASTRUCTURE ONLY (imported by the tests and the benchmark's baseline leg).

Plain numpy in FP64, each step in the order of the method's definition; the probe vectors and the MINRES starting
vector are inputs (the paper draws them at random: Rademacher probes, a random start), so the CUDA path can be
given the same ones. A library routine serves one step: numpy.linalg.eigh for the eigenpairs of the small Lanczos
tridiagonal matrix.

- slq_logdet: stochastic Lanczos quadrature (Ubaru, Chen and Saad, 2017), the estimator the paper uses for the
  log-determinant above 100k points: for each probe v, k steps of the Lanczos process from v / |v| (no
  reorthogonalisation) give the tridiagonal T_k = U diag(theta) U^T, and v^T log(C) v is estimated by
  |v|^2 sum_i U_{1i}^2 log(theta_i); the log-determinant tr log(C) is the mean of these over the probes.
- minres: the minimum-residual method of Paige and Saunders (1975) that the paper uses for the solve, here in its
  Lanczos form with Givens rotations, stopped when the residual estimate |phibar| falls to tol |r|.
"""
from __future__ import annotations

import math

import numpy as np


def csr_matvec(rowptr, col, val):
    """x -> C x for a CSR matrix (rows in index order)."""
    n = rowptr.shape[0] - 1
    rows = np.repeat(np.arange(n), np.diff(rowptr))

    def mv(x):
        return np.bincount(rows, weights=val * x[col], minlength=n) if x.ndim == 1 else \
            np.stack([np.bincount(rows, weights=val * x[col, p], minlength=n) for p in range(x.shape[1])], 1)
    return mv


def lanczos(matvec, v, k):
    """k steps of the Lanczos process from q_1 = v / |v|: returns (alpha[k'], beta[k' - 1]) of T_k' (k' <= k; the
    process stops early if beta vanishes: the Krylov space is then invariant)."""
    q_prev = np.zeros_like(v)
    q = v / np.linalg.norm(v)
    alpha, beta = [], []
    b_prev = 0.0
    for j in range(k):
        w = matvec(q)
        a = float(q @ w)
        w = w - a * q - b_prev * q_prev
        alpha.append(a)
        b = float(np.linalg.norm(w))
        if j == k - 1:
            break
        if b <= 1e-14 * max(abs(a), 1e-300):
            break
        beta.append(b)
        q_prev, q, b_prev = q, w / b, b
    return np.array(alpha), np.array(beta)


def quadrature(alpha, beta, vnorm2):
    """|v|^2 sum_i U_{1i}^2 log(theta_i) for T = tridiag(beta, alpha, beta) = U diag(theta) U^T."""
    k = alpha.shape[0]
    Tm = np.diag(alpha)
    if k > 1:
        Tm += np.diag(beta, 1) + np.diag(beta, -1)
    theta, U = np.linalg.eigh(Tm)
    if np.any(theta <= 0):
        raise np.linalg.LinAlgError("a Ritz value is not positive")
    return vnorm2 * float(np.sum(U[0, :] ** 2 * np.log(theta)))


def slq_logdet(matvec, probes, k):
    """Stochastic Lanczos quadrature estimate of log det C over the probe vectors (columns of probes, n x P).
    Returns (estimate, per-probe quadratures)."""
    gam = []
    for p in range(probes.shape[1]):
        v = probes[:, p]
        a, b = lanczos(matvec, v, k)
        gam.append(quadrature(a, b, float(v @ v)))
    gam = np.array(gam)
    return float(gam.mean()), gam


def minres(matvec, b, x0, tol, maxiter):
    """MINRES for C x = b from x0 (C symmetric), stopped when |b - C x| (the recurrence's estimate) <= tol |b|.
    Returns (x, iterations, residual estimates per iteration)."""
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - matvec(x)
    bnorm = float(np.linalg.norm(b))
    beta = float(np.linalg.norm(r))
    hist = [beta]
    if beta <= tol * bnorm:
        return x, 0, hist
    v_prev = np.zeros_like(b)
    v = r / beta
    c2, s2, c1, s1 = 1.0, 0.0, 1.0, 0.0       # rotations j - 2 and j - 1
    d2 = np.zeros_like(b)
    d1 = np.zeros_like(b)
    phibar = beta
    it = 0
    while it < maxiter:
        it += 1
        # Lanczos: p = C v_j - beta_j v_{j-1}, alpha_j = v_j . p, p -= alpha_j v_j, beta_{j+1} = |p|
        p = matvec(v) - beta * v_prev
        alpha = float(v @ p)
        p = p - alpha * v
        beta_next = float(np.linalg.norm(p))
        # column j of the tridiagonal (beta_j, alpha_j, beta_{j+1}) through rotations j - 2 and j - 1
        eps = s2 * beta
        dbar = c2 * beta
        delta = c1 * dbar + s1 * alpha
        gbar = -s1 * dbar + c1 * alpha
        # rotation j zeroes beta_{j+1}
        gamma = math.hypot(gbar, beta_next)
        if gamma == 0.0:
            raise np.linalg.LinAlgError("MINRES breakdown")
        c, s = gbar / gamma, beta_next / gamma
        phi = c * phibar
        phibar = -s * phibar
        d = (v - delta * d1 - eps * d2) / gamma
        x = x + phi * d
        hist.append(abs(phibar))
        if abs(phibar) <= tol * bnorm or beta_next == 0.0:
            break
        v_prev, v = v, p / beta_next
        d2, d1 = d1, d
        c2, s2, c1, s1 = c1, s1, c, s
        beta = beta_next
    return x, it, hist


def iterative_loglik(rowptr, col, val, resid, probes, k, x0, tol=1e-8, maxiter=10000):
    """The paper's iterative log-likelihood (Sec. 3.3): -1/2 (SLQ log det) - 1/2 r^T x (x from MINRES) - n/2 log 2 pi."""
    mv = csr_matvec(rowptr, col, val)
    logdet, gam = slq_logdet(mv, probes, k)
    x, it, hist = minres(mv, resid, x0, tol, maxiter)
    quad = float(resid @ x)
    n = resid.shape[0]
    return {"loglik": -0.5 * logdet - 0.5 * quad - 0.5 * n * math.log(2 * math.pi), "logdet": logdet,
            "quad": quad, "x": x, "iters": it, "relres": hist[-1] / float(np.linalg.norm(resid)), "gam": gam}
