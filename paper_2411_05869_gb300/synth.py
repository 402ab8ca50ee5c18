"""Seeded synthetic inputs for the exact sparse GP (no kernel, likelihood or factorization arithmetic here).

This module is the only code shared by the CUDA path, the CPU oracle, the tests and the benchmark. It draws
point sets, hyperparameters and residual vectors; it evaluates none of the method's formulas (no bump
function, no Wendland polynomial, no covariance, no Cholesky). Where a workload wants a residual "drawn from
the GP", the caller draws it (the oracle does, from the standard-normal vector returned here).

Workloads follow the shapes of the paper's experiments: 2-D spatial points (Sec. 5.1) and space-time
station-by-day layouts (Sec. 5.2, N about 1e6, d = 3, bumps in the spatial coordinates only), bump radii and
Wendland support sized from the user-parameter table (Appendix, supplemental table of user parameters).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

SEED_BASE = 2411_05869


@dataclasses.dataclass
class Hyper:
    """One hyperparameter setting of C_z = C_core * C_sparse + tau^2 I (Sec. 2, Eq. C_sparse; Sec. 3.1, Eq. Zcov).

    C_core(x, x') = core_var * W(q_c), q_c the anisotropic distance with radii core_radius[d].
    C_sparse(x, x') = s0 * W(q_0) + sum_i f_i(x) f_i(x'), q_0 with radii r0[d];
    f_i(x) = sum_j g_ij(x), g_ij a bump with centre h_ij (bump_dims coords), amplitude a_ij, shape b_ij, radius r_ij.
    Arrays h (n1*n2*bump_dims), a, b, r (n1*n2) are row-major over (i, j).
    """
    d: int
    n1: int
    n2: int
    bump_dims: int
    core_var: float
    core_radius: np.ndarray
    s0: float
    r0: np.ndarray
    h: np.ndarray
    a: np.ndarray
    b: np.ndarray
    r: np.ndarray
    noise_var: float
    # core kind: 0 the compact Wendland-type core core_var * f0(q; core_radius); 1 the parametric nonstationary
    # Matern core of App. B (Eq. PScov, smoothness 3/2) with log sigma(x) = log sigma0 + phi_sigma . x and
    # log Sigma(x) = log Sigma0 + phi_Sigma . x (the coordinates as basis functions); then core_var and core_radius
    # are unused and the support is that of C_sparse
    core_kind: int = 0
    sigma0: float = 1.0
    Sigma0: float = 1.0
    phi_sigma: Optional[np.ndarray] = None
    phi_Sigma: Optional[np.ndarray] = None

    def copy(self) -> "Hyper":
        cp = lambda a: None if a is None else a.copy()
        return dataclasses.replace(self, core_radius=self.core_radius.copy(), r0=self.r0.copy(), h=self.h.copy(),
                                   a=self.a.copy(), b=self.b.copy(), r=self.r.copy(), phi_sigma=cp(self.phi_sigma),
                                   phi_Sigma=cp(self.phi_Sigma))

    def validate(self) -> None:
        nb = self.n1 * self.n2
        assert self.core_radius.shape == (self.d,) and self.r0.shape == (self.d,)
        assert self.h.shape == (nb * self.bump_dims,) and self.a.shape == (nb,) and self.b.shape == (nb,)
        assert self.r.shape == (nb,) and 0 <= self.bump_dims <= self.d


def sparse_param_count(d: int, n1: int, n2: int, anisotropic_r0: bool = False) -> int:
    """Length of theta_sparse = (s0, r0, {h_ij, a_ij, b_ij, r_ij}) with h in R^d (Sec. 2.1, count below Eq. C_sparse).

    With coordinate-specific Wendland radii (Sec. 5.1 and 5.2) r0 carries d entries instead of one."""
    return 1 + (d if anisotropic_r0 else 1) + n1 * n2 * (d + 3)


def pack_sparse(hp: Hyper) -> np.ndarray:
    """Flat theta_sparse in the paper's order: s0, r0, then per bump (h_ij, a_ij, b_ij, r_ij)."""
    nb = hp.n1 * hp.n2
    bumps = np.concatenate([hp.h.reshape(nb, hp.bump_dims), hp.a[:, None], hp.b[:, None], hp.r[:, None]], axis=1)
    r0 = hp.r0[:1] if np.all(hp.r0 == hp.r0[0]) else hp.r0
    return np.concatenate([[hp.s0], r0, bumps.ravel()])


@dataclasses.dataclass
class Workload:
    name: str
    X: np.ndarray            # n x d float64, row-major
    Xtest: np.ndarray        # m x d float64
    hyper: Hyper
    resid: Optional[np.ndarray] = None     # r = z - mu (n,)
    mu_test: Optional[np.ndarray] = None   # mu* at test points (m,)
    normals: Optional[np.ndarray] = None   # iid N(0,1) (n,) for a GP draw by the caller
    noise: Optional[np.ndarray] = None     # iid N(0,1) (n,) observation noise draw
    thetas: Optional[List[Hyper]] = None   # batched proposals
    info: dict = dataclasses.field(default_factory=dict)


def _bumps(rng, n1, n2, bump_dims, lo, hi, rlo=0.1, rhi=0.3, alo=0.5, ahi=2.0):
    nb = n1 * n2
    h = rng.uniform(lo, hi, size=(nb, bump_dims)).ravel()
    r = rng.uniform(rlo, rhi, size=nb)
    a = rng.uniform(alo, ahi, size=nb)
    b = np.ones(nb)                    # shape fixed to 1 (Sec. 3.1, prior paragraph)
    return h, a, b, r


def _split_bumps(nbumps: int):
    """n1 x n2 split of a bump count with n1 <= n2 (supplemental table of user parameters)."""
    return {4: (2, 2), 8: (2, 4), 16: (4, 4)}[nbumps]


# ---------------------------------------------------------------------------------------------------------
# support radius calibration by closed-form expected neighbour counts (no pair enumeration)
# ---------------------------------------------------------------------------------------------------------

def _p_within_unit_square(rho: float) -> float:
    """P(|s - s'| < rho) for s, s' iid uniform on [0,1]^2 (exact for rho <= 1)."""
    return math.pi * rho * rho - 8.0 / 3.0 * rho ** 3 + 0.5 * rho ** 4


def expected_row_nnz_uniform_spacetime(n: int, ndays: int, rs: float, rt_days: float) -> float:
    """Expected nonzeros per row for (x,y) ~ U[0,1]^2, day k ~ U{0..ndays-1}, ellipsoidal support (rs, rt)."""
    p = 0.0
    for lag in range(-int(math.ceil(rt_days)), int(math.ceil(rt_days)) + 1):
        frac = 1.0 - (lag / rt_days) ** 2
        if frac <= 0 or abs(lag) >= ndays:
            continue
        p += (ndays - abs(lag)) / ndays ** 2 * _p_within_unit_square(rs * math.sqrt(frac))
    return 1.0 + (n - 1) * p


def _bisect(f, lo, hi, target, iters=80):
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if f(mid) < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def calibrate_rs_uniform(n: int, ndays: int, rt_days: float, nnz_row: float) -> float:
    return _bisect(lambda rs: expected_row_nnz_uniform_spacetime(n, ndays, rs, rt_days), 1e-5, 0.5, nnz_row)


def _mixture_self_overlap(w, mu, sd) -> float:
    """int p(s)^2 ds for an isotropic 2-D Gaussian mixture (closed form)."""
    s2 = sd[:, None] ** 2 + sd[None, :] ** 2
    d2 = ((mu[:, None, :] - mu[None, :, :]) ** 2).sum(-1)
    return float((w[:, None] * w[None, :] * np.exp(-d2 / (2 * s2)) / (2 * math.pi * s2)).sum())


# ---------------------------------------------------------------------------------------------------------
# residual fields: a smooth random Fourier field plus white noise (stands in for a GP draw at large n)
# ---------------------------------------------------------------------------------------------------------

def _fourier_field(rng, X: np.ndarray, scales: np.ndarray, nfeat: int = 64, amp: float = 1.0) -> np.ndarray:
    om = rng.standard_normal((nfeat, X.shape[1])) / scales[None, :]
    ph = rng.uniform(0, 2 * math.pi, nfeat)
    out = np.empty(X.shape[0])
    step = 1 << 16
    for s in range(0, X.shape[0], step):
        out[s:s + step] = np.cos(X[s:s + step] @ om.T + ph).sum(1)
    return out * (amp * math.sqrt(2.0 / nfeat))


# ---------------------------------------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------------------------------------

def spatial_2d(n: int = 2000, m: int = 500, seed: int = SEED_BASE + 1, nbumps: int = 4, rho: float = 0.05,
               noise_var: float = 1e-2, name: str = "spatial2d") -> Workload:
    """2-D points uniform in [0,1]^2 with bumps h ~ U[0,1]^2, r ~ U[0.1,0.3], a ~ U[0.5,2] and a compact core.

    The residual is left for the caller to draw from the GP (``normals``, ``noise``)."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, size=(n, 2))
    Xt = rng.uniform(0.0, 1.0, size=(m, 2))
    n1, n2 = _split_bumps(nbumps)
    h, a, b, r = _bumps(rng, n1, n2, 2, 0.0, 1.0)
    hp = Hyper(d=2, n1=n1, n2=n2, bump_dims=2, core_var=1.0, core_radius=np.full(2, rho), s0=1.0,
               r0=np.full(2, rho), h=h, a=a, b=b, r=r, noise_var=noise_var)
    return Workload(name=name, X=X, Xtest=Xt, hyper=hp, normals=rng.standard_normal(n),
                    noise=rng.standard_normal(n), mu_test=np.zeros(m),
                    info=dict(n=n, m=m, d=2, nbumps=nbumps, rho=rho))


def uniform_spacetime(n: int, m: int, nnz_row: float, nbumps: int, seed: int, ndays: int = 365,
                      rt_days: float = 3.8, noise_var: float = 1e-2, name: str = "spacetime") -> Workload:
    """(x,y) ~ U[0,1]^2, t = k/(ndays-1) with k ~ U{0..ndays-1}; bumps in the spatial coordinates only (Sec. 5.2).

    Temporal truncation r_t = 3.8 days (posterior median, Sec. 5.2 results); the spatial radius is set for the
    requested mean row count by the closed-form expectation above."""
    rng = np.random.default_rng(seed)
    rs = calibrate_rs_uniform(n, ndays, rt_days, nnz_row)
    rt = rt_days / (ndays - 1)

    def draw(k):
        xy = rng.uniform(0.0, 1.0, size=(k, 2))
        day = rng.integers(0, ndays, size=k)
        return np.concatenate([xy, (day / (ndays - 1))[:, None]], axis=1)

    X = draw(n)
    Xt = draw(m)
    n1, n2 = _split_bumps(nbumps)
    h, a, b, r = _bumps(rng, n1, n2, 2, 0.0, 1.0)
    rad = np.array([rs, rs, rt])
    hp = Hyper(d=3, n1=n1, n2=n2, bump_dims=2, core_var=1.0, core_radius=rad, s0=1.0, r0=rad.copy(),
               h=h, a=a, b=b, r=r, noise_var=noise_var)
    field = _fourier_field(rng, X, np.array([0.08, 0.08, 4.0 / (ndays - 1)]))
    resid = field + math.sqrt(noise_var) * rng.standard_normal(n)
    return Workload(name=name, X=X, Xtest=Xt, hyper=hp, resid=resid, mu_test=np.zeros(m),
                    info=dict(n=n, m=m, d=3, nbumps=nbumps, rs=rs, rt=rt, ndays=ndays, nnz_row_target=nnz_row))


def perturb(rng, base: Hyper, rel: float = 0.1) -> Hyper:
    """Proposal: amplitudes, bump radii and noise variance each scaled by (1 + rel * N(0,1)), kept > 0. With the
    non-compact core the bump radii stay (they fix the point set's pattern) and sigma0, Sigma0 move instead."""
    hp = base.copy()
    nb = hp.n1 * hp.n2
    hp.a = np.maximum(base.a * (1.0 + rel * rng.standard_normal(nb)), 1e-3)
    if hp.core_kind == 1:
        hp.sigma0 = base.sigma0 * math.exp(rel * rng.standard_normal())
        hp.Sigma0 = base.Sigma0 * math.exp(rel * rng.standard_normal())
    else:
        hp.r = np.maximum(base.r * (1.0 + rel * rng.standard_normal(nb)), 1e-3)
    hp.noise_var = max(base.noise_var * (1.0 + rel * rng.standard_normal()), 1e-6)
    return hp


def batched_spacetime(n: int = 200_000, B: int = 64, nnz_row: float = 80.0, seed: int = SEED_BASE + 3,
                      m: int = 0) -> Workload:
    """n space-time points, B MCMC-style proposals around one base setting (each +-10% Gaussian)."""
    w = uniform_spacetime(n, m, nnz_row, 8, seed, name=f"batched_spacetime_n{n}_B{B}")
    rng = np.random.default_rng(seed + 1000)
    w.thetas = [perturb(rng, w.hyper) for _ in range(B)]
    w.info["B"] = B
    return w


def station_spacetime(nsites: int = 5000, ndays: int = 240, ncomp: int = 50, nnz_row: float = 100.0,
                      grid: int = 200, grid_days: int = 30, seed: int = SEED_BASE + 5, noise_var: float = 0.25,
                      nbumps: int = 16, rt_days: float = 3.8, with_test: bool = True) -> Workload:
    """Station sites from a seeded isotropic Gaussian mixture on [0,1]^2 times ndays daily steps.

    Values: a temperature-like field 15 + 10 sin(2 pi (k-100)/365) - 8 (lat - 0.5) + smooth field + noise. The
    caller receives r = z - mu with mu the seasonal and latitude terms. Test points are the cell centres of a
    grid x grid lattice times grid_days evenly spaced days."""
    rng = np.random.default_rng(seed)
    w = rng.dirichlet(np.ones(ncomp))
    mu = rng.uniform(0.1, 0.9, size=(ncomp, 2))
    sd = rng.uniform(0.02, 0.1, size=ncomp)
    comp = rng.choice(ncomp, size=nsites, p=w)
    sites = mu[comp] + sd[comp, None] * rng.standard_normal((nsites, 2))
    bad = ~np.all((sites >= 0) & (sites <= 1), axis=1)
    while bad.any():                                   # resample sites that fall outside the unit square
        c = comp[bad]
        sites[bad] = mu[c] + sd[c, None] * rng.standard_normal((int(bad.sum()), 2))
        bad = ~np.all((sites >= 0) & (sites <= 1), axis=1)
    t = np.arange(ndays) / (ndays - 1)
    X = np.empty((nsites * ndays, 3))
    X[:, 0] = np.repeat(sites[:, 0], ndays)
    X[:, 1] = np.repeat(sites[:, 1], ndays)
    X[:, 2] = np.tile(t, nsites)
    # spatial radius: expected rows = sum over lags of (1 + (nsites-1) pi rs^2 (1 - (lag/rt)^2) int p^2)
    ov = _mixture_self_overlap(w, mu, sd)

    def rows(rs):
        tot = 0.0
        for lag in range(-int(math.ceil(rt_days)), int(math.ceil(rt_days)) + 1):
            fr = 1.0 - (lag / rt_days) ** 2
            if fr > 0:
                tot += (ndays - abs(lag)) / ndays * (1.0 + (nsites - 1) * math.pi * rs * rs * fr * ov)
        return tot

    rs = _bisect(rows, 1e-5, 0.5, nnz_row)
    rt = rt_days / (ndays - 1)
    n1, n2 = _split_bumps(nbumps)
    h, a, b, r = _bumps(rng, n1, n2, 2, 0.0, 1.0)
    rad = np.array([rs, rs, rt])
    hp = Hyper(d=3, n1=n1, n2=n2, bump_dims=2, core_var=1.0, core_radius=rad, s0=1.0, r0=rad.copy(),
               h=h, a=a, b=b, r=r, noise_var=noise_var)
    k = np.tile(np.arange(ndays), nsites)
    field = 2.0 * _fourier_field(rng, X, np.array([0.05, 0.05, 3.0 / (ndays - 1)]))
    resid = field + math.sqrt(noise_var) * rng.standard_normal(X.shape[0])
    mean = 15.0 + 10.0 * np.sin(2 * math.pi * (k - 100) / 365.0) - 8.0 * (X[:, 1] - 0.5)
    Xt = np.zeros((0, 3))
    mu_t = np.zeros(0)
    if with_test:
        cc = (np.arange(grid) + 0.5) / grid
        days = np.linspace(0, ndays - 1, grid_days)
        gx, gy, gd = np.meshgrid(cc, cc, days, indexing="ij")
        Xt = np.stack([gx.ravel(), gy.ravel(), gd.ravel() / (ndays - 1)], axis=1)
        mu_t = 15.0 + 10.0 * np.sin(2 * math.pi * (Xt[:, 2] * (ndays - 1) - 100) / 365.0) - 8.0 * (Xt[:, 1] - 0.5)
    return Workload(name=f"station_spacetime_{nsites}x{ndays}", X=X, Xtest=Xt, hyper=hp, resid=resid,
                    mu_test=mu_t, info=dict(n=X.shape[0], m=Xt.shape[0], d=3, nbumps=nbumps, rs=rs, rt=rt,
                                            nsites=nsites, ndays=ndays, nnz_row_target=nnz_row,
                                            z_mean=mean.mean()))


def serving_pointsets(count: int = 20, nmin: int = 5000, nmax: int = 500_000, nnz_row: float = 60.0,
                      seed: int = SEED_BASE + 4, scale: float = 1.0) -> List[Workload]:
    """Point sets with n log-uniform in [nmin, nmax] (scaled by ``scale``), 16 bumps, ~nnz_row per row."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=count)) * scale
    return [uniform_spacetime(int(max(ni, 100)), 0, nnz_row, 16, seed * 100 + i, name=f"serve_set{i}")
            for i, ni in enumerate(ns)]


def noncompact_spatial(n: int = 50_000, m: int = 0, seed: int = SEED_BASE + 6, nbumps: int = 4,
                       noise_var: float = 0.05) -> Workload:
    """2-D points U[0,1]^2 with the non-compact core of App. B (core_kind 1: sigma0 = 1.2, Sigma0 = 0.01, sigma and
    Sigma log-linear in the coordinates), 2 x 2 bumps with radii U[0.04, 0.08] (each family covers a few per cent of
    the domain, so its points form a dense block of the pattern), r0 = 0.02 for about 60 nonzeros per row from f0 at
    n = 50k. The residual is a smooth random Fourier field plus white noise."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, size=(n, 2))
    Xt = rng.uniform(0.0, 1.0, size=(m, 2))
    n1, n2 = _split_bumps(nbumps)
    h, a, b, r = _bumps(rng, n1, n2, 2, 0.1, 0.9, rlo=0.04, rhi=0.08)
    hp = Hyper(d=2, n1=n1, n2=n2, bump_dims=2, core_var=1.0, core_radius=np.full(2, 1.0), s0=0.9,
               r0=np.full(2, 0.02), h=h, a=a, b=b, r=r, noise_var=noise_var, core_kind=1, sigma0=1.2, Sigma0=0.01,
               phi_sigma=np.array([0.4, 0.4]), phi_Sigma=np.array([-0.8, 0.6]))
    field = _fourier_field(rng, X, np.array([0.05, 0.05]))
    resid = field + math.sqrt(noise_var) * rng.standard_normal(n)
    return Workload(name=f"noncompact_{n}", X=X, Xtest=Xt, hyper=hp, resid=resid, mu_test=np.zeros(m),
                    info=dict(n=n, m=m, d=2, nbumps=nbumps))


def config(idx: int, **kw) -> Workload:
    """The five workload shapes: 1 spatial n=2000; 2 space-time n=100k; 3 batched n=200k B=64;
    5 station space-time n=1.2M (4, the serving mix, is built by serving_pointsets)."""
    if idx == 1:
        return spatial_2d(seed=SEED_BASE + 1, **kw)
    if idx == 2:
        kw.setdefault("n", 100_000)
        kw.setdefault("m", 10_000)
        return uniform_spacetime(nnz_row=50.0, nbumps=8, seed=SEED_BASE + 2, name="spacetime_100k", **kw)
    if idx == 3:
        return batched_spacetime(seed=SEED_BASE + 3, **kw)
    if idx == 5:
        return station_spacetime(seed=SEED_BASE + 5, **kw)
    raise ValueError(idx)
