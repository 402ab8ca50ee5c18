"""Pins of the oracle's kernel arithmetic against what the paper fixes (Sec. 2.1, Sec. 2.3, Prop. 1, Appendix S2).

None of these re-type the oracle's formula: they check closed forms, asymptotic coefficients, symmetry,
positive definiteness, special cases and the paper's printed counts.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2411_05869_gb300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def _hyper(d=2, n1=2, n2=2, bump_dims=None, rho=0.2, s0=1.0, core_var=1.0, noise=1e-2, seed=0):
    rng = np.random.default_rng(seed)
    bd = d if bump_dims is None else bump_dims
    nb = n1 * n2
    return synth.Hyper(d=d, n1=n1, n2=n2, bump_dims=bd, core_var=core_var, core_radius=np.full(d, rho), s0=s0,
                       r0=np.full(d, rho), h=rng.uniform(0, 1, nb * bd), a=rng.uniform(0.5, 2, nb),
                       b=np.ones(nb), r=rng.uniform(0.1, 0.3, nb), noise_var=noise)


# ------------------------------------------------------------------ Wendland f0 (Eq. compSupp)

def test_wendland_support_and_origin():
    assert oracle.wendland(0.0) == 1.0
    assert oracle.wendland(1.0) == 0.0
    assert oracle.wendland(1.0 + 1e-12) == 0.0
    assert oracle.wendland(7.0) == 0.0
    qs = np.linspace(1e-6, 1 - 1e-6, 101)
    assert all(oracle.wendland(q) > 0 for q in qs)
    vals = [oracle.wendland(q) for q in qs]
    assert all(a > b for a, b in zip(vals, vals[1:])), "f0 must decrease on (0,1)"


def test_wendland_taylor_coefficients_pin_printed_constants():
    """Expanding (1-q)^8 (c3 q^3 + 25 q^2 + 8 q + 1) gives 1 - 11 q^2 + (c3 - 32) q^3 + 42 q^4 + ... at c3 = 35.

    So the q^2 coefficient pins 25 and 8, the q^3 coefficient pins the printed 35 (a 32 would leave 0)."""
    c3 = GOLD["wendland_cubic_coefficient"]["c3"]
    q = 1e-3
    w = oracle.wendland(q)
    assert (w - 1.0) / q ** 2 == pytest.approx(-11.0, abs=1e-2)
    assert (w - 1.0 + 11.0 * q * q) / q ** 3 == pytest.approx(c3 - 32 + 42 * q, abs=5e-3)


def test_wendland_edge_behaviour():
    """Near q = 1, f0 ~ (1-q)^8 p(1) with p(1) = 35 + 25 + 8 + 1 = 69."""
    eps = 1e-3
    assert oracle.wendland(1 - eps) / eps ** 8 == pytest.approx(69.0 - 163.0 * eps, rel=1e-4)


def test_wendland_positive_definite_fourier_3d():
    """Prop. 1 needs f0 strictly PD in R^d; its radial Fourier transform in R^3 must be positive."""
    q = np.linspace(0, 1, 20001)
    w = np.array([oracle.wendland(x) for x in q])
    for om in np.linspace(0.5, 120.0, 60):
        integrand = w * q * np.sin(om * q)
        ft = 4 * math.pi / om * np.trapezoid(integrand, q)
        assert ft > 0, om


# ------------------------------------------------------------------ bump function g (Eq. bumpFcn)

def test_bump_centre_and_support():
    h = np.array([0.3, 0.6])
    assert oracle.bump(h, h, 1.7, 1.0, 0.2) == 1.7          # exp(0) = 1: g(h) = a
    assert oracle.bump(h + [0.2, 0.0], h, 1.7, 1.0, 0.2) == 0.0   # |x - h| = r: exactly zero
    assert oracle.bump(h + [0.15, 0.15], h, 1.7, 1.0, 0.2) == 0.0  # beyond r
    assert oracle.bump(h + [0.0, 0.19], h, 1.7, 1.0, 0.2) > 0.0   # exp(-9.3): tiny but nonzero


@pytest.mark.parametrize("b", [0.1, 1.0, 3.0])
def test_bump_half_radius_closed_form(b):
    """At |x - h| = r/2: 1 - (1 - 1/4)^(-1) = -1/3, so g = a exp(-b/3)."""
    h = np.array([0.5, 0.5])
    x = h + np.array([0.06, 0.08])   # |x-h| = 0.1 = r/2
    g = oracle.bump(x, h, 0.8, b, 0.2)
    assert g == pytest.approx(0.8 * math.exp(-b / 3.0), rel=1e-14)


def test_bump_dims_ignore_trailing_coordinates():
    """Space-time bumps live in the spatial coordinates only (Sec. 5.2)."""
    hp = _hyper(d=3, bump_dims=2)
    X = np.array([[0.4, 0.5, 0.0], [0.4, 0.5, 0.9]])
    F = oracle.features(hp, X)
    assert np.array_equal(F[0], F[1])


# ------------------------------------------------------------------ C_y, C_z (Eq. C_sparse, Eq. Zcov)

def test_cy_diagonal_closed_form():
    """C_y(x,x) = core_var f0(0) (s0 f0(0) + sum_i f_i(x)^2) = core_var (s0 + |F(x)|^2)."""
    hp = _hyper(n1=3, n2=2, s0=0.7, core_var=2.5)
    X = np.random.default_rng(1).uniform(0, 1, (20, 2))
    F = oracle.features(hp, X)
    for k in range(20):
        assert oracle.cy(hp, X[k], X[k]) == pytest.approx(2.5 * (0.7 + (F[k] ** 2).sum()), rel=1e-15)


def test_cz_symmetric_and_zero_beyond_support():
    hp = _hyper(rho=0.15)
    X = np.random.default_rng(2).uniform(0, 1, (150, 2))
    C = oracle.dense_cov(hp, X)
    assert np.array_equal(C, C.T), "C_z must be bitwise symmetric"
    dist = np.sqrt(((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))
    assert np.all(C[dist > 0.15 * (1 + 1e-9)] == 0.0)
    assert np.all(np.diag(C) > hp.noise_var)


@pytest.mark.parametrize("d,seed", [(1, 3), (2, 4), (3, 5)])
def test_prop1_positive_definite(d, seed):
    """Prop. 1: C_y is PD, so lambda_min(C_z) >= tau^2."""
    hp = _hyper(d=d, n1=2, n2=3, rho=0.3, seed=seed, noise=1e-3)
    X = np.random.default_rng(seed).uniform(0, 1, (250, d))
    C = oracle.dense_cov(hp, X)
    lam = np.linalg.eigvalsh(C)
    assert lam[0] >= hp.noise_var - 1e-12 * abs(lam[-1])
    Cy = oracle.dense_cov(hp, X, noise=False)
    assert np.linalg.eigvalsh(Cy)[0] >= -1e-12 * abs(lam[-1])


def test_stationary_limit_is_scenario_s2():
    """Sec. 2.3 case 1 and Appendix S2: no bumps, r0 -> infinity gives C_y = sigma^2 f0(|x-x'|; r0).

    The reference value uses the expanded Wendland polynomial (numpy.polynomial), not the oracle's form."""
    s2 = GOLD["scenario_S2"]
    poly = np.polynomial.polynomial.polymul(np.polynomial.polynomial.polypow([1.0, -1.0], 8),
                                            [1.0, 8.0, 25.0, float(GOLD["wendland_cubic_coefficient"]["c3"])])
    hp = synth.Hyper(d=1, n1=1, n2=1, bump_dims=1, core_var=s2["sigma2"], core_radius=np.array([s2["r0"]]), s0=1.0,
                     r0=np.array([1e150]), h=np.array([5.0]), a=np.array([0.0]), b=np.array([1.0]),
                     r=np.array([1.0]), noise_var=0.1)
    rng = np.random.default_rng(7)
    for _ in range(200):
        x, y = rng.uniform(*s2["domain"], 2)
        q = abs(x - y) / s2["r0"]
        ref = s2["sigma2"] * np.polynomial.polynomial.polyval(q, poly) if q < 1 else 0.0
        # the expanded monomial form cancels near q = 1 (coefficients up to ~1e4), hence the absolute slack
        assert oracle.cy(hp, [x], [y]) == pytest.approx(ref, rel=1e-11, abs=1e-11)


def test_sparse_stationary_special_case():
    """Sec. 2.3 case 1: C_core = 1 (core support far wider than r0) and all amplitudes zero gives s0 f0."""
    hp = synth.Hyper(d=2, n1=2, n2=2, bump_dims=2, core_var=1.0, core_radius=np.array([1e150, 1e150]), s0=2.0,
                     r0=np.array([0.3, 0.3]), h=np.full(8, 0.5), a=np.zeros(4), b=np.ones(4), r=np.full(4, 0.4),
                     noise_var=0.0)
    x, y = np.array([0.1, 0.2]), np.array([0.2, 0.3])
    assert oracle.cy(hp, x, y) == 2.0 * oracle.wendland(math.sqrt(0.02) / 0.3) or \
        oracle.cy(hp, x, y) == pytest.approx(2.0 * oracle.wendland(math.sqrt(0.02) / 0.3), rel=1e-14)


def test_illustrative_1d_example_structure():
    """Sec. 2.1 example (n1 = 2, n2 = 3, r0 = 0.15): far points share a bump family only through f_i."""
    ex = GOLD["illustrative_1d"]
    h = np.array([0.17, 0.70, 0.45,      # family 1: covers 0.17 and 0.7
                  0.17, 0.90, 0.45])     # family 2: covers 0.17 and 0.9, not 0.7
    r = np.array([0.1, 0.1, 0.05, 0.1, 0.1, 0.05])
    hp = synth.Hyper(d=1, n1=2, n2=3, bump_dims=1, core_var=1.0, core_radius=np.array([1e150]), s0=1.0,
                     r0=np.array([ex["r0"]]), h=h, a=np.ones(6), b=np.ones(6), r=r, noise_var=0.0)
    for x, y in ex["pairs_positive"]:
        assert oracle.csparse(hp, [x], [y]) > 0
    for x, y in ex["pairs_zero"]:
        assert oracle.csparse(hp, [x], [y]) == 0.0
    F = oracle.features(hp, np.array([[0.17], [0.7], [0.9]]))
    assert F[0, 0] > 0 and F[1, 0] > 0 and F[0, 1] > 0 and F[2, 1] > 0 and F[1, 1] == 0


def test_hyperparameter_counts():
    for d, n1, n2, cnt in GOLD["hyperparameter_count"]["cases"]:
        assert synth.sparse_param_count(d, n1, n2) == cnt
        hp = synth.Hyper(d=d, n1=n1, n2=n2, bump_dims=d, core_var=1.0, core_radius=np.ones(d), s0=1.0,
                         r0=np.full(d, 0.2), h=np.zeros(n1 * n2 * d), a=np.ones(n1 * n2), b=np.ones(n1 * n2),
                         r=np.ones(n1 * n2), noise_var=0.1)
        assert synth.pack_sparse(hp).shape[0] == cnt
    for d, n1, n2, cnt in GOLD["hyperparameter_count_anisotropic"]["cases"]:
        assert synth.sparse_param_count(d, n1, n2, anisotropic_r0=True) == cnt


# ------------------------------------------------------------------ features f_i = sum_j g_ij (Sec. 2.1)

def _two_family_hyper():
    """n1 = 2 families of n2 = 3 bumps in 2-D, placed around x = (0.4, 0.5) at distances with closed forms.

    Family 1: bump 0 at distance r/2 (g = a e^{-b/3}), bump 1 at distance r/sqrt(2) (t = 1/2, so
    1 - (1 - t)^{-1} = -1 and g = a e^{-b}), bump 2 beyond its radius (g = 0).
    Family 2: bump 0 centred on x (g = a), bumps 1 and 2 beyond their radii."""
    x = np.array([0.4, 0.5])
    h = np.array([[0.46, 0.58],    # |x - h| = 0.1, r = 0.2: t = 1/4
                  [0.3, 0.4],      # |x - h|^2 = 0.02, r = 0.2: t = 1/2
                  [0.9, 0.9],      # far outside r = 0.2
                  [0.4, 0.5],      # on x
                  [0.0, 0.0],
                  [0.8, 0.1]])
    a = np.array([1.3, 0.7, 1.9, 1.6, 1.1, 0.9])
    b = np.array([0.5, 2.0, 1.0, 1.0, 1.0, 1.0])
    r = np.array([0.2, 0.2, 0.2, 0.25, 0.3, 0.3])
    hp = synth.Hyper(d=2, n1=2, n2=3, bump_dims=2, core_var=1.7, core_radius=np.array([0.3, 0.3]), s0=0.8,
                     r0=np.array([0.25, 0.25]), h=h.ravel(), a=a, b=b, r=r, noise_var=1e-2)
    return hp, x


def test_features_sum_of_bumps_closed_form():
    """f_1(x) = a_11 e^{-b_11/3} + a_12 e^{-b_12} + 0 and f_2(x) = a_21, written out by hand: a maximum over j,
    a sum of squares, a dropped bump or a family mix-up all give other numbers."""
    hp, x = _two_family_hyper()
    F = oracle.features(hp, x[None, :])[0]
    f1 = 1.3 * math.exp(-0.5 / 3.0) + 0.7 * math.exp(-2.0)
    f2 = 1.6
    assert F[0] == pytest.approx(f1, rel=1e-13)
    assert F[1] == pytest.approx(f2, rel=1e-15)
    assert F[0] != pytest.approx(max(1.3 * math.exp(-0.5 / 3.0), 0.7 * math.exp(-2.0)), rel=1e-6)


def test_csparse_and_cy_of_a_pair_by_hand():
    """C_sparse(x, y) = s0 f0(|x - y| / r0) + f_1(x) f_1(y) + f_2(x) f_2(y) (Eq. C_sparse) and
    C_y = core_var f0(|x - y| / rho) C_sparse, at a pair whose features are closed forms: y = x + (0.06, 0.08)
    sits on bump 11 (g = a), at |y - h_12| = sqrt(0.0436) from bump 12, on nothing of family 2 but bump 21 (at
    |y - h_21| = 0.1 of r = 0.25: t = 0.16). f0 comes from the expanded polynomial (numpy), not from the oracle."""
    hp, x = _two_family_hyper()
    y = x + np.array([0.06, 0.08])
    c3 = float(GOLD["wendland_cubic_coefficient"]["c3"])
    poly = np.polynomial.polynomial.polymul(np.polynomial.polynomial.polypow([1.0, -1.0], 8), [1.0, 8.0, 25.0, c3])

    def f0(q):
        return float(np.polynomial.polynomial.polyval(q, poly)) if q < 1 else 0.0

    def g(dist2, a, b, r):
        t = dist2 / (r * r)
        return a * math.exp(b * (1.0 - 1.0 / (1.0 - t))) if t < 1 else 0.0

    fx = [1.3 * math.exp(-0.5 / 3.0) + 0.7 * math.exp(-2.0), 1.6]
    d12 = (0.46 - 0.3) ** 2 + (0.58 - 0.4) ** 2
    fy = [1.3 + g(d12, 0.7, 2.0, 0.2), g(0.01, 1.6, 1.0, 0.25)]
    assert oracle.features(hp, y[None, :])[0] == pytest.approx(fy, rel=1e-13)
    q0 = 0.1 / 0.25
    cs = 0.8 * f0(q0) + fx[0] * fy[0] + fx[1] * fy[1]
    assert oracle.csparse(hp, x, y) == pytest.approx(cs, rel=1e-12)
    qc = 0.1 / 0.3
    assert oracle.cy(hp, x, y) == pytest.approx(1.7 * f0(qc) * cs, rel=1e-12)
    # the diagonal: C_y(x, x) = core_var (s0 + f_1^2 + f_2^2) with the hand-computed features
    assert oracle.cy(hp, x, x) == pytest.approx(1.7 * (0.8 + fx[0] ** 2 + fx[1] ** 2), rel=1e-13)
