"""GPU parity on the method's edge cases, against the oracle.

- Pairs exactly on the support boundary: integer lattices with integer radii put many pairs at q^2 = 1 exactly
  (excluded: the support is open, Eq. compSupp), and a radius of 3 puts pairs near q^2 = 1 after the rounding of
  x / 3. Pattern, prediction gather and values must take the same strict decision on both sides.
- Duplicated inputs: noise enters on the observation index only (Eq. Zcov), so duplicates are distinct rows of
  C_z with identical C_y entries; ordering keys tie and are broken by index.
- Test points outside the training points' bounding box and grid: no training neighbour, so m* = mu* exactly.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2411_05869_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def ctx():
    from paper_2411_05869_gb300 import gp
    return gp.Context(0)


def _hyper(d, rho, lo, hi, seed, bump_dims=None, noise=0.05):
    rng = np.random.default_rng(seed)
    bd = d if bump_dims is None else bump_dims
    n1, n2 = 2, 2
    span = hi - lo
    return synth.Hyper(d=d, n1=n1, n2=n2, bump_dims=bd, core_var=1.3, core_radius=np.asarray(rho, float), s0=0.9,
                       r0=np.asarray(rho, float) * 1.1, h=rng.uniform(lo, hi, n1 * n2 * bd),
                       a=rng.uniform(0.5, 2.0, n1 * n2), b=np.ones(n1 * n2), r=rng.uniform(0.2, 0.5, n1 * n2) * span,
                       noise_var=noise)


def _check(ctx, X, hp, Xt, mu=None, rtol_mixed=1e-6):
    from paper_2411_05869_gb300 import gp
    n = X.shape[0]
    rng = np.random.default_rng(n)
    r = rng.standard_normal(n)
    rp, col = oracle.pattern(X, hp.core_radius)
    perm = oracle.fill_order(X, hp.core_radius, rp, col)
    sym = oracle.symbolic(rp, col, perm)
    ref = oracle.sparse_loglik(hp, X, rp, col, perm, r, want_alpha=True)
    ps = ctx.assemble(_dev(X), hp.core_radius)
    assert np.array_equal(ps.export("rowptr"), rp) and np.array_equal(ps.export("col"), col)
    assert np.array_equal(ps.export("perm"), perm)
    assert np.array_equal(ps.export("eta"), sym["eta"]) and np.array_equal(ps.export("sn_first"), sym["sn_first"])
    m_ref = oracle.predict(hp, X, ref["alpha"], Xt, mu)
    out = {}
    for prec, tol in ((gp.GP_FP64, 1e-10), (gp.GP_MIXED, rtol_mixed)):
        f = ctx.factor(ps, [hp], prec)
        ll = float(f.loglik(_dev(r)).cpu()[0])
        assert abs(ll - ref["loglik"]) <= tol * abs(ref["loglik"]), (prec, ll, ref["loglik"])
        m = f.predict(_dev(Xt), None if mu is None else _dev(mu)).cpu().numpy()
        assert np.abs(m - m_ref).max() <= 1e-9 * max(1.0, np.abs(m_ref).max()), prec
        out[prec] = m
        f.free()
    ps.free()
    return rp, col, m_ref, out


@pytest.mark.parametrize("d,side,rho", [(2, 24, (2.0, 2.0)), (3, 11, (2.0, 2.0, 3.0)), (1, 300, (2.0,))])
def test_lattice_pairs_exactly_on_the_boundary(ctx, d, side, rho):
    g = np.stack(np.meshgrid(*[np.arange(side, dtype=float)] * d, indexing="ij"), -1).reshape(-1, d)
    hp = _hyper(d, rho, 0.0, side - 1.0, seed=side)
    # test points on the lattice, half-way between lattice points, and at exactly one radius from a lattice point
    Xt = np.concatenate([g[::7], g[::11] + 0.5, g[::13] + np.asarray(rho)[None, :] * np.eye(d)[0]], axis=0)
    rp, col, _, _ = _check(ctx, g, hp, Xt)
    # axis neighbours two apart sit at q^2 = 1 exactly for radius 2 and are excluded; diagonal ones are included
    i = int(np.ravel_multi_index(tuple([side // 2] * d), [side] * d))
    row = set(col[rp[i]:rp[i + 1]].tolist())
    step = int(np.prod([side] * (d - 1)))   # the lattice neighbour along the first coordinate
    assert i + step in row and i + 2 * step not in row


def test_duplicated_inputs(ctx):
    rng = np.random.default_rng(21)
    X = rng.uniform(0, 1, (1500, 2))
    dup = rng.choice(1500, 200, replace=False)
    X = np.concatenate([X, X[dup], X[dup[:40]]], axis=0)   # 200 pairs and 40 triples of identical points
    X = X[rng.permutation(X.shape[0])]
    hp = _hyper(2, (0.06, 0.06), 0.0, 1.0, seed=22, noise=0.02)
    Xt = np.concatenate([X[:50], rng.uniform(0, 1, (100, 2))], axis=0)
    _check(ctx, X, hp, Xt)


def test_test_points_outside_the_training_box(ctx):
    rng = np.random.default_rng(23)
    X = rng.uniform(0.2, 0.8, (3000, 3))
    X[:, 2] = rng.integers(0, 40, 3000) / 39.0 * 0.6 + 0.2
    hp = _hyper(3, (0.07, 0.07, 0.05), 0.2, 0.8, seed=24, bump_dims=2)
    far = np.array([[-5.0, -5.0, -5.0], [5.0, 5.0, 5.0], [0.5, 0.5, 3.0], [-0.3, 0.5, 0.5], [0.5, 1.2, 0.5],
                    [1e6, -1e6, 0.5], [0.9, 0.9, 0.9], [0.1, 0.1, 0.1]])
    inside = rng.uniform(0.2, 0.8, (100, 3))
    edge = np.array([[0.2 - 0.0699, 0.5, 0.5], [0.8 + 0.0699, 0.5, 0.5], [0.13, 0.13, 0.5]])
    Xt = np.concatenate([far, inside, edge], axis=0)
    mu = np.linspace(-1.0, 1.0, Xt.shape[0])
    _, _, m_ref, out = _check(ctx, X, hp, Xt, mu)
    for m in out.values():   # no training neighbour: exactly the prior mean
        assert np.array_equal(m[:6], mu[:6])
    assert np.array_equal(m_ref[:6], mu[:6])
