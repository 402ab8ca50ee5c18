"""GPU parity with the non-compact core of App. B (Eq. PScov: the parametric nonstationary Matern core) against the
oracle: the pattern is the support of C_sparse (q0 < 1 for r0, or a shared bump family; bit for bit), the ordering
and symbolic structure bit for bit, the log-likelihood to 1e-10 (FP64) and 1e-6 (mixed), predictive means to 1e-9
of their scale, predictive variances to 1e-9 (FP64) of the prior scale.
"""
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


def _workload(n, seed, d=2):
    """Points U[0,1]^d, 2 x 2 bumps with radii 0.04-0.08 (families cover part of the domain), r0 = 0.035,
    nonstationary core with sigma, Sigma log-linear in the coordinates."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, (n, d))
    nb = 4
    hp = synth.Hyper(d=d, n1=2, n2=2, bump_dims=d, core_var=1.0, core_radius=np.full(d, 1.0), s0=0.9,
                     r0=np.full(d, 0.035), h=rng.uniform(0.1, 0.9, nb * d), a=rng.uniform(0.5, 2.0, nb),
                     b=np.ones(nb), r=rng.uniform(0.04, 0.08, nb), noise_var=0.05, core_kind=1, sigma0=1.2,
                     Sigma0=0.01, phi_sigma=np.full(d, 0.4), phi_Sigma=np.linspace(-0.8, 0.6, d))
    resid = rng.standard_normal(n)
    Xt = np.concatenate([rng.uniform(0, 1, (300, d)), X[:20], np.full((2, d), 3.0)], axis=0)
    return X, resid, Xt, hp


@pytest.mark.parametrize("n,seed", [(3000, 91), (12000, 92)])
def test_noncompact_core_matches_oracle(ctx, n, seed):
    from paper_2411_05869_gb300 import gp
    X, r, Xt, hp = _workload(n, seed)
    rp, col = oracle.pattern_sparse(hp, X)
    perm = oracle.fill_order(X, hp.r0, rp, col)
    sym = oracle.symbolic(rp, col, perm)
    ref = oracle.sparse_loglik(hp, X, rp, col, perm, r, want_alpha=True)
    ps = ctx.assemble_sparse_support(_dev(X), hp)
    assert np.array_equal(ps.export("rowptr"), rp) and np.array_equal(ps.export("col"), col)
    assert np.array_equal(ps.export("perm"), perm)
    assert np.array_equal(ps.export("eta"), sym["eta"]) and np.array_equal(ps.export("sn_first"), sym["sn_first"])
    m_ref = oracle.predict(hp, X, ref["alpha"], Xt)
    rng = np.random.default_rng(seed + 1)
    hp2 = hp.copy()   # another setting on the same support: amplitudes, core and noise move, r0, h, r stay
    hp2.a = hp.a * 1.1
    hp2.sigma0, hp2.Sigma0, hp2.noise_var = 0.9, 0.02, 0.07
    hp2.phi_sigma = -hp.phi_sigma
    ref2 = oracle.sparse_loglik(hp2, X, rp, col, perm, r)
    for prec, tol in ((gp.GP_FP64, 1e-10), (gp.GP_MIXED, 1e-6)):
        f = ctx.factor(ps, [hp, hp2], prec)
        ll = f.loglik(_dev(np.stack([r, r]))).cpu().numpy()
        assert abs(ll[0] - ref["loglik"]) <= tol * abs(ref["loglik"]), (prec, ll[0], ref["loglik"])
        assert abs(ll[1] - ref2["loglik"]) <= tol * abs(ref2["loglik"]), (prec, ll[1], ref2["loglik"])
        m = f.predict(_dev(Xt), b=0).cpu().numpy()
        assert np.abs(m - m_ref).max() <= 1e-9 * max(1.0, np.abs(m_ref).max()), prec
        f.free()
    if n <= 3000:   # the dense variance oracle
        v_ref = oracle.predictive_variance(hp, X, Xt)
        f = ctx.factor(ps, [hp], gp.GP_FP64)
        v = f.predict_var(_dev(Xt)).cpu().numpy()
        scale = max(oracle.cy(hp, x, x) for x in Xt)
        assert np.abs(v - v_ref).max() <= 1e-9 * scale
        f.free()
    ps.free()


def test_noncompact_core_refusals(ctx):
    from paper_2411_05869_gb300 import gp
    X, r, Xt, hp = _workload(500, 93)
    ps = ctx.assemble_sparse_support(_dev(X), hp)
    bad = hp.copy()
    bad.r = hp.r * 1.01   # a different support
    with pytest.raises(gp.GpError):
        ctx.factor(ps, [bad], gp.GP_FP64)
    compact = hp.copy()
    compact.core_kind = 0
    with pytest.raises(gp.GpError):   # the compact core on a support point set
        ctx.factor(ps, [compact], gp.GP_FP64)
    ps.free()
