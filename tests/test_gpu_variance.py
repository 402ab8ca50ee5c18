"""GPU parity of the predictive variance (Sec. 3.2, the diagonal of C_{y|z} = C_y - C_{y,z} C_z^{-1} C_{z,y}) against the
oracle's dense computation, element by element, and its defining bounds at full size.

FP64 factor: within 1e-9 of the prior variance's scale. Mixed factor: FP32 forward solves with the FP32 panels,
within 1e-5 of that scale (|w|^2 carries the mixed factor's relative accuracy, about 1e-6).
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


def _cases():
    return {
        "spatial_2d_n2000": lambda: synth.spatial_2d(n=2000, m=300, seed=synth.SEED_BASE + 1),
        "spacetime_n4000": lambda: synth.uniform_spacetime(4000, 400, 40.0, 8, seed=77, ndays=60),
        "station_300x16": lambda: synth.station_spacetime(nsites=300, ndays=16, ncomp=10, nnz_row=60.0, grid=8,
                                                          grid_days=3, seed=78, nbumps=16),
    }


@pytest.mark.parametrize("name", list(_cases().keys()))
def test_variance_matches_oracle(ctx, name):
    from paper_2411_05869_gb300 import gp
    w = _cases()[name]()
    hp = w.hyper
    rng = np.random.default_rng(3)
    # test points: the workload's, some training inputs themselves, and points far outside the data
    far = np.full((3, w.X.shape[1]), 5.0)
    Xt = np.concatenate([w.Xtest, w.X[rng.choice(w.X.shape[0], 37, replace=False)], far], axis=0)
    ref = oracle.predictive_variance(hp, w.X, Xt)
    prior = np.array([oracle.cy(hp, x, x) for x in Xt])
    scale = prior.max()
    ps = ctx.assemble(_dev(w.X), hp.core_radius)
    for prec, tol in ((gp.GP_FP64, 1e-9), (gp.GP_MIXED, 1e-5)):
        f = ctx.factor(ps, [hp], prec)
        v = f.predict_var(_dev(Xt)).cpu().numpy()
        assert np.abs(v - ref).max() <= tol * scale, (prec, np.abs(v - ref).max(), scale)
        assert np.array_equal(v[-3:], prior[-3:]) or np.allclose(v[-3:], prior[-3:], rtol=1e-15)
        v2 = f.predict_var(_dev(Xt)).cpu().numpy()   # a second call reuses the workspace: same bits
        assert v.tobytes() == v2.tobytes()
        f.free()
    ps.free()


def test_variance_batches_and_proposals(ctx):
    """Many chunks of 32 test points (a ragged last one), and proposal b of a batched factor."""
    from paper_2411_05869_gb300 import gp
    w = synth.uniform_spacetime(3000, 0, 40.0, 8, seed=81, ndays=50)
    rng = np.random.default_rng(4)
    Xt = np.concatenate([rng.uniform(0, 1, (1077, 2)), rng.integers(0, 50, (1077, 1)) / 49.0], axis=1)
    th = [w.hyper, synth.perturb(rng, w.hyper)]
    ps = ctx.assemble(_dev(w.X), w.hyper.core_radius)
    f = ctx.factor(ps, th, gp.GP_FP64)
    for b in range(2):
        ref = oracle.predictive_variance(th[b], w.X, Xt)
        v = f.predict_var(_dev(Xt), b=b).cpu().numpy()
        scale = max(oracle.cy(th[b], x, x) for x in Xt[:50])
        assert np.abs(v - ref).max() <= 1e-9 * max(scale, 1.0), b
    f.free()
    ps.free()


def test_variance_bounds_at_100k(ctx):
    """The full 100k space-time workload (no dense oracle at this size): 0 < var <= C_y(x*, x*) at test points,
    var <= tau^2 at training inputs (Sec. 3.2: conditioning on a noisy observation at x* itself), FP64 and mixed
    agreeing to 1e-5 of the prior scale."""
    from paper_2411_05869_gb300 import gp
    w = synth.config(2, m=3000)
    hp = w.hyper
    rng = np.random.default_rng(5)
    tr = w.X[rng.choice(w.X.shape[0], 200, replace=False)]
    Xt = np.concatenate([w.Xtest, tr], axis=0)
    ps = ctx.assemble(_dev(w.X), hp.core_radius)
    out = {}
    for prec in (gp.GP_FP64, gp.GP_MIXED):
        f = ctx.factor(ps, [hp], prec)
        out[prec] = f.predict_var(_dev(Xt)).cpu().numpy()
        f.free()
    v = out[gp.GP_FP64]
    prior = np.array([oracle.cy(hp, x, x) for x in Xt])
    assert np.all(v > 0) and np.all(v <= prior * (1 + 1e-12))
    assert np.all(v[-200:] <= hp.noise_var * (1 + 1e-9))
    assert np.abs(out[gp.GP_MIXED] - v).max() <= 1e-5 * prior.max()
    ps.free()
