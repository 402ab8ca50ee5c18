"""The App. C sampler driven by the library (GpEvaluator, FP64 path) against the same sampler driven by the oracle:
with one seed the chains must take the same accept/reject decisions and reach the same states, and the
log-likelihoods the chains carry must agree to the FP64 parity tolerance. The mean block reuses the factor of
the current settings (solves only), which this comparison checks as well: a stale factor would change its
log-likelihoods."""
import numpy as np
import pytest

import oracle
from paper_2411_05869_gb300 import mcmc, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_library_chains_match_oracle_chains():
    from paper_2411_05869_gb300 import gp
    w = synth.spatial_2d(n=2000, m=10, seed=synth.SEED_BASE + 41)
    hp = w.hyper
    z = np.random.default_rng(8).standard_normal(w.X.shape[0]) + 0.5
    rp, col = oracle.pattern(w.X, hp.core_radius)
    perm = oracle.fill_order(w.X, hp.core_radius, rp, col)
    bounds = mcmc.Bounds(r0=(0.01, 0.1), r=(0.05, 0.5))

    def oracle_ev(thetas, resid, refactor):
        return np.array([oracle.sparse_loglik(t, w.X, rp, col, perm, resid[k])["loglik"]
                         for k, t in enumerate(thetas)])

    ctx = gp.Context(0)
    ps = ctx.assemble(torch.as_tensor(w.X, dtype=torch.float64, device="cuda"), hp.core_radius)
    gev = mcmc.GpEvaluator(ctx, ps, 4, gp.GP_FP64)
    runs = []
    for ev in (gev, oracle_ev):
        s = mcmc.BlockMCMC(ev, z, hp, 4, seed=9, bounds=bounds)
        acc = []
        s.run(4, callback=lambda smp, a: acc.append({k: v.copy() for k, v in a.items()}))
        runs.append((s, acc))
    (sg, ag), (so, ao) = runs
    for a, b in zip(ag, ao):
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    for c in range(4):
        assert np.array_equal(sg.state.beta[c], so.state.beta[c])
        tg, to = sg.state.theta[c], so.state.theta[c]
        for f in ("core_var", "noise_var", "s0"):
            assert getattr(tg, f) == getattr(to, f)
        for f in ("r0", "h", "a", "r"):
            assert np.array_equal(getattr(tg, f), getattr(to, f))
        assert abs(sg.state.loglik[c] - so.state.loglik[c]) <= 1e-10 * abs(so.state.loglik[c])
    assert gev.factorizations >= 1 + 3 * 4 and gev.calls == 1 + 4 * 4
    gev.free()
    ps.free()
