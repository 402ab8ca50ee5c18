"""Failure detection without a GPU fault: the tensor-core kernels' bounded waits, made to run out on purpose.

A context whose wait limits are one poll and zero nanoseconds (GP_OPT_WAIT_POLLS / GP_OPT_WAIT_NS) gives factors
whose first wait that is not already satisfied gives up: the kernel records the failure, waits (with the default
limits) for the operand copies and MMAs it already issued, frees its tensor memory and returns; later tensor-core
launches of the factorization skip their tiles. The factor must then report GP_ERR_TIMEOUT (gp_factor_info,
gp_loglik), its log-likelihood must be NaN, and the context must stay usable: a factor with the default limits on
the same context and point set matches the oracle. Both update-tile kinds run: 128-column tiles of one CTA, and
256 x 256 tiles of a CTA pair (whose copies complete on the even CTA's barriers).
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
def setup():
    from paper_2411_05869_gb300 import gp
    w = synth.uniform_spacetime(20000, 0, 60.0, 8, seed=79, ndays=120)
    hp = w.hyper
    rp, col = oracle.pattern(w.X, hp.core_radius)
    perm = oracle.fill_order(w.X, hp.core_radius, rp, col)
    ref = oracle.sparse_loglik(hp, w.X, rp, col, perm, w.resid)["loglik"]
    ctx = gp.Context(0)
    ps = ctx.assemble(_dev(w.X), hp.core_radius)
    yield dict(gp=gp, w=w, ref=ref, ctx=ctx, ps=ps)
    ps.free()


@pytest.mark.parametrize("blocking", [(8, 128), (16, 256)], ids=["tiles128", "pairs256"])
def test_waits_that_run_out_report_timeout_and_the_context_recovers(setup, blocking):
    gp, w, ctx, ps = setup["gp"], setup["w"], setup["ctx"], setup["ps"]
    ps.set_blocking(*blocking)
    r = _dev(w.resid)
    ctx.set_option("wait_polls", 1)
    ctx.set_option("wait_ns", 0)
    try:
        f = ctx.factor(ps, [w.hyper], gp.GP_MIXED)
    finally:
        ctx.set_option("wait_polls", 1 << 26)
        ctx.set_option("wait_ns", 1_000_000_000)
    info = f.info(allow_timeout=True)
    assert info["timed_out"] == 1
    with pytest.raises(gp.GpError) as e:
        f.info()
    assert e.value.status == 5
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(gp.GpError) as e:
        f.loglik(r, out=out)
    assert e.value.status == 5
    torch.cuda.synchronize()
    assert np.isnan(float(out.cpu()[0]))
    f.free()
    # the same context and point set, default limits
    f2 = ctx.factor(ps, [w.hyper], gp.GP_MIXED)
    assert f2.info()["timed_out"] == 0
    ll = float(f2.loglik(r).cpu()[0])
    assert abs(ll - setup["ref"]) <= 1e-6 * abs(setup["ref"]), (ll, setup["ref"])
    f2.free()
