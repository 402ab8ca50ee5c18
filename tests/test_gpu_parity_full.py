"""GPU parity at full size, against the oracle's stored results (tests/golden/fullsize.json, written by
tests/golden/make_fullsize.py from the oracle alone; the oracle takes minutes at these sizes).

spacetime_100k: the full 100k-point space-time workload. station_5000x12: the 1.2M station field's 5000 sites over
12 days, with the update blocking the autotuner picks at 1.2M (groups of 16 blocks of 64 columns, 256 x 256
CTA-pair group-end tiles): fronts wider than one group, so multi-group fronts, the paired block steps and the
CTA-pair group-end updates all run. Structure bit for bit (fingerprints), FP64 log-likelihood to 1e-10 relative,
mixed precision (FP64 and FP32 diagonal-block factorization) to 1e-6, predictive means to 1e-9 of their scale.
"""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_2411_05869_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fullsize.json")))
NTEST = 500


def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _inputs(name):
    """The same seeded inputs make_fullsize.py gave the oracle."""
    if name == "spacetime_100k":
        w = synth.config(2, m=NTEST)
        rng = np.random.default_rng(2411)
        return w.X, w.resid, w.Xtest[:NTEST], w.hyper, synth.perturb(rng, w.hyper, 0.1)
    s = synth.config(5, with_test=True)
    ns, nd, days = s.info["nsites"], s.info["ndays"], 12
    idx = (np.arange(ns)[:, None] * nd + np.arange(days)[None, :]).ravel()
    t = s.Xtest[s.Xtest[:, 2] <= (days - 1) / (nd - 1)]
    Xt = t[np.linspace(0, t.shape[0] - 1, NTEST).astype(np.int64)]
    rng = np.random.default_rng(2412)
    return s.X[idx], s.resid[idx], Xt, s.hyper, synth.perturb(rng, s.hyper, 0.1)


@pytest.fixture(scope="module")
def ctx():
    from paper_2411_05869_gb300 import gp
    return gp.Context(0)


@pytest.fixture(scope="module", params=["spacetime_100k", "station_5000x12"])
def case(request, ctx):
    name = request.param
    g = GOLD[name]
    X, r, Xt, hp, hp2 = _inputs(name)
    assert _sha(X) == g["inputs"]["X"], "inputs differ from the ones the oracle saw"
    assert [float(v).hex() for v in hp.core_radius] == g["inputs"]["core_radius"]
    assert _sha(Xt) == g["inputs"]["Xtest"]
    assert r.sum() == pytest.approx(g["inputs"]["resid_sum"], rel=1e-12, abs=1e-9)
    assert (r * r).sum() == pytest.approx(g["inputs"]["resid_sumsq"], rel=1e-12)
    ps = ctx.assemble(_dev(X), hp.core_radius)
    if name == "station_5000x12":
        ps.set_blocking(16, 256)
    yield dict(name=name, g=g, X=X, r=r, Xt=Xt, thetas=[hp, hp2], ps=ps)
    ps.free()


def test_structure_bit_exact_full_size(case):
    ps, g = case["ps"], case["g"]
    inf = ps.info()
    assert inf["nnz"] == g["nnz"] and inf["nnzL"] == g["nnzL"] and inf["nsuper"] == g["nsuper"]
    for name in ("rowptr", "col", "perm", "parent", "eta", "sn_first", "sn_rows"):
        assert _sha(ps.export(name)) == g["structure"][name], name


def test_fp64_full_size(case, ctx):
    g, ps = case["g"], case["ps"]
    f = ctx.factor(ps, case["thetas"])
    r = _dev(case["r"])
    ll = f.loglik(_dev(np.stack([case["r"], case["r"]]))).cpu().numpy()
    for b in range(2):
        assert abs(ll[b] - g["loglik"][b]) <= 1e-10 * abs(g["loglik"][b]), (b, ll[b], g["loglik"][b])
    ref = np.array(g["predict_mean"])
    m = f.predict(_dev(case["Xt"]), b=0).cpu().numpy()
    assert np.abs(m - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())
    del r
    f.free()


@pytest.mark.parametrize("diag_fp32,split_f16", [(0, 1), (1, 1), (0, 0)])
def test_mixed_full_size(case, ctx, diag_fp32, split_f16):
    from paper_2411_05869_gb300 import gp
    g, ps = case["g"], case["ps"]
    if case["name"] == "station_5000x12":
        assert g["max_width"] > 16 * 64   # a front spans more than one 1024-column update group
    split0 = ctx.get_option("split_f16")
    ctx.set_option("diag_fp32", diag_fp32)
    ctx.set_option("split_f16", split_f16)
    try:
        f = ctx.factor(ps, case["thetas"], gp.GP_MIXED)
    finally:
        ctx.set_option("diag_fp32", 0)
        ctx.set_option("split_f16", split0)
    err = torch.empty(2, dtype=torch.float64, device="cuda")
    ll = f.loglik(_dev(np.stack([case["r"], case["r"]])), err=err).cpu().numpy()
    for b in range(2):
        assert abs(ll[b] - g["loglik"][b]) <= 1e-6 * abs(g["loglik"][b]), (b, ll[b], g["loglik"][b])
    assert float(err.max().cpu()) <= 1e-10   # gp_loglik's default stopping residual; predict refines to 1e-12
    ref = np.array(g["predict_mean"])
    m = f.predict(_dev(case["Xt"]), b=0).cpu().numpy()
    assert np.abs(m - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())
    f.free()
