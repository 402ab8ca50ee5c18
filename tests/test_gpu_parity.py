"""GPU parity: the CUDA path through the C-ABI against the oracle, element by element.

Structure (pattern, order, etree, column counts, supernodes, row structures) must match bit for bit;
FP64 log-likelihoods to 1e-10 relative; alpha and predictive means to 1e-9 of their scale (the same
factorization carried through two triangular solves and one more product).
"""
import copy
import math

import numpy as np
import pytest

import oracle
from paper_2411_05869_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LOGLIK_RTOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    from paper_2411_05869_gb300 import gp
    return gp.Context(0)


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _cases():
    return {
        "spatial_2d_n2000": lambda: synth.spatial_2d(n=2000, m=300, seed=synth.SEED_BASE + 1),
        "spacetime_n6000": lambda: synth.uniform_spacetime(6000, 400, 40.0, 8, seed=77, ndays=60),
        "station_600x20": lambda: synth.station_spacetime(nsites=600, ndays=20, ncomp=10, nnz_row=60.0, grid=12,
                                                          grid_days=3, seed=78, nbumps=16),
    }


@pytest.fixture(scope="module", params=list(_cases().keys()))
def case(request, ctx):
    w = _cases()[request.param]()
    hp = w.hyper
    if w.resid is None:
        y = oracle.sample_dense(hp, w.X, w.normals)
        w.resid = y + math.sqrt(hp.noise_var) * w.noise
    rp, col = oracle.pattern(w.X, hp.core_radius)
    perm = oracle.fill_order(w.X, hp.core_radius, rp, col)
    sym = oracle.symbolic(rp, col, perm)
    ps = ctx.assemble(_dev(w.X), hp.core_radius)
    return dict(name=request.param, w=w, rp=rp, col=col, perm=perm, sym=sym, ps=ps)


def test_pattern_bit_exact(case):
    ps = case["ps"]
    assert np.array_equal(ps.export("rowptr"), case["rp"])
    assert np.array_equal(ps.export("col"), case["col"])


def test_cell_list_sorted_by_cell_then_index(case):
    w = case["w"]
    key = oracle.cell_keys(w.X, w.hyper.core_radius)
    cp = case["ps"].export("cell_perm")
    ref = np.lexsort((np.arange(len(key)), key))
    assert np.array_equal(cp, ref)


def test_order_and_symbolic_bit_exact(case):
    ps, sym = case["ps"], case["sym"]
    assert np.array_equal(ps.export("perm"), case["perm"])
    assert np.array_equal(ps.export("parent"), sym["parent"])
    assert np.array_equal(ps.export("eta"), sym["eta"])
    assert np.array_equal(ps.export("sn_first"), sym["sn_first"])
    assert np.array_equal(ps.export("sn_rowptr"), sym["sn_rowptr"])
    assert np.array_equal(ps.export("sn_rows"), sym["sn_rows"])
    assert np.array_equal(ps.export("sn_parent"), sym["sn_parent"])
    assert np.array_equal(ps.export("sn_level"), sym["sn_level"])
    inf = ps.info()
    assert inf["nnzL"] == sym["nnzL"]


def test_loglik_fp64_matches_oracle(case, ctx):
    w, ps = case["w"], case["ps"]
    ref = oracle.sparse_loglik(w.hyper, w.X, case["rp"], case["col"], case["perm"], w.resid, want_alpha=True)
    f = ctx.factor(ps, [w.hyper])
    err = torch.empty(1, dtype=torch.float64, device="cuda")
    ll = f.loglik(_dev(w.resid), err=err)
    got = float(ll.cpu()[0])
    assert abs(got - ref["loglik"]) <= LOGLIK_RTOL * abs(ref["loglik"]), (got, ref["loglik"])
    assert float(err.cpu()[0]) < 1e-12
    # predictive mean at test points (and alpha through it)
    mu = np.linspace(-0.5, 0.5, w.Xtest.shape[0])
    m_ref = oracle.predict(w.hyper, w.X, ref["alpha"], w.Xtest, mu)
    m_gpu = f.predict(_dev(w.Xtest), _dev(mu)).cpu().numpy()
    scale = max(1.0, np.abs(m_ref).max())
    assert np.abs(m_gpu - m_ref).max() <= 1e-9 * scale
    f.free()


def test_batched_proposals_each_match_oracle(case, ctx):
    w, ps = case["w"], case["ps"]
    rng = np.random.default_rng(5)
    thetas = [w.hyper] + [synth.perturb(rng, w.hyper) for _ in range(2)]
    f = ctx.factor(ps, thetas)
    R = np.stack([w.resid, w.resid * 0.5 + 0.1, np.roll(w.resid, 7)])
    ll = f.loglik(_dev(R)).cpu().numpy()
    for b, hp in enumerate(thetas):
        ref = oracle.sparse_loglik(hp, w.X, case["rp"], case["col"], case["perm"], R[b])
        assert abs(ll[b] - ref["loglik"]) <= LOGLIK_RTOL * abs(ref["loglik"]), (b, ll[b], ref["loglik"])
    f.free()


def test_repeatable_bitwise(case, ctx):
    w, ps = case["w"], case["ps"]
    f = ctx.factor(ps, [w.hyper])
    r = _dev(w.resid)
    a = f.loglik(r).cpu().numpy().copy()
    f.update([w.hyper])
    b = f.loglik(r).cpu().numpy().copy()
    assert a.tobytes() == b.tobytes()
    f.free()


def test_not_positive_definite_is_flagged(ctx):
    w = synth.spatial_2d(n=500, m=1, seed=31)
    hp = w.hyper.copy()
    hp.noise_var = -50.0
    ps = ctx.assemble(_dev(w.X), hp.core_radius)
    f = ctx.factor(ps, [w.hyper, hp])
    ll = f.loglik(_dev(np.ones((2, 500)))).cpu().numpy()
    assert np.isfinite(ll[0]) and ll[1] == -np.inf
    inf = f.info()
    assert inf["not_pd_count"] == 1 and inf["not_pd_column"][0] == -1 and inf["not_pd_column"][1] >= 0


@pytest.mark.parametrize("n,d", [(1, 2), (7, 1), (64, 3), (65, 2), (300, 1)])
def test_edge_sizes(ctx, n, d):
    rng = np.random.default_rng(n + d)
    X = rng.uniform(0, 1, (n, d))
    rho = np.full(d, 0.3)
    nb = 2
    hp = synth.Hyper(d=d, n1=1, n2=nb, bump_dims=d, core_var=1.2, core_radius=rho, s0=0.9, r0=rho.copy(),
                     h=rng.uniform(0, 1, nb * d), a=np.array([1.0, 0.7]), b=np.ones(nb), r=np.array([0.4, 0.3]),
                     noise_var=0.05)
    r = rng.standard_normal(n)
    rp, col = oracle.pattern(X, rho)
    perm = oracle.fill_order(X, rho, rp, col)
    ref = oracle.sparse_loglik(hp, X, rp, col, perm, r, want_alpha=True)
    ps = ctx.assemble(_dev(X), rho)
    assert np.array_equal(ps.export("col"), col)
    assert np.array_equal(ps.export("perm"), perm)
    f = ctx.factor(ps, [hp])
    ll = float(f.loglik(_dev(r)).cpu()[0])
    assert abs(ll - ref["loglik"]) <= LOGLIK_RTOL * abs(ref["loglik"])


MIXED_RTOL = 1e-6


@pytest.mark.parametrize("split_f16", [0, 1])
@pytest.mark.parametrize("diag_fp32", [0, 1])
def test_loglik_mixed_matches_oracle(case, ctx, diag_fp32, split_f16):
    """GP_MIXED: tensor-core updates on TF32 operand pairs (default) or FP16 pairs (GP_OPT_SPLIT_F16),
    FP64-accumulated diagonal tiles factored in FP64 (default) or in FP32 (GP_OPT_DIAG_FP32), FP64 refinement;
    loglik within 1e-6."""
    from paper_2411_05869_gb300 import gp
    w, ps = case["w"], case["ps"]
    ref = oracle.sparse_loglik(w.hyper, w.X, case["rp"], case["col"], case["perm"], w.resid, want_alpha=True)
    split0 = ctx.get_option("split_f16")
    ctx.set_option("diag_fp32", diag_fp32)
    ctx.set_option("split_f16", split_f16)
    try:
        f = ctx.factor(ps, [w.hyper], gp.GP_MIXED)
    finally:
        ctx.set_option("diag_fp32", 0)
        ctx.set_option("split_f16", split0)
    assert f.info()["diag_fp32"] == diag_fp32 and f.info()["split_f16"] == split_f16
    err = torch.empty(1, dtype=torch.float64, device="cuda")
    ll = float(f.loglik(_dev(w.resid), err=err).cpu()[0])
    assert abs(ll - ref["loglik"]) <= MIXED_RTOL * abs(ref["loglik"]), (ll, ref["loglik"])
    assert float(err.cpu()[0]) <= 1e-10   # gp_loglik's default stopping residual (GP_OPT_REFINE_EXP = 10)
    # the prediction first refines alpha to 1e-12
    mu = np.zeros(w.Xtest.shape[0])
    m_ref = oracle.predict(w.hyper, w.X, ref["alpha"], w.Xtest, mu)
    m_gpu = f.predict(_dev(w.Xtest), _dev(mu)).cpu().numpy()
    assert np.abs(m_gpu - m_ref).max() <= 1e-9 * max(1.0, np.abs(m_ref).max())
    f.free()


def test_mixed_refinement_tolerance(case, ctx):
    """The mixed log-likelihood's quadratic form is second order in the refinement residual (alpha^T (2 r - C alpha)),
    so stopping at 1e-10 (the default) or at 1e-12 (GP_OPT_REFINE_EXP = 12) gives the same log-likelihood to far
    below the 1e-6 bound; the stricter setting reaches its residual."""
    from paper_2411_05869_gb300 import gp
    w, ps = case["w"], case["ps"]
    out = {}
    for e in (10, 12):
        ctx.set_option("refine_exp", e)
        try:
            f = ctx.factor(ps, [w.hyper], gp.GP_MIXED)
        finally:
            ctx.set_option("refine_exp", 10)
        err = torch.empty(1, dtype=torch.float64, device="cuda")
        out[e] = float(f.loglik(_dev(w.resid), err=err).cpu()[0])
        assert float(err.cpu()[0]) <= 10.0 ** -e
        f.free()
    assert abs(out[10] - out[12]) <= 1e-11 * abs(out[12]), out


def test_mixed_batched_each_proposal(case, ctx):
    from paper_2411_05869_gb300 import gp
    w, ps = case["w"], case["ps"]
    rng = np.random.default_rng(9)
    thetas = [synth.perturb(rng, w.hyper) for _ in range(3)]
    f = ctx.factor(ps, thetas, gp.GP_MIXED)
    ll = f.loglik(_dev(np.stack([w.resid] * 3))).cpu().numpy()
    for b, hp in enumerate(thetas):
        ref = oracle.sparse_loglik(hp, w.X, case["rp"], case["col"], case["perm"], w.resid)
        assert abs(ll[b] - ref["loglik"]) <= MIXED_RTOL * abs(ref["loglik"]), (b, ll[b], ref["loglik"])
    f.free()


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_matches_direct_launches(case, ctx, precision):
    """On an explicit stream the factor and solve launch sequences are captured once as CUDA graphs and
    replayed; results must equal the directly launched ones (default stream) bit for bit."""
    from paper_2411_05869_gb300 import gp
    w, ps = case["w"], case["ps"]
    rng = np.random.default_rng(11)
    th = [synth.perturb(rng, w.hyper) for _ in range(2)]
    r = _dev(np.stack([w.resid, 0.5 * w.resid]))
    f0 = ctx.factor(ps, th, precision)
    direct = f0.loglik(r).cpu().numpy().copy()
    s = torch.cuda.Stream()
    ctx2 = gp.Context(0, stream=s)
    with torch.cuda.stream(s):
        X2 = _dev(w.X)
        ps2 = ctx2.assemble(X2, w.hyper.core_radius)
        f2 = ctx2.factor(ps2, th, precision)      # captures and replays the factor graph
        a = f2.loglik(r).cpu().numpy().copy()     # captures and replays the solve graph(s)
        f2.update(th)                             # replays
        b = f2.loglik(r).cpu().numpy().copy()
    s.synchronize()
    assert a.tobytes() == direct.tobytes() and b.tobytes() == direct.tobytes()
    f2.free()
    f0.free()


def test_every_update_blocking_and_the_autotuner_match_oracle(ctx):
    """The mixed path's update blocking (G blocks of 64 columns per deferred group, 128 x TN group tiles) only
    reorders FP32 sums: every blocking, and the autotuner's choice, must give the oracle's log-likelihood to
    1e-6. Fronts here span many 64-column blocks, so the left-looking and group-end updates all occur."""
    from paper_2411_05869_gb300 import gp
    w = synth.uniform_spacetime(20000, 0, 60.0, 8, seed=79, ndays=120)
    hp = w.hyper
    rp, col = oracle.pattern(w.X, hp.core_radius)
    perm = oracle.fill_order(w.X, hp.core_radius, rp, col)
    ref = oracle.sparse_loglik(hp, w.X, rp, col, perm, w.resid)["loglik"]
    ps = ctx.assemble(_dev(w.X), hp.core_radius)
    assert ps.info()["max_front"] > 8 * 64
    r = _dev(w.resid)
    split0 = ctx.get_option("split_f16")
    for G in (1, 4, 8, 16, 32):
        for TN in (128, 256):
            ps.set_blocking(G, TN)
            for split in (0, 1):   # TF32 and FP16 operand pairs
                ctx.set_option("split_f16", split)
                try:
                    f = ctx.factor(ps, [hp], gp.GP_MIXED)
                finally:
                    ctx.set_option("split_f16", split0)
                ll = float(f.loglik(r).cpu()[0])
                f.free()
                assert abs(ll - ref) <= MIXED_RTOL * abs(ref), (G, TN, split, ll, ref)
    tried = ps.autotune([hp], reps=1)
    assert len(tried) == 7 and all(t["ms"] > 0 for t in tried)
    f = ctx.factor(ps, [hp], gp.GP_MIXED)
    ll = float(f.loglik(r).cpu()[0])
    assert abs(ll - ref) <= MIXED_RTOL * abs(ref), (ll, ref)
    with pytest.raises(gp.GpError):   # the schedule of live factors is not re-planned under them
        ps.autotune([hp], reps=1)
    f.free()
    ps.free()


@pytest.mark.parametrize("c", [1e-9, 1e9])
def test_mixed_f16_pairs_scale_with_the_covariance(ctx, c):
    """The FP16 operand pairs take a power-of-two scale from max_i C_ii: with C_z and r multiplied by c and
    sqrt(c) (core and noise variances times c), every L entry moves by sqrt(c), far outside FP16's range for
    c = 1e9 and below its normal range for c = 1e-9 without the scale. The log-likelihood must still match the
    oracle's on the scaled problem within 1e-6, on fronts wide enough for every update mode."""
    from paper_2411_05869_gb300 import gp
    w = synth.uniform_spacetime(8000, 0, 60.0, 8, seed=83, ndays=80)
    hp = copy.deepcopy(w.hyper)
    hp.core_var *= c
    hp.noise_var *= c
    r = w.resid * math.sqrt(c)
    rp, col = oracle.pattern(w.X, hp.core_radius)
    perm = oracle.fill_order(w.X, hp.core_radius, rp, col)
    ref = oracle.sparse_loglik(hp, w.X, rp, col, perm, r)["loglik"]
    ps = ctx.assemble(_dev(w.X), hp.core_radius)
    assert ps.info()["max_front"] > 4 * 64
    split0 = ctx.get_option("split_f16")
    ctx.set_option("split_f16", 1)
    try:
        f = ctx.factor(ps, [hp], gp.GP_MIXED)
    finally:
        ctx.set_option("split_f16", split0)
    ll = float(f.loglik(_dev(r)).cpu()[0])
    assert abs(ll - ref) <= MIXED_RTOL * abs(ref), (c, ll, ref)
    f.free()
    ps.free()


def test_left_updates_beside_the_potrf_match_one_launch(ctx):
    """On an explicit stream the mixed factorization runs the left-looking update of a block step in two launches
    (the rows of the step's diagonal tiles first, the rows below on a second stream beside the step's POTRF); on
    the legacy default stream it is one launch. Every tile computes the same sums either way, so the
    log-likelihoods must agree bit for bit, for both operand splits, on fronts wide enough for left updates at
    every level of the chain."""
    from paper_2411_05869_gb300 import gp
    w = synth.uniform_spacetime(20000, 0, 60.0, 8, seed=79, ndays=120)
    hp = w.hyper
    rng = np.random.default_rng(13)
    th = [synth.perturb(rng, hp) for _ in range(2)]
    r = np.stack([w.resid, 0.5 * w.resid])
    s = torch.cuda.Stream()
    ctx2 = gp.Context(0, stream=s)
    ps = ctx.assemble(_dev(w.X), hp.core_radius)
    with torch.cuda.stream(s):
        ps2 = ctx2.assemble(_dev(w.X), hp.core_radius)
    s.synchronize()
    assert ps.info()["max_front"] > 8 * 64
    split0 = ctx.get_option("split_f16")
    for split in (1, 0):
        ctx.set_option("split_f16", split)
        ctx2.set_option("split_f16", split)
        try:
            f = ctx.factor(ps, th, gp.GP_MIXED)
            a = f.loglik(_dev(r)).cpu().numpy().copy()
            with torch.cuda.stream(s):
                f2 = ctx2.factor(ps2, th, gp.GP_MIXED)
                b = f2.loglik(_dev(r)).cpu().numpy().copy()
            s.synchronize()
        finally:
            ctx.set_option("split_f16", split0)
            ctx2.set_option("split_f16", split0)
        assert a.tobytes() == b.tobytes(), (split, a, b)
        f.free()
        f2.free()
    ps.free()
    ps2.free()
