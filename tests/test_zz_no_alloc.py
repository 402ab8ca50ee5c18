"""gp_pattern_counts_noalloc: the support-pattern row counts for callers that must not allocate device memory.

It must give the same counts as the pattern gp_assemble builds (integers: bit for bit), on two calls in a row
(the static scratch array is shared and reused), and refuse sizes beyond its fixed limits. This file is
collected last on purpose, and also runs alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2411_05869_gb300 import gp, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    L = gp.load()
    f = L.gp_pattern_counts_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                  ctypes.c_void_p]
    return f


def _counts_noalloc(ctx, X, rho):
    fn = _lib()
    Xd = torch.as_tensor(np.ascontiguousarray(X), dtype=torch.float64, device="cuda")
    out = torch.full((X.shape[0],), -1, dtype=torch.int64, device="cuda")
    r = np.ascontiguousarray(rho, dtype=np.float64)
    st = fn(ctx.h, Xd.data_ptr(), X.shape[0], X.shape[1], r.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            out.data_ptr())
    torch.cuda.synchronize()
    return st, out.cpu().numpy()


@pytest.mark.parametrize("kind", ["spatial", "spacetime"])
def test_noalloc_counts_match_assembled_pattern_twice(kind):
    ctx = gp.Context(0)
    if kind == "spatial":
        w = synth.spatial_2d(n=3000, m=1, seed=41)
    else:
        w = synth.uniform_spacetime(5000, 1, 40.0, 8, seed=42, ndays=50)
    rho = w.hyper.core_radius
    ps = ctx.assemble(torch.as_tensor(w.X, dtype=torch.float64, device="cuda"), rho)
    ref = np.diff(ps.export("rowptr"))
    for _ in range(2):
        st, cnt = _counts_noalloc(ctx, w.X, rho)
        assert st == 0, ctx.lib.gp_last_error(ctx.h)
        assert np.array_equal(cnt, ref)
    # a different, smaller input in between leaves no trace in the next call
    st, small = _counts_noalloc(ctx, w.X[:700], rho)
    assert st == 0
    ps_small = ctx.assemble(torch.as_tensor(w.X[:700], dtype=torch.float64, device="cuda"), rho)
    assert np.array_equal(small, np.diff(ps_small.export("rowptr")))
    st, cnt = _counts_noalloc(ctx, w.X, rho)
    assert st == 0 and np.array_equal(cnt, ref)


def test_noalloc_rejects_sizes_beyond_its_limits():
    ctx = gp.Context(0)
    X = np.random.default_rng(3).uniform(0, 1, (65537, 2))
    st, _ = _counts_noalloc(ctx, X, np.array([0.05, 0.05]))
    assert st == 1   # GP_ERR_ARG: n above 65536
    X = np.random.default_rng(4).uniform(0, 1, (1000, 3))
    st, _ = _counts_noalloc(ctx, X, np.array([1e-3, 1e-3, 1e-3]))
    assert st == 1   # GP_ERR_ARG: more than 2^20 cells
