"""Step A6 of the library on the host (gp_symbolic_host): the symbolic analysis gp_assemble runs on the device
pattern, here from a host pattern with no device call. It must match the oracle's independent analysis bit for
bit: the postorder relabelling of the elimination tree, the etree, the exact column counts, the relaxed
supernodes, their row structures, parents and levels. The oracle itself is pinned against brute-force elimination
(test_oracle_structure.py). Malformed inputs must be refused with GP_ERR_ARG.
"""
import numpy as np
import pytest

import oracle
from paper_2411_05869_gb300 import gp, synth

GP_ERR_ARG = 1


def _workloads():
    return {
        "spatial_2d_n2000": lambda: synth.spatial_2d(n=2000, m=300, seed=synth.SEED_BASE + 1),
        "spacetime_n6000": lambda: synth.uniform_spacetime(6000, 400, 40.0, 8, seed=77, ndays=60),
        "station_600x20": lambda: synth.station_spacetime(nsites=600, ndays=20, ncomp=10, nnz_row=60.0, grid=12,
                                                          grid_days=3, seed=78, nbumps=16),
        "uniform_3d_n1500": lambda: synth.uniform_spacetime(1500, 100, 25.0, 4, seed=5, ndays=30),
    }


@pytest.fixture(scope="module", params=list(_workloads().keys()))
def case(request):
    w = _workloads()[request.param]()
    rp, col = oracle.pattern(w.X, w.hyper.core_radius)
    nd = oracle.nd_order(w.X, w.hyper.core_radius, rp, col)
    return rp, col, nd


def test_host_symbolic_matches_oracle(case):
    rp, col, nd = case
    got = gp.symbolic_host(rp, col, nd)
    perm = oracle.etree_postorder(rp, col, nd)
    ref = oracle.symbolic(rp, col, perm)
    assert np.array_equal(got["perm"], perm)
    for name in ["parent", "eta", "sn_first", "sn_rowptr", "sn_rows", "sn_parent", "sn_level"]:
        assert np.array_equal(got[name], ref[name]), name
    assert got["nnzL"] == ref["nnzL"] == int(ref["eta"].astype(np.int64).sum())
    assert got["nsuper"] == ref["sn_first"].shape[0] - 1
    assert got["nnz"] == rp[-1]
    # sum_j eta_j^2, the algorithmic flop count of the factorization
    assert got["flops"] == pytest.approx(float((ref["eta"].astype(np.float64) ** 2).sum()), rel=1e-12)


def test_host_symbolic_single_point_and_diagonal_pattern():
    got = gp.symbolic_host(np.array([0, 1]), np.array([0]), np.array([0]))
    assert got["nsuper"] == 1 and got["nnzL"] == 1 and list(got["parent"]) == [-1]
    n = 40   # no coupling: a forest of single columns, each column count 1
    rp = np.arange(n + 1, dtype=np.int64)
    col = np.arange(n, dtype=np.int32)
    nd = np.random.default_rng(3).permutation(n).astype(np.int32)
    got = gp.symbolic_host(rp, col, nd)
    perm = oracle.etree_postorder(rp, col, nd)
    ref = oracle.symbolic(rp, col, perm)
    assert got["nnzL"] == n and np.all(got["eta"] == 1) and np.all(got["parent"] == -1)
    for name in ["perm", "sn_first", "sn_parent", "sn_level"]:
        want = perm if name == "perm" else ref[name]
        assert np.array_equal(got[name], want), name


def _malformed():
    rp = np.array([0, 2, 4], dtype=np.int64)
    col = np.array([0, 1, 0, 1], dtype=np.int32)
    nd = np.array([1, 0], dtype=np.int32)
    yield "ok", rp, col, nd
    yield "missing diagonal", rp, np.array([0, 1, 0, 0], dtype=np.int32), nd
    yield "column out of range", rp, np.array([0, 2, 0, 1], dtype=np.int32), nd
    yield "columns not ascending", rp, np.array([1, 0, 0, 1], dtype=np.int32), nd
    yield "not a permutation", rp, col, np.array([1, 1], dtype=np.int32)
    yield "decreasing rowptr", np.array([0, 3, 2], dtype=np.int64), np.array([0, 1, 1], dtype=np.int32), nd


@pytest.mark.parametrize("what,rp,col,nd", list(_malformed()))
def test_host_symbolic_refuses_malformed_input(what, rp, col, nd):
    if what == "ok":
        got = gp.symbolic_host(rp, col, nd)
        assert got["nnzL"] == 3
        return
    with pytest.raises(gp.GpError) as e:
        gp.symbolic_host(rp, col, nd)
    assert e.value.status == GP_ERR_ARG, what
