"""Pins of the oracle's structural outputs: support pattern, nested-dissection order and symbolic analysis.

Pattern: a k-d tree range search (scipy, a library routine with its own distance arithmetic) brackets the
brute-force pattern, and lattice inputs give exact counts (integer points in a ball) within Prop. 4's bound.
Ordering: the rule is the build's (the paper is silent); it is pinned by its defining properties.
Symbolic: etree and column counts against a brute-force boolean dense elimination.
"""
import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
from paper_2411_05869_gb300 import synth


def _pattern_sets(rowptr, col):
    return [set(col[rowptr[i]:rowptr[i + 1]].tolist()) for i in range(rowptr.shape[0] - 1)]


@pytest.mark.parametrize("d,n,seed", [(2, 800, 1), (3, 900, 2)])
def test_pattern_brackets_kdtree(d, n, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, (n, d))
    rho = np.array([0.11, 0.07, 0.2][:d])
    rp, col = oracle.pattern(X, rho)
    assert np.all(np.diff(rp) >= 1)
    for i in range(n):
        row = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(row) > 0) and i in row
    sets = _pattern_sets(rp, col)
    t = cKDTree(X / rho)
    inner = t.query_pairs(1.0 - 1e-9)
    outer = t.query_pairs(1.0 + 1e-9)
    for (a, b) in inner:
        assert b in sets[a] and a in sets[b]
    outer_sets = [set() for _ in range(n)]
    for (a, b) in outer:
        outer_sets[a].add(b)
        outer_sets[b].add(a)
    for i in range(n):
        assert sets[i] - {i} <= outer_sets[i]
    # symmetric
    for i in range(n):
        for j in sets[i]:
            assert i in sets[j]


@pytest.mark.parametrize("d,rho,count", [(2, 2.5, 21), (3, 1.5, 19), (1, 3.5, 7)])
def test_pattern_lattice_counts_and_prop4_bound(d, rho, count):
    """Unit lattice: interior rows hold #{v in Z^d : |v|^2 < rho^2}; Prop. 4 bounds rows by (4 r / delta + 1)^d."""
    side = {1: 40, 2: 15, 3: 9}[d]
    g = np.stack(np.meshgrid(*[np.arange(side)] * d, indexing="ij"), -1).reshape(-1, d).astype(float)
    rp, col = oracle.pattern(g, np.full(d, rho))
    cnt = np.diff(rp)
    interior = np.all((g >= np.ceil(rho)) & (g <= side - 1 - np.ceil(rho)), axis=1)
    ball = sum(1 for v in np.ndindex(*[int(2 * np.ceil(rho) + 1)] * d)
               if sum((np.array(v) - np.ceil(rho)) ** 2) < rho * rho)
    assert ball == count
    assert np.all(cnt[interior] == count)
    assert cnt.max() <= (4 * rho / 1.0 + 1) ** d


def _nd_reference(U, key, rows, verts):
    """The ordering rule restated with Python lists, for tiny inputs."""
    if len(verts) == 0:
        return []
    if len(verts) <= 64:
        return sorted(verts, key=lambda v: (key[v], v))
    d = U.shape[1]
    ext = [max(U[v, k] for v in verts) - min(U[v, k] for v in verts) for k in range(d)]
    k = max(range(d), key=lambda kk: (ext[kk], -kk))
    s = sorted(verts, key=lambda v: (U[v, k], v))
    L, R = s[:len(s) // 2], s[len(s) // 2:]
    Rset = set(R)
    S = [v for v in L if any(w in Rset for w in rows[v])]
    Sset = set(S)
    Lrest = [v for v in L if v not in Sset]
    return _nd_reference(U, key, rows, Lrest) + _nd_reference(U, key, rows, R) + S


@pytest.mark.parametrize("d,n,seed", [(2, 700, 3), (3, 900, 4)])
def test_nd_order_rule(d, n, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, (n, d))
    if d == 3:
        X[:, 2] = rng.integers(0, 30, n) / 29.0         # many ties along time, as in daily data
    rho = np.array([0.12, 0.12, 0.08][:d])
    rp, col = oracle.pattern(X, rho)
    perm, lo, hi, kind = oracle.nd_order(X, rho, rp, col, with_tree=True)
    assert np.array_equal(np.sort(perm), np.arange(n))
    rows = [col[rp[i]:rp[i + 1]].tolist() for i in range(n)]
    ref = _nd_reference(X / rho, oracle.cell_keys(X, rho), rows, list(range(n)))
    assert perm.tolist() == ref
    assert np.all((hi - lo)[kind == 0] <= 64)
    assert (hi - lo).sum() == n


def test_cell_keys_grid():
    X = np.array([[0.0, 0.0], [0.99, 0.0], [1.0, 0.0], [0.0, 2.5], [3.2, 1.1]])
    key = oracle.cell_keys(X, np.array([1.0, 1.0]))
    # nc_0 = 4 (cells 0..3 along x): key = c_0 + 4 c_1
    assert key.tolist() == [0, 0, 1, 8, 3 + 4]


def _boolean_elimination(M):
    M = M.copy()
    n = M.shape[0]
    for k in range(n):
        nz = np.nonzero(M[k + 1:, k])[0] + k + 1
        M[np.ix_(nz, nz)] = True
    return np.tril(M)


@pytest.mark.parametrize("d,n,seed", [(2, 180, 5), (3, 200, 6)])
def test_symbolic_against_boolean_elimination(d, n, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, (n, d))
    rho = np.array([0.2, 0.2, 0.25][:d])
    rp, col = oracle.pattern(X, rho)
    perm = oracle.nd_order(X, rho, rp, col)
    pinv = np.empty(n, int); pinv[perm] = np.arange(n)
    M = np.zeros((n, n), bool)
    for i in range(n):
        M[pinv[i], pinv[col[rp[i]:rp[i + 1]]]] = True
    Lb = _boolean_elimination(M)
    s = oracle.symbolic(rp, col, perm)
    eta = Lb.sum(0)
    parent = np.array([(np.nonzero(Lb[j + 1:, j])[0][0] + j + 1) if Lb[j + 1:, j].any() else -1 for j in range(n)])
    assert np.array_equal(s["eta"], eta)
    assert np.array_equal(s["parent"], parent)
    assert s["nnzL"] == Lb.sum()
    # supernodes: contiguous partition; each supernode's rows = structure of its last column
    snf = s["sn_first"]
    assert snf[0] == 0 and snf[-1] == n and np.all(np.diff(snf) > 0)
    for k in range(len(snf) - 1):
        f, l = snf[k], snf[k + 1] - 1
        rows = s["sn_rows"][s["sn_rowptr"][k]:s["sn_rowptr"][k + 1]]
        assert rows.tolist() == (np.nonzero(Lb[l + 1:, l])[0] + l + 1).tolist()
        for j in range(f, l + 1):           # every column's structure fits in the panel
            below = set((np.nonzero(Lb[l + 1:, j])[0] + l + 1).tolist())
            assert below <= set(rows.tolist())


def test_fundamental_supernodes_and_relaxation_rule():
    """Fundamental rule on a hand-built etree, then relaxation by width <= 16."""
    # chain 0->1->2->3 with eta 4,3,2,1 is one fundamental supernode; node 4 alone (root of its own tree)
    parent = np.array([1, 2, 3, -1, -1], np.int32)
    eta = np.array([4, 3, 2, 1, 1], np.int32)
    assert oracle.supernodes(parent, eta).tolist() == [0, 4, 5]
    # two leaves 0, 1 under 2: 1 -> 2 is contiguous, merged by width; 0 ends at 0 and next supernode starts at 1
    parent = np.array([2, 2, -1], np.int32)
    eta = np.array([2, 2, 1], np.int32)
    snf = oracle.supernodes(parent, eta)
    assert snf.tolist() == [0, 3]           # 1 merges into 2 (width 2), then 0 merges into {1,2} (width 3)


def test_symbolic_levels_and_parents_consistent():
    w = synth.spatial_2d(n=1500, m=10, seed=11)
    rp, col = oracle.pattern(w.X, w.hyper.core_radius)
    perm = oracle.nd_order(w.X, w.hyper.core_radius, rp, col)
    s = oracle.symbolic(rp, col, perm)
    sp, lev = s["sn_parent"], s["sn_level"]
    ns = len(sp)
    for k in range(ns):
        if sp[k] >= 0:
            assert sp[k] > k and lev[sp[k]] > lev[k]
    assert (np.diff(s["sn_rowptr"]) == s["eta"][s["sn_first"][1:] - 1] - 1).all()


# ------------------------------------------------------------------ etree postorder relabelling (fill_order)

def _elimination_tree(rp, col, perm):
    """Boolean dense elimination of P C P^T (tiny n): the lower pattern of L, its etree and its column counts."""
    n = perm.shape[0]
    pinv = np.empty(n, int)
    pinv[perm] = np.arange(n)
    M = np.zeros((n, n), bool)
    for i in range(n):
        M[pinv[i], pinv[col[rp[i]:rp[i + 1]]]] = True
    Lb = _boolean_elimination(M)
    parent = np.array([(np.nonzero(Lb[j + 1:, j])[0][0] + j + 1) if Lb[j + 1:, j].any() else -1 for j in range(n)])
    return Lb, parent, Lb.sum(0)


@pytest.mark.parametrize("d,n,seed", [(2, 220, 8), (3, 240, 9)])
def test_etree_postorder_keeps_fill_and_makes_subtrees_contiguous(d, n, seed):
    """The relabelling of the nested-dissection order by a postorder of its elimination tree (the build's rule;
    the paper is silent) must (i) be a permutation, (ii) keep the fill: the same nnz(L) and the same multiset of
    column counts as the order it relabels, (iii) make every subtree a contiguous range of columns ending at its
    root, and (iv) visit children in increasing index order and roots in increasing order. Each property is
    checked on the etree of a brute-force boolean elimination, not on the oracle's own analysis."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, (n, d))
    rho = np.array([0.2, 0.2, 0.25][:d])
    rp, col = oracle.pattern(X, rho)
    nd = oracle.nd_order(X, rho, rp, col)
    po = oracle.fill_order(X, rho, rp, col)
    assert np.array_equal(np.sort(po), np.arange(n))
    Lnd, par_nd, eta_nd = _elimination_tree(rp, col, nd)
    Lpo, par_po, eta_po = _elimination_tree(rp, col, po)
    assert Lpo.sum() == Lnd.sum()
    assert np.array_equal(np.sort(eta_po), np.sort(eta_nd))
    # subtree sizes from the relabelled etree: children precede parents
    size = np.ones(n, int)
    for j in range(n):
        if par_po[j] >= 0:
            assert par_po[j] > j
            size[par_po[j]] += size[j]
    for j in range(n):   # descendants of j are exactly the columns j - size_j + 1 .. j
        k, anc = j - size[j] + 1, True
        for c in range(k, j):
            p = c
            while p >= 0 and p != j:
                p = par_po[p]
            anc = anc and p == j
        assert anc, j
    # the same tree: relabelled node new = old position post[new] in the nd order, with the edges preserved
    pos_nd = np.empty(n, int)
    pos_nd[nd] = np.arange(n)
    post = pos_nd[po]               # new label -> nd label
    for j in range(n):
        pj = par_po[j]
        assert (par_nd[post[j]] == -1) if pj < 0 else (par_nd[post[j]] == post[pj])
    # the traversal rule, restated as a recursive walk over the nd etree (tiny n)
    kids = [[] for _ in range(n)]
    for v in range(n):
        if par_nd[v] >= 0:
            kids[par_nd[v]].append(v)
    walk = []

    def visit(v):
        for c in sorted(kids[v]):
            visit(c)
        walk.append(v)

    import sys
    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 4 * n))
    try:
        for v in range(n):
            if par_nd[v] < 0:
                visit(v)
    finally:
        sys.setrecursionlimit(old)
    assert post.tolist() == walk


@pytest.mark.parametrize("d,n,seed", [(2, 190, 10), (3, 210, 11)])
def test_symbolic_on_fill_order_against_boolean_elimination(d, n, seed):
    """The symbolic analysis of the relabelled (factorization) order against a boolean dense elimination."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, (n, d))
    rho = np.array([0.2, 0.2, 0.25][:d])
    rp, col = oracle.pattern(X, rho)
    perm = oracle.fill_order(X, rho, rp, col)
    Lb, parent, eta = _elimination_tree(rp, col, perm)
    s = oracle.symbolic(rp, col, perm)
    assert np.array_equal(s["eta"], eta)
    assert np.array_equal(s["parent"], parent)
    assert s["nnzL"] == Lb.sum()
    snf = s["sn_first"]
    for k in range(len(snf) - 1):
        f, l = snf[k], snf[k + 1] - 1
        rows = s["sn_rows"][s["sn_rowptr"][k]:s["sn_rowptr"][k + 1]]
        assert rows.tolist() == (np.nonzero(Lb[l + 1:, l])[0] + l + 1).tolist()
        # a (relaxed) supernode is a contiguous piece of the tree rooted at its last column
        assert np.all((parent[f:l] > np.arange(f, l)) & (parent[f:l] <= l)), "supernode columns must hang off its last"


# ------------------------------------------------------------------ relaxed amalgamation: the explicit-zeros branch

def _two_chain_etree(a, b, k, r):
    """Columns 0..a-1 (child chain c) then a..a+b-1 (parent chain p), one path, p's last column with r rows below.
    Within each chain eta drops by one per column (fundamental supernodes); between them column a-1 has k fewer
    rows than a fundamental merge would need, so merging c into p stores a * k explicit zeros."""
    n = a + b
    parent = np.arange(1, n + 1, dtype=np.int32)
    parent[-1] = -1
    eta = np.empty(n, np.int32)
    for j in range(a, n):
        eta[j] = r + 1 + (n - 1 - j)
    for j in range(a):
        eta[j] = eta[a] + 1 - k + (a - 1 - j)
    return parent, eta


def _merged_panel(a, b, r):
    w = a + b
    return w * (w + 1) // 2 + w * r


def test_relaxation_explicit_zeros_branch_at_exactly_ten_percent():
    """A merge wider than 16 columns is taken iff the merged panel holds at most 10 % explicit zeros: the
    boundary case (zeros = 10 % of the panel's entries exactly) merges, one more zero row per column does not."""
    found = None
    for a in range(2, 30):
        for b in range(2, 30):
            if a + b <= 16:
                continue
            for r in range(0, 60):
                ent = _merged_panel(a, b, r)
                if ent % (10 * a) == 0:
                    k = ent // (10 * a)
                    if 1 <= k <= r + b - 1:
                        found = (a, b, k, r)
                        break
            if found:
                break
        if found:
            break
    assert found is not None
    a, b, k, r = found
    parent, eta = _two_chain_etree(a, b, k, r)
    # the panel bookkeeping: explicit zeros = entries - sum of the exact column counts = a * k
    assert _merged_panel(a, b, r) - int(eta.sum()) == a * k
    assert 10 * a * k == _merged_panel(a, b, r)
    # without relaxation these are two fundamental supernodes
    assert oracle.supernodes(parent, eta).tolist() == [0, a + b]
    parent2, eta2 = _two_chain_etree(a, b, k + 1, r)
    assert oracle.supernodes(parent2, eta2).tolist() == [0, a, a + b]
    # and width alone decides at or below 16 columns, whatever the zeros
    a3, b3 = 8, 8
    parent3, eta3 = _two_chain_etree(a3, b3, b3 + 5, 5)
    assert oracle.supernodes(parent3, eta3).tolist() == [0, a3 + b3]
