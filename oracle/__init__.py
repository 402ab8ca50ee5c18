"""The oracle: plain FP64 CPU reference for the exact sparse GP (arXiv 2411.05869). TEST INFRASTRUCTURE ONLY.

Only the tests, the package smoke check and the benchmark's CPU-baseline / reference leg import this module.
It wraps ``gp_oracle.c`` (compiled with gcc, -ffp-contract=off) through ctypes and numpy, shares no code with
the CUDA library, and is never called by the product path.

Every function names the passage it follows; see gp_oracle.c for the arithmetic. Parity of the structural
outputs (pattern, ordering, symbolic analysis) is pinned by the tests in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libgp_oracle.so")
_lib = None

c_i64 = ctypes.c_int64
c_dbl = ctypes.c_double
P = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no vectorisation assumptions, no FMA contraction). The brute-force
    pattern's independent rows run on OpenMP threads when gcc has OpenMP (same results); otherwise serially."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
        try:
            subprocess.check_call(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        L.or_wendland.restype = c_dbl
        L.or_wendland.argtypes = [c_dbl]
        L.or_bump.restype = c_dbl
        L.or_bump.argtypes = [P, ctypes.c_int, P, c_dbl, c_dbl, c_dbl]
        L.or_csparse.restype = c_dbl
        L.or_csparse.argtypes = [P, P, P, P]
        L.or_cy.restype = c_dbl
        L.or_cy.argtypes = [P, P, P, P]
        L.or_features.argtypes = [c_i64, P, P, P, P]
        L.or_dense_cov.argtypes = [c_i64, P, P, P, ctypes.c_int, P]
        L.or_pattern_count.restype = c_i64
        L.or_pattern_count.argtypes = [c_i64, ctypes.c_int, P, P, P]
        L.or_pattern_fill.argtypes = [c_i64, ctypes.c_int, P, P, P, P]
        L.or_pattern_row.restype = c_i64
        L.or_pattern_row.argtypes = [c_i64, ctypes.c_int, P, P, c_i64, P, c_i64]
        L.or_cell_keys.argtypes = [c_i64, ctypes.c_int, P, P, P]
        L.or_nd_order.restype = c_i64
        L.or_nd_order.argtypes = [c_i64, ctypes.c_int, P, P, P, P, P, P, P, P]
        L.or_etree_postorder.argtypes = [c_i64, P, P, P, P]
        L.or_supernodes.restype = c_i64
        L.or_supernodes.argtypes = [c_i64, P, P, P]
        L.or_symbolic.restype = c_i64
        L.or_symbolic.argtypes = [c_i64, P, P, P, P, P, P, P, P, c_i64, P, P, P]
        L.or_dense_chol.restype = c_i64
        L.or_dense_chol.argtypes = [c_i64, P]
        L.or_dense_loglik.restype = c_i64
        L.or_dense_loglik.argtypes = [c_i64, P, P, P, P, P, P]
        L.or_sample_dense.restype = c_i64
        L.or_sample_dense.argtypes = [c_i64, P, P, P, P, P]
        L.or_sparse_loglik.restype = c_i64
        L.or_sparse_loglik.argtypes = [c_i64, P, P, P, P, P, P, P, P, P, P]
        L.or_sparse_factor.restype = c_i64
        L.or_sparse_factor.argtypes = [c_i64, P, P, P, P, P, P, P, P, P, c_i64]
        L.or_predict.argtypes = [c_i64, c_i64, P, P, P, P, P, P, P]
        L.or_csr_values.argtypes = [c_i64, P, P, P, P, P, P]
        L.or_pattern_count_sparse.restype = c_i64
        L.or_pattern_count_sparse.argtypes = [c_i64, P, P, P, P]
        L.or_pattern_fill_sparse.argtypes = [c_i64, P, P, P, P, P]
        _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(P)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def theta_block(hp):
    """(dims int32[5], theta float64[]) in the oracle's layout from a synth.Hyper."""
    kind = int(getattr(hp, "core_kind", 0))
    dims = np.array([hp.d, hp.n1, hp.n2, hp.bump_dims, kind], dtype=np.int32)
    parts = [[hp.core_var], hp.core_radius, [hp.s0], hp.r0, [hp.noise_var], hp.h, hp.a, hp.b, hp.r]
    if kind == 1:
        parts += [[hp.sigma0, hp.Sigma0], hp.phi_sigma, hp.phi_Sigma]
    th = np.concatenate(parts).astype(np.float64)
    return dims, th


# ------------------------------------------------------------------ kernel pieces (Sec. 2.1)

def wendland(q: float) -> float:
    """f0 as a function of q = |x-x'|/r0 (Eq. compSupp, cubic coefficient 35 as printed)."""
    return lib().or_wendland(float(q))


def bump(x, h, a, b, r) -> float:
    """g(x) of Eq. bumpFcn."""
    x = _f64(x); h = _f64(h)
    return lib().or_bump(_p(x), int(h.shape[0]), _p(h), float(a), float(b), float(r))


def features(hp, X) -> np.ndarray:
    """F[k, i] = f_i(x_k) = sum_j g_ij(x_k)."""
    X = _f64(X)
    dims, th = theta_block(hp)
    F = np.zeros((X.shape[0], max(hp.n1, 1)))
    lib().or_features(X.shape[0], _p(dims), _p(th), _p(X), _p(F))
    return F[:, :hp.n1]


def csparse(hp, x, y) -> float:
    dims, th = theta_block(hp)
    return lib().or_csparse(_p(dims), _p(th), _p(_f64(x)), _p(_f64(y)))


def cy(hp, x, y) -> float:
    dims, th = theta_block(hp)
    return lib().or_cy(_p(dims), _p(th), _p(_f64(x)), _p(_f64(y)))


def dense_cov(hp, X, noise: bool = True) -> np.ndarray:
    """C_z (noise=True) or C_y over all pairs (Eq. Zcov)."""
    X = _f64(X)
    n = X.shape[0]
    dims, th = theta_block(hp)
    C = np.empty((n, n))
    lib().or_dense_cov(n, _p(dims), _p(th), _p(X), int(noise), _p(C))
    return C


# ------------------------------------------------------------------ pattern and ordering

def pattern(X, rho):
    """Full symmetric support pattern by brute force: (rowptr int64[n+1], col int32[nnz]), columns ascending."""
    X = _f64(X); rho = _f64(rho)
    n, d = X.shape
    cnt = np.zeros(n, dtype=np.int64)
    lib().or_pattern_count(n, d, _p(X), _p(rho), _p(cnt))
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt, out=rowptr[1:])
    col = np.empty(int(rowptr[-1]), dtype=np.int32)
    lib().or_pattern_fill(n, d, _p(X), _p(rho), _p(rowptr), _p(col))
    return rowptr, col


def pattern_sparse(hp, X):
    """The support of C_sparse by brute force (the pattern with the non-compact core of App. B): pairs with q0 < 1
    for the radii r0, or both inside one bump family's support. (rowptr int64[n+1], col int32[nnz])."""
    X = _f64(X)
    n = X.shape[0]
    dims, th = theta_block(hp)
    cnt = np.zeros(n, dtype=np.int64)
    lib().or_pattern_count_sparse(n, _p(dims), _p(th), _p(X), _p(cnt))
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt, out=rowptr[1:])
    col = np.empty(int(rowptr[-1]), dtype=np.int32)
    lib().or_pattern_fill_sparse(n, _p(dims), _p(th), _p(X), _p(rowptr), _p(col))
    return rowptr, col


def pattern_row(X, rho, i: int) -> np.ndarray:
    X = _f64(X); rho = _f64(rho)
    n, d = X.shape
    out = np.empty(4096, dtype=np.int32)
    c = lib().or_pattern_row(n, d, _p(X), _p(rho), int(i), _p(out), out.shape[0])
    if c > out.shape[0]:
        out = np.empty(c, dtype=np.int32)
        lib().or_pattern_row(n, d, _p(X), _p(rho), int(i), _p(out), out.shape[0])
    return out[:c].copy()


def cell_keys(X, rho) -> np.ndarray:
    X = _f64(X); rho = _f64(rho)
    key = np.empty(X.shape[0], dtype=np.int64)
    lib().or_cell_keys(X.shape[0], X.shape[1], _p(X), _p(rho), _p(key))
    return key


def nd_order(X, rho, rowptr, col, with_tree: bool = False):
    """Nested-dissection order perm[new] = old (the build's geometric rule; the paper is silent)."""
    X = _f64(X); rho = _f64(rho)
    n, d = X.shape
    perm = np.empty(n, dtype=np.int32)
    lo = np.empty(max(n, 1), dtype=np.int32); hi = np.empty_like(lo); kind = np.empty_like(lo)
    nn = lib().or_nd_order(n, d, _p(X), _p(rho), _p(rowptr.astype(np.int64)), _p(col.astype(np.int32)),
                           _p(perm), _p(lo), _p(hi), _p(kind))
    if with_tree:
        return perm, lo[:nn].copy(), hi[:nn].copy(), kind[:nn].copy()
    return perm


def etree_postorder(rowptr, col, perm) -> np.ndarray:
    """Relabel an ordering by a postorder of its elimination tree (same fill, subtrees contiguous)."""
    n = perm.shape[0]
    out = np.empty(n, dtype=np.int32)
    lib().or_etree_postorder(n, _p(np.ascontiguousarray(rowptr, np.int64)), _p(np.ascontiguousarray(col, np.int32)),
                             _p(np.ascontiguousarray(perm, np.int32)), _p(out))
    return out


def fill_order(X, rho, rowptr, col) -> np.ndarray:
    """The factorization order: nested dissection, then the etree postorder relabelling."""
    return etree_postorder(rowptr, col, nd_order(X, rho, rowptr, col))


def symbolic(rowptr, col, perm, want_rows: bool = True):
    """etree, column counts, relaxed supernodes and their below-diagonal row structures of P C P^T."""
    n = perm.shape[0]
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    parent = np.empty(n, dtype=np.int32); eta = np.empty(n, dtype=np.int32)
    snf = np.empty(n + 1, dtype=np.int32)
    snrp = np.empty(n + 1, dtype=np.int64)
    snpar = np.empty(n + 1, dtype=np.int32); snlev = np.empty(n + 1, dtype=np.int32)
    nnzL = np.zeros(1, dtype=np.int64)
    L = lib()
    ns = L.or_symbolic(n, _p(rowptr), _p(col), _p(perm), _p(parent), _p(eta), _p(snf), _p(snrp), None, 0,
                       _p(snpar), _p(snlev), _p(nnzL))
    out = dict(parent=parent, eta=eta, sn_first=snf[:ns + 1].copy(), sn_parent=snpar[:ns].copy(),
               sn_level=snlev[:ns].copy(), sn_rowptr=snrp[:ns + 1].copy(), nnzL=int(nnzL[0]))
    if want_rows:
        rows = np.empty(int(snrp[ns]), dtype=np.int32)
        L.or_symbolic(n, _p(rowptr), _p(col), _p(perm), _p(parent), _p(eta), _p(snf), _p(snrp), _p(rows),
                      rows.shape[0], None, None, None)
        out["sn_rows"] = rows
    return out


def supernodes(parent, eta) -> np.ndarray:
    n = parent.shape[0]
    snf = np.empty(n + 1, dtype=np.int32)
    ns = lib().or_supernodes(n, _p(np.ascontiguousarray(parent, np.int32)), _p(np.ascontiguousarray(eta, np.int32)),
                             _p(snf))
    return snf[:ns + 1].copy()


# ------------------------------------------------------------------ likelihood and prediction

def dense_chol(A) -> np.ndarray:
    A = np.array(A, dtype=np.float64, order="C")
    fail = lib().or_dense_chol(A.shape[0], _p(A))
    if fail >= 0:
        raise np.linalg.LinAlgError(f"not positive definite at column {fail}")
    return np.tril(A)


def dense_loglik(hp, X, resid, want_alpha: bool = False):
    """Exact log-likelihood with the full density constant (Sec. 3.3), dense Cholesky.
    Returns dict(loglik, logdet, quad[, alpha])."""
    X = _f64(X); r = _f64(resid)
    n = X.shape[0]
    dims, th = theta_block(hp)
    out = np.zeros(3)
    alpha = np.empty(n) if want_alpha else None
    fail = lib().or_dense_loglik(n, _p(dims), _p(th), _p(X), _p(r), _p(out), _p(alpha))
    if fail >= 0:
        raise np.linalg.LinAlgError(f"not positive definite at column {fail}")
    res = dict(loglik=out[0], logdet=out[1], quad=out[2])
    if want_alpha:
        res["alpha"] = alpha
    return res


def sample_dense(hp, X, normals) -> np.ndarray:
    """y = chol(C_y) o: a GP draw for small n (Sec. 3.2, unconditional simulation)."""
    X = _f64(X); o = _f64(normals)
    dims, th = theta_block(hp)
    y = np.empty(X.shape[0])
    fail = lib().or_sample_dense(X.shape[0], _p(dims), _p(th), _p(X), _p(o), _p(y))
    if fail >= 0:
        raise np.linalg.LinAlgError(f"not positive definite at column {fail}")
    return y


def sparse_loglik(hp, X, rowptr, col, perm, resid, want_alpha: bool = False, want_diag: bool = False):
    """Exact log-likelihood through the left-looking sparse Cholesky of P C_z P^T."""
    X = _f64(X); r = _f64(resid)
    n = X.shape[0]
    dims, th = theta_block(hp)
    out = np.zeros(4)
    alpha = np.empty(n) if want_alpha else None
    diag = np.empty(n) if want_diag else None
    fail = lib().or_sparse_loglik(n, _p(dims), _p(th), _p(X), _p(np.ascontiguousarray(rowptr, np.int64)),
                                  _p(np.ascontiguousarray(col, np.int32)), _p(np.ascontiguousarray(perm, np.int32)),
                                  _p(r), _p(out), _p(alpha), _p(diag))
    if fail >= 0:
        raise np.linalg.LinAlgError(f"not positive definite at permuted column {fail}")
    res = dict(loglik=out[0], logdet=out[1], quad=out[2], nnzL=int(out[3]))
    if want_alpha:
        res["alpha"] = alpha
    if want_diag:
        res["Ldiag"] = diag
    return res


def sparse_factor_dense(hp, X, rowptr, col, perm) -> np.ndarray:
    """The sparse factor L of P C_z P^T expanded to a dense n x n array (small n only)."""
    X = _f64(X)
    n = X.shape[0]
    dims, th = theta_block(hp)
    rp = np.ascontiguousarray(rowptr, np.int64); cc = np.ascontiguousarray(col, np.int32)
    pm = np.ascontiguousarray(perm, np.int32)
    cap = n * n
    ri = np.empty(cap, np.int32); ci = np.empty(cap, np.int32); v = np.empty(cap)
    nnz = lib().or_sparse_factor(n, _p(dims), _p(th), _p(X), _p(rp), _p(cc), _p(pm), _p(ri), _p(ci), _p(v), cap)
    if nnz < 0:
        raise np.linalg.LinAlgError("not positive definite")
    Ld = np.zeros((n, n))
    Ld[ri[:nnz], ci[:nnz]] = v[:nnz]
    return Ld


def predictive_variance(hp, X, Xtest) -> np.ndarray:
    """diag(C_{y|z}) at the test inputs: C_y(x*, x*) - c^T C_z^{-1} c with c = C_y(X, x*) (Sec. 3.2, the
    conditional covariance C_{y|z} = C_y - C_{y,z} C_z^{-1} C_{z,y}; no noise at the test inputs). Dense: C_y over
    the stacked training and test inputs gives the cross block and the test diagonal, and the Cholesky factor L of
    C_z turns each term into |L^{-1} c|^2. Small n only (n <= 8000)."""
    X = _f64(X); Xt = _f64(Xtest)
    n, m = X.shape[0], Xt.shape[0]
    if n > 8000:
        raise ValueError("predictive_variance is dense: n <= 8000")
    Cz = dense_cov(hp, X, noise=True)
    Ly = dense_cov(hp, np.vstack([X, Xt]), noise=False)
    cross = Ly[:n, n:]                 # n x m
    prior = np.diag(Ly[n:, n:]).copy()
    L = dense_chol(Cz)
    W = np.linalg.solve(np.tril(L), cross)   # L^{-1} C_{z,y}
    return prior - np.einsum("ij,ij->j", W, W)


def predict(hp, X, alpha, Xtest, mu_test=None) -> np.ndarray:
    """m* = mu* + C_y(X*, X) alpha with alpha = C_z^{-1} r (Sec. 3.2), brute force over training points."""
    X = _f64(X); Xt = _f64(Xtest); a = _f64(alpha)
    dims, th = theta_block(hp)
    m = Xt.shape[0]
    mean = np.empty(m)
    mu = None if mu_test is None else _f64(mu_test)
    lib().or_predict(X.shape[0], m, _p(dims), _p(th), _p(X), _p(a), _p(Xt), _p(mu), _p(mean))
    return mean


def csr_values(hp, X, rowptr, col) -> np.ndarray:
    """C_z (Eq. Zcov) at the entries of a CSR pattern, rows in index order."""
    X = _f64(X)
    dims, th = theta_block(hp)
    rp = np.ascontiguousarray(rowptr, np.int64)
    cc = np.ascontiguousarray(col, np.int32)
    val = np.empty(cc.shape[0])
    lib().or_csr_values(X.shape[0], _p(dims), _p(th), _p(X), _p(rp), _p(cc), _p(val))
    return val
