"""Thin ctypes binding of libgp.so (include/gp.h). Argument marshalling only: every step runs in the library.

PyTorch supplies device memory (CUDA tensors) and streams. The library is the only compute path; when it is
missing or cannot load, these calls raise, there is no fallback.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import weakref
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build

c_i64 = ctypes.c_int64
c_int = ctypes.c_int
c_dbl = ctypes.c_double
P = ctypes.c_void_p
DP = ctypes.POINTER(ctypes.c_double)

GP_FP64, GP_MIXED = 0, 1
STATUS = {0: "GP_OK", 1: "GP_ERR_ARG", 2: "GP_ERR_NOMEM", 3: "GP_ERR_NOT_PD", 4: "GP_ERR_CUDA",
          5: "GP_ERR_TIMEOUT", 6: "GP_ERR_STATE"}
EXPORTS = {"perm": (0, np.int32), "parent": (1, np.int32), "eta": (2, np.int32), "rowptr": (3, np.int64),
           "col": (4, np.int32), "sn_first": (5, np.int32), "sn_rowptr": (6, np.int64), "sn_rows": (7, np.int32),
           "sn_parent": (8, np.int32), "sn_level": (9, np.int32), "cell_perm": (10, np.int32)}


class GpHyper(ctypes.Structure):
    _fields_ = [("d", c_int), ("n1", c_int), ("n2", c_int), ("bump_dims", c_int), ("core_var", c_dbl),
                ("core_radius", DP), ("s0", c_dbl), ("r0", DP), ("h", DP), ("a", DP), ("b", DP), ("r", DP),
                ("noise_var", c_dbl)]


class GpCore(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("sigma0", c_dbl), ("Sigma0", c_dbl), ("phi_sigma", DP), ("phi_Sigma", DP)]


GP_CORE_WENDLAND, GP_CORE_PACIOREK = 0, 1


class PointsetInfo(ctypes.Structure):
    _fields_ = [("n", c_i64), ("d", c_int), ("nnz", c_i64), ("ncells", c_i64), ("nnzL", c_i64),
                ("nsuper", c_i64), ("panel_entries", c_i64), ("update_entries", c_i64), ("nlevels", ctypes.c_int32),
                ("max_front", ctypes.c_int32), ("flops", c_dbl)]


class FactorInfo(ctypes.Structure):
    _fields_ = [("B", c_int), ("precision", c_int), ("bytes", c_i64), ("not_pd_count", ctypes.c_int32),
                ("diag_fp32", ctypes.c_int32), ("timed_out", ctypes.c_int32), ("split_f16", ctypes.c_int32)]


GP_OPT_DIAG_FP32, GP_OPT_WAIT_POLLS, GP_OPT_WAIT_NS, GP_OPT_REFINE_EXP, GP_OPT_SPLIT_F16 = 0, 1, 2, 3, 4
OPTIONS = {"diag_fp32": GP_OPT_DIAG_FP32, "wait_polls": GP_OPT_WAIT_POLLS, "wait_ns": GP_OPT_WAIT_NS,
           "refine_exp": GP_OPT_REFINE_EXP, "split_f16": GP_OPT_SPLIT_F16}


class GpRequest(ctypes.Structure):
    _fields_ = [("kind", c_int), ("pointset", ctypes.c_int32), ("precision", c_int), ("theta", ctypes.POINTER(GpHyper)),
                ("d_resid", P), ("d_Xtest", P), ("m", c_i64), ("d_mu_test", P), ("d_out", P), ("d_err", P)]


class GpCompletion(ctypes.Structure):
    _fields_ = [("id", c_i64), ("status", c_int), ("slot", ctypes.c_int32), ("t_submit", c_dbl), ("t_start", c_dbl),
                ("t_done", c_dbl)]


class GpServerStats(ctypes.Structure):
    _fields_ = [("budget", ctypes.c_size_t), ("held", ctypes.c_size_t), ("peak", ctypes.c_size_t),
                ("cached_factors", ctypes.c_int32), ("queued", ctypes.c_int32), ("running", ctypes.c_int32),
                ("max_running", ctypes.c_int32), ("completed", c_i64)]


class IterativeOpts(ctypes.Structure):
    _fields_ = [("probes", ctypes.c_int32), ("lanczos_steps", ctypes.c_int32), ("tol", c_dbl),
                ("max_iter", ctypes.c_int32)]


class IterativeResult(ctypes.Structure):
    _fields_ = [("loglik", c_dbl), ("logdet", c_dbl), ("quad", c_dbl), ("minres_iters", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("minres_relres", c_dbl), ("true_relres", c_dbl)]


class GpTuneCandidate(ctypes.Structure):
    _fields_ = [("group_blocks", ctypes.c_int32), ("group_tile_n", ctypes.c_int32), ("ms", c_dbl)]


GP_REQ_LOGLIK, GP_REQ_PREDICT = 0, 1

SYMBOLS = ["gp_create", "gp_destroy", "gp_last_error", "gp_assemble", "gp_pointset_free", "gp_pointset_info",
           "gp_pointset_export", "gp_factor", "gp_factor_update", "gp_factor_free", "gp_factor_info", "gp_loglik",
           "gp_predict", "gp_launch_count", "gp_profile", "gp_profile_read", "gp_factor_bytes",
           "gp_pointset_prepare", "gp_autotune", "gp_pointset_set_blocking", "gp_symbolic_host", "gp_symbolic_info",
           "gp_symbolic_export", "gp_symbolic_free", "gp_server_create", "gp_server_add_pointset", "gp_server_submit",
           "gp_server_poll", "gp_server_wait", "gp_server_stats", "gp_server_last_error", "gp_server_destroy",
           "gp_set_option", "gp_get_option", "gp_predict_var", "gp_loglik_iterative", "gp_assemble_sparse_support",
           "gp_factor_core", "gp_factor_update_core", "gp_profile_read_level"]
KCLASS = {"values": 0, "extend_add": 1, "front_small": 2, "potrf": 3, "trsm": 4, "update": 5, "solve": 6,
          "predict": 7, "update_left": 9}

_lib = None
_LIVE = {"server": weakref.WeakSet(), "factor": weakref.WeakSet(), "pointset": weakref.WeakSet(),
         "context": weakref.WeakSet()}
_EXIT_HOOKED = False


def _free_all():
    """Free the library handles still alive at interpreter exit, factors first, while CUDA is still up."""
    for kind in ("server", "factor", "pointset", "context"):
        for obj in list(_LIVE[kind]):
            try:
                obj.close() if kind in ("context", "server") else obj.free()
            except Exception:
                pass


def _hook_exit():
    global _EXIT_HOOKED
    if not _EXIT_HOOKED:
        atexit.register(_free_all)   # registered after torch initialised CUDA, so it runs before its teardown
        _EXIT_HOOKED = True


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Open libgp.so (building it with nvcc when absent or stale) and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libgp.so not found at {_build.LIB}; run paper_2411_05869_gb300.build")
    L = ctypes.CDLL(_build.LIB)
    L.gp_create.restype = c_int
    L.gp_create.argtypes = [ctypes.POINTER(P), c_int, P, ctypes.c_size_t]
    L.gp_destroy.argtypes = [P]
    L.gp_destroy.restype = None
    L.gp_last_error.restype = ctypes.c_char_p
    L.gp_last_error.argtypes = [P]
    L.gp_assemble.restype = c_int
    L.gp_assemble.argtypes = [P, P, c_i64, c_int, DP, ctypes.POINTER(P)]
    L.gp_pointset_free.argtypes = [P]
    L.gp_pointset_free.restype = None
    L.gp_pointset_info.restype = c_int
    L.gp_pointset_info.argtypes = [P, ctypes.POINTER(PointsetInfo)]
    L.gp_pointset_export.restype = c_int
    L.gp_pointset_export.argtypes = [P, c_int, P, ctypes.c_size_t]
    L.gp_factor.restype = c_int
    L.gp_factor.argtypes = [P, P, ctypes.POINTER(GpHyper), c_int, c_int, ctypes.POINTER(P)]
    L.gp_factor_update.restype = c_int
    L.gp_factor_update.argtypes = [P, P, ctypes.POINTER(GpHyper)]
    L.gp_assemble_sparse_support.restype = c_int
    L.gp_assemble_sparse_support.argtypes = [P, P, c_i64, c_int, ctypes.POINTER(GpHyper), ctypes.POINTER(P)]
    L.gp_factor_core.restype = c_int
    L.gp_factor_core.argtypes = [P, P, ctypes.POINTER(GpHyper), ctypes.POINTER(GpCore), c_int, c_int,
                                 ctypes.POINTER(P)]
    L.gp_factor_update_core.restype = c_int
    L.gp_factor_update_core.argtypes = [P, P, ctypes.POINTER(GpHyper), ctypes.POINTER(GpCore)]
    L.gp_factor_free.argtypes = [P]
    L.gp_factor_free.restype = None
    L.gp_factor_info.restype = c_int
    L.gp_factor_info.argtypes = [P, ctypes.POINTER(FactorInfo), P]
    L.gp_loglik.restype = c_int
    L.gp_loglik.argtypes = [P, P, P, P, P]
    L.gp_predict.restype = c_int
    L.gp_predict.argtypes = [P, P, c_int, P, c_i64, P, P]
    L.gp_predict_var.restype = c_int
    L.gp_predict_var.argtypes = [P, P, c_int, P, c_i64, P]
    L.gp_loglik_iterative.restype = c_int
    L.gp_loglik_iterative.argtypes = [P, P, c_int, P, P, P, ctypes.POINTER(IterativeOpts),
                                      ctypes.POINTER(IterativeResult)]
    L.gp_launch_count.restype = c_i64
    L.gp_launch_count.argtypes = [P]
    L.gp_set_option.restype = c_int
    L.gp_set_option.argtypes = [P, c_int, c_i64]
    L.gp_get_option.restype = c_int
    L.gp_get_option.argtypes = [P, c_int, ctypes.POINTER(c_i64)]
    L.gp_profile.restype = c_int
    L.gp_profile.argtypes = [P, c_int]
    L.gp_profile_read.restype = c_int
    L.gp_profile_read.argtypes = [P, c_int, ctypes.POINTER(c_dbl), ctypes.POINTER(c_i64), ctypes.POINTER(c_dbl)]
    L.gp_profile_read_level.restype = c_int
    L.gp_profile_read_level.argtypes = [P, c_int, c_int, ctypes.POINTER(c_dbl), ctypes.POINTER(c_i64)]
    L.gp_factor_bytes.restype = c_int
    L.gp_factor_bytes.argtypes = [P, ctypes.POINTER(GpHyper), c_int, c_int, ctypes.POINTER(ctypes.c_size_t)]
    L.gp_autotune.restype = c_int
    L.gp_autotune.argtypes = [P, P, ctypes.POINTER(GpHyper), c_int, c_int, ctypes.POINTER(GpTuneCandidate),
                              ctypes.POINTER(c_int)]
    L.gp_pointset_set_blocking.restype = c_int
    L.gp_pointset_set_blocking.argtypes = [P, P, c_int, c_int]
    L.gp_symbolic_host.restype = c_int
    L.gp_symbolic_host.argtypes = [c_i64, P, P, P, ctypes.POINTER(P)]
    L.gp_symbolic_info.restype = c_int
    L.gp_symbolic_info.argtypes = [P, ctypes.POINTER(PointsetInfo)]
    L.gp_symbolic_export.restype = c_int
    L.gp_symbolic_export.argtypes = [P, c_int, P, ctypes.c_size_t]
    L.gp_symbolic_free.argtypes = [P]
    L.gp_symbolic_free.restype = None
    L.gp_pointset_prepare.restype = c_int
    L.gp_pointset_prepare.argtypes = [P, P, c_int]
    L.gp_server_create.restype = c_int
    L.gp_server_create.argtypes = [c_int, c_int, ctypes.c_size_t, ctypes.POINTER(P)]
    L.gp_server_add_pointset.restype = c_int
    L.gp_server_add_pointset.argtypes = [P, P, c_i64, c_int, DP, ctypes.POINTER(ctypes.c_int32)]
    L.gp_server_submit.restype = c_int
    L.gp_server_submit.argtypes = [P, ctypes.POINTER(GpRequest), ctypes.POINTER(c_i64)]
    L.gp_server_poll.restype = c_int
    L.gp_server_poll.argtypes = [P, ctypes.POINTER(GpCompletion), c_int]
    L.gp_server_wait.restype = c_int
    L.gp_server_wait.argtypes = [P, c_dbl]
    L.gp_server_stats.restype = c_int
    L.gp_server_stats.argtypes = [P, ctypes.POINTER(GpServerStats)]
    L.gp_server_last_error.restype = ctypes.c_char_p
    L.gp_server_last_error.argtypes = [P]
    L.gp_server_destroy.restype = None
    L.gp_server_destroy.argtypes = [P]
    _lib = L
    return L


class GpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _dp(a: np.ndarray):
    return a.ctypes.data_as(DP)


class _HyperPack:
    """Keeps the numpy arrays behind a ctypes gp_hyper array (and, for settings with the non-compact core, a
    gp_core array) alive for the duration of a call."""

    def __init__(self, thetas: Sequence):
        self.keep: List[np.ndarray] = []
        self.arr = (GpHyper * len(thetas))()
        self.cores = None
        if any(int(getattr(hp, "core_kind", 0)) != 0 for hp in thetas):
            self.cores = (GpCore * len(thetas))()
        for k, hp in enumerate(thetas):
            def arr(x):
                a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
                if a.size == 0:
                    a = np.zeros(1)
                self.keep.append(a)
                return _dp(a)
            self.arr[k] = GpHyper(hp.d, hp.n1, hp.n2, hp.bump_dims, float(hp.core_var), arr(hp.core_radius),
                                  float(hp.s0), arr(hp.r0), arr(hp.h), arr(hp.a), arr(hp.b), arr(hp.r),
                                  float(hp.noise_var))
            if self.cores is not None:
                kind = int(getattr(hp, "core_kind", 0))
                zeros = np.zeros(hp.d)
                self.cores[k] = GpCore(kind, float(getattr(hp, "sigma0", 1.0)), float(getattr(hp, "Sigma0", 1.0)),
                                       arr(hp.phi_sigma if kind else zeros), arr(hp.phi_Sigma if kind else zeros))


class Context:
    """A library context on one CUDA device and stream (gp_create)."""

    def __init__(self, device: int = 0, stream=None, mem_budget_bytes: int = 0):
        import torch
        self.lib = load()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = P()
        st = self.lib.gp_create(ctypes.byref(h), device, P(stream.cuda_stream), mem_budget_bytes)
        if st != 0:
            raise GpError(st, "gp_create failed")
        self.h = h
        _hook_exit()
        _LIVE["context"].add(self)

    def check(self, st: int):
        if st != 0:
            raise GpError(st, self.lib.gp_last_error(self.h).decode())

    def launches(self) -> int:
        return int(self.lib.gp_launch_count(self.h))

    def set_option(self, name: str, value: int):
        """gp_set_option by name (OPTIONS): applies to the context's later calls."""
        self.check(self.lib.gp_set_option(self.h, OPTIONS[name], int(value)))

    def get_option(self, name: str) -> int:
        v = c_i64()
        self.check(self.lib.gp_get_option(self.h, OPTIONS[name], ctypes.byref(v)))
        return int(v.value)

    def profile(self, enable: bool):
        """Start (clearing counters) or stop the per-kernel-class launch profiler."""
        self.check(self.lib.gp_profile(self.h, int(enable)))

    def profile_read(self) -> dict:
        """{class: (total ms, launches, useful flops)} accumulated since profile(True)."""
        out = {}
        for name, k in KCLASS.items():
            ms, n, fl = c_dbl(), c_i64(), c_dbl()
            self.check(self.lib.gp_profile_read(self.h, k, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(fl)))
            out[name] = (ms.value, n.value, fl.value)
        return out

    def profile_read_levels(self, nlevels: int) -> dict:
        """{class: [(ms, launches) per elimination-tree level]} for the classes a factorization issues per level."""
        out = {}
        for name in ("extend_add", "front_small", "potrf", "trsm", "update", "update_left"):
            rows = []
            for lev in range(min(nlevels, 64)):
                ms, n = c_dbl(), c_i64()
                self.check(self.lib.gp_profile_read_level(self.h, KCLASS[name], lev, ctypes.byref(ms),
                                                          ctypes.byref(n)))
                rows.append((ms.value, n.value))
            out[name] = rows
        return out

    def assemble(self, X, core_radius) -> "PointSet":
        """Steps A1, A2, A5, A6 for a CUDA float64 tensor X (n x d)."""
        import torch
        assert X.is_cuda and X.dtype == torch.float64 and X.dim() == 2
        X = X.contiguous()
        rad = np.ascontiguousarray(np.asarray(core_radius, dtype=np.float64))
        h = P()
        self.check(self.lib.gp_assemble(self.h, P(X.data_ptr()), X.shape[0], X.shape[1], _dp(rad), ctypes.byref(h)))
        return PointSet(self, h)

    def factor(self, ps: "PointSet", thetas: Sequence, precision: int = GP_FP64) -> "Factor":
        """Steps A3, A4, A7 for B = len(thetas) settings (gp_factor_core when they carry the non-compact core)."""
        pack = _HyperPack(thetas)
        h = P()
        if pack.cores is not None:
            self.check(self.lib.gp_factor_core(self.h, ps.h, pack.arr, pack.cores, len(thetas), precision,
                                               ctypes.byref(h)))
        else:
            self.check(self.lib.gp_factor(self.h, ps.h, pack.arr, len(thetas), precision, ctypes.byref(h)))
        return Factor(self, ps, h, len(thetas))

    def assemble_sparse_support(self, X, theta) -> "PointSet":
        """Steps A1, A2, A5, A6 with the support of C_sparse of theta (r0, bump centres and radii) as the pattern:
        the point set of the non-compact core."""
        import torch
        assert X.is_cuda and X.dtype == torch.float64 and X.dim() == 2
        X = X.contiguous()
        pack = _HyperPack([theta])
        h = P()
        self.check(self.lib.gp_assemble_sparse_support(self.h, P(X.data_ptr()), X.shape[0], X.shape[1], pack.arr,
                                                       ctypes.byref(h)))
        return PointSet(self, h)

    def close(self):
        if getattr(self, "h", None):
            self.lib.gp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def symbolic_host(rowptr, col, nd_perm) -> dict:
    """gp_symbolic_host: step A6 alone on the host (no device) for a host CSR pattern and a nested-dissection
    order; returns the sizes and the structural arrays (the names of PointSet.export)."""
    lib = load()
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    pm = np.ascontiguousarray(nd_perm, dtype=np.int32)
    h = P()
    st = lib.gp_symbolic_host(pm.shape[0], rp.ctypes.data_as(P), cl.ctypes.data_as(P), pm.ctypes.data_as(P),
                              ctypes.byref(h))
    if st != 0:
        raise GpError(st, "gp_symbolic_host failed")
    try:
        inf = PointsetInfo()
        if lib.gp_symbolic_info(h, ctypes.byref(inf)) != 0:
            raise GpError(1, "gp_symbolic_info failed")
        out = {k: getattr(inf, k) for k, _ in PointsetInfo._fields_}
        n, ns = out["n"], out["nsuper"]
        sizes = {"perm": n, "parent": n, "eta": n, "sn_first": ns + 1, "sn_rowptr": ns + 1, "sn_parent": ns,
                 "sn_level": ns}
        for name in ["perm", "parent", "eta", "sn_first", "sn_rowptr", "sn_parent", "sn_level", "sn_rows"]:
            what, dt = EXPORTS[name]
            size = int(out["sn_rowptr"][-1]) if name == "sn_rows" else sizes[name]
            arr = np.empty(size, dtype=dt)
            st = lib.gp_symbolic_export(h, what, arr.ctypes.data_as(P), arr.nbytes)
            if st != 0:
                raise GpError(st, f"gp_symbolic_export({name}) failed")
            out[name] = arr
        return out
    finally:
        lib.gp_symbolic_free(h)


class PointSet:
    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h
        _LIVE["pointset"].add(self)

    def info(self) -> dict:
        inf = PointsetInfo()
        self.ctx.check(self.ctx.lib.gp_pointset_info(self.h, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in PointsetInfo._fields_}

    def export(self, name: str) -> np.ndarray:
        what, dt = EXPORTS[name]
        inf = self.info()
        n, nnz, ns = inf["n"], inf["nnz"], inf["nsuper"]
        if name == "sn_rows":
            size = int(self.export("sn_rowptr")[-1])
        else:
            size = {"perm": n, "parent": n, "eta": n, "rowptr": n + 1, "col": nnz, "sn_first": ns + 1,
                    "sn_rowptr": ns + 1, "sn_parent": ns, "sn_level": ns, "cell_perm": n}[name]
        out = np.empty(size, dtype=dt)
        self.ctx.check(self.ctx.lib.gp_pointset_export(self.h, what, out.ctypes.data_as(P), out.nbytes))
        return out

    def autotune(self, thetas: Sequence, reps: int = 2) -> list:
        """gp_autotune: time the mixed factorization under each update blocking and keep the fastest; returns
        [{"group_blocks", "group_tile_n", "ms"}] in candidate order."""
        pack = _HyperPack(thetas)
        tried = (GpTuneCandidate * 16)()
        nt = c_int()
        self.ctx.check(self.ctx.lib.gp_autotune(self.ctx.h, self.h, pack.arr, len(thetas), reps, tried,
                                                ctypes.byref(nt)))
        return [{"group_blocks": tried[i].group_blocks, "group_tile_n": tried[i].group_tile_n, "ms": tried[i].ms}
                for i in range(nt.value)]

    def set_blocking(self, group_blocks: int, group_tile_n: int):
        """gp_pointset_set_blocking: plan a given mixed-path update blocking."""
        self.ctx.check(self.ctx.lib.gp_pointset_set_blocking(self.ctx.h, self.h, group_blocks, group_tile_n))

    def factor_bytes(self, theta, B: int = 1, precision: int = GP_FP64) -> int:
        """Device bytes a factor of B settings of theta's shape takes (gp_factor_bytes)."""
        pack = _HyperPack([theta])
        out = ctypes.c_size_t()
        self.ctx.check(self.ctx.lib.gp_factor_bytes(self.h, pack.arr, B, precision, ctypes.byref(out)))
        return int(out.value)

    def free(self):
        if self.h:
            self.ctx.lib.gp_pointset_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Factor:
    def __init__(self, ctx: Context, ps: PointSet, h, B: int):
        self.ctx, self.ps, self.h, self.B = ctx, ps, h, B
        _LIVE["factor"].add(self)

    def update(self, thetas: Sequence):
        """Re-run A3, A4, A7 in place with new settings (same B)."""
        assert len(thetas) == self.B
        pack = _HyperPack(thetas)
        if pack.cores is not None:
            self.ctx.check(self.ctx.lib.gp_factor_update_core(self.ctx.h, self.h, pack.arr, pack.cores))
        else:
            self.ctx.check(self.ctx.lib.gp_factor_update(self.ctx.h, self.h, pack.arr))

    def info(self, allow_timeout: bool = False):
        """gp_factor_info; with allow_timeout a GP_ERR_TIMEOUT status still returns the filled info."""
        inf = FactorInfo()
        cols = np.empty(self.B, dtype=np.int32)
        st = self.ctx.lib.gp_factor_info(self.h, ctypes.byref(inf), cols.ctypes.data_as(P))
        if not (allow_timeout and st == 5):
            self.ctx.check(st)
        d = {k: getattr(inf, k) for k, _ in FactorInfo._fields_}
        d["not_pd_column"] = cols
        return d

    def loglik(self, resid, out=None, err=None):
        """Steps A8-A11: resid is a CUDA float64 tensor (n,) or (B, n); returns the B log-likelihoods."""
        import torch
        r = resid.contiguous()
        assert r.is_cuda and r.dtype == torch.float64
        if out is None:
            out = torch.empty(self.B, dtype=torch.float64, device=r.device)
        self.ctx.check(self.ctx.lib.gp_loglik(self.ctx.h, self.h, P(r.data_ptr()), P(out.data_ptr()),
                                              P(_ptr(err)) if err is not None else None))
        return out

    def predict(self, Xtest, mu_test=None, b: int = 0, out=None):
        """Step A12 for proposal b at CUDA float64 test points (m x d)."""
        import torch
        Xt = Xtest.contiguous()
        m = Xt.shape[0]
        if out is None:
            out = torch.empty(m, dtype=torch.float64, device=Xt.device)
        mu = None if mu_test is None else mu_test.contiguous()
        self.ctx.check(self.ctx.lib.gp_predict(self.ctx.h, self.h, b, P(Xt.data_ptr()), m,
                                               P(mu.data_ptr()) if mu is not None else None, P(out.data_ptr())))
        return out

    def loglik_iterative(self, resid, probes, x0=None, b: int = 0, lanczos_steps: int = 30, tol: float = 1e-8,
                         max_iter: int = 10000) -> dict:
        """The paper's approximate log-likelihood (stochastic Lanczos log-det, MINRES) with C_z of proposal b;
        probes: CUDA float64 (P, n)."""
        import torch
        r = resid.contiguous()
        pr = probes.contiguous()
        assert r.is_cuda and pr.is_cuda and r.dtype == torch.float64 and pr.dtype == torch.float64
        o = IterativeOpts(pr.shape[0], lanczos_steps, tol, max_iter)
        res = IterativeResult()
        x = None if x0 is None else x0.contiguous()
        self.ctx.check(self.ctx.lib.gp_loglik_iterative(self.ctx.h, self.h, b, P(r.data_ptr()), P(pr.data_ptr()),
                                                        P(x.data_ptr()) if x is not None else None,
                                                        ctypes.byref(o), ctypes.byref(res)))
        return {k: getattr(res, k) for k, _ in IterativeResult._fields_}

    def predict_var(self, Xtest, b: int = 0, out=None):
        """Predictive variance diag(C_{y|z}) for proposal b at CUDA float64 test points (m x d)."""
        import torch
        Xt = Xtest.contiguous()
        m = Xt.shape[0]
        if out is None:
            out = torch.empty(m, dtype=torch.float64, device=Xt.device)
        self.ctx.check(self.ctx.lib.gp_predict_var(self.ctx.h, self.h, b, P(Xt.data_ptr()), m, P(out.data_ptr())))
        return out

    def free(self):
        if self.h:
            self.ctx.lib.gp_factor_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Server:
    """The continuous-batching request server (gp_server_*): cached point sets, `slots` concurrent workers,
    admission by a device-memory budget. Device buffers passed to submit() must stay alive until their
    completion has been polled; the server keeps a reference to them until then."""

    def __init__(self, device: int = 0, slots: int = 4, mem_budget_bytes: int = 0):
        self.lib = load()
        h = P()
        st = self.lib.gp_server_create(device, slots, mem_budget_bytes, ctypes.byref(h))
        if st != 0:
            raise GpError(st, "gp_server_create failed")
        self.h = h
        self._keep = {}
        _hook_exit()
        _LIVE["server"].add(self)

    def check(self, st: int):
        if st != 0:
            raise GpError(st, self.lib.gp_server_last_error(self.h).decode())

    def add_pointset(self, X, core_radius) -> int:
        import torch
        assert X.is_cuda and X.dtype == torch.float64 and X.dim() == 2
        X = X.contiguous()
        rad = np.ascontiguousarray(np.asarray(core_radius, dtype=np.float64))
        pid = ctypes.c_int32()
        self.check(self.lib.gp_server_add_pointset(self.h, P(X.data_ptr()), X.shape[0], X.shape[1], _dp(rad),
                                                   ctypes.byref(pid)))
        return int(pid.value)

    def submit(self, pointset: int, theta, resid, out, precision: int = GP_MIXED, Xtest=None, mu_test=None,
               err=None) -> int:
        """Queue a log-likelihood request (Xtest None: out holds 1 value) or a predictive-mean request
        (out holds Xtest.shape[0] values)."""
        pack = _HyperPack([theta])
        req = GpRequest(GP_REQ_PREDICT if Xtest is not None else GP_REQ_LOGLIK, pointset, precision, pack.arr,
                        P(resid.data_ptr()), P(Xtest.data_ptr()) if Xtest is not None else None,
                        0 if Xtest is None else Xtest.shape[0],
                        P(mu_test.data_ptr()) if mu_test is not None else None, P(out.data_ptr()),
                        P(err.data_ptr()) if err is not None else None)
        rid = c_i64()
        self.check(self.lib.gp_server_submit(self.h, ctypes.byref(req), ctypes.byref(rid)))
        self._keep[int(rid.value)] = (resid, out, Xtest, mu_test, err)
        return int(rid.value)

    def poll(self, max_n: int = 256) -> list:
        buf = (GpCompletion * max_n)()
        k = self.lib.gp_server_poll(self.h, buf, max_n)
        out = []
        for i in range(k):
            c = buf[i]
            out.append({"id": c.id, "status": c.status, "slot": c.slot, "t_submit": c.t_submit,
                        "t_start": c.t_start, "t_done": c.t_done})
            self._keep.pop(int(c.id), None)
        return out

    def wait(self, timeout_s: float = 0.0):
        self.check(self.lib.gp_server_wait(self.h, timeout_s))

    def stats(self) -> dict:
        st = GpServerStats()
        self.check(self.lib.gp_server_stats(self.h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in GpServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.lib.gp_server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
