"""Writes tests/golden/fullsize.json: the oracle's results on two large workloads, for the GPU parity tests at
sizes where running the oracle inside the test would take minutes.

Only the oracle (plain C, FP64) and the seeded input generators run here; nothing comes from the CUDA path.
Workloads:
  spacetime_100k   n = 100,000 space-time points, (x, y) ~ U[0,1]^2, day ~ U{0..364}, ~50 nonzeros per row, 8 bumps
                   (the full 100k space-time workload), its base setting and one perturbed setting;
  station_5000x12  the 1.2M station field's 5000 sites over its first 12 days (60,000 points, ~91 nonzeros per row,
                   16 bumps): fronts wider than 1024 columns, so a 1024-column update group does not cover them.
Stored per workload: fingerprints of the inputs (SHA-256 of the float64 bytes of X, the core radii, the first
500 test points), fingerprints of the structural outputs (pattern, order, etree, column counts, supernodes and
their row structures), nnz(L), the log-likelihood of each setting (Sec. 3.3, with the -n/2 log 2 pi term) and
the predictive mean (Sec. 3.2) of the base setting at the 500 test points, with the residual's sum and sum of
squares (the residual comes from cosines, whose last bit may differ between C libraries).

Run: python tests/golden/make_fullsize.py   (about ten minutes on eight cores)
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2411_05869_gb300 import synth  # noqa: E402

NTEST = 500


def sha(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def workloads():
    """name -> (X, resid, Xtest[:NTEST], base setting, perturbed setting)."""
    out = {}
    w = synth.config(2, m=NTEST)
    rng = np.random.default_rng(2411)
    out["spacetime_100k"] = (w.X, w.resid, w.Xtest[:NTEST], w.hyper, synth.perturb(rng, w.hyper, 0.1))
    s = synth.config(5, with_test=True)
    ns, nd, days = s.info["nsites"], s.info["ndays"], 12
    idx = (np.arange(ns)[:, None] * nd + np.arange(days)[None, :]).ravel()
    # test points: every 2400th point of the prediction grid inside the first 12 days, then the first NTEST
    t = s.Xtest[s.Xtest[:, 2] <= (days - 1) / (nd - 1)]
    Xt = t[np.linspace(0, t.shape[0] - 1, NTEST).astype(np.int64)]
    rng = np.random.default_rng(2412)
    out["station_5000x12"] = (s.X[idx], s.resid[idx], Xt, s.hyper, synth.perturb(rng, s.hyper, 0.1))
    return out


def main():
    res = {}
    for name, (X, r, Xt, hp, hp2) in workloads().items():
        t0 = time.time()
        rp, col = oracle.pattern(X, hp.core_radius)
        perm = oracle.fill_order(X, hp.core_radius, rp, col)
        sym = oracle.symbolic(rp, col, perm)
        lls = []
        for k, h in enumerate((hp, hp2)):
            o = oracle.sparse_loglik(h, X, rp, col, perm, r, want_alpha=(k == 0))
            lls.append(float(o["loglik"]))
            if k == 0:
                alpha = o["alpha"]
        mean = oracle.predict(hp, X, alpha, Xt)
        res[name] = {
            "n": int(X.shape[0]), "nnz": int(col.shape[0]), "nnzL": int(sym["nnzL"]),
            "nsuper": int(len(sym["sn_first"]) - 1), "max_width": int(np.diff(sym["sn_first"]).max()),
            "inputs": {"X": sha(X), "core_radius": [float(v).hex() for v in hp.core_radius], "Xtest": sha(Xt),
                       "resid_sum": float(r.sum()), "resid_sumsq": float((r * r).sum())},
            "structure": {"rowptr": sha(rp), "col": sha(col), "perm": sha(perm), "parent": sha(sym["parent"]),
                          "eta": sha(sym["eta"]), "sn_first": sha(sym["sn_first"]), "sn_rows": sha(sym["sn_rows"])},
            "loglik": lls,
            "predict_mean": [float(v) for v in mean],
            "oracle_seconds": round(time.time() - t0, 1),
        }
        print(name, res[name]["n"], res[name]["nnzL"], lls, res[name]["oracle_seconds"], flush=True)
    with open(os.path.join(HERE, "fullsize.json"), "w") as fh:
        json.dump(res, fh, indent=1)


if __name__ == "__main__":
    main()
