"""The request server (gp_server_*): continuous batching over cached point sets with memory admission.

Each request's results must be the same whether it runs alone or in a mix of concurrent requests of uneven
sizes, and the same as the direct library calls; the factor bytes the server admits against must be the
bytes gp_factor allocates; the server must never hold more factor memory than its budget.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _sets():
    from paper_2411_05869_gb300 import synth
    return [synth.uniform_spacetime(n, 40, 30.0, 8, seed=synth.SEED_BASE + 700 + i, name=f"srv{i}")
            for i, n in enumerate([2500, 5000, 9000])]


def _requests(ws, count=12):
    from paper_2411_05869_gb300 import gp, synth
    rng = np.random.default_rng(77)
    reqs = []
    for k in range(count):
        i = k % len(ws)
        prec = gp.GP_MIXED if k % 3 else gp.GP_FP64
        reqs.append({"set": i, "theta": synth.perturb(rng, ws[i].hyper, 0.1), "prec": prec,
                     "predict": k % 4 == 3})
    return reqs


def _run_server(ws, reqs, slots, budget, order=None):
    import torch
    from paper_2411_05869_gb300 import gp
    srv = gp.Server(0, slots=slots, mem_budget_bytes=budget)
    ids = [srv.add_pointset(torch.as_tensor(w.X, device="cuda"), w.hyper.core_radius) for w in ws]
    resid = [torch.as_tensor(w.resid, device="cuda") for w in ws]
    xt = [torch.as_tensor(w.Xtest, device="cuda") for w in ws]
    outs = [None] * len(reqs)
    done = {}
    batch = [list(range(len(reqs)))] if order is None else [[k] for k in order]
    for group in batch:
        rid = {}
        for k in group:
            q = reqs[k]
            i = q["set"]
            if q["predict"]:
                outs[k] = torch.full((xt[i].shape[0],), float("nan"), dtype=torch.float64, device="cuda")
                rid[srv.submit(ids[i], q["theta"], resid[i], outs[k], q["prec"], Xtest=xt[i])] = k
            else:
                outs[k] = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
                rid[srv.submit(ids[i], q["theta"], resid[i], outs[k], q["prec"])] = k
        srv.wait(600.0)
        for c in srv.poll(1024):
            done[rid[c["id"]]] = c
    stats = srv.stats()
    res = [o.cpu().numpy().copy() for o in outs]
    srv.close()
    return res, done, stats


def test_server_mix_equals_alone_and_direct_calls():
    import torch
    from paper_2411_05869_gb300 import gp
    ws = _sets()
    reqs = _requests(ws)
    mix, done_mix, st_mix = _run_server(ws, reqs, slots=3, budget=1 << 36)
    alone, done_alone, _ = _run_server(ws, reqs, slots=1, budget=1 << 36, order=range(len(reqs)))
    assert all(c["status"] == 0 for c in done_mix.values()) and len(done_mix) == len(reqs)
    assert all(c["status"] == 0 for c in done_alone.values())
    assert st_mix["max_running"] >= 2, "requests should have overlapped on the device"
    for k in range(len(reqs)):
        assert np.all(np.isfinite(mix[k])), k
        np.testing.assert_array_equal(mix[k], alone[k], err_msg=f"request {k} differs alone vs in the mix")
    # the direct library calls give the same numbers
    ctx = gp.Context(0)
    for k, q in enumerate(reqs):
        w = ws[q["set"]]
        ps = ctx.assemble(torch.as_tensor(w.X, device="cuda"), w.hyper.core_radius)
        f = ctx.factor(ps, [q["theta"]], q["prec"])
        ll = f.loglik(torch.as_tensor(w.resid, device="cuda"))
        ref = f.predict(torch.as_tensor(w.Xtest, device="cuda")) if q["predict"] else ll
        torch.cuda.synchronize()
        np.testing.assert_array_equal(mix[k], ref.cpu().numpy(), err_msg=f"request {k} differs from direct calls")
        f.free()
        ps.free()


def test_server_memory_admission_and_factor_bytes():
    import torch
    from paper_2411_05869_gb300 import gp
    ws = _sets()
    ctx = gp.Context(0)
    need = []
    for w in ws:   # the admission size is what gp_factor allocates
        ps = ctx.assemble(torch.as_tensor(w.X, device="cuda"), w.hyper.core_radius)
        for prec in (gp.GP_FP64, gp.GP_MIXED):
            f = ctx.factor(ps, [w.hyper], prec)
            assert f.info()["bytes"] == ps.factor_bytes(w.hyper, 1, prec)
            need.append(f.info()["bytes"])
            f.free()
        ps.free()
    reqs = _requests(ws, 9)
    budget = int(max(need) * 1.5)   # room for one large factor at a time plus a small one
    res, done, st = _run_server(ws, reqs, slots=3, budget=budget)
    assert len(done) == len(reqs) and all(c["status"] == 0 for c in done.values())
    assert st["peak"] <= budget and st["held"] <= budget
    assert all(np.all(np.isfinite(r)) for r in res)
    # a request whose factor could never fit is refused at submission
    srv = gp.Server(0, slots=1, mem_budget_bytes=min(need) // 2)
    pid = srv.add_pointset(torch.as_tensor(ws[0].X, device="cuda"), ws[0].hyper.core_radius)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(gp.GpError):
        srv.submit(pid, ws[0].hyper, torch.as_tensor(ws[0].resid, device="cuda"), out, gp.GP_MIXED)
    srv.close()
