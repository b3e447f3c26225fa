"""Serving loop (include/ca_serve.h) on the GPU: each request's result is the
same alone and in the mix, the admitted footprint stays within the budget,
and a request larger than the budget is refused."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ca():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1612_04003_gb300 as mod
    mod.build()
    return mod


def _dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    return (t.to(dtype) if dtype is not None else t).cuda().contiguous()


def _requests():
    """A mix of primal / dual, FP64 / FP32, Gram modes, s and stopping."""
    out = []
    t = synth.tiny_primal(d=64, n=1024, seed=1)
    out.append(dict(method="primal", X=_dev(t.X), y=_dev(t.y), xs=64, auxs=1024,
                    kw=dict(b=4, s=4, H=200, lam=1e-3, seed=42, prec="f64")))
    m = synth.dense_primal(d=256, n=4096, cond=1e2, seed=3)
    for prec, s, ce in (("bf16x3", 16, 0), ("3xtf32", 8, 4), ("tf32", 4, 0), ("fp16_scaled", 16, 2)):
        out.append(dict(method="primal", X=_dev(m.X), y=_dev(m.y), xs=256, auxs=4096,
                        kw=dict(b=8, s=s, H=512, lam=1e-3, seed=5, prec=prec, check_every=ce)))
    w = synth.dense_dual(d=300, n=120, seed=4)
    out.append(dict(method="dual", X=_dev(np.ascontiguousarray(w.X.T)), y=_dev(w.y), xs=120,
                    auxs=300, kw=dict(b=6, s=5, H=150, lam=1e-2, seed=9, prec="f64")))
    p = synth.dense_dual(d=1028, n=400, seed=6)
    XT32 = np.ascontiguousarray(p.X.astype(np.float32).T)
    for prec in ("bf16x3", "3xtf32"):
        out.append(dict(method="dual", X=_dev(XT32), y=_dev(p.y), xs=400, auxs=1028,
                        kw=dict(b=8, s=16, H=256, lam=1e-2, seed=2, prec=prec)))
    return out


def _run_alone(ca, r):
    ctx = ca.Context(0)
    x = torch.zeros(r["xs"], dtype=torch.float64, device="cuda")
    aux = torch.zeros(r["auxs"], dtype=torch.float64, device="cuda")
    if r["method"] == "primal":
        ctx.ca_bcd_solve(r["X"], r["y"], x, aux, **r["kw"])
    else:
        ctx.ca_bdcd_solve(r["X"], r["y"], x, aux, **r["kw"])
    info = ctx.solve_info()
    ctx.close()
    return x.cpu().numpy(), aux.cpu().numpy(), info


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("workers,budget_mb", [(4, 4096), (3, 0)])
def test_served_equals_alone(ca, workers, budget_mb):
    reqs = _requests()
    alone = [_run_alone(ca, r) for r in reqs]
    # budget 0: just above the largest single need (requests then queue)
    ctx = ca.Context(0)
    needs = []
    for r in reqs:
        o = ca.Context._opts(r["kw"]["b"], r["kw"]["s"], r["kw"]["H"], r["kw"]["lam"], 0,
                             r["kw"]["prec"], 0, 0, 0.0, r["kw"].get("check_every", 0))
        rows, cols = r["X"].shape
        d, n = (rows, cols) if r["method"] == "primal" else (cols, rows)
        nb = ctypes.c_size_t()
        st = ctx._lib.ca_solve_scratch_bytes(ctx.handle, 0 if r["method"] == "primal" else 1,
                                             ca._xfmt(r["X"]), d, n, ctypes.byref(o),
                                             ctypes.byref(nb))
        assert st == ca.CA_OK
        needs.append(nb.value)
    ctx.close()
    budget = budget_mb << 20 if budget_mb else int(max(needs) * 1.5)
    srv = ca.Server(0, workers=workers, budget_bytes=budget)
    outs, ids = [], []
    for r in reqs:
        x = torch.zeros(r["xs"], dtype=torch.float64, device="cuda")
        aux = torch.zeros(r["auxs"], dtype=torch.float64, device="cuda")
        ids.append(srv.submit(r["method"], r["X"], r["y"], x, aux, **r["kw"]))
        outs.append((x, aux))
    results = [srv.wait(i) for i in ids]
    st = srv.stats()
    srv.close()
    for k, (r, res, (x, aux), (xa, auxa, info)) in enumerate(zip(reqs, results, outs, alone)):
        assert res["status"] == ca.CA_OK, (k, res)
        assert res["h_done"] == info["h_done"] and res["scratch_bytes"] == needs[k]
        assert _rel(x.cpu().numpy(), xa) < 1e-12, k
        assert _rel(aux.cpu().numpy(), auxa) < 1e-12, k
        assert abs(res["res"] - info["res"]) <= 1e-9 * max(info["res"], 1e-300)
    assert st["completed"] == len(reqs) and st["rejected"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    assert st["peak_footprint"] <= budget and 1 <= st["peak_concurrency"] <= workers
    # the FP64 primal request also against the oracle
    t = synth.tiny_primal(d=64, n=1024, seed=1)
    w_ref, _ = oracle.ca_bcd(t.X, t.y, 1e-3, b=4, s=4, H=200, seed=42)
    assert _rel(outs[0][0].cpu().numpy(), w_ref) < 1e-10


def test_request_larger_than_budget_is_refused(ca):
    m = synth.dense_primal(d=256, n=4096, cond=1e2, seed=3)
    X, y = _dev(m.X), _dev(m.y)
    srv = ca.Server(0, workers=2, budget_bytes=1 << 20)  # 1 MiB: below any real need
    x = torch.zeros(256, dtype=torch.float64, device="cuda")
    rid = srv.submit("primal", X, y, x, None, b=8, s=16, H=64, lam=1e-3, prec="bf16x3")
    res = srv.wait(rid)
    assert res["status"] == ca.CA_ERR_OOM and res["worker"] == -1
    assert srv.stats()["rejected"] == 1
    assert float(x.abs().max()) == 0.0  # never ran
    srv.close()


def test_served_batches_share_launches(ca):
    """Continuous batching: with ca_server_set_batching the scheduler starts
    the queue's head with the batchable requests queued right behind it (one
    Gram mode, FP32 X, b <= 16, s b <= 128) as one batched solve.  Each
    batched result is held to the same request alone at the FP32-path
    tolerance (the shared plan splits its Gram sums differently); requests
    that do not batch (FP64 X, a second Gram mode) run alone and equal the
    solve alone to 1e-12; more requests run at once than there are workers."""
    reqs = []
    for i, (d, n, b, s) in enumerate([(256, 4096, 8, 16), (512, 2048, 4, 16), (128, 8192, 16, 8),
                                      (384, 4000, 8, 8), (200, 1024, 4, 32), (640, 3000, 8, 16),
                                      (96, 2048, 16, 4), (300, 5000, 8, 16)]):
        m = synth.dense_primal(d=d, n=n, cond=1e2, seed=30 + i)
        reqs.append(dict(method="primal", X=_dev(np.ascontiguousarray(m.X[:, :n])),
                         y=_dev(m.y[:n]), xs=d, auxs=n,
                         kw=dict(b=b, s=s, H=256, lam=1e-3, seed=40 + i, prec="bf16x3")))
    p = synth.dense_dual(d=1028, n=400, seed=6)
    reqs.insert(3, dict(method="dual", X=_dev(np.ascontiguousarray(p.X.astype(np.float32).T)),
                        y=_dev(p.y), xs=400, auxs=1028,
                        kw=dict(b=8, s=16, H=256, lam=1e-2, seed=2, prec="bf16x3")))
    t = synth.tiny_primal(d=64, n=1024, seed=1)
    reqs.insert(5, dict(method="primal", X=_dev(t.X), y=_dev(t.y), xs=64, auxs=1024,
                        kw=dict(b=4, s=4, H=200, lam=1e-3, seed=42, prec="f64")))
    alone = [_run_alone(ca, r) for r in reqs]
    workers = 2
    srv = ca.Server(0, workers=workers, budget_bytes=8 << 30, batch=8)
    outs, ids = [], []
    for r in reqs:
        x = torch.zeros(r["xs"], dtype=torch.float64, device="cuda")
        aux = torch.zeros(r["auxs"], dtype=torch.float64, device="cuda")
        ids.append(srv.submit(r["method"], r["X"], r["y"], x, aux, **r["kw"]))
        outs.append((x, aux))
    results = [srv.wait(i) for i in ids]
    st = srv.stats()
    srv.close()
    for k, (r, res, (x, aux), (xa, auxa, info)) in enumerate(zip(reqs, results, outs, alone)):
        assert res["status"] == ca.CA_OK and res["h_done"] == info["h_done"], (k, res)
        tol = 1e-12 if r["kw"]["prec"] == "f64" else 1e-5
        assert _rel(x.cpu().numpy(), xa) < tol, k
        assert _rel(aux.cpu().numpy(), auxa) < tol, k
    assert st["completed"] == len(reqs)
    assert st["peak_concurrency"] > workers  # some requests ran as a group
