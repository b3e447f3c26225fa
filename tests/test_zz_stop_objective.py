"""The certified stopping rule (stop = "objective") on the GPU, against the
oracle's duality gaps (Sec. 2.2 duality, Sec. 5.1.5 stopping).

At a check the library forms the full residual r and from its norm the
duality gap in closed form (primal: ||r||^2/(2 lambda) at alpha = X^T w - y;
dual: ||r||^2/(2n) at w = -X alpha/(lambda n)), and f(w) of the model from
the maintained vectors; the solve ends at the first check with
gap <= tol (f(w) - gap), which certifies (f(w) - f(w*))/f(w*) <= tol.
Checked here: gap and f(w) against the oracle at the GPU's own iterate; the
update count of the stop against the oracle's certified run (tolerance
chosen between two clearly separated checks); the certificate against the
closed-form optimum; the stop at the first check under the tolerance.
Also the per-check trace (f non-increasing under BCD, D under BDCD) and,
for the serving loop, a certified request and requests whose unrolling
depth s the server picks by measured cost.  Collected after the parity and
serving suites.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import synth  # noqa: E402

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-5


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1612_04003_gb300 as ca
    ca.build()
    c = ca.Context(0)
    yield c
    c.close()


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda().contiguous()


def _np(t):
    return t.detach().cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _bound(f, g):
    return g / (f - g) if f > g else float("inf")


def _tol_between(bounds, sep=2.0):
    """A tolerance first met at check j and by no earlier check, with a
    factor sep between bounds[j] and every earlier bound."""
    for j in range(1, len(bounds)):
        hi = min(bounds[:j])
        if bounds[j] * sep < hi:
            return (float(np.sqrt(bounds[j] * hi)) if np.isfinite(hi) else 2.0 * bounds[j]), j
    raise AssertionError("no clear crossing")


@pytest.fixture(scope="module")
def tiny():
    return synth.tiny_primal(d=64, n=1024, seed=1)


def test_primal_f64_gap_and_stop(ctx, tiny):
    X, y, lam = tiny.X, tiny.y, 1e-3
    n = X.shape[1]
    kw = dict(b=4, s=4, H=400, seed=42)
    _, _, trace = oracle.ca_bcd_certified(X, y, lam, tol=0.0, check_every=5, **kw)
    Xd, yd = _dev(X), _dev(y)
    w = torch.zeros(64, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(Xd, yd, w, lam=lam, prec="f64", check_every=5, stop="objective", **kw)
    info = ctx.solve_info()
    assert info["h_done"] == 400 and info["checks"] == len(trace) == 20
    wg = _np(w)
    r = oracle.primal_residual(X, y, lam, wg)
    scale = oracle.primal_objective(X, y, lam, wg) + y @ y / (2 * n)
    assert abs(info["gap"] - r @ r / (2 * lam)) <= 1e-6 * (r @ r / (2 * lam)) + 1e-14 * scale
    assert abs(info["fval"] - oracle.primal_objective(X, y, lam, wg)) <= 1e-10 * info["fval"]
    assert abs(info["fval"] - trace[-1][0]) <= 1e-9 * trace[-1][0]
    tol, j = _tol_between([_bound(f, g) for f, g in trace])
    w_ref, h_ref, _ = oracle.ca_bcd_certified(X, y, lam, tol=tol, check_every=5, **kw)
    assert h_ref == 20 * (j + 1)
    w = torch.zeros(64, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(Xd, yd, w, lam=lam, prec="f64", check_every=5, stop="objective", tol=tol,
                     **kw)
    info = ctx.solve_info()
    assert info["h_done"] == h_ref and info["checks"] == j + 1
    assert _rel(_np(w), w_ref) < TOL64
    assert info["bound"] is not None and info["bound"] <= tol
    fstar = oracle.primal_objective(X, y, lam, oracle.closed_form(X, y, lam))
    assert (oracle.primal_objective(X, y, lam, _np(w)) - fstar) / fstar <= tol


@pytest.fixture(scope="module")
def mid():
    """Dense primal 512 x 8192 FP32 (cond 1e3 row scaling), lambda 1e-4, with
    its closed-form optimum."""
    m = synth.dense_primal(d=512, n=8205, cond=1e3, seed=2)
    X32 = np.ascontiguousarray(m.X[:, :8192])
    X64, y = X32.astype(np.float64), m.y[:8192].copy()
    fstar = oracle.primal_objective(X64, y, 1e-4, oracle.closed_form(X64, y, 1e-4))
    return X32, X64, y, fstar


@pytest.mark.parametrize("prec", ["bf16x3", "3xtf32", "f64"])
def test_primal_certified_relative_objective_error(ctx, mid, prec):
    """Stop at a certified relative objective error of 1e-6 (the tensor-core
    path with b = 8, s = 16, and the FP64 path on the same data): the true
    error from the closed form is within it, gap and f(w) are those of the
    GPU's own iterate, and the check before the stop was above it."""
    X32, X64, y, fstar = mid
    lam, tol = 1e-4, 1e-6
    kw = dict(b=8, s=16, seed=7, check_every=2, stop="objective")
    Xd = _dev(X64) if prec == "f64" else _dev(X32)
    yd = _dev(y)
    w = torch.zeros(512, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(Xd, yd, w, lam=lam, prec=prec, H=8192, tol=tol, **kw)
    info = ctx.solve_info()
    h = info["h_done"]
    assert h < 8192 and h % 32 == 0 and info["bound"] is not None and info["bound"] <= tol
    wg = _np(w)
    f = oracle.primal_objective(X64, y, lam, wg)
    r = oracle.primal_residual(X64, y, lam, wg)
    # f(w) from rho; FP32 X: rho rebuilt at the check with exact products
    # summed in double-float (emulated within 1e-12 f along a run in
    # test_split_precision_cpu.py; 1e-10 f here)
    assert abs(info["fval"] - f) <= 1e-10 * f
    assert abs(info["bound"] - info["gap"] / (info["fval"] - info["gap"])) <= 1e-14 * info["bound"]
    g_own = r @ r / (2 * lam)
    # FP32 X: the residual pass forms exact products summed in double-float;
    # its gap is within 1e-6 g + 1e-13 f by the same emulation (1e-4 g +
    # 1e-12 f here)
    rtol, atol = (1e-6, 1e-14) if prec == "f64" else (1e-4, 1e-12)
    assert abs(info["gap"] - g_own) <= rtol * g_own + atol * f
    assert (f - fstar) / fstar <= tol
    # the same solve stopped one check earlier: its bound was above tol
    w = torch.zeros(512, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(Xd, yd, w, lam=lam, prec=prec, H=h - 32, tol=0.0, **kw)
    prev = ctx.solve_info()
    assert prev["h_done"] == h - 32
    assert prev["bound"] is None or prev["bound"] > tol


@pytest.fixture(scope="module")
def wide():
    return synth.dense_dual(d=300, n=120, seed=4)


def test_dual_dense_gap_and_stop(ctx, wide):
    X, y, lam = wide.X, wide.y, 1e-2
    d, n = X.shape
    kw = dict(b=6, s=3, H=150, seed=9)
    _, _, _, trace = oracle.ca_bdcd_certified(X, y, lam, tol=0.0, check_every=5, **kw)
    XT, yd = _dev(X.T), _dev(y)
    a = torch.zeros(n, dtype=torch.float64, device="cuda")
    w = torch.zeros(d, dtype=torch.float64, device="cuda")
    ctx.ca_bdcd_solve(XT, yd, a, w, lam=lam, prec="f64", check_every=5, stop="objective", **kw)
    info = ctx.solve_info()
    assert info["h_done"] == 150 and info["checks"] == len(trace) == 10
    ag, wg = _np(a), _np(w)
    r = oracle.dual_residual(X, y, ag, wg)
    scale = y @ y / (2 * n)
    assert abs(info["gap"] - r @ r / (2 * n)) <= 1e-6 * (r @ r / (2 * n)) + 1e-14 * scale
    f = oracle.primal_objective(X, y, lam, wg)
    assert abs(info["fval"] - f) <= 1e-9 * f + 1e-13 * scale
    tol, j = _tol_between([_bound(f, g) for f, g in trace])
    a_ref, w_ref, h_ref, _ = oracle.ca_bdcd_certified(X, y, lam, tol=tol, check_every=5, **kw)
    assert h_ref == 15 * (j + 1)
    a.zero_()
    w.zero_()
    ctx.ca_bdcd_solve(XT, yd, a, w, lam=lam, prec="f64", check_every=5, stop="objective",
                      tol=tol, **kw)
    info = ctx.solve_info()
    assert info["h_done"] == h_ref and info["checks"] == j + 1
    assert _rel(_np(a), a_ref) < TOL64 and _rel(_np(w), w_ref) < TOL64
    fstar = oracle.primal_objective(X, y, lam, oracle.closed_form(X, y, lam))
    assert (oracle.primal_objective(X, y, lam, _np(w)) - fstar) / fstar <= tol


def test_dual_csr_gap(ctx):
    sp = synth.sparse_dual(d=4000, n=600, density=0.01, seed=3)
    A = oracle.CSR(sp.rowptr, sp.col, sp.val.astype(np.float64), sp.d)
    lam = 1e-3
    kw = dict(b=8, s=8, H=192, seed=4)
    _, _, _, trace = oracle.ca_bdcd_certified(A, sp.y, lam, tol=0.0, check_every=3, **kw)
    a = torch.zeros(sp.n, dtype=torch.float64, device="cuda")
    w = torch.zeros(sp.d, dtype=torch.float64, device="cuda")
    csr = (_dev(sp.rowptr), _dev(sp.col), _dev(sp.val))
    ctx.ca_bdcd_solve(csr, _dev(sp.y), a, w, lam=lam, d=sp.d, check_every=3, stop="objective",
                      **kw)
    info = ctx.solve_info()
    assert info["h_done"] == 192 and info["checks"] == len(trace) == 8
    ag, wg = _np(a), _np(w)
    r = oracle.dual_residual(A, sp.y, ag, wg)
    scale = sp.y @ sp.y / (2 * sp.n)
    assert abs(info["gap"] - r @ r / (2 * sp.n)) <= 1e-6 * (r @ r / (2 * sp.n)) + 1e-14 * scale
    f, g = trace[-1]
    assert abs(info["fval"] - f) <= 1e-9 * f + 1e-13 * scale
    assert abs(info["gap"] - g) <= 1e-6 * g + 1e-13 * scale


def test_served_certified_request_equals_alone(ctx, tiny):
    import paper_1612_04003_gb300 as ca
    X, y = _dev(tiny.X), _dev(tiny.y)
    kw = dict(b=4, s=4, H=2000, lam=1e-3, seed=42, prec="f64", check_every=5, tol=1e-9,
              stop="objective")
    w = torch.zeros(64, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(X, y, w, **kw)
    alone = ctx.solve_info()
    assert alone["h_done"] < 2000
    srv = ca.Server(0, workers=2, budget_bytes=1 << 30)
    w2 = torch.zeros(64, dtype=torch.float64, device="cuda")
    res = srv.wait(srv.submit("primal", X, y, w2, None, **kw))
    srv.close()
    assert res["status"] == ca.CA_OK and res["h_done"] == alone["h_done"]
    assert abs(res["gap"] - alone["gap"]) <= 1e-9 * alone["gap"]
    assert abs(res["fval"] - alone["fval"]) <= 1e-12 * alone["fval"]
    assert _rel(_np(w2), _np(w)) < 1e-12


def test_trace_primal_objective_non_increasing(ctx, tiny):
    """Sec. 3.1: each BCD step minimises f exactly over its block, so f never
    increases; the per-check trace (every outer step here) gives f(w_h) and
    the gap, each against the oracle's iterate of the same length."""
    X, y, lam = tiny.X, tiny.y, 1e-3
    kw = dict(b=4, s=4, H=200, seed=42)
    w = torch.zeros(64, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(_dev(X), _dev(y), w, lam=lam, prec="f64", check_every=1, stop="objective",
                     **kw)
    info, tr = ctx.solve_info(), ctx.solve_trace()
    assert len(tr) == info["checks"] + 1 == 51
    assert [c["h"] for c in tr] == list(range(0, 201, 4))
    assert tr[0]["res"] == info["res0"] and tr[-1]["res"] == info["res"]
    assert tr[-1]["gap"] == info["gap"] and tr[-1]["fval"] == info["fval"]
    fs = [c["fval"] for c in tr]
    assert all(b <= a * (1 + 1e-13) for a, b in zip(fs, fs[1:]))
    for c in tr[::10]:
        wh, _ = oracle.ca_bcd(X, y, lam, H=c["h"], **{k: v for k, v in kw.items() if k != "H"}) \
            if c["h"] else (np.zeros(64), None)
        f = oracle.primal_objective(X, y, lam, wh)
        r = oracle.primal_residual(X, y, lam, wh)
        assert abs(c["fval"] - f) <= 1e-10 * f
        assert abs(c["gap"] - r @ r / (2 * lam)) <= 1e-6 * (r @ r / (2 * lam)) + 1e-14 * f


def test_trace_dual_objective_non_increasing(ctx, wide):
    """Sec. 3.2: BDCD minimises D exactly over its block, so D never
    increases (the primal objective of w(alpha) need not decrease).  From
    the trace, D = ||y||^2/(2n) + gap - f(w)."""
    X, y, lam = wide.X, wide.y, 1e-2
    d, n = X.shape
    a = torch.zeros(n, dtype=torch.float64, device="cuda")
    w = torch.zeros(d, dtype=torch.float64, device="cuda")
    ctx.ca_bdcd_solve(_dev(X.T), _dev(y), a, w, lam=lam, prec="f64", b=6, s=3, H=150, seed=9,
                      check_every=1, stop="objective")
    tr = ctx.solve_trace()
    assert len(tr) == 51
    scale = y @ y / (2 * n)
    D = [scale + c["gap"] - c["fval"] for c in tr]
    assert all(b <= a + 1e-13 * scale for a, b in zip(D, D[1:]))
    assert abs(D[-1] - oracle.dual_objective(X, y, lam, _np(a))) <= 1e-10 * scale


def test_trace_residual_rule_records_norms(ctx, tiny):
    X, y = _dev(tiny.X), _dev(tiny.y)
    w = torch.zeros(64, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(X, y, w, b=4, s=4, H=200, lam=1e-3, seed=42, prec="f64", check_every=5)
    info, tr = ctx.solve_info(), ctx.solve_trace()
    assert len(tr) == info["checks"] + 1 == 11
    assert [c["h"] for c in tr] == list(range(0, 201, 20))
    assert all(c["fval"] == 0.0 for c in tr)
    assert all(abs(c["gap"] - c["res"] ** 2 / 2e-3) <= 1e-12 * c["gap"] for c in tr)
    w = torch.zeros(64, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(X, y, w, b=4, s=4, H=200, lam=1e-3, seed=42, prec="f64")
    assert ctx.solve_trace() == []


def test_served_s_by_measured_cost(ctx, tiny):
    """Serving: requests submitted with s = 0 get their unrolling depth from
    measured cost -- each candidate s (s*b <= 256, in the order 8, 16, 4, 32,
    2, 1, 64) once per shape class, then the cheapest so far; every result
    equals the same solve made alone with the s it reports."""
    import paper_1612_04003_gb300 as ca
    X, y = _dev(tiny.X), _dev(tiny.y)
    kw = dict(b=4, H=96, lam=1e-3, seed=42, prec="f64")
    srv = ca.Server(0, workers=1, budget_bytes=1 << 30)
    outs = []
    for _ in range(9):  # one after another: each choice sees the earlier costs
        w = torch.zeros(64, dtype=torch.float64, device="cuda")
        outs.append((srv.wait(srv.submit("primal", X, y, w, None, s=0, **kw)), w))
    srv.close()
    cands = [8, 16, 4, 32, 2, 1, 64]
    assert [r["s"] for r, _ in outs[:7]] == cands
    assert all(r["s"] in cands for r, _ in outs[7:])
    for r, w in outs:
        assert r["status"] == ca.CA_OK and r["h_done"] == 96
        w_alone = torch.zeros(64, dtype=torch.float64, device="cuda")
        ctx.ca_bcd_solve(X, y, w_alone, s=r["s"], **kw)
        assert _rel(_np(w), _np(w_alone)) < 1e-12


def test_unknown_stopping_rule_is_refused(ctx, tiny):
    import paper_1612_04003_gb300 as ca
    X, y = _dev(tiny.X), _dev(tiny.y)
    w = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(ca.CaError) as e:
        ctx.ca_bcd_solve(X, y, w, b=4, s=4, H=40, lam=1e-3, prec="f64", check_every=2, stop=2)
    assert e.value.status == ca.CA_ERR_ARG
    assert float(w.abs().max()) == 0.0
