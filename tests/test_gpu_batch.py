"""Batched solves (ca_batch_solve) on the GB300, through the C ABI: uneven
problems -- primal and dual, different d, n, b, s and H -- solved together
in shared launches (one Gram pass over all problems' atoms, one reduction,
one chain CTA per problem per round).

Each problem computes what the same solve computes alone except for the
split-K partition of its Gram sums (the shared plan splits its atoms
differently), so a batched problem is held to the oracle at the FP32-path
tolerance 1e-5, and to its solo solve at the same 1e-5: both are FP32-Gram
roundings of one exact path, each within 1e-5 of it (measured: batch vs
solo 1.2e-7 .. 1.05e-6, each vs the oracle 8e-8 .. 2.5e-6).  The
graph-captured and the plainly launched batch run the same kernels on the
same data and agree up to the order of FP64 atomic additions (1e-13).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import synth  # noqa: E402

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module")
def ca_ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1612_04003_gb300 as ca
    ca.build()
    stream = torch.cuda.Stream()
    c = ca.Context(0, stream=stream.cuda_stream)
    yield ca, c, stream
    c.close()


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda().contiguous()


def _rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    b = b.detach().cpu().numpy() if hasattr(b, "detach") else np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# uneven problems: (method, d, n, b, s, H, lambda); H not always a multiple
# of s (short last steps), K from 1 to a few hundred atoms
SPECS = [("primal", 256, 4096, 8, 16, 512, 1e-3),
         ("dual", 1536, 384, 4, 16, 300, 1e-2),
         ("primal", 512, 8224, 16, 8, 256, 1e-4),
         ("dual", 640, 200, 8, 4, 202, 1e-1),
         ("primal", 96, 1000, 4, 32, 130, 1e-2),
         ("primal", 300, 20000, 8, 8, 64, 1e-3)]


def _problems(specs, prec="bf16x3", recompute_every=0):
    out = []
    for i, (method, d, n, b, s, H, lam) in enumerate(specs):
        if method == "primal":
            m = synth.dense_primal(d=d, n=n, cond=1e2, seed=10 + i)
            X32 = np.ascontiguousarray(m.X[:, :n]).astype(np.float32)
            y = m.y[:n].copy()
            out.append(dict(method=method, X=_dev(X32), X64=X32.astype(np.float64), y=_dev(y),
                            yh=y, x=torch.zeros(d, dtype=torch.float64, device="cuda"),
                            aux=torch.zeros(n, dtype=torch.float64, device="cuda"),
                            b=b, s=s, H=H, lam=lam, seed=100 + i, prec=prec,
                            recompute_every=recompute_every))
        else:
            p = synth.dense_dual(d=d, n=n, seed=20 + i)
            X32 = p.X.astype(np.float32)
            out.append(dict(method=method, X=_dev(X32.T), X64=X32.astype(np.float64),
                            y=_dev(p.y), yh=p.y,
                            x=torch.zeros(n, dtype=torch.float64, device="cuda"),
                            aux=torch.zeros(d, dtype=torch.float64, device="cuda"),
                            b=b, s=s, H=H, lam=lam, seed=100 + i, prec=prec,
                            recompute_every=recompute_every))
    return out


def _solo(ctx, p):
    x = torch.zeros_like(p["x"])
    aux = torch.zeros_like(p["aux"])
    kw = dict(b=p["b"], s=p["s"], H=p["H"], lam=p["lam"], seed=p["seed"], prec=p["prec"],
              recompute_every=p["recompute_every"])
    if p["method"] == "primal":
        ctx.ca_bcd_solve(p["X"], p["y"], x, aux, **kw)
    else:
        ctx.ca_bdcd_solve(p["X"], p["y"], x, aux, **kw)
    return x, aux


def _oracle(p, s=None):
    kw = dict(b=p["b"], H=p["H"], seed=p["seed"], recompute_every=p["recompute_every"])
    if p["method"] == "primal":
        if s is None:
            return oracle.ca_bcd(p["X64"], p["yh"], p["lam"], s=p["s"], **kw)
        return oracle.bcd(p["X64"], p["yh"], p["lam"], **kw)
    if s is None:
        return oracle.ca_bdcd(p["X64"], p["yh"], p["lam"], s=p["s"], **kw)
    return oracle.bdcd(p["X64"], p["yh"], p["lam"], **kw)


@pytest.mark.parametrize("prec", ["bf16x3", "3xtf32"])
def test_uneven_batch_equals_solo_and_oracle(ca_ctx, prec):
    ca, ctx, _ = ca_ctx
    probs = _problems(SPECS, prec=prec)
    res = ctx.ca_batch_solve(probs, graph=True)
    for p, r in zip(probs, res):
        assert r["status"] == ca.CA_OK and r["h_done"] == p["H"] and r["s"] == p["s"]
        x_ref, aux_ref = _oracle(p)
        xs, auxs = _solo(ctx, p)
        e_or = _rel(p["x"], x_ref)
        e_solo = _rel(p["x"], xs)
        print(f"{p['method']} {tuple(p['X'].shape)} b={p['b']} s={p['s']} H={p['H']}: "
              f"oracle {e_or:.2e} solo {e_solo:.2e}")
        assert e_or < TOL32 and _rel(p["aux"], aux_ref) < TOL32
        assert e_solo < TOL32 and _rel(p["aux"], auxs) < TOL32


def test_graph_and_plain_launches_agree_bitwise(ca_ctx):
    ca, ctx, _ = ca_ctx
    a = _problems(SPECS[:4])
    b = _problems(SPECS[:4])
    ctx.ca_batch_solve(a, graph=True)
    ctx.ca_batch_solve(b, graph=False)
    for pa, pb in zip(a, b):
        # the same kernels on the same data: equal up to the order of FP64
        # atomic additions (an index recurring across the blocks of an outer
        # step is updated atomically; z = X^T w_H adds row splits atomically)
        assert _rel(pa["x"], pb["x"]) < 1e-13
        assert _rel(pa["aux"], pb["aux"]) < 1e-13


def test_batch_periodic_recompute(ca_ctx):
    ca, ctx, _ = ca_ctx
    probs = _problems(SPECS[:4], recompute_every=3)
    res = ctx.ca_batch_solve(probs)
    for p, r in zip(probs, res):
        assert r["status"] == ca.CA_OK
        x_ref, aux_ref = _oracle(p)
        assert _rel(p["x"], x_ref) < TOL32 and _rel(p["aux"], aux_ref) < TOL32


def test_depth_by_measured_cost(ca_ctx):
    """s = 0: a warm-up round and one timed round each at s b = 128, 64, 32,
    then the cheapest; s changes between outer steps, so every problem is
    held to the oracle's Algorithm 1 / 3 (the s = 1 iterates, which CA-BCD
    reproduces for any sequence of depths in exact arithmetic)."""
    ca, ctx, _ = ca_ctx
    specs = [(m, d, n, b, 0, H, lam) for (m, d, n, b, _, H, lam) in SPECS]
    probs = _problems(specs)
    res = ctx.ca_batch_solve(probs)
    for p, r in zip(probs, res):
        assert r["status"] == ca.CA_OK and r["h_done"] == p["H"]
        assert r["s"] * p["b"] in (32, 64, 128) or r["s"] == 1
        x_ref, aux_ref = _oracle(p, s=1)
        assert _rel(p["x"], x_ref) < TOL32 and _rel(p["aux"], aux_ref) < TOL32


def test_batch_refusals(ca_ctx):
    ca, ctx, _ = ca_ctx
    p = _problems(SPECS[:1])[0]
    for bad, st in ((dict(b=32, s=2), ca.CA_ERR_UNSUPPORTED), (dict(s=32), ca.CA_ERR_UNSUPPORTED)):
        q = dict(p, **bad)
        with pytest.raises(ca.CaError) as e:
            ctx.ca_batch_solve([q])
        assert e.value.status == st
    q = dict(p, prec="3xtf32")
    with pytest.raises(ca.CaError) as e:  # one Gram mode per batch
        ctx.ca_batch_solve([p, q])
    assert e.value.status == ca.CA_ERR_ARG
    q = dict(p, y=p["yh"])  # host array
    with pytest.raises(ca.CaError) as e:
        ctx.ca_batch_solve([q])
    assert e.value.status == ca.CA_ERR_ARG


def test_batch_certified_stop_matches_solo(ca_ctx):
    """The stopping test inside a batch (Sec. 5.1.5 with the duality gap of
    Sec. 2.2): a problem checked every 2 outer steps stops at the same check
    as alone, with a tolerance chosen between two clearly separated checks
    of the solo run, while the other problems of the batch run to H."""
    ca, ctx, _ = ca_ctx
    m = synth.dense_primal(d=512, n=8205, cond=1e3, seed=2)
    X32 = np.ascontiguousarray(m.X[:, :8192]).astype(np.float32)
    y = m.y[:8192].copy()
    kw = dict(b=8, s=16, H=4096, lam=1e-4, seed=7, prec="bf16x3", check_every=2,
              stop="objective")
    Xd, yd = _dev(X32), _dev(y)
    w = torch.zeros(512, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(Xd, yd, w, **kw)
    bounds = [c["gap"] / (c["fval"] - c["gap"]) if c["fval"] > c["gap"] else float("inf")
              for c in ctx.solve_trace()]
    tol, j = None, None
    for jj in range(1, len(bounds)):
        hi = min(bounds[:jj])
        if bounds[jj] * 3.0 < hi and np.isfinite(hi) and bounds[jj] < 1e-4:
            tol, j = float(np.sqrt(bounds[jj] * hi)), jj
            break
    assert tol is not None
    w.zero_()
    ctx.ca_bcd_solve(Xd, yd, w, tol=tol, **kw)
    alone = ctx.solve_info()
    assert alone["h_done"] == 32 * j
    others = _problems(SPECS[2:5])
    wb = torch.zeros(512, dtype=torch.float64, device="cuda")
    mine = dict(method="primal", X=Xd, y=yd, x=wb, aux=None, tol=tol, **kw)
    res = ctx.ca_batch_solve([mine] + others)
    r = res[0]
    assert r["status"] == ca.CA_OK and r["h_done"] == alone["h_done"]
    assert r["bound"] is not None and r["bound"] <= tol
    assert abs(r["gap"] - alone["gap"]) <= 1e-3 * alone["gap"]
    assert _rel(wb, w) < TOL32
    for p, q in zip(others, res[1:]):
        assert q["h_done"] == p["H"] and q["bound"] is None
