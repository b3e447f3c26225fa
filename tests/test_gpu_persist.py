"""CUDA path vs the FP64 oracle (GB300, through the C ABI): the persistent
launch of consecutive outer steps, in which the s unrolled solves of step k
(eq. "recur", Algorithms 2 / 4) run while the Gram pass of step k+1 already
streams its rows, and that pass corrects the projection of its first columns
by the cross Gram C = Y_{k+1,A} Y_{k,A}^T:
    p_{k+1} = Y_{k+1,A} v_k[A] - cU C Delta_k + Y_{k+1,B} v_{k+1}[B],
the same sum as Y_{k+1} v_{k+1} in exact arithmetic (Sec. 3.1's deferred
update v_{k+1} = v_k - cU Y_k^T Delta_k).

Each case runs the same solve with the persistent launches (at several
overlaps: 0 = no region A, the default, all columns in region A) and with one
launch per step, and compares both with the oracle at the FP32-path
tolerance 1e-5, and with each other at 2e-6 (they differ only in the
rounding of the Gram sums of region A's correction: BF16x3 carries 3 2^-16
of |x||y| per product, scaled FP16 2^-10 -- those runs stay within the
FP32-path tolerance of the exact path, not within FP64 rounding).  The
problems have K >= 32768 so that every Gram CTA owns more atoms than its load
ring holds (region A is used).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import synth  # noqa: E402

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1612_04003_gb300 as ca
    ca.build()
    c = ca.Context(0)
    yield c
    c.ca_set_tuning(persistent=True, overlap=0.4)
    c.close()


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda().contiguous()


def _rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    b = b.detach().cpu().numpy() if hasattr(b, "detach") else np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def primal():
    """X 256 x 32768 FP32 (cond 1e3 rows), lambda 1e-4."""
    m = synth.dense_primal(d=256, n=32768, cond=1e3, seed=11)
    X32 = np.ascontiguousarray(m.X[:, :32768]).astype(np.float32)
    return X32, m.y[:32768].copy()


def _launches(ctx, fn):
    """Kernels the solve in fn launched (the profiling hooks' count)."""
    ctx.ca_profile_enable(True)
    fn()
    n = ctx.ca_profile_read()["kernel_launches"]
    ctx.ca_profile_enable(False)
    return n


def _primal_run(ctx, X, y, *, persistent, overlap=0.4, **kw):
    ctx.ca_set_tuning(persistent=persistent, overlap=overlap)
    w = torch.zeros(X.shape[0], dtype=torch.float64, device="cuda")
    z = torch.zeros(X.shape[1], dtype=torch.float64, device="cuda")
    n = _launches(ctx, lambda: ctx.ca_bcd_solve(_dev(X), _dev(y), w, z, **kw))
    ctx.ca_set_tuning(persistent=True, overlap=0.4)
    return w, z, n


@pytest.mark.parametrize("prec", ["bf16x3", "fp16_scaled"])
def test_persistent_primal_equals_per_step_and_oracle(ctx, primal, prec):
    X, y = primal
    kw = dict(b=8, s=16, H=512, lam=1e-4, seed=42, prec=prec)
    w_ref, z_ref = oracle.ca_bcd(X.astype(np.float64), y, 1e-4, b=8, s=16, H=512, seed=42)
    w1, z1, n1 = _primal_run(ctx, X, y, persistent=False, **kw)
    for ov in (0.0, 0.4, 1.0):
        w, z, n = _primal_run(ctx, X, y, persistent=True, overlap=ov, **kw)
        assert n < n1 / 4  # (32 outer steps: a handful of launches instead of 2 per step)
        print(f"{prec} overlap {ov}: oracle w {_rel(w, w_ref):.2e} z {_rel(z, z_ref):.2e}, "
              f"per-step w {_rel(w, w1):.2e}")
        assert _rel(w, w_ref) < TOL32 and _rel(z, z_ref) < TOL32
        assert _rel(w, w1) < 2e-6 and _rel(z, z1) < 2e-6


def test_persistent_runs_split_by_checks_recompute_and_short_step(ctx, primal):
    """Runs end at every check (stopping test every 3 outer steps), before
    every due recomputation (every 5) and before the short last step
    (H = 500 = 31 * 16 + 4)."""
    X, y = primal
    kw = dict(b=8, s=16, H=500, lam=1e-4, seed=7, prec="bf16x3", recompute_every=5,
              check_every=3, tol=0.0)
    w, z, n = _primal_run(ctx, X, y, persistent=True, **kw)
    w_ref, z_ref = oracle.ca_bcd(X.astype(np.float64), y, 1e-4, b=8, s=16, H=500, seed=7,
                                 recompute_every=5)
    w1, _, n1 = _primal_run(ctx, X, y, persistent=False, **kw)
    assert n < n1
    print(f"checks/recompute: oracle {_rel(w, w_ref):.2e}, per-step {_rel(w, w1):.2e}")
    assert _rel(w, w_ref) < TOL32 and _rel(z, z_ref) < TOL32
    assert _rel(w, w1) < 2e-6


@pytest.fixture(scope="module")
def dual():
    p = synth.dense_dual(d=65536, n=512, seed=5)
    return p.X.astype(np.float32), p.y


@pytest.mark.parametrize("b,s", [(8, 8), (4, 16), (2, 16)])
def test_persistent_dual_dense(ctx, dual, b, s):
    """Dual CA-BDCD on FP32 X^T 512 x 65536 (A = X^T, N = n = 512 rows,
    K = d = 65536): s*b = 64 and 32 (smaller tiles), b < 8."""
    X32, y = dual
    kw = dict(b=b, s=s, H=24 * s, lam=1e-2, seed=3, prec="bf16x3")

    def run(persistent):
        ctx.ca_set_tuning(persistent=persistent)
        a = torch.zeros(512, dtype=torch.float64, device="cuda")
        w = torch.zeros(65536, dtype=torch.float64, device="cuda")
        n = _launches(ctx, lambda: ctx.ca_bdcd_solve(_dev(X32.T), _dev(y), a, w, **kw))
        ctx.ca_set_tuning(persistent=True)
        return a, w, n

    a, w, n = run(True)
    a1, w1, n1 = run(False)
    a_ref, w_ref = oracle.ca_bdcd(X32.astype(np.float64), y, 1e-2, b=b, s=s, H=24 * s, seed=3)
    print(f"dual b={b} s={s}: oracle a {_rel(a, a_ref):.2e} w {_rel(w, w_ref):.2e}, "
          f"per-step a {_rel(a, a1):.2e}; launches {n} vs {n1}")
    assert n < n1 / 4
    assert _rel(a, a_ref) < TOL32 and _rel(w, w_ref) < TOL32
    assert _rel(a, a1) < 2e-6 and _rel(w, w1) < 2e-6


def test_tuning_refuses_bad_values(ctx):
    import paper_1612_04003_gb300 as ca
    for kw in (dict(overlap=1.5), dict(overlap=-0.1)):
        with pytest.raises(ca.CaError) as e:
            ctx.ca_set_tuning(**kw)
        assert e.value.status == ca.CA_ERR_ARG
