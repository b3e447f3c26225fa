"""CUDA path vs the FP64 oracle, through the C ABI (GB300).

Element-wise comparisons on the same seeded inputs.  Tolerances (relative
2-norm error of the iterates after H block updates):
  * 1e-10 for FP64 X with the FP64 Gram;
  * 1e-5  for FP32 X with the 3xTF32 and the BF16x3 tensor-core Gram (FP32
    products in the projection / update, FP64 vectors and solves).  3xTF32
    drops terms below ~2^-20 |x||y| per product; BF16x3 (x = b0 + b1 in
    BF16, unit roundoff 2^-8) drops b1 c1 and the split remainders, at most
    3 * 2^-16 |x||y| per product (random signs keep the Gram entries near
    3e-6 sqrt(G_ii G_jj)), and the iterates (measured 2e-7 .. 4e-6 on these
    cases) stay inside the FP32 bound;
  * TF32 Gram (inputs rounded to 11 significant bits) and the scaled FP16
    Gram (each row times a power of two, rounded to FP16's 11 significant
    bits; the scales come off exactly): each Gram entry is off
    by ~2^-11 relative, which perturbs the path of the iteration but not its
    fixed point (the projection and vectors stay FP32/FP64-accurate).  The
    deviation from the exact path is ~1e-3 after a few sweeps and decays as
    the iteration converges: held to 2e-3 at H = 256 on the mid-size problem
    and to 1e-5 once converged (H = 2048).
Sampled indices must match bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import synth  # noqa: E402

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-5
TOL_TF32_SHORT = 2e-3


def _tol(prec):
    return {"3xtf32": TOL32, "bf16x3": TOL32, "tf32": TOL_TF32_SHORT,
            "fp16_scaled": TOL_TF32_SHORT}[prec]


def _rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1612_04003_gb300 as ca
    ca.build()
    c = ca.Context(0)
    yield c
    c.close()


def _dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda().contiguous()


# ---------------------------------------------------------------------------
# a1 sampler: bit-exact against the oracle's implementation
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed,h0,H,b,N", [
    (42, 0, 200, 4, 64), (1, 12345, 64, 8, 4096), (7, 2**40, 16, 3, 10), (9, 0, 5, 64, 64),
    (3, 5, 40, 37, 100), (11, 0, 3, 1, 1), (2024, 77, 50, 128, 131072), (5, 0, 4, 300, 301)])
def test_sampler_bit_exact(ctx, seed, h0, H, b, N):
    out = torch.empty((H, b), dtype=torch.int32, device="cuda")
    ctx.ca_sample_indices(seed, h0, H, b, N, out)
    ref = oracle.sample_blocks(seed, h0, H, b, N)
    assert np.array_equal(out.cpu().numpy(), ref)


def test_sampler_host_output(ctx):
    out = np.zeros((10, 8), dtype=np.int32)
    ctx.ca_sample_indices(42, 3, 10, 8, 4096, out)
    assert np.array_equal(out, oracle.sample_blocks(42, 3, 10, 8, 4096))


# ---------------------------------------------------------------------------
# Primal CA-BCD, FP64 X (tiny dense workload: X 64 x 1024, lambda 1e-3, b 4, H 200)
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def tiny():
    return synth.tiny_primal(d=64, n=1024, seed=1)


@pytest.mark.parametrize("s", [1, 4, 7, 16])
def test_primal_f64_tiny(ctx, tiny, s):
    X, y = _dev(tiny.X), _dev(tiny.y)
    w = torch.zeros(64, dtype=torch.float64, device="cuda")
    z = torch.zeros(1024, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(X, y, w, z, b=4, s=s, H=200, lam=1e-3, seed=42, prec="f64")
    w_ref, z_ref = oracle.ca_bcd(tiny.X, tiny.y, 1e-3, b=4, s=s, H=200, seed=42)
    assert _rel(w, w_ref) < TOL64
    assert _rel(z, z_ref) < TOL64


def test_primal_f64_full_block_is_closed_form(ctx, tiny):
    X, y = _dev(tiny.X), _dev(tiny.y)
    w = torch.zeros(64, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(X, y, w, b=64, s=1, H=1, lam=1e-3, seed=42, prec="f64")
    assert _rel(w, oracle.closed_form(tiny.X, tiny.y, 1e-3)) < 1e-10


def test_primal_f64_repeats_short_last_step_resume(ctx, tiny):
    """Indices repeating across blocks (b = 40 of d = 64), H not a multiple of
    s, a non-zero w0 / h0, and periodic recomputation."""
    X, y = _dev(tiny.X), _dev(tiny.y)
    w0 = np.random.default_rng(3).standard_normal(64)
    w = _dev(w0)
    ctx.ca_bcd_solve(X, y, w, b=40, s=6, H=31, lam=1e-3, seed=3, h0=17, prec="f64",
                     recompute_every=2)
    w_ref, _ = oracle.ca_bcd(tiny.X, tiny.y, 1e-3, b=40, s=6, H=31, seed=3, h0=17, w0=w0,
                             recompute_every=2)
    assert _rel(w, w_ref) < TOL64


def test_primal_f64_ragged_ld(ctx):
    """n not a multiple of the 32-column chunk, leading dimension > n, sb
    spanning several 64-row tiles."""
    p = synth.dense_primal(d=200, n=1500, cond=1e2, seed=4, dtype=np.float64)
    ld = 1537
    Xp = np.zeros((200, ld))
    Xp[:, :1500] = p.X
    X = _dev(Xp)
    y = _dev(p.y)
    w = torch.zeros(200, dtype=torch.float64, device="cuda")
    z = torch.zeros(1500, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(X[:, :1500].contiguous(), y, w, z, b=10, s=15, H=120, lam=1e-3, seed=8,
                     prec="f64")
    w_ref, z_ref = oracle.ca_bcd(p.X, p.y, 1e-3, b=10, s=15, H=120, seed=8)
    assert _rel(w, w_ref) < TOL64 and _rel(z, z_ref) < TOL64
    # the same through an explicit leading dimension
    w2 = torch.zeros(200, dtype=torch.float64, device="cuda")
    import paper_1612_04003_gb300 as ca
    o = ca.Context._opts(10, 15, 120, 1e-3, 8, "f64", 0, 0)
    import ctypes
    st = ctx._lib.ca_bcd_solve(ctx.handle, ca.CA_DENSE_F64, X.data_ptr(), 200, 1500, ld,
                               y.data_ptr(), ctypes.byref(o), w2.data_ptr(), None)
    assert st == 0
    assert _rel(w2, w_ref) < TOL64


# ---------------------------------------------------------------------------
# Primal CA-BCD, FP32 X, tensor-core Gram (TF32 and 3xTF32)
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def mid32():
    """Dense primal, geometric row scaling (cond 1e3), lambda 1e-4; n with a
    ragged 32-column tail."""
    return synth.dense_primal(d=512, n=8205, cond=1e3, seed=2)


@pytest.mark.parametrize("prec", ["tf32", "3xtf32", "bf16x3", "fp16_scaled"])
@pytest.mark.parametrize("b,s", [(8, 1), (8, 4), (8, 13), (8, 16), (8, 17), (8, 32), (32, 4),
                                 (32, 8), (3, 7)])
def test_primal_f32_tc(ctx, mid32, prec, b, s):
    X64 = mid32.X.astype(np.float64)
    d, n = mid32.X.shape
    # keep the leading dimension a multiple of 4 (16-byte rows for cp.async)
    ld = (n + 3) // 4 * 4
    Xp = np.zeros((d, ld), dtype=np.float32)
    Xp[:, :n] = mid32.X
    X = _dev(Xp)
    y = _dev(mid32.y)
    w = torch.zeros(d, dtype=torch.float64, device="cuda")
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    H = 256
    ctx.ca_bcd_solve(X, y, w, z, b=b, s=s, H=H, lam=1e-4, seed=42, prec=prec, n=n)
    w_ref, z_ref = oracle.ca_bcd(X64, mid32.y, 1e-4, b=b, s=s, H=H, seed=42)
    tol = _tol(prec)
    print(f"mid32 {prec} b={b} s={s}: w {_rel(w, w_ref):.3e} z {_rel(z, z_ref):.3e}")
    assert _rel(w, w_ref) < tol
    assert _rel(z, z_ref) < tol


@pytest.mark.parametrize("prec", ["tf32", "bf16x3", "fp16_scaled"])
@pytest.mark.parametrize("s", [8, 32])
def test_primal_tf32_converged(ctx, mid32, s, prec):
    """TF32 Gram: once the iteration has converged (H = 2048, 32 sweeps of
    d = 512) the iterates agree with the oracle's Algorithm 1 to 1e-5."""
    X = _dev(mid32.X[:, :8192])
    y = _dev(mid32.y[:8192])
    w = torch.zeros(512, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(X, y, w, b=8, s=s, H=2048, lam=1e-4, seed=7, prec=prec)
    w_ref, _ = oracle.bcd(mid32.X[:, :8192].astype(np.float64), mid32.y[:8192], 1e-4, b=8,
                          H=2048, seed=7)
    print(f"converged {prec} s={s}: w {_rel(w, w_ref):.3e}")
    assert _rel(w, w_ref) < TOL32


@pytest.fixture(scope="module")
def long_k():
    """d = 512 features, n = 262144 samples: every CTA streams ~54 32-column
    stages, more than any stage ring holds (deep-pipeline paths)."""
    return synth.dense_primal(d=512, n=262144, cond=1e3, seed=5)


@pytest.fixture(scope="module")
def long_k_oracle(long_k):
    w_ref, z_ref = oracle.bcd(long_k.X.astype(np.float64), long_k.y, 1e-4, b=8, H=256, seed=3)
    return w_ref, z_ref


@pytest.mark.parametrize("prec,s", [("3xtf32", 16), ("3xtf32", 8), ("3xtf32", 32), ("3xtf32", 3),
                                    ("tf32", 16), ("tf32", 32), ("tf32", 4),
                                    ("bf16x3", 16), ("bf16x3", 32), ("bf16x3", 5),
                                    ("fp16_scaled", 16), ("fp16_scaled", 32)])
def test_primal_f32_long_k(ctx, long_k, long_k_oracle, prec, s):
    """Fused update (s*b <= 128) and the plain Gram pass with deep stage rings,
    against the oracle's Algorithm 1 (s = 1)."""
    X, y = _dev(long_k.X), _dev(long_k.y)
    w = torch.zeros(512, dtype=torch.float64, device="cuda")
    z = torch.zeros(262144, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(X, y, w, z, b=8, s=s, H=256, lam=1e-4, seed=3, prec=prec)
    w_ref, z_ref = long_k_oracle
    print(f"long_k {prec} s={s}: w {_rel(w, w_ref):.3e} z {_rel(z, z_ref):.3e}")
    assert _rel(w, w_ref) < _tol(prec) and _rel(z, z_ref) < _tol(prec)


def test_primal_f32_simt_f64_gram(ctx, mid32):
    X = _dev(mid32.X)
    d, n = mid32.X.shape
    y = _dev(mid32.y)
    w = torch.zeros(d, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(X, y, w, b=8, s=8, H=128, lam=1e-4, seed=42, prec="f64")
    w_ref, _ = oracle.ca_bcd(mid32.X.astype(np.float64), mid32.y, 1e-4, b=8, s=8, H=128, seed=42)
    assert _rel(w, w_ref) < TOL32


def test_primal_tc_s_equals_1_iterates(ctx, mid32):
    """Sec. 3.1: CA-BCD (s = 16) and BCD (s = 1) give the same iterates up to
    rounding on the device as well."""
    X = _dev(mid32.X[:, :8192])
    y = _dev(mid32.y[:8192])
    outs = []
    for s in (1, 16):
        w = torch.zeros(512, dtype=torch.float64, device="cuda")
        ctx.ca_bcd_solve(X, y, w, b=8, s=s, H=256, lam=1e-4, seed=5, prec="3xtf32")
        outs.append(w.cpu().numpy())
    assert _rel(outs[1], outs[0]) < TOL32


def test_primal_host_buffers_match_device(ctx, mid32):
    """Host (numpy) arrays are staged by the library: same result."""
    Xh = np.ascontiguousarray(mid32.X[:, :8192])
    yh = np.ascontiguousarray(mid32.y[:8192])
    wh = np.zeros(512)
    zh = np.zeros(8192)
    ctx.ca_bcd_solve(Xh, yh, wh, zh, b=8, s=8, H=128, lam=1e-4, seed=5, prec="3xtf32")
    w = torch.zeros(512, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(_dev(Xh), _dev(yh), w, b=8, s=8, H=128, lam=1e-4, seed=5, prec="3xtf32")
    assert np.array_equal(wh, w.cpu().numpy())
    w_ref, z_ref = oracle.ca_bcd(Xh.astype(np.float64), yh, 1e-4, b=8, s=8, H=128, seed=5)
    assert _rel(wh, w_ref) < TOL32 and _rel(zh, z_ref) < TOL32


def test_pinned_host_x_is_read_in_place(ctx, mid32):
    """Page-locked host X is repacked straight from host memory (no staging
    copy): the iterates equal those of the device-resident X, primal and dual."""
    d, n = 512, 8192
    Xh = torch.from_numpy(np.ascontiguousarray(mid32.X[:, :n])).pin_memory()
    y = _dev(np.ascontiguousarray(mid32.y[:n]))
    kw = dict(b=8, s=8, H=128, lam=1e-4, seed=5, prec="3xtf32")
    w_host = torch.zeros(d, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(Xh, y, w_host, **kw)
    w_dev = torch.zeros(d, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(Xh.cuda(), y, w_dev, **kw)
    assert _rel(w_host, w_dev.cpu().numpy()) < 1e-12
    XTh = torch.from_numpy(np.ascontiguousarray(mid32.X[:64, :1024].T)).pin_memory()  # 1024 x 64
    ys = _dev(np.ascontiguousarray(mid32.y[:1024]))
    kw2 = dict(b=8, s=4, H=64, lam=1e-2, seed=2, prec="3xtf32")
    a1 = torch.zeros(1024, dtype=torch.float64, device="cuda")
    w1 = torch.zeros(64, dtype=torch.float64, device="cuda")
    ctx.ca_bdcd_solve(XTh, ys, a1, w1, **kw2)
    a2 = torch.zeros(1024, dtype=torch.float64, device="cuda")
    w2 = torch.zeros(64, dtype=torch.float64, device="cuda")
    ctx.ca_bdcd_solve(XTh.cuda(), ys, a2, w2, **kw2)
    assert _rel(a1, a2.cpu().numpy()) < 1e-12 and _rel(w1, w2.cpu().numpy()) < 1e-12


# ---------------------------------------------------------------------------
# Dual CA-BDCD
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def wide():
    return synth.dense_dual(d=300, n=120, seed=4)


@pytest.mark.parametrize("s", [1, 5, 13])
def test_dual_dense_f64(ctx, wide, s):
    XT = _dev(wide.X.T)
    y = _dev(wide.y)
    a = torch.zeros(120, dtype=torch.float64, device="cuda")
    w = torch.zeros(300, dtype=torch.float64, device="cuda")
    ctx.ca_bdcd_solve(XT, y, a, w, b=6, s=s, H=150, lam=1e-2, seed=9, prec="f64")
    a_ref, w_ref = oracle.ca_bdcd(wide.X, wide.y, 1e-2, b=6, s=s, H=150, seed=9)
    assert _rel(a, a_ref) < TOL64 and _rel(w, w_ref) < TOL64


def test_dual_dense_f64_full_block(ctx, wide):
    XT = _dev(wide.X.T)
    y = _dev(wide.y)
    a = torch.zeros(120, dtype=torch.float64, device="cuda")
    w = torch.zeros(300, dtype=torch.float64, device="cuda")
    ctx.ca_bdcd_solve(XT, y, a, w, b=120, s=1, H=1, lam=1e-2, seed=1, prec="f64")
    X = wide.X
    wstar = np.linalg.solve(X @ X.T / 120 + 1e-2 * np.eye(300), X @ wide.y / 120)
    assert _rel(w, wstar) < 1e-9
    assert _rel(a, X.T @ wstar - wide.y) < 1e-9


@pytest.mark.parametrize("prec", ["tf32", "3xtf32", "bf16x3", "fp16_scaled"])
def test_dual_dense_f32_tc(ctx, prec):
    p = synth.dense_dual(d=1028, n=400, seed=6)
    X32 = p.X.astype(np.float32)
    XT = _dev(np.ascontiguousarray(X32.T))
    y = _dev(p.y)
    a = torch.zeros(400, dtype=torch.float64, device="cuda")
    w = torch.zeros(1028, dtype=torch.float64, device="cuda")
    ctx.ca_bdcd_solve(XT, y, a, w, b=8, s=16, H=256, lam=1e-2, seed=2, prec=prec)
    a_ref, w_ref = oracle.ca_bdcd(X32.astype(np.float64), p.y, 1e-2, b=8, s=16, H=256, seed=2)
    print(f"dual {prec}: a {_rel(a, a_ref):.3e} w {_rel(w, w_ref):.3e}")
    assert _rel(a, a_ref) < _tol(prec) and _rel(w, w_ref) < _tol(prec)


# ---------------------------------------------------------------------------
# 32-column panel storage of X (the tensor-core path reads X this way)
# ---------------------------------------------------------------------------
def _panels_ref(A, K):
    """Panels of the first K columns of A by their definition:
    out[a, r, c] = A[r, 32 a + c], zero where 32 a + c >= K."""
    N = A.shape[0]
    na = (K + 31) // 32
    out = np.zeros((na, N, 32), dtype=np.float32)
    for a in range(na):
        w = min(32, K - 32 * a)
        out[a, :, :w] = A[:, 32 * a:32 * a + w]
    return out.reshape(-1)


@pytest.mark.parametrize("N,K,ld", [(1, 1, 4), (37, 77, 80), (300, 1024, 1024), (5, 33, 36),
                                    (3, 4100, 4100)])
def test_pack_panels_layout(ctx, N, K, ld):
    rng = np.random.default_rng(N + K)
    A = rng.standard_normal((N, ld)).astype(np.float32)
    out = torch.full(((K + 31) // 32 * N * 32,), float("nan"), dtype=torch.float32, device="cuda")
    ctx.ca_pack_panels(_dev(A), out, K=K)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), _panels_ref(A, K))


def test_primal_prepacked_panels_match(ctx, mid32):
    """X handed over already packed gives the iterates of the row-major X that
    the solve packs itself (same kernels on the same panels; only the
    order of FP64 atomic additions may differ)."""
    d, n = mid32.X.shape
    ld = (n + 3) // 4 * 4
    Xp = np.zeros((d, ld), dtype=np.float32)
    Xp[:, :n] = mid32.X
    X = _dev(Xp)
    y = _dev(mid32.y)
    kw = dict(b=8, s=16, H=128, lam=1e-4, seed=3, prec="3xtf32")
    w1 = torch.zeros(d, dtype=torch.float64, device="cuda")
    z1 = torch.zeros(n, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(X, y, w1, z1, n=n, **kw)
    P = torch.empty(((n + 31) // 32 * d * 32,), dtype=torch.float32, device="cuda")
    ctx.ca_pack_panels(X, P, K=n)
    w2 = torch.zeros(d, dtype=torch.float64, device="cuda")
    z2 = torch.zeros(n, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(P, y, w2, z2, panels=(d, n), **kw)
    assert _rel(w2, w1.cpu().numpy()) < 1e-12 and _rel(z2, z1.cpu().numpy()) < 1e-12
    import paper_1612_04003_gb300 as ca
    with pytest.raises(ca.CaError) as ei:  # panels need a tensor-core Gram mode
        ctx.ca_bcd_solve(P, y, w2, panels=(d, n), b=8, s=4, H=8, lam=1e-4, prec="f64")
    assert ei.value.status == ca.CA_ERR_ARG


def test_dual_prepacked_panels_match(ctx):
    p = synth.dense_dual(d=1028, n=400, seed=6)
    XT = _dev(np.ascontiguousarray(p.X.astype(np.float32).T))
    y = _dev(p.y)
    kw = dict(b=8, s=16, H=256, lam=1e-2, seed=2, prec="3xtf32")
    a1 = torch.zeros(400, dtype=torch.float64, device="cuda")
    w1 = torch.zeros(1028, dtype=torch.float64, device="cuda")
    ctx.ca_bdcd_solve(XT, y, a1, w1, **kw)
    P = torch.empty(((1028 + 31) // 32 * 400 * 32,), dtype=torch.float32, device="cuda")
    ctx.ca_pack_panels(XT, P)
    a2 = torch.zeros(400, dtype=torch.float64, device="cuda")
    w2 = torch.zeros(1028, dtype=torch.float64, device="cuda")
    ctx.ca_bdcd_solve(P, y, a2, w2, panels=(400, 1028), **kw)
    assert _rel(a2, a1.cpu().numpy()) < 1e-12 and _rel(w2, w1.cpu().numpy()) < 1e-12


@pytest.fixture(scope="module")
def sparse_small():
    return synth.sparse_dual(d=4000, n=600, density=0.01, seed=3)


# (s*b >= 128 runs the diagonal-block inverses on the second stream and the
# chain alone on the library stream: b = 8, 13, 16 there)
@pytest.mark.parametrize("b,s", [(8, 1), (8, 8), (8, 32), (5, 3), (16, 8), (13, 12), (16, 16)])
def test_dual_csr(ctx, sparse_small, b, s):
    sp = sparse_small
    rp, col, val = _dev(sp.rowptr), _dev(sp.col), _dev(sp.val)
    y = _dev(sp.y)
    a = torch.zeros(sp.n, dtype=torch.float64, device="cuda")
    w = torch.zeros(sp.d, dtype=torch.float64, device="cuda")
    ctx.ca_bdcd_solve((rp, col, val), y, a, w, b=b, s=s, H=96, lam=1e-3, seed=4, d=sp.d)
    A = oracle.CSR(sp.rowptr, sp.col, sp.val.astype(np.float64), sp.d)
    a_ref, w_ref = oracle.ca_bdcd(A, sp.y, 1e-3, b=b, s=s, H=96, seed=4)
    assert _rel(a, a_ref) < TOL64 and _rel(w, w_ref) < TOL64


def test_dual_csr_host_arrays_and_recompute(ctx, sparse_small):
    sp = sparse_small
    a = np.zeros(sp.n)
    w = np.zeros(sp.d)
    ctx.ca_bdcd_solve((sp.rowptr, sp.col, sp.val), sp.y, a, w, b=8, s=8, H=96, lam=1e-3, seed=4,
                      d=sp.d, recompute_every=3)
    A = oracle.CSR(sp.rowptr, sp.col, sp.val.astype(np.float64), sp.d)
    a_ref, w_ref = oracle.ca_bdcd(A, sp.y, 1e-3, b=8, s=8, H=96, seed=4, recompute_every=3)
    assert _rel(a, a_ref) < TOL64 and _rel(w, w_ref) < TOL64


# ---------------------------------------------------------------------------
# Error paths
# ---------------------------------------------------------------------------
def test_errors(ctx, tiny):
    import paper_1612_04003_gb300 as ca
    X, y = _dev(tiny.X), _dev(tiny.y)
    w = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(ca.CaError) as e:
        ctx.ca_bcd_solve(X, y, w, b=65, s=1, H=10, lam=1e-3)
    assert e.value.status == ca.CA_ERR_ARG
    with pytest.raises(ca.CaError) as e:
        ctx.ca_bcd_solve(X, y, w, b=4, s=1, H=10, lam=0.0)
    assert e.value.status == ca.CA_ERR_ARG
    with pytest.raises(ca.CaError) as e:
        ctx.ca_bcd_solve(X, y, w, b=4, s=1, H=0, lam=1e-3)
    assert e.value.status == ca.CA_ERR_ARG
    X32 = X.float().contiguous()
    with pytest.raises(ca.CaError) as e:  # s*b beyond the tensor-core tile
        ctx.ca_bcd_solve(X32, y, w, b=32, s=9, H=288, lam=1e-3, prec="tf32")
    assert e.value.status == ca.CA_ERR_UNSUPPORTED
    Xbad = X.clone()
    Xbad[:, 5] = float("nan")
    with pytest.raises(ca.CaError) as e:
        ctx.ca_bcd_solve(Xbad, y, w, b=64, s=1, H=1, lam=1e-3, prec="f64")
    assert e.value.status in (ca.CA_ERR_NONFINITE, ca.CA_ERR_NOT_SPD)
    # the context stays usable after errors
    w = torch.zeros(64, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(X, y, w, b=4, s=4, H=200, lam=1e-3, seed=42, prec="f64")
    w_ref, _ = oracle.ca_bcd(tiny.X, tiny.y, 1e-3, b=4, s=4, H=200, seed=42)
    assert _rel(w, w_ref) < TOL64


def test_bounded_wait_times_out_and_context_survives(ctx, tiny):
    import paper_1612_04003_gb300 as ca
    assert ctx.ca_selftest_wait_timeout(50_000_000) == ca.CA_ERR_TIMEOUT
    X, y = _dev(tiny.X), _dev(tiny.y)
    w = torch.zeros(64, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(X, y, w, b=4, s=4, H=40, lam=1e-3, seed=42, prec="f64")
    w_ref, _ = oracle.ca_bcd(tiny.X, tiny.y, 1e-3, b=4, s=4, H=40, seed=42)
    assert _rel(w, w_ref) < TOL64


# ---------------------------------------------------------------------------
# a2+a3 alone: Gram matrix and projection of given rows vs a float64 reference
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def gram_data():
    rng = np.random.default_rng(17)
    N, K = 700, 8205                      # K has a ragged 32-column tail
    ld = 8208
    A = np.zeros((N, ld), dtype=np.float32)
    A[:, :K] = (rng.standard_normal((N, K)) * (10.0 ** rng.uniform(-2, 1, size=(N, 1)))).astype(
        np.float32)
    v = rng.standard_normal(K)
    return A, K, ld, v


# Gram tolerances relative to sqrt(G_ii G_jj): FP64 rounding; 3xTF32: the
# dropped lo*lo term (2^-22) plus FP32 accumulation of up to ~1000 same-sign
# terms per split (1000 * 2^-24 ~ 6e-5 worst case, 2e-5 used); TF32: 2^-11
# input rounding; BF16x3: the dropped b1 c1 and split remainders, 3 * 2^-16
# ~ 4.6e-5 (unit roundoff 2^-8; Cauchy-Schwarz over the sum), plus the same
# FP32 accumulation allowance: 1e-4; scaled FP16: each scaled element rounded to 11
# significant bits (2^-11 relative), a product within ~2^-10, as TF32: 3e-3.
@pytest.mark.parametrize("prec,tolG,tolp", [("f64", 1e-13, 1e-13), ("3xtf32", 2e-5, 1e-6),
                                            ("tf32", 3e-3, 1e-6), ("bf16x3", 1e-4, 1e-6),
                                            ("fp16_scaled", 3e-3, 1e-6)])
@pytest.mark.parametrize("sb", [1, 8, 32, 100, 128, 129, 136, 256])
def test_gram_project_kernel(ctx, gram_data, prec, tolG, tolp, sb):
    A, K, ld, v = gram_data
    rng = np.random.default_rng(sb)
    idx = rng.integers(0, A.shape[0], size=sb).astype(np.int32)  # repeats allowed
    if sb > 4:
        idx[3] = idx[1]
    Ad, idx_d, v_d = _dev(A), _dev(idx), _dev(v)   # keep the device arrays alive
    G = torch.zeros((sb, sb), dtype=torch.float64, device="cuda")
    p = torch.zeros(sb, dtype=torch.float64, device="cuda")
    import paper_1612_04003_gb300 as ca
    st = ctx._lib.ca_gram_project(ctx.handle, ca.CA_DENSE_F32, ca.PREC[prec], Ad.data_ptr(),
                                  A.shape[0], K, ld, idx_d.data_ptr(), sb, v_d.data_ptr(),
                                  G.data_ptr(), p.data_ptr())
    assert st == 0, ca.status_str(st)
    Y = A[idx, :K].astype(np.float64)
    G_ref = Y @ Y.T
    p_ref = Y @ v
    nrm = np.sqrt(np.diag(G_ref))
    Gerr = np.abs(G.cpu().numpy() - G_ref) / np.outer(nrm, nrm)
    print(f"gram {prec} sb={sb}: G {Gerr.max():.3e}")
    assert Gerr.max() < tolG, Gerr.max()
    perr = np.abs(p.cpu().numpy() - p_ref) / (nrm * np.linalg.norm(v))
    assert perr.max() < tolp, perr.max()


@pytest.mark.parametrize("prec", ["fp16_scaled", "bf16x3"])
def test_gram_project_wide_magnitudes(ctx, prec):
    """Rows whose magnitudes span 1e-12 .. 1e12 (far outside FP16's range of
    6e-8 .. 65504 unscaled): the per-row power-of-two scaling keeps every
    entry within the bound of the mode."""
    rng = np.random.default_rng(5)
    N, K = 96, 4104  # the last 4 columns zero (a ragged 32-column tail)
    A = np.zeros((N, K), dtype=np.float32)
    A[:, :4100] = (rng.standard_normal((N, 4100)) *
                   (10.0 ** rng.uniform(-12, 12, size=(N, 1)))).astype(np.float32)
    v = np.zeros(K)
    v[:4100] = rng.standard_normal(4100)
    idx = rng.permutation(N)[:64].astype(np.int32)
    Ad, idx_d, v_d = _dev(A), _dev(idx), _dev(v)
    G = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    p = torch.zeros(64, dtype=torch.float64, device="cuda")
    ctx.ca_gram_project(Ad, idx_d, v_d, G, p, prec=prec)
    Y = A[idx].astype(np.float64)
    G_ref = Y @ Y.T
    nrm = np.sqrt(np.diag(G_ref))
    Gerr = np.abs(G.cpu().numpy() - G_ref) / np.outer(nrm, nrm)
    assert np.isfinite(G.cpu().numpy()).all()
    assert Gerr.max() < (3e-3 if prec == "fp16_scaled" else 1e-4), Gerr.max()


def test_noalloc_refuses_scaled_fp16(ctx, gram_data):
    """The fixed-scratch entry has no room for per-row scales."""
    import paper_1612_04003_gb300 as ca
    A, K, ld, v = gram_data
    Ad, v_d = _dev(A), _dev(v)
    idx_d = _dev(np.arange(8, dtype=np.int32))
    G = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    p = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = ctx._lib.ca_gram_project_noalloc(None, ca.CA_DENSE_F32, ca.CA_GRAM_FP16_SCALED,
                                          Ad.data_ptr(), A.shape[0], K, ld, idx_d.data_ptr(), 8,
                                          v_d.data_ptr(), G.data_ptr(), p.data_ptr())
    assert st == ca.CA_ERR_UNSUPPORTED


# ---------------------------------------------------------------------------
# Stopping test (Sec. 5.1.5): full residuals every check_every outer steps,
# the early end once ||r|| <= tol ||r_0||
# ---------------------------------------------------------------------------
def _tol_between(norms, r0, gap=1.1):
    """A tolerance whose first crossing is unambiguous: between two checks
    j, j+1 with norms[j+1] < norms[j] / gap and every earlier norm above."""
    for j in range(1, len(norms) - 1):
        if norms[j + 1] * gap < norms[j] and min(norms[:j + 1]) > norms[j + 1] * gap:
            return float(np.sqrt(norms[j] * norms[j + 1]) / r0), j + 1
    raise AssertionError("no clear crossing")


def test_stopping_primal_f64(ctx, tiny):
    X, y, lam = tiny.X, tiny.y, 1e-3
    kw = dict(b=4, s=4, H=400, seed=42)
    _, _, r0, norms = oracle.ca_bcd_stopped(X, y, lam, tol=0.0, check_every=5, **kw)
    w = torch.zeros(64, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(_dev(X), _dev(y), w, lam=lam, prec="f64", check_every=5, **kw)
    info = ctx.solve_info()
    assert info["h_done"] == 400 and info["checks"] == len(norms) == 20
    assert abs(info["res0"] - r0) < 1e-12 * r0
    assert abs(info["res"] - norms[-1]) < 1e-8 * norms[-1]
    tol, jstop = _tol_between(norms, r0)
    w_ref, h_ref, _, _ = oracle.ca_bcd_stopped(X, y, lam, tol=tol, check_every=5, **kw)
    assert h_ref == 20 * (jstop + 1)
    w = torch.zeros(64, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(_dev(X), _dev(y), w, lam=lam, prec="f64", check_every=5, tol=tol, **kw)
    info = ctx.solve_info()
    assert info["h_done"] == h_ref and info["checks"] == jstop + 1
    assert _rel(w, w_ref) < TOL64


@pytest.mark.parametrize("prec", ["bf16x3", "3xtf32"])
def test_stopping_primal_tensor_core(ctx, mid32, prec):
    """The fused tensor-core path (b = 8, s = 16, s*b = 128): the deferred
    update is applied before each check.  The residual of the GPU's own
    iterate, formed on the CPU in FP64, checks the residual pass itself."""
    X32 = mid32.X[:, :8192]
    X64, y = X32.astype(np.float64), mid32.y[:8192]
    lam = 1e-4
    kw = dict(b=8, s=16, H=1024, seed=7)
    _, _, r0, norms = oracle.ca_bcd_stopped(X64, y, lam, tol=0.0, check_every=2, **kw)
    w = torch.zeros(512, dtype=torch.float64, device="cuda")
    Xd, yd = _dev(X32), _dev(y)
    ctx.ca_bcd_solve(Xd, yd, w, lam=lam, prec=prec, check_every=2, **kw)
    info = ctx.solve_info()
    assert info["h_done"] == 1024 and info["checks"] == len(norms) == 32
    assert abs(info["res0"] - r0) < 1e-6 * r0
    r_own = np.linalg.norm(oracle.primal_residual(X64, y, lam, w.cpu().numpy()))
    assert abs(info["res"] - r_own) < 1e-4 * r_own
    assert abs(info["res"] - norms[-1]) < 1e-3 * norms[-1]
    tol, jstop = _tol_between(norms, r0, gap=1.3)
    w_ref, h_ref, _, _ = oracle.ca_bcd_stopped(X64, y, lam, tol=tol, check_every=2, **kw)
    w = torch.zeros(512, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(Xd, yd, w, lam=lam, prec=prec, check_every=2, tol=tol, **kw)
    info = ctx.solve_info()
    assert info["h_done"] == h_ref and info["checks"] == jstop + 1
    assert _rel(w, w_ref) < TOL32


def test_stopping_dual_dense_and_csr(ctx, wide, sparse_small):
    lam = 1e-2
    X, y = wide.X, wide.y
    d, n = X.shape
    kw = dict(b=6, s=3, H=150, seed=9)
    _, _, _, r0, norms = oracle.ca_bdcd_stopped(X, y, lam, tol=0.0, check_every=5, **kw)
    a = torch.zeros(n, dtype=torch.float64, device="cuda")
    w = torch.zeros(d, dtype=torch.float64, device="cuda")
    XT = _dev(np.ascontiguousarray(X.T))
    ctx.ca_bdcd_solve(XT, _dev(y), a, w, lam=lam, prec="f64", check_every=5, **kw)
    info = ctx.solve_info()
    assert info["h_done"] == 150 and info["checks"] == len(norms) == 10
    assert abs(info["res0"] - r0) < 1e-12 * r0 and abs(info["res"] - norms[-1]) < 1e-8 * norms[-1]
    tol, jstop = _tol_between(norms, r0)
    a_ref, w_ref, h_ref, _, _ = oracle.ca_bdcd_stopped(X, y, lam, tol=tol, check_every=5, **kw)
    a.zero_()
    w.zero_()
    ctx.ca_bdcd_solve(XT, _dev(y), a, w, lam=lam, prec="f64", check_every=5, tol=tol, **kw)
    info = ctx.solve_info()
    assert info["h_done"] == h_ref and _rel(a, a_ref) < TOL64 and _rel(w, w_ref) < TOL64
    # sparse dual (CSR of X^T)
    sp = sparse_small
    A = oracle.CSR(sp.rowptr, sp.col, sp.val.astype(np.float64), sp.d)
    kw = dict(b=8, s=8, H=192, seed=4)
    _, _, _, r0, norms = oracle.ca_bdcd_stopped(A, sp.y, 1e-3, tol=0.0, check_every=3, **kw)
    a = torch.zeros(sp.n, dtype=torch.float64, device="cuda")
    w = torch.zeros(sp.d, dtype=torch.float64, device="cuda")
    csr = (_dev(sp.rowptr), _dev(sp.col), _dev(sp.val))
    ctx.ca_bdcd_solve(csr, _dev(sp.y), a, w, lam=1e-3, d=sp.d, check_every=3, **kw)
    info = ctx.solve_info()
    assert info["h_done"] == 192 and info["checks"] == len(norms) == 8
    assert abs(info["res0"] - r0) < 1e-12 * r0 and abs(info["res"] - norms[-1]) < 1e-8 * norms[-1]


# ---------------------------------------------------------------------------
# Full size, in the configuration bench.py times: X 4096 x 262144 FP32
# (cond 1e3), lambda 1e-4, b = 8, s = 32, H = 4096.  The oracle runs its
# Algorithm 1 (s = 1), which the s-step method reproduces (Sec. 3.1).
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def full_size():
    X, y, _ = synth.dense_primal_torch(4096, 262144, cond=1e3, seed=1, device="cuda")
    yield X, y
    del X


@pytest.fixture(scope="module")
def full_size_oracle(full_size):
    X, y = full_size
    w_ref, z_ref = oracle.bcd(X.cpu().numpy().astype(np.float64), y.cpu().numpy(), 1e-4, b=8,
                              H=4096, seed=42)
    return w_ref, z_ref


@pytest.mark.parametrize("prec,tol,s", [("3xtf32", TOL32, 32), ("3xtf32", TOL32, 16),
                                        ("tf32", TOL_TF32_SHORT, 32), ("tf32", TOL_TF32_SHORT, 16),
                                        ("bf16x3", TOL32, 16), ("bf16x3", TOL32, 32)])
def test_full_size_bench_config(ctx, full_size, full_size_oracle, prec, tol, s):
    """BF16x3 (the benchmarked mode) and 3xTF32 meet 1e-5; TF32 is held to its stated
    bound (8 sweeps of d = 4096 are not enough for its path deviation to
    decay below 1e-5: measured 1.3e-4)."""
    X, y = full_size
    w_ref, z_ref = full_size_oracle
    w = torch.zeros(4096, dtype=torch.float64, device="cuda")
    z = torch.zeros(262144, dtype=torch.float64, device="cuda")
    ctx.ca_bcd_solve(X, y, w, z, b=8, s=s, H=4096, lam=1e-4, seed=42, prec=prec)
    err_w, err_z = _rel(w, w_ref), _rel(z, z_ref)
    print(f"full size {prec} s={s}: rel err w {err_w:.3e} z {err_z:.3e}")
    assert err_w < tol and err_z < tol
