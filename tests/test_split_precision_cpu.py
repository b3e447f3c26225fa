"""The error bounds behind the Gram-mode tolerances, checked by emulating the
splits on the CPU (numpy; no GPU, no library code):

* BF16 has 8 significant bits, unit roundoff u = 2^-8.  BF16x3 splits
  x = b0 + b1 + r with b0 = bf16(x), b1 = bf16(x - b0) (x - b0 is exact in
  FP32): |x - b0| <= u|x|, |r| <= u|x - b0| <= u^2 |x|.  The three products
  b0 c0 + b0 c1 + b1 c0 drop b1 c1, b0 r_y + r_x c0 and smaller terms: each
  product is within 3 u^2 (1 + 2u) |x||y| ~ 4.6e-5 |x||y|, and so a Gram entry
  within that of sqrt(G_ii G_jj) (Cauchy-Schwarz).
* Scaled FP16 rounds x s_r (s_r a power of two, the row's largest magnitude
  in [2^14, 2^15)) to 11 significant bits: u = 2^-11, a product within
  (2u + u^2) |x||y|.
* 3xTF32: hi = x rounded to TF32 (11 significant bits: |x - hi| <= 2^-11 |x|),
  lo = x - hi exact in FP32; the tensor core reads lo with its low 13
  mantissa bits dropped (|lo - lo'| < 2^-10 |lo|).  hi hi + hi lo' + lo' hi
  drops lo lo and the two truncation errors: within ~(2^-22 + 2 * 2^-21)
  |x||y| ~ 1.2e-6 |x||y|.
"""
import numpy as np


def _bf16_rn(x):
    """Round float32 to BF16 (nearest, ties to even), as float32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def _tf32_head(x):
    """TF32 head by rounding at bit 13 (half up in magnitude), as float32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return (((u + 0x1000) & 0xFFFFE000) & 0xFFFFFFFF).astype(np.uint32).view(np.float32)


def _tf32_trunc(x):
    u = np.asarray(x, dtype=np.float32).view(np.uint32)
    return (u & np.uint32(0xFFFFE000)).view(np.float32)


def _data(rng, shape):
    # magnitudes over many binades, mantissas uniform
    return (rng.standard_normal(shape) * 2.0 ** rng.uniform(-20, 20, size=shape)).astype(np.float32)


def test_bf16_split_bounds():
    rng = np.random.default_rng(1)
    x = _data(rng, 200000)
    b0 = _bf16_rn(x)
    b1 = _bf16_rn(x - b0)  # x - b0 exact in FP32
    ax = np.abs(x.astype(np.float64))
    e0 = np.abs(x.astype(np.float64) - b0)
    r = x.astype(np.float64) - b0 - b1
    assert np.all(e0 <= 2.0 ** -8 * ax)
    assert np.all(np.abs(r) <= 2.0 ** -16 * ax)
    assert np.max(e0 / ax) > 0.9 * 2.0 ** -8  # the bound is attained: u = 2^-8, not 2^-9


def test_bf16x3_product_and_gram_bounds():
    rng = np.random.default_rng(2)
    x, y = _data(rng, 100000), _data(rng, 100000)
    def split(v):
        h = _bf16_rn(v)
        return h.astype(np.float64), _bf16_rn(v - h).astype(np.float64)
    (b0, b1), (c0, c1) = split(x), split(y)
    prod = b0 * c0 + b0 * c1 + b1 * c0
    exact = x.astype(np.float64) * y.astype(np.float64)
    bound = 3 * 2.0 ** -16 * (1 + 2 * 2.0 ** -8)
    assert np.all(np.abs(prod - exact) <= bound * np.abs(exact))
    # a Gram of rows with one scale per row (as a sampled block of X)
    Y = (rng.standard_normal((48, 4096)) * 10.0 ** rng.uniform(-3, 3, size=(48, 1))).astype(np.float32)
    H0 = _bf16_rn(Y).astype(np.float64)
    H1 = _bf16_rn(Y - H0.astype(np.float32)).astype(np.float64)
    G = H0 @ H0.T + H0 @ H1.T + H1 @ H0.T
    Ge = Y.astype(np.float64) @ Y.T.astype(np.float64)
    nrm = np.sqrt(np.diag(Ge))
    err = np.abs(G - Ge) / np.outer(nrm, nrm)
    assert err.max() <= bound
    assert err.max() < 1e-5  # random signs: far inside the worst case (GPU: 2.8e-6 .. 3.4e-6)


def test_scaled_fp16_product_bound():
    rng = np.random.default_rng(3)
    Y = (rng.standard_normal((32, 2048)) * 10.0 ** rng.uniform(-12, 12, size=(32, 1))).astype(np.float32)
    m = np.abs(Y).max(axis=1)
    e = np.frexp(m)[1]
    s = np.ldexp(1.0, 15 - e).astype(np.float32)
    Z = (Y * s[:, None]).astype(np.float16)  # round to nearest, 11 significant bits
    assert np.isfinite(Z).all() and np.abs(Z).max() < 2.0 ** 15
    back = Z.astype(np.float64) / s[:, None]
    rel = np.abs(back - Y) / np.maximum(np.abs(Y), 1e-300)
    normal = np.abs(Y * s[:, None]) >= 2.0 ** -14  # FP16 normal range
    assert rel[normal].max() <= 2.0 ** -11
    G = back @ back.T
    Ge = Y.astype(np.float64) @ Y.T.astype(np.float64)
    nrm = np.sqrt(np.diag(Ge))
    assert (np.abs(G - Ge) / np.outer(nrm, nrm)).max() <= 2 * 2.0 ** -11 + 2.0 ** -22


def test_3xtf32_product_bound():
    rng = np.random.default_rng(4)
    x, y = _data(rng, 100000), _data(rng, 100000)
    def split(v):
        h = _tf32_head(v)
        lo = (v - h).astype(np.float32)  # exact
        return h.astype(np.float64), _tf32_trunc(lo).astype(np.float64)
    (h0, l0), (g0, m0) = split(x), split(y)
    prod = h0 * g0 + h0 * m0 + l0 * g0
    exact = x.astype(np.float64) * y.astype(np.float64)
    assert np.all(np.abs(prod - exact) <= (2.0 ** -22 + 2 * 2.0 ** -21) * 1.01 * np.abs(exact))


def test_fp32_residual_pass_precision_at_a_certified_stop():
    """The tolerance of the GPU gap at a certified stop (FP32 X): the
    residual pass multiplies FP32 X by the FP32 (hi, lo) pair of the FP64
    vector with FP32 fused multiply-adds, 8 atoms per lane into an FP32
    partial, partials summed compensated.  Its error is a fixed fraction of
    sum |x_k v_k|, so relative to r it grows as r shrinks.  Emulated on a
    dense 512 x 1024 problem (cond 1e3 rows) along a BCD run: the gap's
    relative error stays below 1e-3 while the certified bound is above 1e-8,
    and everywhere within 1e-2 of the gap plus 1e-10 of f (the cross term
    2 r.dr grows relative to r as r shrinks; at convergence the gap it gives
    levels off near 1.2e-13 f): certificates on FP32 X are sound down to
    ~1e-10."""
    import oracle
    import synth
    m = synth.dense_primal(d=128, n=1024, cond=1e3, seed=2)
    X32 = np.ascontiguousarray(m.X[:, :1024]).astype(np.float32)
    X64, y, lam = X32.astype(np.float64), m.y[:1024], 1e-4
    d, n = X64.shape

    def device_like_r(w):
        rho = y - X64.T @ w
        hi = rho.astype(np.float32)
        lo = (rho - hi).astype(np.float32)
        A = X32.reshape(d, n // 32, 32).astype(np.float64)
        pacc = np.zeros((d, 32), dtype=np.float32)
        tot = np.zeros((d, 32))
        for a in range(n // 32):  # fmaf(x, hi, fmaf(x, lo, pacc)), one rounding each
            t = (A[:, a, :] * lo.reshape(-1, 32)[a] + pacc).astype(np.float32)
            pacc = (A[:, a, :] * hi.reshape(-1, 32)[a] + t).astype(np.float32)
            if a % 8 == 7:
                tot += pacc
                pacc[:] = 0
        tot += pacc
        return tot.sum(axis=1) / n - lam * w

    w = np.zeros(d)
    h, seen = 0, 0
    while h < 2048:
        w, _ = oracle.ca_bcd(X64, y, lam, 8, 8, 64, 7, h0=h, w0=w)
        h += 64
        r = oracle.primal_residual(X64, y, lam, w)
        f, g = oracle.primal_objective(X64, y, lam, w), r @ r / (2 * lam)
        rd = device_like_r(w)
        gd = rd @ rd / (2 * lam)
        if f > g and g / (f - g) > 1e-8:
            assert abs(gd - g) <= 1e-3 * g
            seen += 1
        assert abs(gd - g) <= 1e-2 * g + 1e-10 * f
    assert seen >= 3
