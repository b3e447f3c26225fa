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
