"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds only input generation (random matrices, labels, sparsity
patterns).  It contains none of the method's arithmetic and is the one module
that both the FP64 oracle's tests and the CUDA library's tests and benchmark
use.

Recipes (the paper's LIBSVM data sets are not available; these stand in for
the shape regimes it studies: n >> d for the primal method, d >> n and sparse
for the dual method, Sec. 5 Tables "dsets" / "perfdsets"):

* ``tiny_primal``: X d x n with iid N(0,1) entries, w_true ~ N(0,1),
  y = X^T w_true + 0.01 N(0,1).
* ``dense_primal``: X d x n, row f = 10^(-log10(cond) f/(d-1)) * N(0,1)
  (geometric singular-value decay; condition about ``cond`` times the
  Marchenko-Pastur factor), y = X^T w_true + noise with
  sigma = noise * rms(X^T w_true).
* ``sparse_dual``: X d x n stored as CSR of X^T (row i = sample i).  Feature
  f appears in k_f = min(n, ceil(k_min / U)) samples, U ~ U(0,1] (a Pareto
  tail with pdf exponent 2), k_min solved so that mean k_f = density * n; the
  k_f sample positions are uniform without replacement; values N(0,1);
  y uniform in {-1, +1}.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class DenseProblem:
    X: np.ndarray          # d x n (rows = features, columns = samples)
    y: np.ndarray          # n, float64
    w_true: np.ndarray     # d, float64


def tiny_primal(d: int = 64, n: int = 1024, seed: int = 1, noise: float = 0.01) -> DenseProblem:
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((d, n))
    w_true = rng.standard_normal(d)
    y = X.T @ w_true + noise * rng.standard_normal(n)
    return DenseProblem(X, y, w_true)


def row_scales(d: int, cond: float) -> np.ndarray:
    """10^(-log10(cond) * f / (d-1)) for f = 0..d-1."""
    if d == 1:
        return np.ones(1)
    return 10.0 ** (-math.log10(cond) * np.arange(d) / (d - 1))


def dense_primal(d: int, n: int, cond: float = 1e3, seed: int = 1, noise: float = 0.01,
                 dtype=np.float32) -> DenseProblem:
    """Dense X with geometrically scaled rows, generated row block by row block."""
    rng = np.random.default_rng(seed)
    X = np.empty((d, n), dtype=dtype)
    scales = row_scales(d, cond)
    step = max(1, (1 << 24) // max(n, 1))
    for f0 in range(0, d, step):
        f1 = min(d, f0 + step)
        blk = rng.standard_normal((f1 - f0, n), dtype=np.float32 if dtype == np.float32
                                  else np.float64)
        X[f0:f1] = blk * scales[f0:f1, None].astype(blk.dtype)
    w_true = rng.standard_normal(d)
    clean = X.T.astype(np.float64) @ w_true if X.size <= (1 << 26) else _xtw_blocked(X, w_true)
    sigma = noise * math.sqrt(float(np.mean(clean * clean)))
    y = clean + sigma * rng.standard_normal(n)
    return DenseProblem(X, y, w_true)


def _xtw_blocked(X: np.ndarray, w: np.ndarray) -> np.ndarray:
    d, n = X.shape
    out = np.zeros(n)
    step = max(1, (1 << 24) // n)
    for f0 in range(0, d, step):
        out += X[f0:f0 + step].T.astype(np.float64) @ w[f0:f0 + step]
    return out


def dense_primal_torch(d: int, n: int, cond: float = 1e3, seed: int = 1, noise: float = 0.01,
                       device: str = "cuda"):
    """Same recipe as ``dense_primal`` drawn with torch's generator on ``device``
    (for matrices of several GiB).  Returns torch tensors (X float32 d x n,
    y float64, w_true float64)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    X = torch.randn(d, n, generator=g, device=device, dtype=torch.float32)
    X.mul_(torch.as_tensor(row_scales(d, cond), dtype=torch.float32, device=device)[:, None])
    w_true = torch.randn(d, generator=g, device=device, dtype=torch.float64)
    clean = torch.zeros(n, dtype=torch.float64, device=device)
    step = max(1, (1 << 24) // n)
    for f0 in range(0, d, step):
        clean += X[f0:f0 + step].T.double() @ w_true[f0:f0 + step]
    sigma = noise * float(torch.sqrt(torch.mean(clean * clean)))
    y = clean + sigma * torch.randn(n, generator=g, device=device, dtype=torch.float64)
    return X, y, w_true


@dataclass
class SparseProblem:
    rowptr: np.ndarray     # n+1 int64, CSR of X^T
    col: np.ndarray        # nnz int32 (feature index)
    val: np.ndarray        # nnz float32
    d: int
    n: int
    y: np.ndarray          # n float64

    def dense_X(self) -> np.ndarray:
        """The d x n matrix X (only for small problems)."""
        X = np.zeros((self.d, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        X[self.col, rows] = self.val
        return X


def pareto_kmin(n: int, mean_k: float) -> float:
    """k_min with E[min(n, ceil(k_min/U))] = mean_k for U ~ U(0,1].

    P(ceil(k_min/U) >= k) = min(1, k_min/(k-1)), so the mean is
    sum_{k=1..n} min(1, k_min/(k-1)) (the k = 1 term is 1); bisection."""
    ks = np.arange(1, n, dtype=np.float64)      # k-1 for k = 2..n

    def mean(kmin):
        return 1.0 + float(np.minimum(1.0, kmin / ks).sum())

    lo, hi = 1e-9, float(n)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mean(mid) < mean_k:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def sparse_dual(d: int = 131072, n: int = 16384, density: float = 0.005, seed: int = 1,
                values_dtype=np.float32) -> SparseProblem:
    rng = np.random.default_rng(seed)
    kmin = pareto_kmin(n, density * n)
    U = 1.0 - rng.random(d)                       # (0, 1]
    k = np.minimum(n, np.ceil(kmin / U)).astype(np.int64)
    # sample positions: for each feature, k_f distinct samples uniformly
    feats = np.repeat(np.arange(d, dtype=np.int64), k)
    pos = np.empty(feats.shape[0], dtype=np.int64)
    starts = np.concatenate([[0], np.cumsum(k)])
    heavy = np.nonzero(k > n // 8)[0]
    light_mask = np.ones(d, dtype=bool)
    light_mask[heavy] = False
    for f in heavy:                                # dense-ish features: a permutation prefix
        pos[starts[f]:starts[f + 1]] = rng.permutation(n)[:k[f]]
    light = np.nonzero(light_mask)[0]
    if light.size:
        sel = np.concatenate([np.arange(starts[f], starts[f + 1]) for f in light]) \
            if light.size < 1000 else np.nonzero(np.repeat(light_mask, k))[0]
        pos[sel] = rng.integers(0, n, size=sel.size)
        # redraw duplicates within a feature until none remain
        for _ in range(1000):
            key = feats[sel] * n + pos[sel]
            order = np.argsort(key, kind="stable")
            dup = np.zeros(sel.size, dtype=bool)
            dup[order[1:]] = key[order[1:]] == key[order[:-1]]
            if not dup.any():
                break
            pos[sel[dup]] = rng.integers(0, n, size=int(dup.sum()))
    vals = rng.standard_normal(feats.shape[0]).astype(values_dtype)
    # CSR of X^T: rows = samples, sorted by (sample, feature)
    order = np.lexsort((feats, pos))
    col = feats[order].astype(np.int32)
    val = vals[order]
    counts = np.bincount(pos, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    y = rng.choice(np.array([-1.0, 1.0]), size=n)
    return SparseProblem(rowptr, col, val, d, n, y)


def dense_dual(d: int, n: int, seed: int = 1, noise: float = 0.01) -> DenseProblem:
    """d >> n dense data for the dual method: iid N(0,1) X, y = X^T w_true + noise."""
    return tiny_primal(d=d, n=n, seed=seed, noise=noise)
