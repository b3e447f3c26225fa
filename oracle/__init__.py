"""FP64 CPU oracle for CA-BCD / CA-BDCD -- TEST INFRASTRUCTURE ONLY.

This package wraps ``ca_oracle.c``, a plain FP64 restatement of Algorithms
1-4 of Devarakonda et al., "Avoiding communication in primal and dual block
coordinate descent methods" (arXiv 1612.04003), plus the closed-form ridge
solution and the primal/dual objectives of Sec. 2.2.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  It shares no code
with the CUDA library in ``paper_1612_04003_gb300`` and never imports it.

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py``
(closed form vs a library solve, one-step exactness at b = d / b' = n, s-step
equivalence, monotone objectives, duality identity, the sampler's generator
against numpy's Philox, Floyd's algorithm by exhaustive enumeration; the
residuals of the stopping test against finite differences of the objectives,
their zeros at the optimum and on the block just solved; the duality gaps
against the closed forms ||r||^2/(2 lambda) and ||r||^2/(2n) of the two
residuals and against the objective error to the closed-form optimum).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ca_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libcaoracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK = 0
ORC_ERR_NOT_SPD = -3


def build(force: bool = False) -> str:
    """Compile ca_oracle.c with gcc (no fused multiply-add contraction)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        c_dp = ctypes.POINTER(ctypes.c_double)
        c_i64p = ctypes.POINTER(ctypes.c_int64)
        c_i32p = ctypes.POINTER(ctypes.c_int32)
        c_u64p = ctypes.POINTER(ctypes.c_uint64)
        i64, u64, dbl, cint = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
        lib.orc_philox4x64_10.argtypes = [c_u64p, c_u64p, c_u64p]
        lib.orc_philox4x64_10.restype = None
        lib.orc_map_to_range.argtypes = [u64, u64]
        lib.orc_map_to_range.restype = u64
        lib.orc_sample_block.argtypes = [u64, i64, cint, i64, c_i32p]
        lib.orc_sample_block.restype = cint
        lib.orc_cholesky_solve.argtypes = [cint, c_dp, c_dp, c_dp]
        lib.orc_cholesky_solve.restype = cint
        lib.orc_primal_objective.argtypes = [c_dp, i64, i64, c_dp, dbl, c_dp]
        lib.orc_primal_objective.restype = dbl
        lib.orc_closed_form.argtypes = [c_dp, i64, i64, c_dp, dbl, c_dp]
        lib.orc_closed_form.restype = cint
        lib.orc_cabcd.argtypes = [c_dp, i64, i64, c_dp, dbl, cint, cint, i64, u64, i64, cint,
                                  c_dp, c_dp]
        lib.orc_cabcd.restype = cint
        lib.orc_bcd.argtypes = [c_dp, i64, i64, c_dp, dbl, cint, i64, u64, i64, cint, c_dp, c_dp]
        lib.orc_bcd.restype = cint
        lib.orc_dual_objective.argtypes = [c_i64p, c_i32p, c_dp, i64, i64, c_dp, dbl, c_dp]
        lib.orc_dual_objective.restype = dbl
        lib.orc_cabdcd.argtypes = [c_i64p, c_i32p, c_dp, i64, i64, c_dp, dbl, cint, cint, i64,
                                   u64, i64, cint, c_dp, c_dp]
        lib.orc_cabdcd.restype = cint
        lib.orc_bdcd.argtypes = [c_i64p, c_i32p, c_dp, i64, i64, c_dp, dbl, cint, i64, u64, i64,
                                 cint, c_dp, c_dp]
        lib.orc_bdcd.restype = cint
        _lib = lib
        return lib


class OracleError(RuntimeError):
    pass


def _check(st: int, what: str):
    if st != ORC_OK:
        raise OracleError(f"{what} failed with status {st}")


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# Sampler (reading R3 in ca_oracle.c)
# --------------------------------------------------------------------------
def philox4x64_10(counter, key) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(np.asarray(counter, dtype=np.uint64).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64).reshape(2))
    out = np.zeros(4, dtype=np.uint64)
    lib.orc_philox4x64_10(_ptr(c, ctypes.c_uint64), _ptr(k, ctypes.c_uint64),
                          _ptr(out, ctypes.c_uint64))
    return out


def map_to_range(u: int, J: int) -> int:
    return int(_load().orc_map_to_range(ctypes.c_uint64(u), ctypes.c_uint64(J)))


def sample_block(seed: int, h: int, b: int, N: int) -> np.ndarray:
    out = np.zeros(b, dtype=np.int32)
    _check(_load().orc_sample_block(seed, h, b, N, _ptr(out, ctypes.c_int32)), "sample_block")
    return out


def sample_blocks(seed: int, h0: int, H: int, b: int, N: int) -> np.ndarray:
    """Blocks h0 .. h0+H-1 as an (H, b) int32 array."""
    return np.stack([sample_block(seed, h0 + h, b, N) for h in range(H)]) if H else \
        np.zeros((0, b), dtype=np.int32)


def cholesky_solve(A, r) -> np.ndarray:
    A = _f64(A)
    r = _f64(r)
    m = r.shape[0]
    x = np.zeros(m)
    _check(_load().orc_cholesky_solve(m, _ptr(A, ctypes.c_double), _ptr(r, ctypes.c_double),
                                      _ptr(x, ctypes.c_double)), "cholesky_solve")
    return x


# --------------------------------------------------------------------------
# Primal (X is d x n, rows = features, columns = samples)
# --------------------------------------------------------------------------
def primal_objective(X, y, lam, w) -> float:
    X, y, w = _f64(X), _f64(y), _f64(w)
    d, n = X.shape
    return float(_load().orc_primal_objective(_ptr(X, ctypes.c_double), d, n,
                                              _ptr(y, ctypes.c_double), lam,
                                              _ptr(w, ctypes.c_double)))


def closed_form(X, y, lam) -> np.ndarray:
    X, y = _f64(X), _f64(y)
    d, n = X.shape
    w = np.zeros(d)
    _check(_load().orc_closed_form(_ptr(X, ctypes.c_double), d, n, _ptr(y, ctypes.c_double),
                                   lam, _ptr(w, ctypes.c_double)), "closed_form")
    return w


def ca_bcd(X, y, lam, b, s, H, seed, h0=0, recompute_every=0, w0=None):
    """Algorithm 2 (Algorithm 1's steps when s == 1).  Returns (w_H, X^T w_H)."""
    X, y = _f64(X), _f64(y)
    d, n = X.shape
    w = np.zeros(d) if w0 is None else _f64(w0).copy()
    z = np.zeros(n)
    _check(_load().orc_cabcd(_ptr(X, ctypes.c_double), d, n, _ptr(y, ctypes.c_double), lam,
                             b, s, H, seed, h0, recompute_every, _ptr(w, ctypes.c_double),
                             _ptr(z, ctypes.c_double)), "ca_bcd")
    return w, z


def bcd(X, y, lam, b, H, seed, h0=0, recompute_every=0, w0=None):
    """Algorithm 1.  Returns (w_H, X^T w_H)."""
    X, y = _f64(X), _f64(y)
    d, n = X.shape
    w = np.zeros(d) if w0 is None else _f64(w0).copy()
    z = np.zeros(n)
    _check(_load().orc_bcd(_ptr(X, ctypes.c_double), d, n, _ptr(y, ctypes.c_double), lam, b, H,
                           seed, h0, recompute_every, _ptr(w, ctypes.c_double),
                           _ptr(z, ctypes.c_double)), "bcd")
    return w, z


# --------------------------------------------------------------------------
# Dual (X given by its columns as CSR of X^T)
# --------------------------------------------------------------------------
class CSR:
    """CSR of X^T: row i holds the non-zeros of column x_i of X."""

    def __init__(self, rowptr, col, val, d: int):
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = _f64(val)
        self.n = self.rowptr.shape[0] - 1
        self.d = int(d)

    @staticmethod
    def from_dense(X) -> "CSR":
        """Every entry of the d x n matrix X stored (dense-as-CSR)."""
        X = _f64(X)
        d, n = X.shape
        rowptr = np.arange(n + 1, dtype=np.int64) * d
        col = np.tile(np.arange(d, dtype=np.int32), n)
        return CSR(rowptr, col, X.T.reshape(-1), d)

    def args(self):
        return (_ptr(self.rowptr, ctypes.c_int64), _ptr(self.col, ctypes.c_int32),
                _ptr(self.val, ctypes.c_double), self.d, self.n)


def _as_csr(X) -> CSR:
    return X if isinstance(X, CSR) else CSR.from_dense(X)


def dual_objective(X, y, lam, alpha) -> float:
    A = _as_csr(X)
    y, alpha = _f64(y), _f64(alpha)
    return float(_load().orc_dual_objective(*A.args(), _ptr(y, ctypes.c_double), lam,
                                            _ptr(alpha, ctypes.c_double)))


def ca_bdcd(X, y, lam, b, s, H, seed, h0=0, recompute_every=0, alpha0=None):
    """Algorithm 4 (Algorithm 3's steps when s == 1).  Returns (alpha_H, w_H)."""
    A = _as_csr(X)
    y = _f64(y)
    alpha = np.zeros(A.n) if alpha0 is None else _f64(alpha0).copy()
    w = np.zeros(A.d)
    _check(_load().orc_cabdcd(*A.args(), _ptr(y, ctypes.c_double), lam, b, s, H, seed, h0,
                              recompute_every, _ptr(alpha, ctypes.c_double),
                              _ptr(w, ctypes.c_double)), "ca_bdcd")
    return alpha, w


def bdcd(X, y, lam, b, H, seed, h0=0, recompute_every=0, alpha0=None):
    """Algorithm 3.  Returns (alpha_H, w_H)."""
    A = _as_csr(X)
    y = _f64(y)
    alpha = np.zeros(A.n) if alpha0 is None else _f64(alpha0).copy()
    w = np.zeros(A.d)
    _check(_load().orc_bdcd(*A.args(), _ptr(y, ctypes.c_double), lam, b, H, seed, h0,
                            recompute_every, _ptr(alpha, ctypes.c_double),
                            _ptr(w, ctypes.c_double)), "bdcd")
    return alpha, w


# --------------------------------------------------------------------------
# Stopping criterion (Sec. 5.1.5): the full primal / dual residual
# --------------------------------------------------------------------------
def primal_residual(X, y, lam, w) -> np.ndarray:
    """The full primal residual of Sec. 5.1.5, the d-vector whose rows at the
    sampled indices are the right-hand side of the BCD subproblem:
    -lam w - (1/n) X (X^T w - y), the negative gradient of the primal objective."""
    X, y, w = _f64(X), _f64(y), _f64(w)
    n = X.shape[1]
    return -lam * w - X @ (X.T @ w - y) / n


def _xt_times(X, w) -> np.ndarray:
    """X^T w for the d x n matrix X, or for X given by the CSR of X^T."""
    if isinstance(X, CSR):
        out = np.zeros(X.n)
        for i in range(X.n):
            a, b = X.rowptr[i], X.rowptr[i + 1]
            out[i] = X.val[a:b] @ w[X.col[a:b]]
        return out
    return _f64(X).T @ w


def dual_residual(X, y, alpha, w) -> np.ndarray:
    """The full dual residual of Sec. 5.1.5, the n-vector -X^T w + alpha + y
    (X dense d x n or the CSR of X^T), whose rows at the sampled indices are
    the BDCD subproblem's right-hand side."""
    return -_xt_times(X, _f64(w)) + _f64(alpha) + _f64(y)


def primal_duality_gap(X, y, lam, w) -> float:
    """Duality gap of the primal point w (Sec. 2.2): f(w) + D(alpha) - ||y||^2/(2n)
    at the dual point alpha = X^T w - y that the optimality conditions pair
    with w (alpha* = X^T w* - y), from the definitions of f and D.  Weak
    duality makes it >= 0 and >= f(w) - f(w*)."""
    X, y, w = _f64(X), _f64(y), _f64(w)
    n = X.shape[1]
    return (primal_objective(X, y, lam, w) + dual_objective(X, y, lam, X.T @ w - y)
            - float(y @ y) / (2 * n))


def dual_duality_gap(X, y, lam, alpha) -> float:
    """Duality gap of the dual point alpha: f(w) + D(alpha) - ||y||^2/(2n) at
    w = -X alpha/(lambda n) (eq. "3"), from the definitions of f and D (X
    dense d x n or the CSR of X^T).  It bounds both D(alpha) - D(alpha*) and
    f(w) - f(w*)."""
    A = _as_csr(X)
    y, alpha = _f64(y), _f64(alpha)
    w = np.zeros(A.d)
    for i in range(A.n):  # w = -X alpha/(lambda n), column by column
        a, b = A.rowptr[i], A.rowptr[i + 1]
        w[A.col[a:b]] -= A.val[a:b] * alpha[i] / (lam * A.n)
    Xd = np.zeros((A.d, A.n))
    for i in range(A.n):
        a, b = A.rowptr[i], A.rowptr[i + 1]
        Xd[A.col[a:b], i] = A.val[a:b]
    return (primal_objective(Xd, y, lam, w) + dual_objective(A, y, lam, alpha)
            - float(y @ y) / (2 * A.n))


def ca_bcd_certified(X, y, lam, b, s, H, seed, tol, check_every):
    """Algorithm 2 with a certified stop: after every check_every outer steps
    the duality gap g of w and the primal objective f(w); since
    f(w*) >= f(w) - g, the relative objective error (f(w) - f(w*))/f(w*) is
    at most g/(f(w) - g), and the run ends at the first check where that
    bound is <= tol (tol = 0: never), or at H.  Returns (w, h_done,
    [(f(w), g) after each check])."""
    X, y = _f64(X), _f64(y)
    w = np.zeros(X.shape[0])
    h, trace = 0, []
    while h < H:
        m = min(check_every * s, H - h)
        w, _ = ca_bcd(X, y, lam, b, s, m, seed, h0=h, w0=w)
        h += m
        f, g = primal_objective(X, y, lam, w), primal_duality_gap(X, y, lam, w)
        trace.append((f, g))
        if h < H and tol > 0 and g <= tol * (f - g):
            break
    return w, h, trace


def ca_bdcd_certified(X, y, lam, b, s, H, seed, tol, check_every):
    """Algorithm 4 with the certified stop of ca_bcd_certified, on the model
    w = -X alpha/(lambda n) and the gap of alpha.  Returns (alpha, w, h_done,
    [(f(w), g) after each check])."""
    A = _as_csr(X)
    y = _f64(y)
    alpha = np.zeros(A.n)
    w = np.zeros(A.d)
    h, trace = 0, []
    while h < H:
        m = min(check_every * s, H - h)
        alpha, w = ca_bdcd(A, y, lam, b, s, m, seed, h0=h, alpha0=alpha)
        h += m
        g = dual_duality_gap(A, y, lam, alpha)
        f = g + float(y @ y) / (2 * A.n) - dual_objective(A, y, lam, alpha)
        trace.append((f, g))
        if h < H and tol > 0 and g <= tol * (f - g):
            break
    return alpha, w, h, trace


def ca_bcd_stopped(X, y, lam, b, s, H, seed, tol, check_every):
    """Algorithm 2 with the stopping test of Sec. 5.1.5: after every
    check_every outer steps (s block updates each) the full primal residual;
    the run ends once ||r|| <= tol ||r_0|| (tol = 0: never), and at H.
    Returns (w, h_done, ||r_0||, [||r|| after each check])."""
    X, y = _f64(X), _f64(y)
    w = np.zeros(X.shape[0])
    r0 = float(np.linalg.norm(primal_residual(X, y, lam, w)))
    h, norms = 0, []
    while h < H:
        m = min(check_every * s, H - h)
        w, _ = ca_bcd(X, y, lam, b, s, m, seed, h0=h, w0=w)
        h += m
        norms.append(float(np.linalg.norm(primal_residual(X, y, lam, w))))
        if h < H and tol > 0 and norms[-1] <= tol * r0:
            break
    return w, h, r0, norms


def ca_bdcd_stopped(X, y, lam, b, s, H, seed, tol, check_every):
    """Algorithm 4 with the stopping test of Sec. 5.1.5 on the full dual
    residual (as ca_bcd_stopped).  Returns (alpha, w, h_done, ||r_0||,
    [||r|| after each check])."""
    A = _as_csr(X)
    y = _f64(y)
    alpha = np.zeros(A.n)
    w = np.zeros(A.d)
    r0 = float(np.linalg.norm(dual_residual(A, y, alpha, w)))
    h, norms = 0, []
    while h < H:
        m = min(check_every * s, H - h)
        alpha, w = ca_bdcd(A, y, lam, b, s, m, seed, h0=h, alpha0=alpha)
        h += m
        norms.append(float(np.linalg.norm(dual_residual(A, y, alpha, w))))
        if h < H and tol > 0 and norms[-1] <= tol * r0:
            break
    return alpha, w, h, r0, norms
