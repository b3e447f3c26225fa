"""GB300 (sm_103a) CA-BCD / CA-BDCD: Python binding of the C ABI in include/ca_bcd.h.

Argument marshalling only: every step of the method runs in the CUDA library
``_build/libcabcd.so``.  There is no CPU path; importing the binding without
the built library raises.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays; they are passed by
pointer.  CUDA tensors are used in place; host arrays are staged by the
library through device buffers it owns.
"""
from __future__ import annotations

import ctypes
import os
import re

from .buildlib import LIB, INCLUDE, build  # noqa: F401

CA_OK = 0
CA_ERR_ARG = -1
CA_ERR_CUDA = -2
CA_ERR_NOT_SPD = -3
CA_ERR_NONFINITE = -4
CA_ERR_TIMEOUT = -5
CA_ERR_OOM = -6
CA_ERR_UNSUPPORTED = -7

CA_DENSE_F64 = 0
CA_DENSE_F32 = 1
CA_CSR_F32 = 2
CA_DENSE_F32_PANELS = 3

CA_GRAM_F64 = 0
CA_GRAM_FP32_EXACT = 1
CA_GRAM_TF32 = 2
CA_GRAM_BF16X3 = 3
CA_GRAM_FP16_SCALED = 4

CA_STOP_RESIDUAL = 0
CA_STOP_OBJECTIVE = 1
STOP = {"residual": CA_STOP_RESIDUAL, "objective": CA_STOP_OBJECTIVE}

CA_BATCH_GRAPH = 1
CA_TUNE_PERSISTENT = 1
CA_TUNE_OVERLAP = 2

CA_SOLVE_DF = 0
CA_SOLVE_F64 = 1
SOLVE = {"df": CA_SOLVE_DF, "f64": CA_SOLVE_F64}

PREC = {"f64": CA_GRAM_F64, "fp32_exact": CA_GRAM_FP32_EXACT, "3xtf32": CA_GRAM_FP32_EXACT,
        "tf32": CA_GRAM_TF32, "bf16x3": CA_GRAM_BF16X3, "fp16_scaled": CA_GRAM_FP16_SCALED}


class ca_opts(ctypes.Structure):
    _fields_ = [("b", ctypes.c_int), ("s", ctypes.c_int), ("H", ctypes.c_longlong),
                ("lam", ctypes.c_double), ("seed", ctypes.c_ulonglong), ("prec", ctypes.c_int),
                ("recompute_every", ctypes.c_int), ("h0", ctypes.c_longlong),
                ("tol", ctypes.c_double), ("check_every", ctypes.c_int), ("stop", ctypes.c_int),
                ("solve", ctypes.c_int)]


class ca_info(ctypes.Structure):
    _fields_ = [("h_done", ctypes.c_longlong), ("checks", ctypes.c_int), ("res0", ctypes.c_double),
                ("res", ctypes.c_double), ("gap", ctypes.c_double), ("fval", ctypes.c_double),
                ("bound", ctypes.c_double)]


class ca_check(ctypes.Structure):
    _fields_ = [("h", ctypes.c_longlong), ("res", ctypes.c_double), ("gap", ctypes.c_double),
                ("fval", ctypes.c_double)]


class ca_request(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("xfmt", ctypes.c_int), ("X", ctypes.c_void_p),
                ("d", ctypes.c_longlong), ("n", ctypes.c_longlong), ("ld", ctypes.c_longlong),
                ("y", ctypes.c_void_p), ("x", ctypes.c_void_p), ("aux", ctypes.c_void_p),
                ("opts", ca_opts)]


class ca_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("worker", ctypes.c_int), ("s", ctypes.c_int),
                ("h_done", ctypes.c_longlong),
                ("res0", ctypes.c_double), ("res", ctypes.c_double), ("gap", ctypes.c_double),
                ("fval", ctypes.c_double), ("bound", ctypes.c_double),
                ("queue_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("scratch_bytes", ctypes.c_size_t)]


class ca_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("rejected", ctypes.c_longlong), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("wall_s", ctypes.c_double),
                ("block_updates_per_s", ctypes.c_double), ("peak_footprint", ctypes.c_size_t),
                ("peak_concurrency", ctypes.c_int)]


class ca_csr(ctypes.Structure):
    _fields_ = [("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class CaError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        extra = f" [{detail}]" if detail else ""
        super().__init__(f"{what}: {status_str(status)} ({status}){extra}")


_lib = None


def load():
    """Load libcabcd.so (built by build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError(f"CUDA library not built: {LIB} is missing (run "
                           "paper_1612_04003_gb300.build.build())")
    lib = ctypes.CDLL(LIB)
    vp, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_ulonglong, \
        ctypes.c_double
    lib.ca_bcd_init.argtypes = [ctypes.POINTER(vp), i32, vp, ctypes.c_size_t]
    lib.ca_bcd_init.restype = i32
    lib.ca_bcd_solve.argtypes = [vp, i32, vp, i64, i64, i64, vp, ctypes.POINTER(ca_opts), vp, vp]
    lib.ca_bcd_solve.restype = i32
    lib.ca_bdcd_solve.argtypes = [vp, i32, vp, i64, i64, i64, vp, ctypes.POINTER(ca_opts), vp, vp]
    lib.ca_bdcd_solve.restype = i32
    lib.ca_sample_indices.argtypes = [vp, u64, i64, i64, i32, i64, vp]
    lib.ca_sample_indices.restype = i32
    lib.ca_status_str.argtypes = [i32]
    lib.ca_status_str.restype = ctypes.c_char_p
    lib.ca_bcd_destroy.argtypes = [vp]
    lib.ca_bcd_destroy.restype = None
    lib.ca_profile_enable.argtypes = [vp, i32]
    lib.ca_profile_enable.restype = i32
    lib.ca_set_tuning.argtypes = [vp, i32, dbl]
    lib.ca_set_tuning.restype = i32
    lib.ca_profile_read.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(i64),
                                    ctypes.POINTER(i64)]
    lib.ca_profile_read.restype = i32
    lib.ca_gram_project_noalloc.argtypes = [vp, i32, i32, vp, i64, i64, i64, vp, i32, vp, vp, vp]
    lib.ca_gram_project_noalloc.restype = i32
    lib.ca_last_error.argtypes = [vp]
    lib.ca_last_error.restype = ctypes.c_char_p
    lib.ca_gram_project.argtypes = [vp, i32, i32, vp, i64, i64, i64, vp, i32, vp, vp, vp]
    lib.ca_solve_info.argtypes = [vp, ctypes.POINTER(ca_info)]
    lib.ca_solve_info.restype = i32
    lib.ca_solve_scratch_bytes.argtypes = [vp, i32, i32, i64, i64, ctypes.POINTER(ca_opts),
                                           ctypes.POINTER(ctypes.c_size_t)]
    lib.ca_solve_scratch_bytes.restype = i32
    lib.ca_bcd_release_scratch.argtypes = [vp]
    lib.ca_bcd_release_scratch.restype = i32
    lib.ca_server_create.argtypes = [ctypes.POINTER(vp), i32, i32, ctypes.c_size_t]
    lib.ca_server_create.restype = i32
    lib.ca_server_submit.argtypes = [vp, ctypes.POINTER(ca_request), ctypes.POINTER(i64)]
    lib.ca_server_submit.restype = i32
    lib.ca_server_wait.argtypes = [vp, i64, ctypes.POINTER(ca_result)]
    lib.ca_server_wait.restype = i32
    lib.ca_server_drain.argtypes = [vp]
    lib.ca_server_drain.restype = i32
    lib.ca_server_get_stats.argtypes = [vp, ctypes.POINTER(ca_server_stats)]
    lib.ca_server_get_stats.restype = i32
    lib.ca_server_destroy.argtypes = [vp]
    lib.ca_server_destroy.restype = None
    lib.ca_gram_project.restype = i32
    lib.ca_pack_panels.argtypes = [vp, vp, i64, i64, i64, vp]
    lib.ca_pack_panels.restype = i32
    lib.ca_selftest_wait_timeout.argtypes = [vp, i64]
    lib.ca_selftest_wait_timeout.restype = i32
    lib.ca_batch_solve.argtypes = [vp, i32, ctypes.POINTER(ca_request), i32,
                                   ctypes.POINTER(ca_result)]
    lib.ca_batch_solve.restype = i32
    lib.ca_batch_scratch_bytes.argtypes = [vp, i32, ctypes.POINTER(ca_request),
                                           ctypes.POINTER(ctypes.c_size_t)]
    lib.ca_batch_scratch_bytes.restype = i32
    lib.ca_server_set_batching.argtypes = [vp, i32]
    lib.ca_server_set_batching.restype = i32
    _lib = lib
    return lib


def header_functions() -> list[str]:
    """Names of the functions declared in include/*.h."""
    names = []
    for fn in sorted(os.listdir(INCLUDE)):
        if fn.endswith(".h"):
            text = open(os.path.join(INCLUDE, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ca_\w+)\s*\(", text, re.M)
    return sorted(set(names))


def gram_project_noalloc(A, idx, v, G, p, *, prec="tf32", ld=None, stream=None):
    """ca_gram_project_noalloc: G = Y Y^T and p = Y v without any device
    allocation (all arrays are device memory on the current device)."""
    N, K = A.shape
    pr = PREC[prec] if isinstance(prec, str) else int(prec)
    st = load().ca_gram_project_noalloc(stream, _xfmt(A), pr, _ptr(A), N, K,
                                        K if ld is None else ld, _ptr(idx), int(idx.shape[0]),
                                        _ptr(v), _ptr(G), _ptr(p))
    if st != CA_OK:
        raise CaError(st, "ca_gram_project_noalloc")
    return G, p


def status_str(status: int) -> str:
    return load().ca_status_str(int(status)).decode()


def _ptr(a):
    """Raw pointer of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("arrays must be contiguous")
        return a.data_ptr()
    if hasattr(a, "ctypes"):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _xfmt(X) -> int:
    name = str(X.dtype)
    if name.endswith("float64"):
        return CA_DENSE_F64
    if name.endswith("float32"):
        return CA_DENSE_F32
    raise TypeError(f"X must be float32 or float64, got {X.dtype}")


def _dtype_is_f64(a) -> bool:
    return str(a.dtype).endswith("float64")


class Context:
    """ca_bcd_init / ca_bcd_destroy around an opaque ca_ctx."""

    def __init__(self, device: int = 0, stream=None, scratch_bytes_max: int = 0):
        self._lib = load()
        h = ctypes.c_void_p()
        s = stream if isinstance(stream, int) or stream is None else getattr(
            stream, "cuda_stream", stream)
        st = self._lib.ca_bcd_init(ctypes.byref(h), device, s, scratch_bytes_max)
        if st != CA_OK:
            raise CaError(st, "ca_bcd_init")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self._lib.ca_bcd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return self._lib.ca_last_error(self.handle).decode()

    @staticmethod
    def _opts(b, s, H, lam, seed, prec, recompute_every, h0, tol=0.0, check_every=0,
              stop="residual", solve="df"):
        p = PREC[prec] if isinstance(prec, str) else int(prec)
        st = STOP[stop] if isinstance(stop, str) else int(stop)
        sv = SOLVE[solve] if isinstance(solve, str) else int(solve)
        return ca_opts(int(b), int(s), int(H), float(lam), int(seed), p, int(recompute_every),
                       int(h0), float(tol), int(check_every), st, sv)

    def solve_info(self) -> dict:
        """Outcome of the last solve: block updates done (h_done), number of
        full-residual checks, ||r_0|| and ||r|| at the last check, the duality
        gap there, f(w) of the model there (objective rule only, else 0) and
        the certified relative objective error gap / (f(w) - gap) the
        library formed (None unless the objective rule ran and f(w) > gap)."""
        info = ca_info()
        st = self._lib.ca_solve_info(self.handle, ctypes.byref(info))
        if st != CA_OK:
            raise CaError(st, "ca_solve_info")
        return {"h_done": info.h_done, "checks": info.checks, "res0": info.res0, "res": info.res,
                "gap": info.gap, "fval": info.fval,
                "bound": info.bound if info.bound >= 0.0 else None}

    def solve_trace(self) -> list:
        """Every check of the last solve, the start first: dicts with the
        block updates done (h), ||r||, the duality gap and f(w) (objective
        rule only, else 0)."""
        cnt = ctypes.c_int()
        st = self._lib.ca_solve_trace(self.handle, None, 0, ctypes.byref(cnt))
        if st != CA_OK:
            raise CaError(st, "ca_solve_trace")
        buf = (ca_check * max(cnt.value, 1))()
        st = self._lib.ca_solve_trace(self.handle, buf, cnt.value, ctypes.byref(cnt))
        if st != CA_OK:
            raise CaError(st, "ca_solve_trace")
        return [{f: getattr(buf[i], f) for f, _ in ca_check._fields_} for i in range(cnt.value)]

    def ca_bcd_solve(self, X, y, w, z=None, *, b, s=1, H, lam, seed=42, prec="tf32",
                     recompute_every=0, h0=0, n=None, ld=None, panels=None, tol=0.0,
                     check_every=0, stop="residual", solve="df"):
        """Primal CA-BCD: w (in: w0, out: w_H) and optionally z = X^T w_H.
        X is d x ld (ld = X.shape[1]); n (default ld) columns are used.
        panels=(d, n): X holds the 32-column panels of a d x n matrix
        (ca_pack_panels)."""
        for a in (y, w) + ((z,) if z is not None else ()):
            if not _dtype_is_f64(a):
                raise TypeError("y, w, z must be float64")
        o = self._opts(b, s, H, lam, seed, prec, recompute_every, h0, tol, check_every, stop,
                       solve)
        if panels is not None:
            d, n = (int(v) for v in panels)
            xf, ld = CA_DENSE_F32_PANELS, 0
        else:
            d, cols = X.shape
            n = cols if n is None else int(n)
            ld = cols if ld is None else int(ld)
            xf = _xfmt(X)
        st = self._lib.ca_bcd_solve(self.handle, xf, _ptr(X), d, n, ld,
                                    _ptr(y), ctypes.byref(o), _ptr(w), _ptr(z))
        if st != CA_OK:
            raise CaError(st, "ca_bcd_solve", self.last_error())
        return w, z

    def ca_bdcd_solve(self, XT, y, alpha, w, *, b, s=1, H, lam, seed=42, prec="tf32",
                      recompute_every=0, h0=0, d=None, ld=None, panels=None, tol=0.0,
                      check_every=0, stop="residual", solve="df"):
        """Dual CA-BDCD.  XT is X^T (n x d, dense), a (rowptr, col, val) CSR
        triple of X^T (then d must be given), or with panels=(n, d) the
        32-column panels of X^T (ca_pack_panels)."""
        for a in (y, alpha, w):
            if not _dtype_is_f64(a):
                raise TypeError("y, alpha, w must be float64")
        o = self._opts(b, s, H, lam, seed, prec, recompute_every, h0, tol, check_every, stop,
                       solve)
        if panels is not None:
            n, dd = (int(v) for v in panels)
            st = self._lib.ca_bdcd_solve(self.handle, CA_DENSE_F32_PANELS, _ptr(XT), dd, n, 0,
                                         _ptr(y), ctypes.byref(o), _ptr(alpha), _ptr(w))
        elif isinstance(XT, (tuple, list)):
            rowptr, col, val = XT
            csr = ca_csr(_ptr(rowptr), _ptr(col), _ptr(val))
            n = int(rowptr.shape[0]) - 1
            st = self._lib.ca_bdcd_solve(self.handle, CA_CSR_F32, ctypes.addressof(csr), int(d), n,
                                         0, _ptr(y), ctypes.byref(o), _ptr(alpha), _ptr(w))
        else:
            n, dd = XT.shape
            st = self._lib.ca_bdcd_solve(self.handle, _xfmt(XT), _ptr(XT), dd, n,
                                         dd if ld is None else ld, _ptr(y), ctypes.byref(o),
                                         _ptr(alpha), _ptr(w))
        if st != CA_OK:
            raise CaError(st, "ca_bdcd_solve", self.last_error())
        return alpha, w

    def ca_sample_indices(self, seed, h0, H, b, N, out):
        st = self._lib.ca_sample_indices(self.handle, int(seed), int(h0), int(H), int(b), int(N),
                                         _ptr(out))
        if st != CA_OK:
            raise CaError(st, "ca_sample_indices", self.last_error())
        return out

    def ca_gram_project(self, A, idx, v, G, p, *, prec="tf32", ld=None):
        """G = Y Y^T and p = Y v for the rows idx of A (all device arrays)."""
        N, K = A.shape
        pr = PREC[prec] if isinstance(prec, str) else int(prec)
        st = self._lib.ca_gram_project(self.handle, _xfmt(A), pr, _ptr(A), N, K,
                                       K if ld is None else ld, _ptr(idx), int(idx.shape[0]),
                                       _ptr(v), _ptr(G), _ptr(p))
        if st != CA_OK:
            raise CaError(st, "ca_gram_project", self.last_error())
        return G, p

    def ca_pack_panels(self, A, out, *, K=None):
        """Write the first K (default all) columns of the FP32 device matrix A
        (N x ld) as 32-column panels into out (ceil(K/32)*N*32 floats,
        device), on the context's stream."""
        N, ld = A.shape
        K = ld if K is None else int(K)
        st = self._lib.ca_pack_panels(self.handle, _ptr(A), N, K, ld, _ptr(out))
        if st != CA_OK:
            raise CaError(st, "ca_pack_panels", self.last_error())
        return out

    def ca_batch_solve(self, problems, *, graph=True):
        """ca_batch_solve: the problems solved together in shared launches.
        problems: dicts with method ("primal" / "dual"), X (FP32 device
        array: primal X d x ld, dual X^T n x ld), y, x (w or alpha: in x0,
        out x_H), aux (primal z or None, dual w), optional panels=(rows,
        cols) for pre-packed panels, n / d (columns used, default ld), and
        the solve keywords b, s (0: by measured cost), H, lam, seed, prec,
        recompute_every, h0, tol, check_every, stop.  Returns one result
        dict per problem (the certified bound is None when not formed)."""
        reqs = (ca_request * len(problems))()
        keep = []
        for i, p in enumerate(problems):
            m = {"primal": 0, "dual": 1}[p["method"]]
            o = self._opts(p["b"], p.get("s", 0), p["H"], p["lam"], p.get("seed", 42),
                           p.get("prec", "bf16x3"), p.get("recompute_every", 0), p.get("h0", 0),
                           p.get("tol", 0.0), p.get("check_every", 0), p.get("stop", "residual"))
            X = p["X"]
            if p.get("panels") is not None:
                rows, cols = (int(v) for v in p["panels"])
                xf, ldv = CA_DENSE_F32_PANELS, 0
            else:
                rows, ldv = X.shape
                xf = _xfmt(X)
                used = p.get("n") if m == 0 else p.get("d")
                cols = ldv if used is None else int(used)
            dd, nn = (rows, cols) if m == 0 else (cols, rows)
            reqs[i] = ca_request(m, xf, _ptr(X), dd, nn, ldv, _ptr(p["y"]), _ptr(p["x"]),
                                 _ptr(p.get("aux")), o)
            keep.append(p)
        outs = (ca_result * len(problems))()
        st = self._lib.ca_batch_solve(self.handle, len(problems), reqs,
                                      CA_BATCH_GRAPH if graph else 0, outs)
        if st != CA_OK:
            raise CaError(st, "ca_batch_solve", self.last_error())
        res = [{f: getattr(outs[i], f) for f, _ in ca_result._fields_}
               for i in range(len(problems))]
        for r in res:
            r["bound"] = r["bound"] if r["bound"] >= 0.0 else None
        return res

    def ca_selftest_wait_timeout(self, limit_ns: int) -> int:
        return int(self._lib.ca_selftest_wait_timeout(self.handle, int(limit_ns)))

    def ca_set_tuning(self, *, persistent=None, overlap=None):
        """ca_set_tuning: persistent launches for runs of outer steps (bool)
        and the share of each Gram CTA's columns streamed before the
        previous step's solve is known (0..1)."""
        for key, val in ((CA_TUNE_PERSISTENT, None if persistent is None else float(bool(persistent))),
                         (CA_TUNE_OVERLAP, overlap)):
            if val is None:
                continue
            st = self._lib.ca_set_tuning(self.handle, key, float(val))
            if st != CA_OK:
                raise CaError(st, "ca_set_tuning")

    def ca_profile_enable(self, on: bool = True):
        st = self._lib.ca_profile_enable(self.handle, 1 if on else 0)
        if st != CA_OK:
            raise CaError(st, "ca_profile_enable")

    PROFILE_CLASSES = ("gram", "reduce", "update", "other", "chain")

    def ca_profile_read(self):
        ms = (ctypes.c_double * 5)()
        n = (ctypes.c_longlong * 5)()
        k = ctypes.c_longlong()
        st = self._lib.ca_profile_read(self.handle, ms, n, ctypes.byref(k))
        if st != CA_OK:
            raise CaError(st, "ca_profile_read")
        out = {"kernel_launches": k.value}
        for i, name in enumerate(self.PROFILE_CLASSES):
            out[f"{name}_ms"] = ms[i]
            out[f"{name}_launches"] = n[i]
        return out


class Server:
    """Serving loop (include/ca_serve.h): `workers` contexts on their own
    streams, FIFO admission by scratch footprint within `budget_bytes`.
    submit() returns at once with an id; wait(id) blocks until that request
    ended.  The arrays of a request stay referenced here until it ended."""

    def __init__(self, device: int = 0, workers: int = 4, budget_bytes: int = 8 << 30,
                 batch: int = 1):
        self._lib = load()
        h = ctypes.c_void_p()
        st = self._lib.ca_server_create(ctypes.byref(h), device, int(workers), int(budget_bytes))
        if st != CA_OK:
            raise CaError(st, "ca_server_create")
        self.handle = h
        self._keep = {}
        if batch > 1:  # groups of up to `batch` requests share launches
            st = self._lib.ca_server_set_batching(self.handle, int(batch))
            if st != CA_OK:
                raise CaError(st, "ca_server_set_batching")

    def submit(self, method, X, y, x, aux=None, *, b, s=1, H, lam, seed=42, prec="tf32",
               recompute_every=0, tol=0.0, check_every=0, stop="residual", solve="df", d=None,
               n=None, ld=None, panels=None) -> int:
        """method "primal" (X d x ld, x = w, aux = z or None) or "dual"
        (X = X^T n x ld, x = alpha, aux = w); panels=(rows, cols) for
        pre-packed FP32 panels.  s = 0: the server picks s by measured cost
        (the result's "s"); stop="objective": end at a certified relative
        objective error tol (the result's "gap" and "fval")."""
        m = {"primal": 0, "dual": 1}[method]
        o = Context._opts(b, s, H, lam, seed, prec, recompute_every, 0, tol, check_every, stop,
                          solve)
        if panels is not None:  # primal (d, n), dual (n, d)
            rows, cols = (int(v) for v in panels)
            xf, ldv = CA_DENSE_F32_PANELS, 0
        else:  # primal X: d x ld (n columns used), dual X^T: n x ld (d used)
            rows, ldv = X.shape
            xf = _xfmt(X)
            used = n if m == 0 else d
            cols = ldv if used is None else int(used)
            ldv = ldv if ld is None else int(ld)
        dd, nn = (rows, cols) if m == 0 else (cols, rows)
        r = ca_request(m, xf, _ptr(X), dd, nn, ldv, _ptr(y), _ptr(x), _ptr(aux), o)
        rid = ctypes.c_longlong()
        st = self._lib.ca_server_submit(self.handle, ctypes.byref(r), ctypes.byref(rid))
        if st != CA_OK:
            raise CaError(st, "ca_server_submit")
        self._keep[rid.value] = (X, y, x, aux)
        return rid.value

    def wait(self, rid: int) -> dict:
        out = ca_result()
        st = self._lib.ca_server_wait(self.handle, int(rid), ctypes.byref(out))
        if st != CA_OK:
            raise CaError(st, "ca_server_wait")
        self._keep.pop(int(rid), None)
        res = {f: getattr(out, f) for f, _ in ca_result._fields_}
        res["bound"] = res["bound"] if res["bound"] >= 0.0 else None  # -1: none formed
        return res

    def drain(self):
        st = self._lib.ca_server_drain(self.handle)
        if st != CA_OK:
            raise CaError(st, "ca_server_drain")

    def stats(self) -> dict:
        out = ca_server_stats()
        st = self._lib.ca_server_get_stats(self.handle, ctypes.byref(out))
        if st != CA_OK:
            raise CaError(st, "ca_server_get_stats")
        return {f: getattr(out, f) for f, _ in ca_server_stats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            self._lib.ca_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
