"""Benchmark: CA-BCD block updates per second on one GB300 (or N replicas).

Workload (the dense primal FP32 configuration): X 4096 x 262144 FP32 with
geometrically scaled rows (condition 1e3), y = X^T w_true + 1% noise,
lambda = 1e-4, b = 8, s = 16, H = 4096 block updates, BF16x3 split-product
Gram on the tensor cores (FP32 accumulation), double-float (~2^-44) b x b
solves and vector updates, FP64 vectors.  One step = one full solve (sampling, H/s outer steps of
gather+Gram+projection, inner solves, deferred update, and the final
z = X^T w_H pass) with X resident in HBM.  X (4 GiB) is larger than L2.
X is resident in the library's 32-column panel layout (packed once, as a
serving process keeps it); the same K solves from row-major X (each one
repacking X first) are reported beside the value.
The value comes from K timed solves without per-kernel events; the roofline
and the per-kernel breakdown from a second timed pass of K solves with CUDA
events around every launch (they cost a few percent of throughput).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  N > 1 runs N independent replicas (one per
GPU, launched by torchrun); value = total block updates / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CA-BCD block-updates/s"
UNIT = "block-updates/s"
D, N_SAMPLES, COND, LAM, B, S, H = 4096, 262144, 1e3, 1e-4, 8, 16, 4096
# Gram mode of the headline: x = b0 + b1 in BF16, three products, FP32
# accumulate (meets the FP32 path's 1e-5 iterate tolerance; the fastest mode
# that does)
PREC = "bf16x3"
_DF = "double-float (~2^-44) b x b solves and vector updates, fp64 vectors"
DTYPE = {"bf16x3": f"bf16x3 Gram (bf16 split products, fp32 accumulate); {_DF}",
         "fp16_scaled": f"fp16 Gram (per-row power-of-two scaling, fp32 accumulate); {_DF}",
         "3xtf32": f"3xtf32 Gram (fp32-faithful split products); {_DF}",
         "tf32": f"tf32 Gram (fp32 accumulate); {_DF}"}


def workload_config(d=D, n=N_SAMPLES, b=B, s=S, h=H, prec=PREC):
    return {
        "workload": f"dense primal CA-BCD, FP32 X {d}x{n} (cond 1e3 geometric rows), "
                    f"lambda 1e-4, b={b}, s={s}, H={h}, {prec} tcgen05 Gram, double-float solves",
        "d": d, "n": n, "b": b, "s": s, "H": h, "lambda": LAM, "gram": prec,
        "l2": "inputs larger than L2 (X is 4 GiB, L2 129 MB); no flush needed",
        "step": "one full solve of H block updates incl. sampling and final z = X^T w_H",
    }


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _traffic_record(kernel_src: str, name: str = "gram_tc_traffic.json"):
    """DRAM traffic of a kernel from the committed ncu summary, if it was
    taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as f:
            rec = json.load(f)
        with open(kernel_src, "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
        if rec.get("src_sha") == sha:
            return rec
    except (OSError, ValueError):
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"],
                    "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in self.rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(self.rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in self.rows)}


def max_over_ranks(value: float, world: int) -> float:
    """Maximum of a per-rank float over the process group (identity at N = 1)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def time_solves(ctx, X, y, w, z, steps, stream, b=B, s=S, h=H, prec=PREC, panels=None,
                solve="df"):
    """Device time (ms) of `steps` back-to-back solves, CUDA events on the
    library's stream.  panels=(d, n): X holds the 32-column panel layout."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        w.zero_()
        ctx.ca_bcd_solve(X, y, w, z, b=b, s=s, H=h, lam=LAM, seed=42, prec=prec, panels=panels,
                         solve=solve)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def certified_race(ctx, XP, y, pan, tol=1e-6, h_cap=1 << 17):
    """The headline solve in each Gram mode, run until its certified relative
    objective error (the duality gap bound gap / (f(w) - gap), a check every
    16 outer steps) is <= tol: wall time of the call (the checks wait for the
    GPU), block updates done, and the bound reached (h_cap block updates at
    most)."""
    import torch
    rows = []
    for prec_ in ("3xtf32", "bf16x3", "fp16_scaled", "tf32"):
        w_ = torch.zeros(D, dtype=torch.float64, device="cuda")
        kw = dict(b=B, s=S, H=h_cap, lam=LAM, seed=42, prec=prec_, panels=pan, tol=tol,
                  check_every=16, stop="objective")
        ctx.ca_bcd_solve(XP, y, w_, **kw)  # warm
        w_.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.ca_bcd_solve(XP, y, w_, **kw)
        dt = time.perf_counter() - t0
        info = ctx.solve_info()
        rows.append({"gram": prec_, "seconds_to_stop": dt, "h_done": info["h_done"],
                     "block_updates_per_s": info["h_done"] / dt,
                     "certified_rel_obj_err": info["bound"],
                     "certified": info["bound"] is not None and info["bound"] <= tol})
    return {"tol": tol, "how": "same solve per Gram mode, stop once gap <= tol (f(w) - gap); "
                               "wall time of the call", "rows": rows}


def cpu_baseline(X_host_f32, y_host, budget_s: float = 30.0):
    """The FP64 oracle as it stands (single thread) on a bounded sample of the
    workload: the first 4 outer steps (4 s block updates) of the same solve."""
    import numpy as np
    import oracle
    X64 = X_host_f32.astype(np.float64)
    h_sample = 4 * S
    t0 = time.perf_counter()
    oracle.ca_bcd(X64, y_host, LAM, b=B, s=S, H=h_sample, seed=42)
    dt = time.perf_counter() - t0
    return {"value": h_sample / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first 4 outer steps ({h_sample} block updates, b={B}, s={S}) of the "
                      f"same {D}x{N_SAMPLES} solve, FP64 C oracle, single thread; {dt:.2f} s"}


def run_reference(args, rank: int, world: int):
    """--impl reference: the FP64 oracle on the host cores, each step the first
    outer step (s block updates) of the workload."""
    if rank != 0:
        return 0
    import numpy as np
    import torch
    import oracle
    import synth
    oracle.build()
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    X, y, _ = synth.dense_primal_torch(D, N_SAMPLES, cond=COND, seed=1, device=dev)
    X64 = X.cpu().numpy().astype(np.float64)
    yh = y.cpu().numpy()
    del X
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.ca_bcd(X64, yh, LAM, b=B, s=S, H=S, seed=42)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    value = S / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"each step: first outer step ({S} block updates) of the "
                                   f"workload, FP64 C oracle, single thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _device_time(stream, fn, reps):
    """Average device time (ms) of fn() over reps calls, CUDA events on stream."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def secondary_workloads(ctx, stream):
    """The other configurations of the benchmark family, measured briefly:
    the sparse dual (CSR of X^T, CUDA-core Gram) and the tiny FP64 primal
    (both latency-bound: reported as block updates/s and us per outer step)."""
    import numpy as np
    import torch
    import synth
    out = []
    sp = synth.sparse_dual()  # d = 131072 features, n = 16384 samples, 0.5%, Pareto nnz
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rp, col, val, ys = dev(sp.rowptr), dev(sp.col), dev(sp.val), dev(sp.y)
    a = torch.zeros(sp.n, dtype=torch.float64, device="cuda")
    w = torch.zeros(sp.d, dtype=torch.float64, device="cuda")
    h_sp = 2048
    for s_ in (1, 8, 16, 32):
        def run():
            a.zero_()
            ctx.ca_bdcd_solve((rp, col, val), ys, a, w, b=8, s=s_, H=h_sp, lam=1e-5, seed=42,
                              d=sp.d, prec="f64")
        run()
        t = _device_time(stream, run, 3)
        out.append({"workload": "sparse dual CA-BDCD, CSR of X^T 16384 x 131072 (0.5%, Pareto "
                                "nnz per feature), lambda 1e-5, b=8, H=2048, CUDA-core FP64 Gram "
                                "(s*b < 32: one warp per row pair; s*b >= 32: dense part of the "
                                "features in at least a quarter of the samples + bucketed pair "
                                "products of the rest), next step's w-independent part on a "
                                "second stream",
                    "nnz": int(sp.rowptr[-1]), "s": s_, "ms_per_solve": t,
                    "block_updates_per_s": h_sp / (t * 1e-3),
                    "us_per_outer_step": t * 1e3 / -(-h_sp // s_)})
    del rp, col, val
    tp = synth.tiny_primal()
    Xt, yt = dev(tp.X), dev(tp.y)
    wt = torch.zeros(64, dtype=torch.float64, device="cuda")
    for s_ in (1, 4):
        def run_t():
            wt.zero_()
            ctx.ca_bcd_solve(Xt, yt, wt, b=4, s=s_, H=200, lam=1e-3, seed=42, prec="f64")
        run_t()
        t = _device_time(stream, run_t, 5)
        out.append({"workload": "tiny dense primal CA-BCD, X 64 x 1024 FP64, lambda 1e-3, b=4, "
                                "H=200, FP64 Gram", "s": s_, "ms_per_solve": t,
                    "block_updates_per_s": 200 / (t * 1e-3),
                    "us_per_outer_step": t * 1e3 / -(-200 // s_)})
    return out


def _uneven_problems(count, seed, d_range, n_range, H_sweeps=4, Hmax=2048, prec="bf16x3",
                     s_rule="fixed"):
    """Uneven dense ridge problems shaped like the served-batch workload:
    d and n log-uniform, FP32 X N(0,1) generated on the device, lambda
    log-uniform in [1e-6, 1e-1], half primal / half dual, b in {4, 8, 16},
    H = min(Hmax, H_sweeps N / b) block updates (N the sampled dimension)."""
    import math
    import numpy as np
    import torch
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        d = int(math.exp(rng.uniform(math.log(d_range[0]), math.log(d_range[1])))) // 32 * 32
        n = int(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))) // 32 * 32
        lam = float(math.exp(rng.uniform(math.log(1e-6), math.log(1e-1))))
        method = "primal" if i % 2 == 0 else "dual"
        b = int(rng.choice([4, 8, 16]))
        N = d if method == "primal" else n
        s_ = 0 if s_rule == "tuned" else max(1, 64 // b)
        H = int(max(b, min(Hmax, H_sweeps * N // b)))
        g = torch.Generator(device="cuda").manual_seed(1000 + i)
        if method == "primal":
            X = torch.randn(d, n, device="cuda", generator=g)
            y = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
            xs, auxs = d, n
        else:
            X = torch.randn(n, d, device="cuda", generator=g)
            y = torch.sign(torch.randn(n, dtype=torch.float64, device="cuda", generator=g))
            xs, auxs = n, d
        out.append(dict(method=method, X=X, y=y, xs=xs, auxs=auxs, d=d, n=n,
                        kw=dict(b=b, s=s_, H=H, lam=lam, seed=7 + i, prec=prec)))
    return out


def batch_study(ctx, stream, count=24):
    """The batched solves (ca_batch_solve) on uneven problems shaped like the
    served-batch workload, scaled to a short run (d 256-2048, n 4096-32768):
    the same problems one after another (each its own solve), in shared
    launches (plain and CUDA-graph-captured), and with the depth chosen by
    measured cost.  Block updates per second of the whole set."""
    import torch
    probs = _uneven_problems(count, 5, (256, 2048), (4096, 32768))
    total_h = sum(p["kw"]["H"] for p in probs)

    def fresh(p):
        return dict(method=p["method"], X=p["X"], y=p["y"],
                    x=torch.zeros(p["xs"], dtype=torch.float64, device="cuda"),
                    aux=torch.zeros(p["auxs"], dtype=torch.float64, device="cuda"), **p["kw"])

    def seq():
        for p in probs:
            x = torch.zeros(p["xs"], dtype=torch.float64, device="cuda")
            aux = torch.zeros(p["auxs"], dtype=torch.float64, device="cuda")
            (ctx.ca_bcd_solve if p["method"] == "primal" else ctx.ca_bdcd_solve)(
                p["X"], p["y"], x, aux, **p["kw"])

    def timed(fn, reps=2):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps

    out = {"problems": count, "block_updates": total_h,
           "workload": "uneven dense ridge problems, d 256-2048 and n 4096-32768 log-uniform, "
                       "FP32 X N(0,1), lambda 1e-6..1e-1, half primal / half dual, b in {4,8,16}, "
                       "s b = 64, H = min(2048, 4 N / b), BF16x3 Gram"}
    t = timed(seq)
    out["one_after_another"] = {"seconds": t, "block_updates_per_s": total_h / t}
    for name, graph in (("shared_launches", False), ("shared_launches_graph", True)):
        t = timed(lambda: ctx.ca_batch_solve([fresh(p) for p in probs], graph=graph))
        out[name] = {"seconds": t, "block_updates_per_s": total_h / t}
    tuned = [dict(fresh(p), s=0) for p in probs]
    t = timed(lambda: ctx.ca_batch_solve([dict(q, x=torch.zeros_like(q["x"]),
                                               aux=torch.zeros_like(q["aux"])) for q in tuned]))
    res = ctx.ca_batch_solve(tuned)
    out["shared_launches_graph_depth_by_cost"] = {
        "seconds": t, "block_updates_per_s": total_h / t,
        "rows_per_step_chosen": sorted({r["s"] * p["kw"]["b"] for r, p in zip(res, probs)})}
    del probs
    return out


def serve_config5(args):
    """The served-batch workload scaled to a bench-length run: a Poisson
    stream (2000 arrivals/s) of dense ridge requests with the configuration's
    distributions -- d log-uniform in [256, 8192], n log-uniform in [4096,
    131072], FP32 X N(0,1), lambda log-uniform in [1e-6, 1e-1], half primal /
    half dual, b in {4, 8, 16}, s by measured cost -- each stopping at a
    certified relative objective error of 1e-6 (duality gap, a check every 4
    outer steps) or after 32 sweeps of its sampled dimension (at most 32768
    block updates; a dual request with n >> d and a small lambda is
    conditioned like 1/lambda and certifies far later); batching on
    (groups of up to 8 requests share launches), 4 workers, 64 GB budget.
    Reports latency percentiles, throughput and how many results are
    certified, beside the same requests run one after another."""
    import numpy as np
    import torch
    import paper_1612_04003_gb300 as ca
    M = args.serve5_requests
    probs = _uneven_problems(M, 11, (256, 8192), (4096, 131072), H_sweeps=32, Hmax=1 << 15,
                             s_rule="tuned")
    for p in probs:
        p["kw"].update(check_every=4, tol=1e-6, stop="objective")
    torch.cuda.synchronize()
    rng = np.random.default_rng(12)
    arrivals = np.cumsum(rng.exponential(1.0 / 2000.0, size=M))

    def fresh(p):
        return (torch.zeros(p["xs"], dtype=torch.float64, device="cuda"),
                torch.zeros(p["auxs"], dtype=torch.float64, device="cuda"))

    # one after another on one context (s = 16 for b <= 8, 8 for b = 16)
    ctx = ca.Context(0)
    t0 = time.perf_counter()
    h_seq, cert_seq = 0, 0
    for p in probs:
        x, aux = fresh(p)
        kw = dict(p["kw"], s=128 // p["kw"]["b"] if p["kw"]["b"] > 8 else 16)
        (ctx.ca_bcd_solve if p["method"] == "primal" else ctx.ca_bdcd_solve)(
            p["X"], p["y"], x, aux, **kw)
        inf = ctx.solve_info()
        h_seq += inf["h_done"]
        cert_seq += inf["bound"] is not None and inf["bound"] <= 1e-6
    seq_s = time.perf_counter() - t0
    ctx.close()
    srv = ca.Server(0, workers=4, budget_bytes=64 << 30, batch=8)
    ids = []
    t0 = time.perf_counter()
    for p, at in zip(probs, arrivals):
        delay = at - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        x, aux = fresh(p)
        ids.append(srv.submit(p["method"], p["X"], p["y"], x, aux, **p["kw"]))
    res = [srv.wait(i) for i in ids]
    st = srv.stats()
    srv.close()
    certified = [r for r in res if r["status"] == ca.CA_OK and r["bound"] is not None
                 and r["bound"] <= 1e-6]
    cert = len(certified)
    lat_c = sorted(r["latency_ms"] for r in certified)
    pct = (lambda q: lat_c[min(len(lat_c), max(1, int(np.ceil(q * len(lat_c))))) - 1]
           if lat_c else None)
    out = {"workload": "served-batch distributions (d 256-8192, n 4096-131072 log-uniform, "
                       "half primal / half dual, b in {4,8,16}, lambda 1e-6..1e-1, FP32 X), "
                       "%d requests (of the configuration's 4000) at 2000/s; stop at a certified "
                       "1e-6 relative objective error or 32 sweeps (<= 32768 block updates); BF16x3 Gram" % M,
           "requests": M, "ok": sum(1 for r in res if r["status"] == ca.CA_OK),
           "certified_1e-6": cert,
           "certified_p50_ms": pct(0.50), "certified_p99_ms": pct(0.99),
           "certified_primal": sum(1 for r, p in zip(res, probs) if p["method"] == "primal"
                                   and r["bound"] is not None and r["bound"] <= 1e-6),
           "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
           "mean_ms": st["mean_ms"], "max_ms": st["max_ms"], "wall_s": st["wall_s"],
           "requests_per_s": st["completed"] / max(st["wall_s"], 1e-9),
           "block_updates_per_s": st["block_updates_per_s"],
           "peak_concurrency": st["peak_concurrency"],
           "peak_footprint_gb": st["peak_footprint"] / 2**30,
           "arrival_span_s": float(arrivals[-1]),
           "sequential": {"wall_s": seq_s, "block_updates_per_s": h_seq / seq_s,
                          "certified_1e-6": cert_seq,
                          "how": "the same requests one after another on one context"}}
    del probs
    return out


def gram_conditioning(ctx, X, lam, b, n_outer=64, s_list=(1, 2, 4, 8, 16)):
    """Condition numbers of the s*b x s*b Gram matrices Y Y^T / n + lambda I
    that the solve factors (the first n_outer outer steps of the seed-42
    index stream, for each s), from the library's sampler and its FP64 Gram
    of the FP32 X; the condition number itself is analysis (torch, FP64).
    Returns min / median / max per s."""
    import torch
    d, n = X.shape
    smax = max(s_list)
    idx_all = torch.empty(n_outer * smax * b, dtype=torch.int32, device="cuda")
    ctx.ca_sample_indices(42, 0, n_outer * smax, b, d, idx_all)
    v0 = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = {}
    for s_ in s_list:
        sb = s_ * b
        G = torch.empty((sb, sb), dtype=torch.float64, device="cuda")
        p = torch.empty(sb, dtype=torch.float64, device="cuda")
        eye = torch.eye(sb, dtype=torch.float64, device="cuda")
        cs = []
        for k in range(n_outer):
            ctx.ca_gram_project(X, idx_all[k * sb:(k + 1) * sb], v0, G, p, prec="f64")
            cs.append(float(torch.linalg.cond(G / n + lam * eye)))
        cs.sort()
        out[f"s={s_}"] = {"min": cs[0], "median": cs[len(cs) // 2], "max": cs[-1]}
    return {"b": b, "outer_steps": n_outer, "cond_gram": out}


def precision_study(args, emit=True):
    """--precision-study: the precision configuration of the benchmark family:
    X 8192 x 131072 FP32 with geometric row scaling (condition 1e2, 1e4, 1e6),
    lambda 1e-6, b = s = 16, H = 8192, recompute every 8 outer steps.  Each
    Gram mode's w_H against the FP64 path on the same data (FP64 X, FP64
    Gram; the path checked against the FP64 oracle), the relative objective
    difference, and block updates/s.  One JSON line."""
    import torch
    import paper_1612_04003_gb300 as ca
    import synth
    ca.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = ca.Context(0, stream=stream.cuda_stream)
    d, n, lam, b, s_, H = 8192, 131072, 1e-6, 16, 16, 8192
    rows, gram_cond = [], []
    for cond in (1e2, 1e4, 1e6):
        X, y, _ = synth.dense_primal_torch(d, n, cond=cond, seed=1, device="cuda")
        kw = dict(b=b, s=s_, H=H, lam=lam, seed=42, recompute_every=8)

        def objective(w):
            r = X.double().T @ w - y
            return float(0.5 * lam * w.dot(w) + 0.5 / n * r.dot(r))

        X64 = X.double()
        w_ref = torch.zeros(d, dtype=torch.float64, device="cuda")
        t64 = _device_time(stream, lambda: ctx.ca_bcd_solve(X64, y, w_ref.zero_(), prec="f64", **kw), 1)
        del X64
        f_ref = objective(w_ref)
        for prec in ("3xtf32", "bf16x3", "tf32", "fp16_scaled"):
            w = torch.zeros(d, dtype=torch.float64, device="cuda")
            ctx.ca_bcd_solve(X, y, w, prec=prec, **kw)
            t = _device_time(stream, lambda: ctx.ca_bcd_solve(X, y, w.zero_(), prec=prec, **kw), 2)
            rel_w = float((w - w_ref).norm() / w_ref.norm())
            f = objective(w)
            # the same solve with one check at its end: the certified relative
            # objective error of w_H (duality gap)
            wc = torch.zeros(d, dtype=torch.float64, device="cuda")
            ctx.ca_bcd_solve(X, y, wc, prec=prec, check_every=H // s_, stop="objective", **kw)
            rows.append({"cond": cond, "gram": prec, "rel_err_w_vs_fp64": rel_w,
                         "rel_objective_diff": abs(f - f_ref) / abs(f_ref),
                         "certified_rel_obj_err": ctx.solve_info()["bound"],
                         "block_updates_per_s": H / (t * 1e-3)})
        rows.append({"cond": cond, "gram": "f64 (FP64 X, reference)", "rel_err_w_vs_fp64": 0.0,
                     "rel_objective_diff": 0.0, "block_updates_per_s": H / (t64 * 1e-3)})
        gram_cond.append({"cond": cond, **gram_conditioning(ctx, X, lam, b)})
        del X, y
    out = {"study": "precision", "workload": "dense primal CA-BCD, X 8192 x 131072 FP32, "
           "lambda 1e-6, b=16, s=16, H=8192, recompute every 8 outer steps",
           "rows": rows, "gram_conditioning": gram_cond}
    ctx.close()
    if emit:
        print(json.dumps(out), flush=True)
        return 0
    return out


def _trajectory(tr, f_star, keep=48):
    """Rows of a check trace: relative residual, certified and true relative
    objective error (f* known to within its own certificate; None: f* not
    certified, no true error); at most keep rows, evenly spaced, the first
    and last included."""
    r0 = tr[0]["res"] if tr and tr[0]["res"] > 0 else 1.0
    idx = sorted(set(int(round(i * (len(tr) - 1) / max(keep - 1, 1))) for i in range(keep)))
    rows = []
    for i in idx:
        c = tr[i]
        f, g = c["fval"], c["gap"]
        rows.append({"h": c["h"], "rel_residual": c["res"] / r0,
                     "certified_rel_obj_err": (g / (f - g)) if f > g else None,
                     "true_rel_obj_err": (f - f_star) / f_star if f_star else None})
    return rows


def stopping_study(args) -> int:
    """--stopping-study: the stopping test along a solve (Sec. 5.1.5; the
    analogue of the paper's stopping-criterion figure).  At every check: the
    relative residual ||r||/||r_0||, the certified relative objective error
    gap/(f - gap) (duality gap) and the true relative objective error
    (f - f*)/f*, with f* from the same solve continued to a certified 1e-13
    (f* taken as f - gap/2 there; reported only when that run certified
    1e-9 or better).  Dense primal CA-BCD on
    the benchmark's X 4096 x 262144 FP32 (BF16x3 Gram, b = 8, s = 16,
    lambda 1e-4, a check every 4 outer steps) and sparse dual CA-BDCD on the
    CSR of X^T 16384 x 131072 (b = 8, s = 8, lambda 1e-5, FP64, f of the model
    w(alpha)).  One JSON line."""
    import numpy as np
    import torch
    import paper_1612_04003_gb300 as ca
    import synth
    ca.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = ca.Context(0, stream=stream.cuda_stream)
    out = {}
    X, y, _ = synth.dense_primal_torch(D, N_SAMPLES, cond=COND, seed=1, device="cuda")
    Xp = torch.empty(((N_SAMPLES + 31) // 32) * D * 32, dtype=torch.float32, device="cuda")
    ctx.ca_pack_panels(X, Xp)
    del X
    w = torch.zeros(D, dtype=torch.float64, device="cuda")
    kw = dict(b=B, s=S, lam=LAM, seed=42, prec=PREC, panels=(D, N_SAMPLES), stop="objective")
    ctx.ca_bcd_solve(Xp, y, w, H=1 << 18, tol=1e-13, check_every=64, **kw)
    fin = ctx.solve_info()
    # f* to within gap/2; unusable unless certified tightly
    certified = fin["bound"] is not None and fin["bound"] <= 1e-9
    f_star = fin["fval"] - fin["gap"] / 2 if certified else None
    w.zero_()
    h_run = max(S, min(1 << 18, fin["h_done"]))
    ctx.ca_bcd_solve(Xp, y, w, H=h_run, tol=0.0, check_every=4, **kw)
    out["primal"] = {"workload": "dense primal CA-BCD, X 4096 x 262144 FP32 (cond 1e3), "
                                 "lambda 1e-4, b=8, s=16, BF16x3 Gram, a check every 4 outer steps",
                     "f_star": f_star, "f_star_certified_rel": fin["bound"],
                     "h_to_certify_1e-13": fin["h_done"],
                     "rows": _trajectory(ctx.solve_trace(), f_star)}
    del Xp, y
    sp = synth.sparse_dual()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    csr = (dev(sp.rowptr), dev(sp.col), dev(sp.val))
    ys = dev(sp.y)
    a = torch.zeros(sp.n, dtype=torch.float64, device="cuda")
    wd = torch.zeros(sp.d, dtype=torch.float64, device="cuda")
    kw = dict(b=8, s=8, lam=1e-5, seed=42, prec="f64", d=sp.d, stop="objective")
    ctx.ca_bdcd_solve(csr, ys, a, wd, H=1 << 17, tol=1e-13, check_every=16, **kw)
    fin = ctx.solve_info()
    certified = fin["bound"] is not None and fin["bound"] <= 1e-9
    f_star = fin["fval"] - fin["gap"] / 2 if certified else None
    a.zero_()
    h_run = max(8, min(1 << 17, fin["h_done"]))
    ctx.ca_bdcd_solve(csr, ys, a, wd, H=h_run, tol=0.0, check_every=4, **kw)
    out["dual"] = {"workload": "sparse dual CA-BDCD, CSR of X^T 16384 x 131072 (0.5%, Pareto "
                               "nnz per feature), lambda 1e-5, b=8, s=8, a check every 4 outer steps",
                   "f_star": f_star, "f_star_certified_rel": fin["bound"],
                   "h_to_certify_1e-13": fin["h_done"],
                   "rows": _trajectory(ctx.solve_trace(), f_star)}
    ctx.close()
    print(json.dumps({"study": "stopping", **out}), flush=True)
    return 0


def serve_study(args) -> int:
    """--serve: the serving loop (include/ca_serve.h) on a Poisson stream of
    dense ridge requests shaped like the served-batch workload, scaled to a
    short run: d log-uniform in [256, 2048], n log-uniform in [4096, 32768],
    FP32 X N(0,1), lambda log-uniform in [1e-6, 1e-1], half primal / half
    dual, b in {4, 8, 16}, s = min(16, 128 / b), H = min(2048, 4 N / b)
    block updates (4 sweeps of the sampled dimension), BF16x3 Gram, the
    stopping test every 8 outer steps at ||r|| <= 1e-6 ||r_0|| (--serve-stop
    residual) or at a certified relative objective error <= 1e-6 (--serve-stop
    objective: duality gap <= 1e-6 (f(w) - gap)).  Reports
    latency percentiles, throughput and peak concurrency, and the same
    requests run one after another on one context.  One JSON line."""
    import math
    import numpy as np
    import torch
    import paper_1612_04003_gb300 as ca
    ca.build()
    rng = np.random.default_rng(11)
    M, rate = args.serve_requests, args.serve_rate
    reqs = []
    for i in range(M):
        # rounded to multiples of 32 (16-byte rows for the tensor-core Gram)
        d = int(math.exp(rng.uniform(math.log(256), math.log(2048)))) // 32 * 32
        n = int(math.exp(rng.uniform(math.log(4096), math.log(32768)))) // 32 * 32
        lam = float(math.exp(rng.uniform(math.log(1e-6), math.log(1e-1))))
        method = "primal" if i % 2 == 0 else "dual"
        b = int(rng.choice([4, 8, 16]))
        N = d if method == "primal" else n
        s_ = min(16, 128 // b)
        H = int(min(2048, 4 * N // b))
        g = torch.Generator(device="cuda").manual_seed(100 + i)
        if method == "primal":
            X = torch.randn(d, n, device="cuda", generator=g)
            y = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
            xs, auxs = d, n
        else:
            X = torch.randn(n, d, device="cuda", generator=g)  # X^T
            y = torch.sign(torch.randn(n, dtype=torch.float64, device="cuda", generator=g))
            xs, auxs = n, d
        reqs.append(dict(method=method, X=X, y=y, xs=xs, auxs=auxs,
                         kw=dict(b=b, s=s_, H=H, lam=lam, seed=7 + i, prec="bf16x3",
                                 check_every=8, tol=1e-6, stop=args.serve_stop)))
    torch.cuda.synchronize()

    def fresh(r):
        return (torch.zeros(r["xs"], dtype=torch.float64, device="cuda"),
                torch.zeros(r["auxs"], dtype=torch.float64, device="cuda"))

    # one after another on one context (the plain form)
    ctx = ca.Context(0)
    for r in reqs[:2]:  # warm
        x, aux = fresh(r)
        (ctx.ca_bcd_solve if r["method"] == "primal" else ctx.ca_bdcd_solve)(
            r["X"], r["y"], x, aux, **r["kw"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h_seq = 0
    for r in reqs:
        x, aux = fresh(r)
        (ctx.ca_bcd_solve if r["method"] == "primal" else ctx.ca_bdcd_solve)(
            r["X"], r["y"], x, aux, **r["kw"])
        h_seq += ctx.solve_info()["h_done"]
    seq_s = time.perf_counter() - t0
    ctx.close()
    # served: Poisson arrivals
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=M))
    srv = ca.Server(0, workers=args.serve_workers, budget_bytes=args.serve_budget_gb << 30)
    outs, ids = [], []
    t0 = time.perf_counter()
    for r, at in zip(reqs, arrivals):
        delay = at - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        x, aux = fresh(r)
        outs.append((x, aux))
        ids.append(srv.submit(r["method"], r["X"], r["y"], x, aux, **r["kw"]))
    res = [srv.wait(i) for i in ids]
    st = srv.stats()
    srv.close()
    ok = sum(1 for v in res if v["status"] == ca.CA_OK)
    print(json.dumps({
        "study": "serve", "workload": "Poisson stream of %d dense ridge requests at %.0f/s "
        "(d 256-2048, n 4096-32768 log-uniform, half primal / half dual, BF16x3 Gram, "
        "stopping at %s)" % (M, rate, {"residual": "1e-6 relative residual",
                                       "objective": "a certified 1e-6 relative objective error"}
                          [args.serve_stop]),
        "workers": args.serve_workers, "budget_gb": args.serve_budget_gb,
        "completed": st["completed"], "ok": ok, "rejected": st["rejected"],
        "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
        "max_ms": st["max_ms"], "wall_s": st["wall_s"],
        "requests_per_s": st["completed"] / max(st["wall_s"], 1e-9),
        "block_updates_per_s": st["block_updates_per_s"],
        "peak_concurrency": st["peak_concurrency"],
        "peak_footprint_gb": st["peak_footprint"] / 2**30,
        "stopped_early": sum(1 for v, r in zip(res, reqs) if v["h_done"] < r["kw"]["H"]),
        "certified_1e-6": (sum(1 for v in res if v["fval"] > v["gap"] and
                               v["gap"] <= 1e-6 * (v["fval"] - v["gap"]))
                           if args.serve_stop == "objective" else None),
        "sequential": {"wall_s": seq_s, "block_updates_per_s": h_seq / seq_s,
                       "how": "the same requests one after another on one context"},
        "arrival_span_s": float(arrivals[-1])}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-sweep", action="store_true", help="skip the s sweep and the other workloads")
    ap.add_argument("--precision-study", action="store_true",
                    help="run the precision study (8192 x 131072, cond 1e2..1e6) instead")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve", action="store_true",
                    help="run the serving study (Poisson stream of ridge requests) instead")
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--serve-rate", type=float, default=400.0, help="arrivals per second")
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--serve-budget-gb", type=int, default=32)
    ap.add_argument("--serve-stop", default="residual", choices=["residual", "objective"],
                    help="stopping rule of the served requests")
    ap.add_argument("--stopping-study", action="store_true",
                    help="relative residual, certified and true objective error along a solve")
    ap.add_argument("--s", type=int, default=None, help="unrolling depth (default %d)" % S)
    ap.add_argument("--n", type=int, default=None,
                    help="samples (columns of X); smaller than the default only for profiler captures")
    ap.add_argument("--h", type=int, default=None, help="block updates per solve (default %d)" % H)
    ap.add_argument("--quick", action="store_true",
                    help="skip the batch, served-stream and precision legs of the default line")
    ap.add_argument("--serve5-requests", type=int, default=160,
                    help="requests of the served-batch leg of the default line")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.precision_study:
        return precision_study(args)
    if args.serve:
        return serve_study(args)
    if args.stopping_study:
        return stopping_study(args)
    s_run = args.s or S
    n_run = args.n or N_SAMPLES
    h_run = args.h or H

    import numpy as np
    import torch
    import paper_1612_04003_gb300 as ca
    import synth

    ca.build()
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    X, y, _ = synth.dense_primal_torch(D, n_run, cond=COND, seed=1, device="cuda")
    w = torch.zeros(D, dtype=torch.float64, device="cuda")
    z = torch.zeros(n_run, dtype=torch.float64, device="cuda")
    ctx = ca.Context(local_rank, stream=stream.cuda_stream)
    # X resident in the library's storage layout (32-column panels), packed
    # once: repeated solves on the same X (the serving case) read only this
    XP = torch.empty(((n_run + 31) // 32 * D * 32,), dtype=torch.float32, device="cuda")
    ctx.ca_pack_panels(X, XP)
    pan = (D, n_run)

    # warm-up
    time_solves(ctx, XP, y, w, z, args.warmup, stream, s=s_run, h=h_run, panels=pan)
    time_solves(ctx, X, y, w, z, 1, stream, s=s_run, h=h_run)
    # timed region (value): K solves, no per-kernel events
    ctx.ca_profile_enable(False)  # resets the launch counter
    clocks = ClockSampler(local_rank)
    clocks.start()
    barrier(world)
    ms = time_solves(ctx, XP, y, w, z, args.steps, stream, s=s_run, h=h_run, panels=pan)
    barrier(world)
    launches = ctx.ca_profile_read()["kernel_launches"]
    # the same K solves from row-major X (each solve repacks X first)
    barrier(world)
    ms_rm = time_solves(ctx, X, y, w, z, args.steps, stream, s=s_run, h=h_run)
    barrier(world)
    # the same K solves with one Gram launch and one solve launch per outer
    # step instead of the persistent launch
    ctx.ca_set_tuning(persistent=False)
    time_solves(ctx, XP, y, w, z, 1, stream, s=s_run, h=h_run, panels=pan)
    barrier(world)
    ms_ps = time_solves(ctx, XP, y, w, z, args.steps, stream, s=s_run, h=h_run, panels=pan)
    barrier(world)
    # ... and its Gram pass alone (events around each launch, two solves)
    ctx.ca_profile_enable(True)
    time_solves(ctx, XP, y, w, z, 2, stream, s=s_run, h=h_run, panels=pan)
    prof_ps = ctx.ca_profile_read()
    ctx.ca_profile_enable(False)
    ctx.ca_set_tuning(persistent=True)
    # second timed pass (roofline, breakdown): the same K solves with CUDA
    # events around every launch, on the library's stream
    ctx.ca_profile_enable(True)
    barrier(world)
    ms_prof = time_solves(ctx, XP, y, w, z, args.steps, stream, s=s_run, h=h_run, panels=pan)
    barrier(world)
    clocks.stop()
    prof = ctx.ca_profile_read()
    ctx.ca_profile_enable(False)
    ms_step = max_over_ranks(ms / args.steps, world)
    value = world * h_run / (ms_step * 1e-3)
    ms_step_rm = max_over_ranks(ms_rm / args.steps, world)

    # roofline of the dominant kernel: the persistent launch of the outer
    # steps (ca_persist.cu) when the solve runs it, else the tcgen05 Gram pass
    # (one launch per outer step)
    peaks, peak_kind = _peaks()
    sb = s_run * B
    n_outer = -(-h_run // s_run)
    gram_launches_per_solve = prof["gram_launches"] / max(1, args.steps)
    persistent = gram_launches_per_solve < n_outer / 2
    fused = sb <= 128 and PREC in ("tf32", "3xtf32", "bf16x3", "fp16_scaled")
    b_gram = sb * n_run * 4 + n_run * 8          # B_G: Y rows + the projection vector
    b_upd = sb * n_run * 4 + 2 * n_run * 8       # B_U: Y rows + read/write of v
    breakdown = {c: {"ms_per_step": prof[f"{c}_ms"] / args.steps,
                     "share": prof[f"{c}_ms"] / max(ms_prof, 1e-9)}
                 for c in ("gram", "reduce", "chain", "update", "other")}
    # algorithmic bytes of the Gram-class launches of one solve: every outer
    # step reads its rows and v (B_G), and every step but the last applies
    # its deferred update inside the next step's pass (B_U)
    solve_bytes = n_outer * b_gram + (n_outer - 1) * b_upd if fused else n_outer * b_gram
    alg_bytes = solve_bytes / gram_launches_per_solve
    gram_ms = prof["gram_ms"] / max(1, prof["gram_launches"])
    achieved = alg_bytes / (gram_ms * 1e-3) / 1e9
    if persistent:
        trec = _traffic_record(os.path.join(ROOT, "paper_1612_04003_gb300", "csrc", "ca_persist.cu"),
                               "persist_traffic.json")
        traffic = (trec["traffic_bytes_per_pass"] * n_outer / gram_launches_per_solve
                   if trec else None)
        kname = (f"k_persist<128,{PREC}> (persistent cooperative launch of the outer steps: "
                 "gather + Gram + cross Gram + projection + deferred updates on 151 CTAs, "
                 "reduction of each step's partials, chain of the s solves on one CTA)")
    else:
        trec = _traffic_record(os.path.join(ROOT, "paper_1612_04003_gb300", "csrc", "ca_gram_tc.cu"))
        traffic = trec["traffic_bytes_per_launch"] if trec else None
        kname = (f"k_gram_tc<{128 if sb <= 128 else 256},{PREC}"
                 f"{',fused update' if fused else ''}> (gather + Gram + projection"
                 f"{' + deferred update of the previous outer step' if fused else ''})")
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "kernel": kname,
            "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": gram_ms,
            "launches": prof["gram_launches"], "peak_source": f"hbm_gbs ({peak_kind})",
            "gram_share_of_step": prof["gram_ms"] / max(ms_prof, 1e-9),
            "measured": "CUDA events around each launch on the library stream, over a second "
                        "timed pass of the same K solves (ms_per_step of that pass: %.3f)"
                        % (ms_prof / args.steps)}
    roof["breakdown"] = breakdown
    # the per-step path's Gram pass (one fused launch per outer step): the
    # roofline of that kernel alone, HBM idle between its launches
    g_ps = prof_ps["gram_ms"] / max(1, prof_ps["gram_launches"])
    per_launch_ps = solve_bytes / max(1.0, prof_ps["gram_launches"] / 2)
    ach_ps = per_launch_ps / (g_ps * 1e-3) / 1e9
    trec_ps = _traffic_record(os.path.join(ROOT, "paper_1612_04003_gb300", "csrc", "ca_gram_tc.cu"))
    roof_gram_pass = {"bound": "hbm", "achieved": ach_ps, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                      "frac": ach_ps / peaks["hbm_gbs"], "avg_launch_ms": g_ps,
                      "algorithmic_bytes_per_launch": per_launch_ps,
                      "traffic": trec_ps["traffic_bytes_per_launch"] if trec_ps else None,
                      "kernel": f"k_gram_tc<128,{PREC},fused update> (launches per step)",
                      "share_of_step": prof_ps["gram_ms"] / max(1e-9, 2 * ms_ps / args.steps)}

    # end to end through the C ABI with host buffers (pinned), copies inside
    Xh = torch.empty((D, n_run), dtype=torch.float32, pin_memory=True)
    Xh.copy_(X)
    yh = torch.empty(n_run, dtype=torch.float64, pin_memory=True)
    yh.copy_(y)
    wh = torch.zeros(D, dtype=torch.float64, pin_memory=True)
    e2e_steps = max(3, min(args.steps, 10))
    ctx.ca_bcd_solve(Xh, yh, wh, None, b=B, s=s_run, H=h_run, lam=LAM, seed=42, prec=PREC)  # warm
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        wh.zero_()
        ctx.ca_bcd_solve(Xh, yh, wh, None, b=B, s=s_run, H=h_run, lam=LAM, seed=42, prec=PREC)
    t_e2e = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world)
    e2e = {"value": world * h_run / t_e2e, "unit": UNIT,
           "h2d_bytes_per_step": int(Xh.numel() * 4 + yh.numel() * 8 + wh.numel() * 8),
           "d2h_bytes_per_step": int(wh.numel() * 8), "ms_per_step": t_e2e * 1e3,
           "how": "ca_bcd_solve on pinned host X, y, w: the library copies them to the device "
                  "and w_H back inside each call; wall clock, synchronous call"}
    del Xh

    # s sweep (same data, fewer steps): s-step against s = 1
    sweep = []
    if not args.no_sweep:
        for prec_ in ("3xtf32", "bf16x3", "tf32", "fp16_scaled"):
            for (b_, s_) in [(8, 1), (8, 4), (8, 8), (8, 16), (8, 32), (32, 1), (32, 4), (32, 8)]:
                nst = 2 if s_ == 1 else 4
                time_solves(ctx, XP, y, w, z, 1, stream, b=b_, s=s_, h=h_run, prec=prec_, panels=pan)
                t = time_solves(ctx, XP, y, w, z, nst, stream, b=b_, s=s_, h=h_run, prec=prec_,
                                panels=pan) / nst
                sweep.append({"gram": prec_, "b": b_, "s": s_, "ms_per_step": t,
                              "block_updates_per_s": h_run / (t * 1e-3)})

    # the b x b solves in FP64 (block Cholesky, CA_SOLVE_F64) against the
    # double-float default, same K solves
    solve_f64 = None
    race = None
    if not args.no_sweep:
        time_solves(ctx, XP, y, w, z, 1, stream, s=s_run, h=h_run, panels=pan, solve="f64")
        t64 = time_solves(ctx, XP, y, w, z, 4, stream, s=s_run, h=h_run, panels=pan,
                          solve="f64") / 4
        solve_f64 = {"ms_per_step": t64, "block_updates_per_s": h_run / (t64 * 1e-3),
                     "how": "same solve with opts.solve = CA_SOLVE_F64 (FP64 Cholesky of each "
                            "diagonal block, FP64 block forward substitution, one CTA)"}
        race = certified_race(ctx, XP, y, pan)

    # the same roofline for the other Gram modes, same K solves
    roof_other = {}
    secondary = []
    if not args.no_sweep:
        for prec_ in [p for p in ("3xtf32", "bf16x3", "tf32", "fp16_scaled") if p != PREC]:
            time_solves(ctx, XP, y, w, z, 1, stream, s=s_run, h=h_run, prec=prec_, panels=pan)
            ctx.ca_profile_enable(True)
            time_solves(ctx, XP, y, w, z, args.steps, stream, s=s_run, h=h_run, prec=prec_,
                        panels=pan)
            p32 = ctx.ca_profile_read()
            ctx.ca_profile_enable(False)
            g32 = p32["gram_ms"] / max(1, p32["gram_launches"])
            per_solve = p32["gram_launches"] / max(1, args.steps)
            ach32 = solve_bytes / per_solve / (g32 * 1e-3) / 1e9
            pers32 = per_solve < n_outer / 2
            roof_other[prec_] = {"bound": "hbm", "achieved": ach32, "peak": peaks["hbm_gbs"],
                                 "unit": "GB/s", "frac": ach32 / peaks["hbm_gbs"],
                                 "avg_launch_ms": g32, "launches_per_solve": per_solve,
                                 "kernel": (f"k_persist<128,{prec_}>" if pers32 else
                                            f"k_gram_tc<128,{prec_},fused update>")}
        secondary = secondary_workloads(ctx, stream)

    batch = serve5 = prec_study = None
    if not args.no_sweep and not args.quick and rank == 0:
        batch = batch_study(ctx, stream)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(X.cpu().numpy(), y.cpu().numpy())

    if not args.no_sweep and not args.quick and rank == 0:
        del X, XP
        torch.cuda.empty_cache()
        serve5 = serve_config5(args)
        torch.cuda.empty_cache()
        prec_study = precision_study(args, emit=False)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[PREC], "data": "synthetic",
            "config": workload_config(n=n_run, s=s_run, h=h_run),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks.summary(), "sweep": sweep,
            "solve_fp64": solve_f64, "time_to_certified_1e-6": race,
            **{f"roofline_{p}_gram": r for p, r in roof_other.items()},
            "other_workloads": secondary,
            "batch": batch, "serve": serve5, "precision_study": prec_study,
            "input_layout": "X resident on the device in the library's 32-column panel layout "
                            "(ca_pack_panels once before the timed region, CA_DENSE_F32_PANELS)",
            "roofline_gram_pass_launches_per_step": roof_gram_pass,
            "value_launches_per_step": {
                "value": world * h_run / (max_over_ranks(ms_ps / args.steps, world) * 1e-3),
                "ms_per_step": max_over_ranks(ms_ps / args.steps, world),
                "how": "same K solves with one Gram launch and one reduce + chain launch per "
                       "outer step (ca_set_tuning persistent off)"},
            "value_rowmajor_input": {"value": world * h_run / (ms_step_rm * 1e-3),
                                     "ms_per_step": ms_step_rm,
                                     "how": "same K solves from row-major X; each solve first "
                                            "repacks X into panels (one pass over X)"},
            "parallelism": "replicas" if world > 1 else "single GPU",
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
