"""Pins for the FP64 oracle against facts fixed outside the oracle itself.

Each test cites the passage of the paper (section / algorithm / equation) or
the mathematical fact it checks.  None re-types the oracle's formulas: the
references are numpy's library routines (Philox bit generator, linalg.solve),
closed forms, exactness properties and statistics.
"""
import math

import numpy as np
import pytest

import oracle
import synth

LAM1 = 1e-3


@pytest.fixture(scope="module")
def tiny():
    """The tiny dense primal workload: X 64 x 1024 iid N(0,1), lambda = 1e-3."""
    return synth.tiny_primal(d=64, n=1024, seed=1)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


# ---------------------------------------------------------------------------
# Sampler (Alg. 1-4: "uniformly at random without replacement")
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("key", [0, 1, 42, 2**64 - 1, 12345678901234567890,
                                 2**100 + 7])
@pytest.mark.parametrize("ctr", [0, 5, 2**64 - 1, 2**130 + 3])
def test_philox_matches_numpy_library(key, ctr):
    """Library pin: numpy's Philox bit generator is Philox4x64-10 (Salmon et al.).
    numpy increments its 256-bit counter before each block of four words."""
    g = np.random.Philox(key=key, counter=ctr)
    raw = g.random_raw(8)
    for blk in range(2):
        c = ctr + 1 + blk
        words = [(c >> (64 * i)) & (2**64 - 1) for i in range(4)]
        mine = oracle.philox4x64_10(words, [key & (2**64 - 1), key >> 64])
        assert [int(x) for x in mine] == [int(x) for x in raw[4 * blk:4 * blk + 4]]


@pytest.mark.parametrize("J", [0, 1, 2, 6, 1000, 2**31 - 2, 2**40 + 11])
def test_map_to_range_preimages(J):
    """floor(u (J+1) / 2^64) sends exactly the u in
    [ceil(t 2^64/(J+1)), ceil((t+1) 2^64/(J+1))) to t: check both edges."""
    M = 2**64
    rng = np.random.default_rng(J)
    ts = {0, J, J // 2} | {int(x) for x in rng.integers(0, J + 1, size=4)}
    for t in ts:
        lo = -((-t * M) // (J + 1))        # ceil(t M / (J+1))
        hi = -((-(t + 1) * M) // (J + 1))  # first u of t+1
        assert oracle.map_to_range(lo, J) == t
        assert oracle.map_to_range(hi - 1, J) == t
        if lo > 0:
            assert oracle.map_to_range(lo - 1, J) == t - 1


def test_sampler_first_draw_is_mapped_philox_word():
    """Draw m = 0 of block h sees an empty set, so it is the first Philox word of
    counter (h, 0, 0, 0) under key (seed, 0) mapped to [0, N-b]."""
    for seed, h, b, N in [(42, 0, 4, 64), (7, 12345, 8, 4096), (1, 2**40, 3, 10)]:
        u = int(oracle.philox4x64_10([h, 0, 0, 0], [seed, 0])[0])
        idx = oracle.sample_block(seed, h, b, N)
        assert idx[0] == (u * (N - b + 1)) >> 64


def test_sampler_draws_use_philox_words_in_counter_order():
    """Library pin of the counter layout (reading of the unspecified RNG): draw
    m of block h is word m % 4 of the block for counter (h, m / 4, 0, 0) (the
    256-bit integer h + (m / 4) 2^64) under key (seed, 0), taken here from
    numpy's Philox.  With N = 2^31 - 1 the b draws do not collide, so Floyd's
    rule keeps every one: idx[m] = floor(u_m (N - b + m + 1) / 2^64)."""
    N, b = 2**31 - 1, 12
    for seed, h in [(42, 1), (7, 777), (2**64 - 5, 2**40 + 3)]:
        t = []
        for m in range(b):
            ctr = h + (m // 4) * 2**64
            u = int(np.random.Philox(key=seed, counter=ctr - 1).random_raw(4)[m % 4])
            t.append((u * (N - b + m + 1)) >> 64)
        assert len(set(t)) == b  # no collision: Floyd's rule keeps each draw
        assert oracle.sample_block(seed, h, b, N).tolist() == t


@pytest.mark.parametrize("b,N", [(1, 1), (3, 3), (4, 64), (8, 4096), (64, 64), (37, 100)])
def test_sampler_distinct_in_range(b, N):
    for h in range(50):
        idx = oracle.sample_block(42, h, b, N)
        assert idx.min() >= 0 and idx.max() < N
        assert len(set(idx.tolist())) == b
    if b == N:  # the whole index set
        assert sorted(oracle.sample_block(3, 9, b, N).tolist()) == list(range(N))


def test_sampler_subsets_uniform_chi2():
    """Without replacement and uniform: every 3-subset of [0,6) equally likely
    (C(6,3) = 20 cells), and every position of the insertion order uniform."""
    N, b, M = 6, 3, 40000
    counts = {}
    pos = np.zeros((b, N))
    for h in range(M):
        idx = oracle.sample_block(2024, h, b, N)
        key = tuple(sorted(idx.tolist()))
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == math.comb(N, b)
    exp = M / math.comb(N, b)
    chi2 = sum((c - exp) ** 2 / exp for c in counts.values())
    # 19 degrees of freedom: P(chi2 > 43.8) = 0.001
    assert chi2 < 43.8, chi2


def test_sampler_marginals_uniform_large():
    N, b, M = 1000, 10, 20000
    hits = np.zeros(N)
    for h in range(M):
        hits[oracle.sample_block(99, h, b, N)] += 1
    exp = M * b / N
    chi2 = float(((hits - exp) ** 2 / exp).sum())
    # 999 dof: mean 999, sd ~ 44.7; 5 sd bound
    assert chi2 < 999 + 5 * 44.7


def test_sampler_rejects_bad_args():
    with pytest.raises(oracle.OracleError):
        oracle.sample_block(1, 0, 5, 4)
    with pytest.raises(oracle.OracleError):
        oracle.sample_block(1, 0, 0, 4)


# ---------------------------------------------------------------------------
# Linear algebra pieces
# ---------------------------------------------------------------------------
def test_cholesky_solve_vs_library():
    rng = np.random.default_rng(5)
    for m in (1, 2, 8, 33):
        B = rng.standard_normal((m, m + 3))
        A = B @ B.T + 0.1 * np.eye(m)
        r = rng.standard_normal(m)
        assert _rel(oracle.cholesky_solve(A, r), np.linalg.solve(A, r)) < 1e-12


def test_cholesky_rejects_indefinite():
    A = np.array([[1.0, 2.0], [2.0, 1.0]])
    with pytest.raises(oracle.OracleError):
        oracle.cholesky_solve(A, np.ones(2))


def test_closed_form_vs_library(tiny):
    """w* solves (X X^T/n + lambda I) w = X y/n (gradient of eq. "primal" = 0)."""
    X, y = tiny.X, tiny.y
    n = X.shape[1]
    ref = np.linalg.solve(X @ X.T / n + LAM1 * np.eye(X.shape[0]), X @ y / n)
    assert _rel(oracle.closed_form(X, y, LAM1), ref) < 1e-13


def test_objectives_against_definitions(tiny):
    """f (eq. "primal") and D (eq. "6") evaluated by numpy from their definitions."""
    X, y = tiny.X, tiny.y
    d, n = X.shape
    rng = np.random.default_rng(0)
    w = rng.standard_normal(d)
    a = rng.standard_normal(n)
    f_np = LAM1 / 2 * w @ w + np.sum((X.T @ w - y) ** 2) / (2 * n)
    v = X @ a / (LAM1 * n)
    D_np = LAM1 / 2 * v @ v + np.sum((a + y) ** 2) / (2 * n)
    assert abs(oracle.primal_objective(X, y, LAM1, w) - f_np) < 1e-12 * abs(f_np)
    assert abs(oracle.dual_objective(X, y, LAM1, a) - D_np) < 1e-12 * abs(D_np)


# ---------------------------------------------------------------------------
# Algorithm 1 / 2 (primal)
# ---------------------------------------------------------------------------
def test_bcd_full_block_one_step_is_closed_form(tiny):
    """With b = d (every feature sampled) Gamma is the whole Hessian
    (Sec. 3.1, the Delta w_h closed form), so one step from w0 = 0 is w*."""
    X, y = tiny.X, tiny.y
    ref = np.linalg.solve(X @ X.T / X.shape[1] + LAM1 * np.eye(64), X @ y / X.shape[1])
    for s in (1, 2):
        w, z = oracle.ca_bcd(X, y, LAM1, b=64, s=s, H=1, seed=42)
        assert _rel(w, ref) < 1e-12
        assert _rel(z, X.T @ w) < 1e-13
    w, _ = oracle.bcd(X, y, LAM1, b=64, H=1, seed=42)
    assert _rel(w, ref) < 1e-12


@pytest.mark.parametrize("s", [2, 3, 4, 7, 50])
def test_ca_bcd_equals_bcd(tiny, s):
    """Sec. 3.1 ("by induction"): the unrolled recurrence eq. "recur" reproduces
    the s = 1 iterates in exact arithmetic for the same sampled indices.
    Algorithm 1 is a separate implementation in the oracle (orc_bcd)."""
    X, y = tiny.X, tiny.y
    w1, z1 = oracle.bcd(X, y, LAM1, b=4, H=200, seed=42)
    ws, zs = oracle.ca_bcd(X, y, LAM1, b=4, s=s, H=200, seed=42)
    assert _rel(ws, w1) < 1e-12
    assert _rel(zs, z1) < 1e-12


def test_ca_bcd_repeats_across_blocks(tiny):
    """With b close to d, indices repeat across the s blocks of one outer step,
    which exercises the lambda I_j^T I_t overlap term of eq. "recur"."""
    X, y = tiny.X, tiny.y
    w1, _ = oracle.bcd(X, y, LAM1, b=40, H=30, seed=3)
    ws, _ = oracle.ca_bcd(X, y, LAM1, b=40, s=6, H=30, seed=3)
    assert _rel(ws, w1) < 1e-12
    I = oracle.sample_blocks(3, 0, 6, 40, 64)
    assert len(set(I.reshape(-1).tolist())) < I.size  # there are repeats


def test_bcd_converges_to_closed_form(tiny):
    X, y = tiny.X, tiny.y
    ref = oracle.closed_form(X, y, LAM1)
    w, _ = oracle.ca_bcd(X, y, LAM1, b=8, s=8, H=6000, seed=5)
    assert _rel(w, ref) < 1e-10


def test_bcd_objective_monotone(tiny):
    """Each BCD step minimises f exactly over the sampled block (Sec. 3.1), so
    f(w_h) is non-increasing."""
    X, y = tiny.X, tiny.y
    w = np.zeros(64)
    f_prev = oracle.primal_objective(X, y, LAM1, w)
    for h in range(60):
        w, _ = oracle.bcd(X, y, LAM1, b=4, H=1, seed=11, h0=h, w0=w)
        f = oracle.primal_objective(X, y, LAM1, w)
        assert f <= f_prev + 1e-14 * abs(f_prev)
        f_prev = f


def test_bcd_block_minimisation_is_exact(tiny):
    """After one step the gradient of f restricted to the sampled block vanishes."""
    X, y = tiny.X, tiny.y
    n = X.shape[1]
    w0 = np.random.default_rng(1).standard_normal(64)
    w, _ = oracle.bcd(X, y, LAM1, b=5, H=1, seed=8, h0=17, w0=w0)
    grad = LAM1 * w + X @ (X.T @ w - y) / n
    I = oracle.sample_block(8, 17, 5, 64)
    assert np.abs(grad[I]).max() < 1e-12 * np.abs(grad).max()
    mask = np.ones(64, bool)
    mask[I] = False
    assert np.array_equal(w[mask], w0[mask])


def test_recompute_is_a_no_op(tiny):
    """Rebuilding z = X^T w from its definition (Sec. 3.1) changes nothing in
    exact arithmetic: Algorithms 1 and 2 with and without it agree."""
    X, y = tiny.X, tiny.y
    wa, _ = oracle.ca_bcd(X, y, LAM1, b=4, s=4, H=200, seed=42)
    wb, _ = oracle.ca_bcd(X, y, LAM1, b=4, s=4, H=200, seed=42, recompute_every=2)
    assert _rel(wb, wa) < 1e-12
    wc, _ = oracle.bcd(X, y, LAM1, b=4, H=200, seed=42)
    wd, _ = oracle.bcd(X, y, LAM1, b=4, H=200, seed=42, recompute_every=3)
    assert _rel(wd, wc) < 1e-12


def test_short_last_outer_step(tiny):
    """Reading of the outer loop bound: H not a multiple of s ends with a short
    outer step; the iterates still equal Algorithm 1's."""
    X, y = tiny.X, tiny.y
    w1, _ = oracle.bcd(X, y, LAM1, b=4, H=203, seed=42)
    ws, _ = oracle.ca_bcd(X, y, LAM1, b=4, s=8, H=203, seed=42)
    assert _rel(ws, w1) < 1e-12


def test_resume_from_h0(tiny):
    """The counter-based sampler makes a split run identical to one run."""
    X, y = tiny.X, tiny.y
    wa, _ = oracle.ca_bcd(X, y, LAM1, b=4, s=4, H=200, seed=42)
    wm, _ = oracle.ca_bcd(X, y, LAM1, b=4, s=4, H=120, seed=42)
    wb, _ = oracle.ca_bcd(X, y, LAM1, b=4, s=4, H=80, seed=42, h0=120, w0=wm)
    assert _rel(wb, wa) < 1e-12


# ---------------------------------------------------------------------------
# Algorithm 3 / 4 (dual)
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def wide():
    """d > n dense data (the dual method's regime): X 96 x 40."""
    return synth.dense_dual(d=96, n=40, seed=4)


def test_bdcd_full_block_one_step(wide):
    """b' = n: Theta is the whole dual Hessian, so one step from alpha0 = 0 gives
    alpha* = X^T w* - y (optimality of eq. "6" with eq. "3"), and w = w*."""
    X, y = wide.X, wide.y
    d, n = X.shape
    lam = 1e-2
    wstar = np.linalg.solve(X @ X.T / n + lam * np.eye(d), X @ y / n)
    astar = X.T @ wstar - y
    a, w = oracle.ca_bdcd(X, y, lam, b=n, s=1, H=1, seed=1)
    assert _rel(a, astar) < 1e-10
    assert _rel(w, wstar) < 1e-10


@pytest.mark.parametrize("s", [2, 5, 13])
def test_ca_bdcd_equals_bdcd(wide, s):
    """Sec. 3.2: the unrolled dual recurrence reproduces Algorithm 3's iterates."""
    X, y = wide.X, wide.y
    a1, w1 = oracle.bdcd(X, y, 1e-2, b=6, H=150, seed=9)
    as_, ws = oracle.ca_bdcd(X, y, 1e-2, b=6, s=s, H=150, seed=9)
    assert _rel(as_, a1) < 1e-12
    assert _rel(ws, w1) < 1e-12


def test_ca_bdcd_repeats_across_blocks(wide):
    X, y = wide.X, wide.y
    a1, w1 = oracle.bdcd(X, y, 1e-2, b=30, H=24, seed=2)
    as_, ws = oracle.ca_bdcd(X, y, 1e-2, b=30, s=6, H=24, seed=2)
    assert _rel(as_, a1) < 1e-12 and _rel(ws, w1) < 1e-12


def test_bdcd_dual_objective_monotone_primal_not_required(wide):
    """BDCD minimises D exactly over each block (Sec. 3.2), so D decreases; the
    primal objective need not (Sec. 5.1, BDCD discussion)."""
    X, y = wide.X, wide.y
    lam = 1e-2
    a = np.zeros(X.shape[1])
    D_prev = oracle.dual_objective(X, y, lam, a)
    for h in range(60):
        a, _ = oracle.bdcd(X, y, lam, b=3, H=1, seed=4, h0=h, alpha0=a)
        D = oracle.dual_objective(X, y, lam, a)
        assert D <= D_prev + 1e-14 * abs(D_prev)
        D_prev = D


def test_bdcd_b1_is_sdca_squared_loss(wide):
    """Sec. 3.2: b' = 1 is SDCA with the squared loss.  In the paper's sign
    convention (w = -X alpha/(lambda n)) the exact coordinate step is
    Delta alpha_i = -(alpha_i + y_i - x_i^T w) / (1 + ||x_i||^2/(lambda n))."""
    X, y = wide.X, wide.y
    d, n = X.shape
    lam = 1e-2
    a0 = np.random.default_rng(6).standard_normal(n)
    w0 = -X @ a0 / (lam * n)
    a1, w1 = oracle.bdcd(X, y, lam, b=1, H=1, seed=5, h0=3, alpha0=a0)
    i = int(oracle.sample_block(5, 3, 1, n)[0])
    xi = X[:, i]
    da = -(a0[i] + y[i] - xi @ w0) / (1 + xi @ xi / (lam * n))
    assert abs((a1[i] - a0[i]) - da) < 1e-12 * abs(da)
    assert _rel(w1, w0 - xi * da / (lam * n)) < 1e-12


def test_bdcd_converges_and_duality(wide):
    """alpha_H -> alpha*, and f(w*) + D(alpha*) = ||y||^2/(2n) (conjugate duality
    of eqs. "primal" and "6")."""
    X, y = wide.X, wide.y
    d, n = X.shape
    lam = 1e-2
    wstar = np.linalg.solve(X @ X.T / n + lam * np.eye(d), X @ y / n)
    astar = X.T @ wstar - y
    a, w = oracle.ca_bdcd(X, y, lam, b=8, s=4, H=4000, seed=12)
    assert _rel(a, astar) < 1e-9 and _rel(w, wstar) < 1e-9
    f = oracle.primal_objective(X, y, lam, wstar)
    D = oracle.dual_objective(X, y, lam, astar)
    assert abs(f + D - y @ y / (2 * n)) < 1e-12 * (y @ y / (2 * n))
    # weak duality: the gap is non-negative anywhere
    rng = np.random.default_rng(1)
    for _ in range(5):
        ww, aa = rng.standard_normal(d), rng.standard_normal(n)
        gap = (oracle.primal_objective(X, y, lam, ww) + oracle.dual_objective(X, y, lam, aa)
               - y @ y / (2 * n))
        assert gap >= -1e-12


def test_dual_recompute_is_a_no_op(wide):
    """Rebuilding w = -X alpha/(lambda n) from its definition (eq. "3")
    changes nothing in exact arithmetic: Algorithms 3 and 4 with and without
    it agree, in alpha and in w."""
    X, y, lam = wide.X, wide.y, 1e-2
    for s in (1, 3):
        a1, w1 = oracle.ca_bdcd(X, y, lam, b=6, s=s, H=120, seed=9)
        a2, w2 = oracle.ca_bdcd(X, y, lam, b=6, s=s, H=120, seed=9, recompute_every=2)
        assert _rel(a2, a1) < 1e-12 and _rel(w2, w1) < 1e-12
    a3, w3 = oracle.bdcd(X, y, lam, b=6, H=120, seed=9)
    a4, w4 = oracle.bdcd(X, y, lam, b=6, H=120, seed=9, recompute_every=5)
    assert _rel(a4, a3) < 1e-12 and _rel(w4, w3) < 1e-12


def test_dual_sparse_csr_equals_dense():
    """The dual oracle reads X through CSR(X^T); a sparse problem gives the same
    iterates as its dense expansion with explicit zeros."""
    sp = synth.sparse_dual(d=300, n=80, density=0.05, seed=3)
    A = oracle.CSR(sp.rowptr, sp.col, sp.val.astype(np.float64), sp.d)
    Xd = sp.dense_X()
    a_s, w_s = oracle.ca_bdcd(A, sp.y, 1e-3, b=4, s=5, H=60, seed=1)
    a_d, w_d = oracle.ca_bdcd(Xd, sp.y, 1e-3, b=4, s=5, H=60, seed=1)
    assert _rel(a_s, a_d) < 1e-13 and _rel(w_s, w_d) < 1e-13


def test_golden_reproduces_on_this_host():
    """The stored oracle output (written by tests/golden/make_golden.py) is
    reproduced here: the oracle is deterministic across hosts."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "tiny_primal_oracle.json")) as f:
        g = json.load(f)
    p = synth.tiny_primal(d=64, n=1024, seed=1)
    w1, _ = oracle.bcd(p.X, p.y, 1e-3, b=4, H=200, seed=42)
    assert _rel(w1, np.array(g["bcd_b4_H200_w"])) < 1e-13
    a4, wd = oracle.ca_bdcd(p.X, p.y, 1e-3, b=8, s=4, H=200, seed=42)
    assert _rel(wd, np.array(g["cabdcd_b8_s4_H200_w"])) < 1e-13
    assert oracle.sample_blocks(42, 0, 8, 4, 64).tolist() == g["first_blocks_seed42_b4_N64"]
