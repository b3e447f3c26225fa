"""Pins of the oracle's stopping-test residuals (Sec. 5.1.5), independent of
their formulas: finite differences of the objectives, the zeros at the
optimum, the zero on the block a step has just solved exactly, and the
stopped runs against plain runs of the same length."""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def tiny():
    return synth.tiny_primal(d=64, n=1024, seed=1)


@pytest.fixture(scope="module")
def wide():
    return synth.dense_dual(d=96, n=40, seed=4)


def _fd_grad(f, x, coords, h):
    g = []
    for i in coords:
        e = np.zeros_like(x)
        e[i] = h
        g.append((f(x + e) - f(x - e)) / (2 * h))
    return np.array(g)


def test_primal_residual_is_negative_gradient(tiny):
    X, y, lam = tiny.X, tiny.y, 1e-3
    rng = np.random.default_rng(3)
    w = rng.standard_normal(X.shape[0])
    coords = rng.choice(X.shape[0], 8, replace=False)
    g = _fd_grad(lambda v: oracle.primal_objective(X, y, lam, v), w, coords, 1e-5)
    r = oracle.primal_residual(X, y, lam, w)
    assert np.allclose(-r[coords], g, rtol=1e-6, atol=1e-9 * np.abs(g).max())


def test_primal_residual_zero_at_optimum(tiny):
    X, y, lam = tiny.X, tiny.y, 1e-3
    wstar = oracle.closed_form(X, y, lam)
    r0 = np.linalg.norm(oracle.primal_residual(X, y, lam, np.zeros(X.shape[0])))
    assert np.linalg.norm(oracle.primal_residual(X, y, lam, wstar)) < 1e-10 * r0


def test_primal_residual_vanishes_on_solved_block(tiny):
    """One BCD step minimises the objective exactly over the sampled block,
    so the residual's rows there vanish (they are the step's right-hand side)."""
    X, y, lam = tiny.X, tiny.y, 1e-3
    rng = np.random.default_rng(4)
    w0 = rng.standard_normal(X.shape[0])
    w1, _ = oracle.bcd(X, y, lam, b=8, H=1, seed=9, w0=w0)
    I = oracle.sample_blocks(9, 0, 1, 8, X.shape[0])[0]
    r0 = oracle.primal_residual(X, y, lam, w0)[I]
    r1 = oracle.primal_residual(X, y, lam, w1)[I]
    assert np.linalg.norm(r1) < 1e-12 * np.linalg.norm(r0)


def test_dual_residual_is_scaled_dual_gradient(wide):
    """With w = -X alpha/(lambda n): -X^T w + alpha + y = n grad D(alpha)."""
    X, y, lam = wide.X, wide.y, 1e-2
    d, n = X.shape
    rng = np.random.default_rng(5)
    a = rng.standard_normal(n)
    w = -X @ a / (lam * n)
    coords = rng.choice(n, 8, replace=False)
    g = _fd_grad(lambda v: oracle.dual_objective(X, y, lam, v), a, coords, 1e-5)
    r = oracle.dual_residual(X, y, a, w)
    assert np.allclose(r[coords], n * g, rtol=1e-6, atol=1e-9 * np.abs(n * g).max())


def test_dual_residual_zero_at_optimum(wide):
    X, y, lam = wide.X, wide.y, 1e-2
    d, n = X.shape
    wstar = oracle.closed_form(X, y, lam)
    astar = X.T @ wstar - y
    assert np.allclose(-X @ astar / (lam * n), wstar, rtol=1e-10)
    r0 = np.linalg.norm(oracle.dual_residual(X, y, np.zeros(n), np.zeros(d)))
    assert np.linalg.norm(oracle.dual_residual(X, y, astar, wstar)) < 1e-10 * r0


def test_dual_residual_vanishes_on_solved_block(wide):
    X, y, lam = wide.X, wide.y, 1e-2
    d, n = X.shape
    rng = np.random.default_rng(6)
    a0 = rng.standard_normal(n)
    a1, w1 = oracle.bdcd(X, y, lam, b=6, H=1, seed=2, alpha0=a0)
    I = oracle.sample_blocks(2, 0, 1, 6, n)[0]
    r0 = oracle.dual_residual(X, y, a0, -X @ a0 / (lam * n))[I]
    r1 = oracle.dual_residual(X, y, a1, w1)[I]
    assert np.linalg.norm(r1) < 1e-12 * np.linalg.norm(r0)


def test_dual_residual_csr_equals_dense(wide):
    X, y = wide.X, wide.y
    rng = np.random.default_rng(7)
    a, w = rng.standard_normal(X.shape[1]), rng.standard_normal(X.shape[0])
    r_dense = oracle.dual_residual(X, y, a, w)
    r_csr = oracle.dual_residual(oracle.CSR.from_dense(X), y, a, w)
    assert np.allclose(r_csr, r_dense, rtol=1e-13, atol=1e-13)
    # a sparse CSR (columns of X^T skipped) against its dense expansion
    sp = synth.sparse_dual(d=300, n=80, density=0.05, seed=3)
    A = oracle.CSR(sp.rowptr, sp.col, sp.val.astype(np.float64), sp.d)
    a, w = rng.standard_normal(sp.n), rng.standard_normal(sp.d)
    r_dense = oracle.dual_residual(sp.dense_X(), sp.y, a, w)
    assert np.allclose(oracle.dual_residual(A, sp.y, a, w), r_dense, rtol=1e-13, atol=1e-13)


def test_primal_stopped_run(tiny):
    """tol = 0 runs to H with one check per check_every outer steps; with a
    tolerance the run ends at the first check below it, with the iterate of
    a plain run of that length."""
    X, y, lam = tiny.X, tiny.y, 1e-3
    w, h, r0, norms = oracle.ca_bcd_stopped(X, y, lam, b=4, s=4, H=200, seed=42, tol=0.0,
                                            check_every=5)
    assert h == 200 and len(norms) == 10  # 200 / (4 * 5)
    w_full, _ = oracle.ca_bcd(X, y, lam, b=4, s=4, H=200, seed=42)
    assert np.allclose(w, w_full, rtol=1e-12, atol=1e-14)
    assert np.isclose(norms[-1], np.linalg.norm(oracle.primal_residual(X, y, lam, w_full)))
    tol = np.sqrt(norms[3] * norms[4]) / r0  # between the 4th and 5th checks
    assert norms[4] < norms[3]
    w2, h2, _, norms2 = oracle.ca_bcd_stopped(X, y, lam, b=4, s=4, H=200, seed=42, tol=tol,
                                              check_every=5)
    assert h2 == 5 * 20 and len(norms2) == 5
    w_part, _ = oracle.ca_bcd(X, y, lam, b=4, s=4, H=h2, seed=42)
    assert np.allclose(w2, w_part, rtol=1e-12, atol=1e-14)


def test_dual_stopped_run(wide):
    X, y, lam = wide.X, wide.y, 1e-2
    a, w, h, r0, norms = oracle.ca_bdcd_stopped(X, y, lam, b=6, s=3, H=150, seed=9, tol=0.0,
                                                check_every=5)
    assert h == 150 and len(norms) == 10
    a_full, w_full = oracle.ca_bdcd(X, y, lam, b=6, s=3, H=150, seed=9)
    assert np.allclose(a, a_full, rtol=1e-12, atol=1e-14)
    assert np.isclose(norms[-1], np.linalg.norm(oracle.dual_residual(X, y, a_full, w_full)))


# ---------------------------------------------------------------------------
# Duality gap (Sec. 2.2) of the iterates: the certified stopping rule
# ---------------------------------------------------------------------------
def _bound(f, g):
    """The certified relative objective error g/(f - g) (vacuous unless f > g)."""
    return g / (f - g) if f > g else float("inf")


def test_primal_gap_equals_residual_closed_form(tiny):
    """At alpha = X^T w - y the gap f(w) + D(alpha) - ||y||^2/(2n) reduces to
    ||r||^2/(2 lambda) with r = -grad f(w) (expand both objectives: the cross
    terms collapse to a perfect square).  Checked at random points and at an
    iterate close to the optimum."""
    X, y, lam = tiny.X, tiny.y, 1e-3
    rng = np.random.default_rng(11)
    w_run, _ = oracle.ca_bcd(X, y, lam, b=4, s=4, H=2000, seed=42)
    for w in [rng.standard_normal(64), 0.1 * rng.standard_normal(64), np.zeros(64), w_run]:
        g = oracle.primal_duality_gap(X, y, lam, w)
        r = oracle.primal_residual(X, y, lam, w)
        # the definition route cancels terms of size ||y||^2/(2n): rounding there
        scale = oracle.primal_objective(X, y, lam, w) + y @ y / (2 * len(y))
        assert abs(g - r @ r / (2 * lam)) <= 1e-10 * abs(g) + 1e-14 * scale


def test_dual_gap_equals_residual_closed_form(wide):
    """At w = -X alpha/(lambda n) the gap reduces to ||r||^2/(2n) with r the
    dual residual X^T w - alpha - y; dense and CSR alike."""
    X, y, lam = wide.X, wide.y, 1e-2
    d, n = X.shape
    rng = np.random.default_rng(12)
    a_run, _ = oracle.ca_bdcd(X, y, lam, b=6, s=3, H=900, seed=9)
    for a in [rng.standard_normal(n), 0.01 * rng.standard_normal(n), a_run]:
        w = -X @ a / (lam * n)
        g = oracle.dual_duality_gap(X, y, lam, a)
        r = oracle.dual_residual(X, y, a, w)
        scale = oracle.dual_objective(X, y, lam, a) + y @ y / (2 * n)
        assert abs(g - r @ r / (2 * n)) <= 1e-10 * abs(g) + 1e-13 * scale
        assert abs(oracle.dual_duality_gap(oracle.CSR.from_dense(X), y, lam, a) - g) <= 1e-12 * scale


def test_gap_bounds_the_objective_error(tiny, wide):
    """Weak and strong duality: f(w) - f(w*) <= gap, D(alpha) - D(alpha*) <= gap,
    hence (f(w) - f*)/f* <= gap/(f(w) - gap), with w* the closed form."""
    X, y, lam = tiny.X, tiny.y, 1e-3
    fstar = oracle.primal_objective(X, y, lam, oracle.closed_form(X, y, lam))
    for H in (8, 40, 200, 1000):
        w, _ = oracle.ca_bcd(X, y, lam, b=4, s=4, H=H, seed=42)
        f, g = oracle.primal_objective(X, y, lam, w), oracle.primal_duality_gap(X, y, lam, w)
        assert f - fstar <= g * (1 + 1e-9) + 1e-14 * (f + y @ y / (2 * len(y)))
        assert (f - fstar) / fstar <= _bound(f, g) * (1 + 1e-9) + 1e-13
    Xw, yw, lw = wide.X, wide.y, 1e-2
    d, n = Xw.shape
    wstar = oracle.closed_form(Xw, yw, lw)
    fstar = oracle.primal_objective(Xw, yw, lw, wstar)
    Dstar = yw @ yw / (2 * n) - fstar  # strong duality
    for H in (6, 60, 600):
        a, w = oracle.ca_bdcd(Xw, yw, lw, b=6, s=3, H=H, seed=9)
        g = oracle.dual_duality_gap(Xw, yw, lw, a)
        assert oracle.dual_objective(Xw, yw, lw, a) - Dstar <= g * (1 + 1e-9) + 1e-13
        assert oracle.primal_objective(Xw, yw, lw, w) - fstar <= g * (1 + 1e-9) + 1e-13


def test_primal_certified_run(tiny):
    """tol = 0 runs to H with one check per check_every outer steps; with a
    tolerance the run ends at the first check whose bound is below it, with
    the iterate of a plain run of that length, and the true relative
    objective error (closed form) is within the tolerance."""
    X, y, lam = tiny.X, tiny.y, 1e-3
    w, h, trace = oracle.ca_bcd_certified(X, y, lam, b=4, s=4, H=400, seed=42, tol=0.0,
                                          check_every=5)
    assert h == 400 and len(trace) == 20
    w_full, _ = oracle.ca_bcd(X, y, lam, b=4, s=4, H=400, seed=42)
    assert np.allclose(w, w_full, rtol=1e-12, atol=1e-14)
    bounds = [_bound(f, g) for f, g in trace]
    j = next(j for j in range(1, len(bounds)) if bounds[j] * 2 < min(bounds[:j]))
    tol = np.sqrt(min(min(bounds[:j]), 1e300) * bounds[j])
    w2, h2, trace2 = oracle.ca_bcd_certified(X, y, lam, b=4, s=4, H=400, seed=42, tol=tol,
                                             check_every=5)
    assert h2 == 20 * (j + 1) and len(trace2) == j + 1
    w_part, _ = oracle.ca_bcd(X, y, lam, b=4, s=4, H=h2, seed=42)
    assert np.allclose(w2, w_part, rtol=1e-12, atol=1e-14)
    fstar = oracle.primal_objective(X, y, lam, oracle.closed_form(X, y, lam))
    assert (oracle.primal_objective(X, y, lam, w2) - fstar) / fstar <= tol


def test_dual_certified_run(wide):
    X, y, lam = wide.X, wide.y, 1e-2
    a, w, h, trace = oracle.ca_bdcd_certified(X, y, lam, b=6, s=3, H=300, seed=9, tol=0.0,
                                              check_every=5)
    assert h == 300 and len(trace) == 20
    a_full, w_full = oracle.ca_bdcd(X, y, lam, b=6, s=3, H=300, seed=9)
    assert np.allclose(a, a_full, rtol=1e-12, atol=1e-14)
    for f, g in trace[-3:]:  # f is the primal objective of w(alpha)
        assert g >= 0
    f_last = oracle.primal_objective(X, y, lam, w_full)
    assert abs(trace[-1][0] - f_last) <= 1e-10 * f_last
    bounds = [_bound(f, g) for f, g in trace]
    j = next(j for j in range(1, len(bounds)) if bounds[j] * 2 < min(bounds[:j]))
    tol = np.sqrt(min(min(bounds[:j]), 1e300) * bounds[j])
    a2, w2, h2, trace2 = oracle.ca_bdcd_certified(X, y, lam, b=6, s=3, H=300, seed=9, tol=tol,
                                                  check_every=5)
    assert h2 == 15 * (j + 1)
    fstar = oracle.primal_objective(X, y, lam, oracle.closed_form(X, y, lam))
    assert (oracle.primal_objective(X, y, lam, w2) - fstar) / fstar <= tol

