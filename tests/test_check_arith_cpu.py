"""The library's host arithmetic of a stopping-test check
(paper_1612_04003_gb300/csrc/ca_check.h, no CUDA): the duality gap and f(w)
it forms from the device's sums of squares, against the oracle's gap and
objectives by their definitions (Sec. 2.2, Sec. 5.1.5)."""
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


def test_host_check_arithmetic_against_the_oracle(tmp_path, tiny, wide):
    """The library's host arithmetic of a check (csrc/ca_check.h: the gap and
    f(w) from the sums of squares the device forms) against the oracle's gap
    and objectives by their definitions, at primal and dual iterates."""
    import os
    import shutil
    import subprocess
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    exe = tmp_path / "check_values_cli"
    subprocess.run(["g++", "-std=c++17", "-O1", "-I",
                    os.path.join(root, "paper_1612_04003_gb300", "csrc"),
                    os.path.join(root, "tests", "check_values_cli.cpp"), "-o", str(exe)],
                   check=True)
    def _line(method, lam, N, K, *sums):
        return f"{method} 1 {float(lam)!r} {N} {K} " + " ".join(repr(float(v)) for v in sums)

    lines, want = [], []
    X, y, lam = tiny.X, tiny.y, 1e-3
    d, n = X.shape
    for H in (0, 40, 400):
        w = oracle.ca_bcd(X, y, lam, b=4, s=4, H=H, seed=42)[0] if H else np.zeros(d)
        r = oracle.primal_residual(X, y, lam, w)
        rho = y - X.T @ w
        lines.append(_line(0, lam, d, n, r @ r, rho @ rho, w @ w, 0.0))
        want.append((np.linalg.norm(r), oracle.primal_duality_gap(X, y, lam, w),
                     oracle.primal_objective(X, y, lam, w), oracle.primal_objective(X, y, lam, w)
                     + y @ y / (2 * n)))
    Xw, yw, lw = wide.X, wide.y, 1e-2
    dw, nw = Xw.shape
    for H in (0, 30, 300):
        a = oracle.ca_bdcd(Xw, yw, lw, b=6, s=3, H=H, seed=9)[0] if H else np.zeros(nw)
        wv = -Xw @ a / (lw * nw)
        r = oracle.dual_residual(Xw, yw, a, wv)
        lines.append(_line(1, lw, nw, dw, r @ r, wv @ wv, (a + yw) @ (a + yw), yw @ yw))
        want.append((np.linalg.norm(r), oracle.dual_duality_gap(Xw, yw, lw, a),
                     oracle.primal_objective(Xw, yw, lw, wv), yw @ yw / (2 * nw)
                     + oracle.dual_objective(Xw, yw, lw, a)))
    out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True,
                         text=True, check=True).stdout.split("\n")
    assert len([o for o in out if o.strip()]) == len(want)
    for line, (res, gap, f, scale) in zip(out, want):
        r_, g_, f_, b_, stop = line.split()
        r_, g_, f_, b_ = float(r_), float(g_), float(f_), float(b_)
        assert abs(r_ - res) <= 1e-14 * res + 1e-300
        assert abs(g_ - gap) <= 1e-9 * gap + 1e-14 * scale
        assert abs(f_ - f) <= 1e-12 * f + 1e-14 * scale
        # the certified bound gap / (f - gap) and the objective rule's stop
        if f_ > g_:
            assert abs(b_ - g_ / (f_ - g_)) <= 1e-15 * b_ + 1e-300
        else:  # far from the optimum the gap can exceed f: no bound
            assert b_ == -1.0
        assert stop == ("1" if g_ <= 1e-6 * (f_ - g_) else "0")


def test_certified_bound_edge_cases(tmp_path):
    """No bound when f(w) <= gap (-1); the residual rule and tol = 0 never
    stop on the objective; the stop at the boundary gap = tol (f - gap)."""
    import os
    import shutil
    import subprocess
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "edge.cpp"
    src.write_text('#include <cstdio>\n#include "ca_check.h"\nint main() {\n'
                   '  std::printf("%g %g\\n", certified_bound(1.0, 1.0), certified_bound(0.5, 1.0));\n'
                   '  std::printf("%d %d %d\\n", (int)check_stops(1, 0.0, 1, 1, 0.0, 1.0),\n'
                   '              (int)check_stops(1, 0.5, 1, 1, 1.0, 3.0),\n'
                   '              (int)check_stops(1, 0.5, 1, 1, 1.0 + 1e-12, 3.0));\n'
                   '  std::printf("%d %d\\n", (int)check_stops(0, 0.5, 2.0, 1.0, 9.0, 1.0),\n'
                   '              (int)check_stops(0, 0.5, 2.0, 1.1, 0.0, 1.0));\n'
                   '  return 0;\n}\n')
    exe = tmp_path / "edge"
    subprocess.run(["g++", "-std=c++17", "-I", os.path.join(root, "paper_1612_04003_gb300", "csrc"),
                    str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert out == ["-1", "-1", "0", "1", "0", "1", "0"]
