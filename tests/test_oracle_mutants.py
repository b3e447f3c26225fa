"""Sensitivity of the oracle's pins: plausible mistakes are planted in a copy
of the oracle (on the CPU: a dropped term, a flipped sign, a wrong index, a
transposed operand, a wrong constant), and each mutated oracle must fail at
least one pin of tests/test_oracle_pins.py or tests/test_oracle_stopping.py.

The stored golden values are left out of these runs: they were written by the
oracle itself, so they would catch every arithmetic change without saying
anything about the paper.  An unmodified copy run the same way must pass
(the control), so that a mutant counts as caught only through a failing pin.

Each mutant runs the pin suite in its own Python process, with the mutated
package imported before pytest starts so that the tests' ``import oracle``
resolves to it.
"""
import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
PIN_FILES = ["tests/test_oracle_pins.py", "tests/test_oracle_stopping.py"]

C, PY = "ca_oracle.c", "__init__.py"

# (name, file, text to replace, replacement, which occurrence (0-based))
MUTANTS = [
    # sampler (reading of "uniformly at random without replacement")
    ("philox_key_schedule", C, "k1 += PHILOX_W1;", "k1 += PHILOX_W0;", 0),
    ("philox_round_word", C, "uint64_t n0 = hi1 ^ c[1] ^ k0;", "uint64_t n0 = hi1 ^ c[3] ^ k0;", 0),
    ("philox_nine_rounds", C, "round < 10", "round < 9", 0),
    ("map_range_off_by_one", C, "(unsigned __int128)(J + 1)", "(unsigned __int128)J", 0),
    ("draw_counter_layout", C, "{(uint64_t)h, (uint64_t)(m / 4), 0, 0}",
     "{(uint64_t)h, 0, (uint64_t)(m / 4), 0}", 0),
    ("draw_word_index", C, "return out[m % 4];", "return out[(m + 1) % 4];", 0),
    ("floyd_swapped_choice", C, "(seen ? J : t)", "(seen ? t : J)", 0),
    ("floyd_range_short", C, "int64_t J = N - b + m;", "int64_t J = N - b + m - 1;", 0),
    # Cholesky solve of the b x b subproblem
    ("cholesky_sign", C, "sum -= L[(size_t)i * m + k] * L[(size_t)j * m + k];",
     "sum += L[(size_t)i * m + k] * L[(size_t)j * m + k];", 0),
    ("cholesky_forward_transposed", C, "sum -= L[(size_t)i * m + k] * u[k];",
     "sum -= L[(size_t)k * m + i] * u[k];", 0),
    ("cholesky_backward_transposed", C, "sum -= L[(size_t)k * m + i] * x[k];",
     "sum -= L[(size_t)i * m + k] * x[k];", 0),
    # objectives and closed form (Sec. 2.2)
    ("z_sign", C, "z[i] += row[i] * w[f];", "z[i] -= row[i] * w[f];", 0),
    ("primal_objective_half", C, "return 0.5 * lam * ww + res / (2.0 * (double)n);",
     "return lam * ww + res / (2.0 * (double)n);", 0),
    ("closed_form_reg_scaled", C, "A[(size_t)i * d + i] += lam;",
     "A[(size_t)i * d + i] += lam / (double)n;", 0),
    ("closed_form_rhs_unscaled", C, "r[i] = dot(X + (size_t)i * n, y, n) / (double)n;",
     "r[i] = dot(X + (size_t)i * n, y, n);", 0),
    ("dual_w_sign", C, "const double c = -1.0 / (lam * (double)n);",
     "const double c = 1.0 / (lam * (double)n);", 0),
    ("dual_objective_no_lambda", C, "return 0.5 * lam * ww + r / (2.0 * (double)n);",
     "return 0.5 * ww + r / (2.0 * (double)n);", 0),
    ("csr_scratch_not_cleared", C,
     "for (int64_t e = A->rowptr[j]; e < A->rowptr[j + 1]; ++e) scratch_d[A->col[e]] = 0.0;",
     "", 0),
    # Algorithm 2 (CA-BCD)
    ("cabcd_overlap_dropped", C, "if (Ij[p] == It[q]) r -= lam * dw[(size_t)t * b + q];",
     "if (Ij[p] == It[q]) r -= 0.0 * dw[(size_t)t * b + q];", 0),
    ("cabcd_projection_sign", C, "r -= inv_n * Yz[(size_t)j * b + p];",
     "r += inv_n * Yz[(size_t)j * b + p];", 0),
    ("cabcd_coupling_dropped", C,
     "r -= G[(size_t)(j * b + p) * sb + (t * b + q)] * dw[(size_t)t * b + q];",
     "r -= 0.0 * G[(size_t)(j * b + p) * sb + (t * b + q)] * dw[(size_t)t * b + q];", 0),
    ("cabcd_coupling_wrong_delta", C,
     "r -= G[(size_t)(j * b + p) * sb + (t * b + q)] * dw[(size_t)t * b + q];",
     "r -= G[(size_t)(j * b + p) * sb + (t * b + q)] * dw[(size_t)t * b + p];", 0),
    ("cabcd_label_term_dropped", C, "r += inv_n * Yy[(size_t)j * b + p];", "", 0),
    ("cabcd_gamma_first_block", C,
     "Gam[(size_t)p * b + q] = G[(size_t)(j * b + p) * sb + (j * b + q)];",
     "Gam[(size_t)p * b + q] = G[(size_t)p * sb + q];", 0),
    ("cabcd_gram_reg_doubled", C, "(p == q ? lam : 0.0);", "(p == q ? 2.0 * lam : 0.0);", 0),
    ("cabcd_w_update_sign", C, "for (int p = 0; p < sb; ++p) w[I[p]] += dw[p];",
     "for (int p = 0; p < sb; ++p) w[I[p]] -= dw[p];", 0),
    ("cabcd_z_update_sign", C, "z[i] += yp[i] * dw[p];", "z[i] -= yp[i] * dw[p];", 0),
    ("cabcd_full_last_step", C,
     "const int sk = (int)((H - (int64_t)s * k) < s ? (H - (int64_t)s * k) : s);",
     "const int sk = s;", 0),
    ("cabcd_same_block_s_times", C, "orc_sample_block(seed, h0 + (int64_t)s * k + j, b, d,",
     "orc_sample_block(seed, h0 + (int64_t)s * k, b, d,", 0),
    ("cabcd_resume_ignores_h0", C, "orc_sample_block(seed, h0 + (int64_t)s * k + j, b, d,",
     "orc_sample_block(seed, (int64_t)s * k + j, b, d,", 0),
    ("cabcd_recompute_clears_z", C,
     "if (recompute_every > 0 && (k + 1) % recompute_every == 0) primal_z(X, d, n, w, z);",
     "if (recompute_every > 0 && (k + 1) % recompute_every == 0) memset(z, 0, (size_t)n * 8);",
     0),
    # Algorithm 1 (BCD)
    ("bcd_rhs_sign", C, "rhs[p] = -lam * w[I[p]] - inv_n * dot(yp, z, n)",
     "rhs[p] = lam * w[I[p]] - inv_n * dot(yp, z, n)", 0),
    ("bcd_gamma_reg_doubled", C, "(p == q ? lam : 0.0);", "(p == q ? 2.0 * lam : 0.0);", 1),
    ("bcd_z_update_sign", C, "z[i] += yp[i] * dw[p];", "z[i] -= yp[i] * dw[p];", 1),
    ("bcd_recompute_clears_z", C,
     "if (recompute_every > 0 && (h + 1) % recompute_every == 0) primal_z(X, d, n, w, z);",
     "if (recompute_every > 0 && (h + 1) % recompute_every == 0) memset(z, 0, (size_t)n * 8);",
     0),
    # Algorithm 4 (CA-BDCD)
    ("cabdcd_gram_scale", C, "/ (ln * (double)n) +\n                                (p == q ? inv_n",
     "/ ln +\n                                (p == q ? inv_n", 0),
    ("cabdcd_theta_reg", C, "(p == q ? inv_n : 0.0);", "(p == q ? lam : 0.0);", 0),
    ("cabdcd_projection_sign", C, "double r = -Yw[(size_t)j * b + p];",
     "double r = Yw[(size_t)j * b + p];", 0),
    ("cabdcd_coupling_sign", C,
     "r += (double)n * G[(size_t)(j * b + p) * sb + (t * b + q)] * da[(size_t)t * b + q];",
     "r -= (double)n * G[(size_t)(j * b + p) * sb + (t * b + q)] * da[(size_t)t * b + q];", 0),
    ("cabdcd_alpha_sign", C, "r += alpha[Ij[p]];", "r -= alpha[Ij[p]];", 0),
    ("cabdcd_overlap_dropped", C, "if (Ij[p] == It[q]) r += da[(size_t)t * b + q];",
     "if (Ij[p] == It[q]) r += 0.0;", 0),
    ("cabdcd_label_sign", C, "r += y[Ij[p]];", "r -= y[Ij[p]];", 0),
    ("cabdcd_step_unscaled", C, "da[(size_t)j * b + p] = -inv_n * sol[p];",
     "da[(size_t)j * b + p] = -sol[p];", 0),
    ("cabdcd_w_update_sign", C, "w[A.col[e]] -= A.val[e] * da[p] / ln;",
     "w[A.col[e]] += A.val[e] * da[p] / ln;", 0),
    ("cabdcd_full_last_step", C,
     "const int sk = (int)((H - (int64_t)s * k) < s ? (H - (int64_t)s * k) : s);",
     "const int sk = s;", 1),
    ("cabdcd_recompute_clears_w", C,
     "if (recompute_every > 0 && (k + 1) % recompute_every == 0) dual_w(&A, d, n, lam, alpha, w);",
     "if (recompute_every > 0 && (k + 1) % recompute_every == 0) memset(w, 0, (size_t)d * 8);",
     0),
    # Algorithm 3 (BDCD)
    ("bdcd_step_sign", C, "const double da = -inv_n * sol[p];", "const double da = inv_n * sol[p];",
     0),
    ("bdcd_theta_reg", C, "(p == q ? inv_n : 0.0);", "(p == q ? lam : 0.0);", 1),
    ("bdcd_rhs_label_dropped", C, "+ alpha[I[p]] + y[I[p]];", "+ alpha[I[p]];", 0),
    ("bdcd_recompute_clears_w", C,
     "if (recompute_every > 0 && (h + 1) % recompute_every == 0) dual_w(&A, d, n, lam, alpha, w);",
     "if (recompute_every > 0 && (h + 1) % recompute_every == 0) memset(w, 0, (size_t)d * 8);",
     0),
    # the stopping test's residuals (Sec. 5.1.5) and the dense-as-CSR input
    ("primal_residual_label_sign", PY, "X @ (X.T @ w - y) / n", "X @ (X.T @ w + y) / n", 0),
    ("primal_residual_unscaled", PY, "X @ (X.T @ w - y) / n", "X @ (X.T @ w - y)", 0),
    ("dual_residual_label_sign", PY, "+ _f64(alpha) + _f64(y)", "+ _f64(alpha) - _f64(y)", 0),
    ("csr_product_ignores_columns", PY, "out[i] = X.val[a:b] @ w[X.col[a:b]]",
     "out[i] = X.val[a:b] @ w[:b - a]", 0),
    ("dense_as_csr_transposed", PY, "return CSR(rowptr, col, X.T.reshape(-1), d)",
     "return CSR(rowptr, col, X.reshape(-1), d)", 0),
    ("stopped_absolute_tolerance", PY, "norms[-1] <= tol * r0", "norms[-1] <= tol", 0),
    # (occurrences of the loop text: 0, 1 the certified runs, 2, 3 the stopped runs)
    ("stopped_check_every_update", PY, "m = min(check_every * s, H - h)",
     "m = min(check_every, H - h)", 2),
    ("stopped_dual_check_every_update", PY, "m = min(check_every * s, H - h)",
     "m = min(check_every, H - h)", 3),
    ("stopped_primal_restarts_sampler", PY, "seed, h0=h, w0=w)", "seed, h0=0, w0=w)", 1),
    ("stopped_dual_drops_iterate", PY, "seed, h0=h, alpha0=alpha)", "seed, h0=h)", 1),
    ("certified_check_every_update", PY, "m = min(check_every * s, H - h)",
     "m = min(check_every, H - h)", 0),
    ("certified_primal_restarts_sampler", PY, "seed, h0=h, w0=w)", "seed, h0=0, w0=w)", 0),
    ("certified_dual_drops_iterate", PY, "seed, h0=h, alpha0=alpha)", "seed, h0=h)", 0),
    # duality gaps and the certified stop (Sec. 2.2 duality, Sec. 5.1.5)
    ("gap_wrong_dual_point", PY, "dual_objective(X, y, lam, X.T @ w - y)",
     "dual_objective(X, y, lam, X.T @ w + y)", 0),
    ("primal_gap_label_norm_unhalved", PY, "- float(y @ y) / (2 * n))", "- float(y @ y) / n)", 0),
    ("dual_gap_label_norm_unhalved", PY, "- float(y @ y) / (2 * A.n))", "- float(y @ y) / A.n)", 0),
    ("dual_gap_model_sign", PY, "w[A.col[a:b]] -= A.val[a:b] * alpha[i] / (lam * A.n)",
     "w[A.col[a:b]] += A.val[a:b] * alpha[i] / (lam * A.n)", 0),
    ("certified_uncertified_bound", PY, "g <= tol * (f - g)", "g <= tol * f", 0),
    ("certified_dual_uncertified_bound", PY, "g <= tol * (f - g)", "g <= tol * f", 1),
    ("certified_dual_objective_drops_gap", PY,
     "f = g + float(y @ y) / (2 * A.n) - dual_objective(A, y, lam, alpha)",
     "f = float(y @ y) / (2 * A.n) - dual_objective(A, y, lam, alpha)", 0),
]


def _run_pins(pkg_parent: str, timeout: float = 300.0):
    """Run the pin suite with the oracle package found under pkg_parent."""
    code = textwrap.dedent(f"""
        import sys
        sys.path.insert(0, {pkg_parent!r})
        import oracle
        assert oracle.__file__.startswith({pkg_parent!r}), oracle.__file__
        oracle.build()
        import pytest
        sys.exit(pytest.main({PIN_FILES + ["-x", "-q", "-p", "no:cacheprovider",
                                           "-k", "not golden"]!r}))
    """)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True,
                       text=True, timeout=timeout)
    failed = re.findall(r"FAILED (\S+)", r.stdout)
    return r.returncode, (failed[0] if failed else ""), r.stdout[-2000:] + r.stderr[-2000:]


def _make_copy(dst: str, mutant=None) -> str:
    pkg = os.path.join(dst, "oracle")
    os.makedirs(pkg)
    for f in (C, PY):
        shutil.copy(os.path.join(ORACLE, f), os.path.join(pkg, f))
    if mutant is not None:
        name, f, old, new, nth = mutant
        path = os.path.join(pkg, f)
        with open(path) as fh:
            text = fh.read()
        pos = -1
        for _ in range(nth + 1):
            pos = text.find(old, pos + 1)
            assert pos >= 0, f"{name}: occurrence {nth} of the target text not found"
        text = text[:pos] + new + text[pos + len(old):]
        with open(path, "w") as fh:
            fh.write(text)
    return dst


def test_mutant_names_unique():
    names = [m[0] for m in MUTANTS]
    assert len(names) == len(set(names))


def test_unmodified_copy_passes(tmp_path):
    rc, failed, tail = _run_pins(_make_copy(str(tmp_path / "control")))
    assert rc == 0, tail


def test_every_planted_mistake_fails_a_pin(tmp_path):
    def one(m):
        d = str(tmp_path / m[0])
        rc, failed, tail = _run_pins(_make_copy(d, m))
        return m[0], rc, failed, tail

    workers = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(one, MUTANTS))
    survivors = [(n, rc, tail) for n, rc, failed, tail in results if rc != 1]
    for n, rc, failed, _ in results:
        print(f"{n:36s} rc={rc} caught by {failed}")
    assert not survivors, "\n\n".join(f"{n} (exit {rc}):\n{tail}" for n, rc, tail in survivors)
