"""CUDA path vs the FP64 oracle (GB300, through the C ABI): the sparse dual's
Gram by the dense-sparse split of the features (Alg. 4 "compute the Gram
matrix" on the CSR of X^T).  Features present in at least a quarter of the
samples go to a small dense matrix whose sampled rows' Gram is formed with
exact products summed in double-float; the others' pair products are added
per feature bucket with FP64 atomics.  Both parts hold exact products of the
FP32 values, so the iterates meet the FP64 path's 1e-10.

Cases: no heavy feature at all (the dense part is empty); heavy features
together with a block of 512 features each in 20% of the samples, whose
entries in one feature range exceed the bucket capacity and make the range
split; s*b = 32, 64, 256.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1612_04003_gb300 as ca
    ca.build()
    c = ca.Context(0)
    yield c
    c.close()


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda().contiguous()


def _rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _csr(n, d, dens, seed):
    """CSR of X^T (n rows = samples, d columns = features): column f is
    present in each row with probability dens[f]; values N(0, 1) in FP32."""
    rng = np.random.default_rng(seed)
    mask = rng.random((n, d)) < dens[None, :]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(mask.sum(axis=1))
    rows, cols = np.nonzero(mask)  # row-major order: columns sorted within a row
    val = rng.standard_normal(len(cols)).astype(np.float32)
    y = np.sign(rng.standard_normal(n))
    return rowptr, cols.astype(np.int32), val, y


CASES = {
    "no heavy feature": (700, 3000, lambda d: np.full(d, 0.02)),
    "heavy + dense block": (1200, 2048, lambda d: np.concatenate(
        [np.full(512, 0.2), np.full(8, 1.0), np.full(d - 520, 0.005)])),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("b,s", [(8, 4), (8, 8), (8, 32)])
def test_split_gram_dual_csr(ctx, case, b, s):
    n, d, dens = CASES[case]
    rowptr, col, val, y = _csr(n, d, dens(d), seed=len(case) + 17 * s)
    lam, H = 1e-3, 8 * s
    a = torch.zeros(n, dtype=torch.float64, device="cuda")
    w = torch.zeros(d, dtype=torch.float64, device="cuda")
    ctx.ca_bdcd_solve((_dev(rowptr), _dev(col), _dev(val)), _dev(y), a, w, b=b, s=s, H=H,
                      lam=lam, seed=5, d=d)
    A = oracle.CSR(rowptr, col, val.astype(np.float64), d)
    a_ref, w_ref = oracle.ca_bdcd(A, y, lam, b=b, s=s, H=H, seed=5)
    print(f"{case} b={b} s={s}: a {_rel(a, a_ref):.2e} w {_rel(w, w_ref):.2e}")
    assert _rel(a, a_ref) < TOL64 and _rel(w, w_ref) < TOL64


@pytest.mark.parametrize("case", list(CASES))
def test_split_gram_dual_csr_short_last_step(ctx, case):
    """s*b = 128 for the first outer steps (the inverses and Rs formed on the
    second stream) and 40 for the short last one (the fused reduction on the
    library stream), with the Gram buffers and Rs alternating by step parity
    across the switch."""
    n, d, dens = CASES[case]
    rowptr, col, val, y = _csr(n, d, dens(d), seed=len(case) + 3)
    lam, b, s, H = 1e-3, 8, 16, 5 * 16 + 5
    a = torch.zeros(n, dtype=torch.float64, device="cuda")
    w = torch.zeros(d, dtype=torch.float64, device="cuda")
    ctx.ca_bdcd_solve((_dev(rowptr), _dev(col), _dev(val)), _dev(y), a, w, b=b, s=s, H=H,
                      lam=lam, seed=9, d=d)
    A = oracle.CSR(rowptr, col, val.astype(np.float64), d)
    a_ref, w_ref = oracle.ca_bdcd(A, y, lam, b=b, s=s, H=H, seed=9)
    print(f"{case} short last step: a {_rel(a, a_ref):.2e} w {_rel(w, w_ref):.2e}")
    assert _rel(a, a_ref) < TOL64 and _rel(w, w_ref) < TOL64
