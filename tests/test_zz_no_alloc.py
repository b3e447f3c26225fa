"""ca_gram_project_noalloc against ca_gram_project (GB300).

The allocation-free entry point serves callers that must not call
cudaMalloc themselves (a framework that owns every device allocation, a
latency-critical path, code that may only enqueue on a given stream).  It
must give the same Gram matrix and projection as the regular entry point, on
two calls in a row (its scratch array keeps the previous call's contents).
This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

# tolerances of the Gram kernel tests (3xTF32: FP32 accumulation of up to
# ~1000 same-sign terms per split, 1000 * 2^-24 ~ 6e-5 worst case), relative to sqrt(G_ii G_jj) and
# ||y_i|| ||v||; the two entry points sum the split-K partials in a different
# order, so FP32-accumulated modes differ at rounding level
TOL = {"f64": (1e-13, 1e-13), "3xtf32": (2e-5, 1e-6), "bf16x3": (2e-5, 1e-6),
       "tf32": (3e-3, 1e-6)}


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1612_04003_gb300 as ca
    ca.build()
    ctx = ca.Context(0)
    yield ca, ctx
    ctx.close()


@pytest.mark.parametrize("prec", ["f64", "3xtf32", "bf16x3", "tf32"])
def test_noalloc_matches_regular_entry_point(setup, prec):
    ca, ctx = setup
    rng = np.random.default_rng(23)
    N, K = 500, 20004          # a multiple of 4 (16-byte rows), ragged vs 32
    A = torch.as_tensor((rng.standard_normal((N, K))).astype(np.float32)).cuda()
    v = torch.as_tensor(rng.standard_normal(K)).cuda()
    tolG, tolp = TOL[prec]
    # calls in a row, different sizes (tile heights 128, 64 and 32)
    for call, sb in enumerate((100, 37, 20)):
        idx = torch.as_tensor(rng.integers(0, N, size=sb).astype(np.int32)).cuda()
        G0 = torch.zeros((sb, sb), dtype=torch.float64, device="cuda")
        p0 = torch.zeros(sb, dtype=torch.float64, device="cuda")
        ctx.ca_gram_project(A, idx, v, G0, p0, prec=prec)
        G1 = torch.full((sb, sb), float("nan"), dtype=torch.float64, device="cuda")
        p1 = torch.full((sb,), float("nan"), dtype=torch.float64, device="cuda")
        ca.gram_project_noalloc(A, idx, v, G1, p1, prec=prec)
        torch.cuda.synchronize()
        g0, g1 = G0.cpu().numpy(), G1.cpu().numpy()
        nrm = np.sqrt(np.abs(np.diag(g0)))
        assert np.all(np.isfinite(g1)) and np.all(np.isfinite(p1.cpu().numpy()))
        assert (np.abs(g1 - g0) / np.outer(nrm, nrm)).max() < tolG, (call, prec)
        pe = np.abs(p1.cpu().numpy() - p0.cpu().numpy()) / (nrm * float(v.norm()))
        assert pe.max() < tolp, (call, prec)


def test_noalloc_rejects_sizes_beyond_its_scratch(setup):
    ca, _ = setup
    A = torch.zeros((300, 64), dtype=torch.float32, device="cuda")
    v = torch.zeros(64, dtype=torch.float64, device="cuda")
    idx = torch.zeros(129, dtype=torch.int32, device="cuda")
    G = torch.zeros((129, 129), dtype=torch.float64, device="cuda")
    p = torch.zeros(129, dtype=torch.float64, device="cuda")
    with pytest.raises(ca.CaError) as e:
        ca.gram_project_noalloc(A, idx, v, G, p, prec="tf32")
    assert e.value.status == ca.CA_ERR_UNSUPPORTED
