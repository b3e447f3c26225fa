"""Host-side checks of the C ABI library (no GPU needed, no compute calls)."""
import ctypes

import pytest

import paper_1612_04003_gb300 as ca
from paper_1612_04003_gb300 import buildlib


@pytest.fixture(scope="module")
def lib():
    buildlib.build()
    return ca.load()


def test_header_declares_the_abi():
    names = ca.header_functions()
    for required in ("ca_bcd_init", "ca_bcd_solve", "ca_bdcd_solve", "ca_sample_indices",
                     "ca_status_str", "ca_bcd_destroy"):
        assert required in names


def test_library_exports_every_header_symbol(lib):
    for name in ca.header_functions():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_status_strings(lib):
    for st in range(-7, 1):
        s = ca.status_str(st)
        assert s.startswith("CA_")
    assert "unknown" in ca.status_str(-99)


def test_null_arguments_rejected_without_gpu(lib):
    o = ca.ca_opts(4, 4, 200, 1e-3, 42, ca.CA_GRAM_F64, 0, 0)
    assert lib.ca_bcd_solve(None, 0, None, 64, 1024, 1024, None, ctypes.byref(o), None, None) == \
        ca.CA_ERR_ARG
    assert lib.ca_bdcd_solve(None, 0, None, 64, 1024, 64, None, ctypes.byref(o), None, None) == \
        ca.CA_ERR_ARG
    assert lib.ca_sample_indices(None, 1, 0, 1, 1, 1, None) == ca.CA_ERR_ARG
    assert lib.ca_profile_enable(None, 1) == ca.CA_ERR_ARG
    lib.ca_bcd_destroy(None)  # no-op


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(ca, "_lib", None)
    monkeypatch.setattr(ca, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        ca.load()


def test_opts_layout_matches_header():
    # b, s (int), H (long long), lam (double), seed (u64), prec, recompute_every (int), h0
    assert ctypes.sizeof(ca.ca_opts) == 4 + 4 + 8 + 8 + 8 + 4 + 4 + 8
    assert ca.ca_opts.H.offset == 8 and ca.ca_opts.lam.offset == 16
    assert ca.ca_opts.prec.offset == 32 and ca.ca_opts.h0.offset == 40
