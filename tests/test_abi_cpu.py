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
    o = ca.ca_opts(4, 4, 200, 1e-3, 42, ca.CA_GRAM_F64, 0, 0, 0.0, 0, 0, 0)
    assert lib.ca_bcd_solve(None, 0, None, 64, 1024, 1024, None, ctypes.byref(o), None, None) == \
        ca.CA_ERR_ARG
    assert lib.ca_bdcd_solve(None, 0, None, 64, 1024, 64, None, ctypes.byref(o), None, None) == \
        ca.CA_ERR_ARG
    assert lib.ca_sample_indices(None, 1, 0, 1, 1, 1, None) == ca.CA_ERR_ARG
    assert lib.ca_profile_enable(None, 1) == ca.CA_ERR_ARG
    assert lib.ca_solve_info(None, None) == ca.CA_ERR_ARG
    assert lib.ca_solve_trace(None, None, 0, None) == ca.CA_ERR_ARG
    assert lib.ca_server_submit(None, None, None) == ca.CA_ERR_ARG
    assert lib.ca_server_create(None, 0, 4, 1 << 20) == ca.CA_ERR_ARG
    h = ctypes.c_void_p()
    assert lib.ca_server_create(ctypes.byref(h), 0, 0, 1 << 20) == ca.CA_ERR_ARG  # no workers
    assert lib.ca_server_create(ctypes.byref(h), 0, 4, 0) == ca.CA_ERR_ARG  # no budget
    assert lib.ca_server_wait(None, 0, None) == ca.CA_ERR_ARG
    assert lib.ca_server_drain(None) == ca.CA_ERR_ARG
    assert lib.ca_solve_scratch_bytes(None, 0, 0, 1, 1, None, None) == ca.CA_ERR_ARG
    assert lib.ca_bcd_release_scratch(None) == ca.CA_ERR_ARG
    assert lib.ca_server_get_stats(None, None) == ca.CA_ERR_ARG
    lib.ca_server_destroy(None)  # no-op
    lib.ca_bcd_destroy(None)  # no-op


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(ca, "_lib", None)
    monkeypatch.setattr(ca, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        ca.load()


def _c_layout(tmp_path, struct, fields):
    """sizeof and offsetof of a header struct, from a C program built with gcc."""
    import os
    import subprocess
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "layout.c"
    body = "".join(f'  printf("%zu\\n", offsetof({struct}, {f}));\n' for f in fields)
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"ca_serve.h\"\n"
                   f"int main(void) {{\n  printf(\"%zu\\n\", sizeof({struct}));\n{body}  return 0;\n}}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    return [int(v) for v in out]


@pytest.mark.parametrize("py,c", [(lambda: ca.ca_opts, "ca_opts"), (lambda: ca.ca_info, "ca_info"),
                                  (lambda: ca.ca_check, "ca_check"),
                                  (lambda: ca.ca_request, "ca_request"),
                                  (lambda: ca.ca_result, "ca_result"),
                                  (lambda: ca.ca_server_stats, "ca_server_stats")])
def test_struct_layout_matches_header(tmp_path, py, c):
    cls = py()
    names = [f[0] for f in cls._fields_]
    got = _c_layout(tmp_path, c, names)
    assert got[0] == ctypes.sizeof(cls)
    assert got[1:] == [getattr(cls, f).offset for f in names]
