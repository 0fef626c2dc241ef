"""The C-ABI library loads and exports every function include/ifmm.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ifmm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text,
                       flags=re.M)
    return sorted(set(n for n in names if not n.startswith("typedef")))


@pytest.fixture(scope="module")
def lib():
    import paper_1508_01835_gb300 as pkg
    from paper_1508_01835_gb300 import build
    build.build()
    return pkg.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("ifmm_factor", "ifmm_solve", "fmm_matvec", "gmres_solve", "ifmm_system_create",
                 "ifmm_sigma0", "gmres_solve_host", "ifmm_factor_batch", "ifmm_server_create",
                 "ifmm_server_register", "ifmm_server_submit", "ifmm_server_wait",
                 "ifmm_server_stats", "ifmm_server_destroy", "ifmm_schur_product",
                 "fmm_matvec_static"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_argument_checks(lib):
    assert lib.ifmm_status_string(0) == b"ok"
    assert lib.ifmm_status_string(4) == b"singular pivot block"
    # NULL handles are rejected before any CUDA call
    assert lib.ifmm_solve(None, None, None, None, 1, 10, None) == 1
    assert lib.fmm_matvec(None, None, 0, None, None, 1, 10, None) == 1
    assert lib.ifmm_factor(None, None, None, None) == 1
    out = ctypes.c_void_p()
    assert lib.ifmm_ctx_create(-1, ctypes.byref(out)) == 1
    # the many-systems and product entry points validate before touching CUDA
    assert lib.ifmm_factor_batch(None, None, 0, None, None) == 1
    # a repeated system handle is refused before the context is touched
    fake = ctypes.c_void_p(0x1000)
    two = (ctypes.c_void_p * 2)(0x2000, 0x2000)
    outs = (ctypes.c_void_p * 2)()
    assert lib.ifmm_factor_batch(fake, two, 2, None, outs) == 1
    assert lib.ifmm_server_create(None, 0, 0, ctypes.byref(out)) == 1
    assert lib.ifmm_server_submit(None, 0, None, None, 1, 1e-10, 10, None) == 1
    assert lib.ifmm_server_wait(None, 1, 0, None, None) == 1
    assert lib.ifmm_server_stats(None, None, None, None, None) == 1
    assert lib.ifmm_schur_product(None, 0, 1, 1, 1, None, 1, 0, None, 1, 0, None, 1,
                                  1.0, 0.0, None) == 1
    assert lib.fmm_matvec_static(None, None, None, None, 1, 10, None) == 1


def test_product_path_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_1508_01835_gb300 as pkg
    monkeypatch.setattr(pkg, "_lib", None)
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        pkg.lib()
