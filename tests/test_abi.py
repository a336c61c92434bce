"""CPU checks of the C ABI library: it loads and exports every entry point
that include/fd.h declares (no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fd.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(fd_[a-z_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2312_13094_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_entry_points():
    names = _declared()
    for must in ("fd_create_grid", "fd_set_model", "fd_forward", "fd_adjoint_gradient",
                 "fd_batch_forward", "fd_destroy_grid", "fd_status_string", "fd_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2312_13094_gb300 import binding
    assert sorted(binding.EXPORTED) == _declared()


def test_status_strings_without_gpu(lib):
    lib.fd_status_string.restype = ctypes.c_char_p
    assert lib.fd_status_string(0) == b"ok"
    assert b"stability" in lib.fd_status_string(4)
    lib.fd_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.fd_last_error(), bytes)
