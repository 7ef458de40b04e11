"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/qpat.h (no GPU needed: nothing is called)."""
import ctypes
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1810_11685_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    from paper_1810_11685_gb300.binding import exported_symbols
    names = exported_symbols()
    for required in ["qpat_create", "qpat_destroy", "qpat_acoustic_forward", "qpat_acoustic_adjoint",
                     "qpat_forward", "qpat_jvp", "qpat_vjp", "qpat_da_solve", "qpat_dot", "qpat_sync",
                     "qpat_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1810_11685_gb300.binding import exported_symbols
    for name in exported_symbols():
        assert hasattr(lib, name), name


def test_binding_loads(lib):
    from paper_1810_11685_gb300 import binding
    assert binding.load() is not None
