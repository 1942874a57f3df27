"""The C ABI library loads and exports every entry point its header declares.

Runs without a GPU: it only loads the shared library and resolves symbols
(no compute call is made).
"""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(ws_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2204_03775_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = _declared("wavestep.h")
    for required in ["ws_create", "ws_set_velocity", "ws_add_source", "ws_set_receivers",
                     "ws_step", "ws_read_traces", "ws_destroy", "ws_last_error"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared("wavestep.h") if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    import paper_2204_03775_gb300.binding as b
    missing = [n for n in _declared("wavestep.h") if not hasattr(b, n)]
    assert not missing, missing


def test_last_error_without_gpu(lib):
    lib.ws_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.ws_last_error(), bytes)
