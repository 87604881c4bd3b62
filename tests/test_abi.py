"""The C-ABI library: it builds, loads, exports what include/qaa.h declares, and
rejects bad arguments before touching a GPU (runs without one)."""

import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared_functions():
    with open(os.path.join(ROOT, "include", "qaa.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qaa_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def q():
    from paper_1103_1399_gb300 import build
    build.build()
    import paper_1103_1399_gb300 as q
    return q


def test_header_and_binding_agree(q):
    declared = _declared_functions()
    assert "qaa_evolve" in declared and "qaa_create" in declared
    assert sorted(q.SIGNATURES) == declared


def test_library_exports_every_declared_symbol(q):
    lib = ctypes.CDLL(q.LIB_PATH)
    for name in _declared_functions():
        assert hasattr(lib, name), name
    assert q.lib.qaa_version() == 1


def _create(q, n, flat, m):
    buf = (ctypes.c_int32 * max(len(flat), 1))(*flat) if flat else (ctypes.c_int32 * 1)(0)
    h = ctypes.c_void_p()
    st = q.lib.qaa_create(n, ctypes.cast(buf, ctypes.c_void_p), m, ctypes.byref(h))
    return st, h, q.lib.qaa_last_error().decode()


@pytest.mark.parametrize(
    "n,flat,m,needle",
    [
        (0, [], 0, "n out of range"),
        (35, [], 0, "n out of range"),
        (3, [1, 2, 4], 1, "literal beyond n"),
        (3, [1, -1, 2], 1, "repeated"),
        (3, [0, 0, 0], 1, "no literals"),
        (3, [1, 2, 3], 1024, "m out of range"),
        (3, [1, 2, 3], -1, "m out of range"),
    ],
)
def test_invalid_arguments_are_rejected(q, n, flat, m, needle):
    st, h, msg = _create(q, n, flat, m)
    assert st == -1, (st, msg)
    assert needle in msg
    assert not h.value


def test_null_handle_is_an_argument_error(q):
    assert q.lib.qaa_evolve(None, None, 1.0, 1) == -1
    assert q.lib.qaa_destroy(None) == 0
    assert "null handle" in q.lib.qaa_last_error().decode()


def test_flatten_pads_short_clauses(q):
    buf, m = q.flatten_clauses([[1], [2, -3], [4, 5, -6]])
    assert m == 3
    assert list(buf) == [1, 0, 0, 2, -3, 0, 4, 5, -6]
    with pytest.raises(ValueError):
        q.flatten_clauses([[1, 2, 3, 4]])
