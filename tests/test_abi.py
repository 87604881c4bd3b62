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


def _compositions(rest, g):
    if g == 0:
        return 1 if rest == 0 else 0
    return sum(_compositions(rest - q, g - 1) for q in range(5, 11) if q <= rest)


def _group_bits(desc):
    """Bit positions of every strided group in a plan description, and how many host the phase."""
    bits, phase = [], 0
    for part in desc.split("; "):
        if not part.startswith("group bits "):
            continue
        for a, b in re.findall(r"\[(\d+),(\d+)\)", part):
            bits.extend(range(int(a), int(b)))
        phase += part.endswith("W.B.W") or " W.B.W " in part
    return sorted(bits), phase


@pytest.mark.parametrize("n", [10, 14, 15, 17, 20, 21, 24, 25, 28, 30, 32, 34])
def test_autotune_candidates_cover_every_split(q, n):
    descs = q.tune_candidates(n)
    if n <= 14:
        assert descs == []
        return
    rest = n - 10
    g = (rest + 9) // 10
    full = _compositions(rest, g) * g
    # the default plan comes first; when it is one of the contiguous splits it is
    # not repeated; with TMA passes, n >= 31 adds a 12-bit low pass candidate
    wide = [d for d in descs if "low pass bits [0,12)" in d]
    assert len(wide) == 0 or n >= 31
    assert len(descs) - len(wide) in (full, full + 1)
    assert len(set(descs)) == len(descs)
    widths = set()
    for d in descs:
        bits, phase = _group_bits(d)
        low = 12 if d in wide else 10
        assert bits == list(range(low, n)), d  # every bit above the low pass exactly once
        assert phase == (0 if "rotation form" in d else 1), d  # W.B.W: one phase group
        widths.add(tuple(int(b) - int(a) for a, b in re.findall(r"group bits \[(\d+),(\d+)\)", d)))
    # every first-half width 5 appears: e.g. n = 25 offers 5+10, 6+9, ..., 10+5
    assert len(descs) >= _compositions(rest, g)


def test_autotune_candidates_argument_check(q):
    with pytest.raises(q.QaaError):
        q.tune_candidates(0)
