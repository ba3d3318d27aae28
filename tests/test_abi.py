"""C-ABI checks that need no GPU: the library loads, exports every entry
point the public header declares, and rejects bad arguments on the host
before any launch."""
import ctypes
import os
import re

import pytest

import paper_2310_19925_b300 as orand

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in ("orand.h",):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(orand_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2310_19925_b300 import build

    build.build()
    return orand._lib()


def test_exports_every_declared_symbol(lib):
    declared = _declared_functions()
    assert "orand_fill_u32" in declared and len(declared) >= 8
    for name in declared:
        assert hasattr(lib, name), name
        assert name in orand._SIGS, "binding lacks " + name


def test_status_strings(lib):
    for code, name in orand.STATUS_NAMES.items():
        assert lib.orand_status_string(code).decode().startswith(name)
    assert lib.orand_version() >= 100


@pytest.mark.parametrize("gen,dtype", [(4, 0), (-1, 0), (0, 4), (0, -2)])
def test_bad_enums_rejected(lib, gen, dtype):
    assert lib.orand_fill(gen, dtype, 1, 0, 4, 4, 16, None) == -1


def test_overflow_rejected(lib):
    assert lib.orand_fill(0, 0, 1, 0, 2**40, 2**30, 16, None) == -2          # n*dps overflows
    assert lib.orand_fill(0, 0, 1, 0, 2**62, 2, 16, None) == -2              # bytes overflow
    assert lib.orand_fill(0, 0, 1, 0, 1, 2**32 + 1, 16, None) == -2          # > 2^32 words
    assert lib.orand_fill(0, 2, 1, 0, 1, 2**31 + 1, 16, None) == -2          # f64 needs 2 words each


def test_null_and_alignment_rejected(lib):
    assert lib.orand_fill(0, 0, 1, 0, 4, 4, None, None) == -1
    assert lib.orand_fill(0, 0, 1, 0, 4, 4, 2, None) == -3                   # u32 at 2-byte offset
    assert lib.orand_fill(0, 2, 1, 0, 4, 4, 4, None) == -3                   # f64 at 4-byte offset


def test_empty_fill_is_a_noop(lib):
    assert lib.orand_fill(0, 0, 1, 0, 0, 5, None, None) == 0
    assert lib.orand_fill(3, 3, 1, 0, 7, 0, None, None) == 0


def test_python_errors_raise(lib):
    with pytest.raises(orand.OrandError):
        orand.orand_fill(9, 0, 1, 0, 1, 1, 16, 0)
