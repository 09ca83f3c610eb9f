"""CPU checks of the C ABI: the library loads, exports every declared entry
point, and validates arguments before touching the GPU."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^(?!typedef)[A-Za-z_][\w \*]*?\b(wz_\w+)\s*\(", src, re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def wz():
    from paper_1005_3276_gb300 import binding
    return binding


def test_library_exports_every_declared_symbol(wz):
    names = declared_symbols()
    assert len(names) >= 6
    lib = ctypes.CDLL(wz.LIBPATH)
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    assert set(wz.EXPORTS) <= set(names)


def test_supported_extents(wz):
    for n in (4, 6, 8, 12, 16, 32):
        assert wz.wz_supported_extent(n)
    for n in (5, 7, 0, -4, 1000):
        assert not wz.wz_supported_extent(n)


@pytest.mark.parametrize("dims,code", [
    ((5, 4, 4, 4), 1),    # odd T: antiperiodic time needs T even (Sec. 3.1)
    ((4, 4, 4, 8), 5),    # X != Y
    ((4, 4, 7, 7), 5),    # extent without kernels
    ((0, 4, 4, 4), 1),
])
def test_create_rejects_bad_lattices(wz, dims, code):
    with pytest.raises(wz.WzError) as e:
        wz.wz_create(wz.make_params(dims))
    assert e.value.code == code
