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


def test_context_calls_reject_a_null_context(wz):
    """Every context call checks its handle before touching the device."""
    L = wz.LIB
    n = None
    calls = {
        "wz_set_phi": lambda: L.wz_set_phi(n, n),
        "wz_get_phi": lambda: L.wz_get_phi(n, n),
        "wz_apply": lambda: L.wz_apply(n, 0, 1, n, n, 1, 0.0),
        "wz_solve": lambda: L.wz_solve(n, n, n, 1, 0.0, 1e-10, 10, 0, n, n),
        "wz_force": lambda: L.wz_force(n, n, 1, 1e-10, 3, n, n, n, n),
        "wz_action": lambda: L.wz_action(n, n, 1, 1e-10, n, n, n),
        "wz_trajectory": lambda: L.wz_trajectory(n, n, n),
        "wz_ward_identity": lambda: L.wz_ward_identity(n, 1e-10, 10, 0, n, n, n),
        "wz_supercurrent": lambda: L.wz_supercurrent(n, n, 1e-10, 10, 0, n, n),
        "wz_aux_vev": lambda: L.wz_aux_vev(n, n),
        "wz_locality": lambda: L.wz_locality(n, n, 0),
        "wz_spectral_bounds": lambda: L.wz_spectral_bounds(n, n, n),
        "wz_apply_mdagm_noalloc": lambda: L.wz_apply_mdagm_noalloc(n, 0, n, n, 1, 0.0),
        "wz_set_workspace_limit": lambda: L.wz_set_workspace_limit(n, 0),
    }
    for name, call in calls.items():
        assert call() == wz.WZ_EINVAL, name
    assert L.wz_destroy(n) == wz.WZ_OK
    assert L.wz_workspace_bytes(n) == 0


def test_product_and_oracle_share_no_code():
    """The product package never imports the oracle (its results must come
    from the library's kernels), and the oracle never imports the product."""
    pat_oracle = re.compile(r"^\s*(import oracle|from oracle\b|from \.\.oracle|import \.\.oracle)", re.M)
    pkg = os.path.join(ROOT, "paper_1005_3276_gb300")
    for fn in os.listdir(pkg):
        if fn.endswith(".py"):
            assert not pat_oracle.search(open(os.path.join(pkg, fn)).read()), fn
    pat_prod = re.compile(r"^\s*(import|from)\s+paper_1005_3276_gb300\b", re.M)
    odir = os.path.join(ROOT, "oracle")
    for fn in os.listdir(odir):
        if fn.endswith(".py"):
            src = open(os.path.join(odir, fn)).read()
            assert not pat_prod.search(src), fn
            assert "ctypes" not in src and "libwz" not in src, fn
