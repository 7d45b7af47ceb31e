"""CPU checks of the C ABI: the library loads, exports every declared symbol,
and validates its arguments (calls that touch no GPU)."""
import ctypes
import os
import re

import pytest

from paper_1910_12979_gb300 import native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "mg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported():
    lib = N.load()
    syms = declared_symbols()
    assert len(syms) >= 12
    for s in syms:
        assert hasattr(lib, s), s
    # and the binding wraps each one under the same name
    wrapped = {name for name, _, _ in N.SIGNATURES}
    assert set(syms) <= wrapped


def _geo(n=(64, 64, 64), loc=N.MG_LOC_CELL, h=None):
    dim = len(n)
    n3 = list(n) + [1] * (3 - dim)
    h3 = list(h or [1.0 / max(v, 1) for v in n]) + [1.0] * (3 - dim)
    return N.mg_geometry(dim, tuple(n3), tuple(h3), loc)


def _bc(lo=(0, 0, 1), hi=(0, 0, 2)):
    return N.mg_bc(lo, hi)


def _bytes(geo, bc, opt=None):
    opt = opt or N.mg_default_options()
    n = ctypes.c_size_t(0)
    rc = N.load().mg_hierarchy_bytes(ctypes.byref(geo), ctypes.byref(bc), ctypes.byref(opt), ctypes.byref(n))
    return rc, n.value


def test_hierarchy_bytes_scales_with_grid():
    rc1, b1 = _bytes(_geo((64, 64, 64)), _bc())
    rc2, b2 = _bytes(_geo((128, 128, 128)), _bc())
    assert rc1 == rc2 == N.MG_OK
    assert 7.0 < b2 / b1 < 8.5
    opt = N.mg_default_options()
    opt.prec = N.MG_PREC_FP64
    rc3, b3 = _bytes(_geo((128, 128, 128)), _bc(), opt)
    assert rc3 == N.MG_OK and b3 != b2


@pytest.mark.parametrize("geo,bc,want", [
    (_geo((64, 64, 64)), _bc((0, 0, 1), (1, 0, 2)), N.MG_ERR_INVALID_ARG),       # unpaired periodic
    (_geo((64, 64, 64)), _bc((0, 0, 7), (0, 0, 2)), N.MG_ERR_INVALID_ARG),       # bad kind
    (_geo((63, 63, 63)), _bc(), N.MG_ERR_UNSUPPORTED),                           # does not coarsen
    (_geo((64, 64, 64), N.MG_LOC_NODAL, (0.1, 0.2, 0.1)), _bc(), N.MG_ERR_INVALID_ARG),  # anisotropic nodal
    (_geo((0, 64, 64)), _bc(), N.MG_ERR_INVALID_ARG),
])
def test_argument_validation(geo, bc, want):
    rc, _ = _bytes(geo, bc)
    assert rc == want
    assert N.mg_last_error()


def test_null_arguments_rejected():
    lib = N.load()
    assert lib.mg_solve(None, None, None, ctypes.c_double(1e-10), None) == N.MG_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert lib.mg_setup(None, None, None, None, None, 0, ctypes.byref(h)) == N.MG_ERR_INVALID_ARG
    assert N.mg_strerror(N.MG_ERR_NOT_CONVERGED) == "not converged"
