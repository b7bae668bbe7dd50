"""CPU checks of the C ABI: the library builds, loads and exports every
function include/dgmg.h declares.  No compute call is made (no GPU here)."""
import ctypes
import os

import pytest

from paper_1805_11930_gb300 import build, dgmg


def _lib_or_skip():
    if not build.up_to_date():
        try:
            build.build()
        except RuntimeError as e:       # no nvcc in this environment
            pytest.skip(str(e))
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = dgmg.exported_symbols()
    for required in ("dgmg_create", "dgmg_destroy", "dgmg_set_mesh", "dgmg_set_coefficients",
                     "dgmg_assemble_rhs", "dgmg_apply", "dgmg_block_apply", "dgmg_block_smooth",
                     "dgmg_restrict", "dgmg_prolong_add", "dgmg_coarse_cycle", "dgmg_vcycle",
                     "dgmg_solve", "dgmg_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = _lib_or_skip()
    for name in dgmg.exported_symbols():
        assert hasattr(lib, name), name
    assert set(dgmg.exported_symbols()) == set(dgmg._SIG), "binding and header disagree"


def test_default_opts_without_gpu():
    _lib_or_skip()
    o = dgmg.default_opts()
    assert o.rtol == 1e-8 and o.restart == 30 and o.eps_inner == 1e-2 and o.npre == 1 and o.npost == 1


def test_create_fails_cleanly_without_device():
    lib = dgmg.load()
    h = ctypes.c_void_p()
    st = lib.dgmg_create(ctypes.byref(h), 10_000, None)
    assert st == 1 and not h.value
