"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads,
and exports every entry point include/dg.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(dg_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def libdg():
    from paper_1506_06140_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared("dg.h")
    for n in ("dg_create", "dg_rhs", "dg_rk_step", "dg_rk_step_adjoint", "dg_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(libdg):
    for name in declared("dg.h"):
        assert hasattr(libdg, name), name


def test_binding_lists_the_same_symbols():
    from paper_1506_06140_gb300 import dg
    assert sorted(dg.EXPORTS) == declared("dg.h")


def test_default_options_host_only(libdg):
    from paper_1506_06140_gb300 import dg
    L = dg.load()
    opt = dg.Options()
    assert L.dg_default_options(ctypes.byref(opt)) == 0
    assert opt.rk_order == 3 and opt.cfl == 0.2 and opt.beta == 1.0 and opt.Mtilde == 0.5
    assert opt.eps == 1e-10 and opt.precision == 0
    assert L.dg_default_options(None) == dg.DG_ERR_ARG


def test_create_rejects_bad_arguments_before_touching_the_device(libdg):
    from paper_1506_06140_gb300 import dg
    L = dg.load()
    h = ctypes.c_void_p()
    md = dg.MeshDesc()
    md.dim = 4
    assert L.dg_create(ctypes.byref(md), 1, 1.4, None, ctypes.byref(h)) == dg.DG_ERR_ARG
    assert b"dim" in L.dg_last_error(None)
    md.dim = 2
    assert L.dg_create(ctypes.byref(md), 1, 0.9, None, ctypes.byref(h)) == dg.DG_ERR_ARG
    opt = dg.Options()
    L.dg_default_options(ctypes.byref(opt))
    opt.rk_order = 7
    assert L.dg_create(ctypes.byref(md), 1, 1.4, ctypes.byref(opt), ctypes.byref(h)) == dg.DG_ERR_ARG
    opt.rk_order = 3
    assert L.dg_create(ctypes.byref(md), 9, 1.4, ctypes.byref(opt), ctypes.byref(h)) == \
        dg.DG_ERR_UNSUPPORTED
    assert not h.value


def test_oracle_exports():
    from oracle import pyoracle
    L = pyoracle.lib()
    text = open(os.path.join(ROOT, "oracle", "oracle.h")).read()
    for name in re.findall(r"\b(orc_\w+)\s*\(", text):
        assert hasattr(L, name), name
