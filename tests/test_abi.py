"""The C-ABI library builds, loads and exports every function that include/dgls.h declares
(no compute calls: these run without a GPU)."""
import os
import re

import pytest

from paper_2511_05233_gb300 import build, dgls

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "dgls.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(build.LIB):
        build.build()
    return dgls.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("dg_setup", "dg_residual", "dg_jvp", "dg_step", "dg_discharge"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_params_default_and_argument_checks(lib):
    p = dgls.default_params(dgls.TRADEOFF, 1)
    assert p.order == 1 and p.chemistry == 1 and p.gmres_restart == 30 and p.newton_rtol == 1e-10
    assert abs(p.T - 298.15) < 1e-12
    assert p.preconditioner == 2 and p.precond_every == 0 and p.reorth == 2 and p.eta_min == 1e-3 and p.newton_stall_rtol == 1e-8
    assert p.species_mg == 2
    import ctypes as C
    bad = dgls.Params()
    assert lib.dg_params_default(C.byref(bad), 7, 0) == dgls.ERR_ARG
    h = C.c_void_p()
    assert lib.dg_setup(None, C.byref(p), None, C.byref(h)) == dgls.ERR_ARG


def test_setup_rejects_out_of_range_solver_switches(lib):
    """Argument checks that dg_setup makes before it touches the device: Gram-Schmidt rule,
    species coarse level, V-cycles per application."""
    import ctypes as C

    import numpy as np

    ph = np.zeros((2, 2, 4), dtype=np.uint8)
    ph[:, :, 0] = 1
    s = dgls.Structure(4, 2, 2, 1e-6, ph.ctypes.data_as(C.POINTER(C.c_uint8)))
    for field, value in (("reorth", 3), ("species_mg", 3), ("species_mg", -1), ("mg_cycles", 0), ("mg_cycles", 17),
                         ("jvp_form", 3), ("jvp_form", -1)):
        p = dgls.default_params(dgls.TRADEOFF, 1)
        setattr(p, field, value)
        h = C.c_void_p()
        assert lib.dg_setup(C.byref(s), C.byref(p), None, C.byref(h)) == dgls.ERR_ARG, (field, value)
        assert not h.value
