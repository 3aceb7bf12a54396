"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/*.h. No GPU needed (no compute call is made)."""

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:int|void|const\s+char\s*\*)\s+(dg_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dg_poisson_setup", "dg_pair_solve_batch", "dg_exchange_build", "dg_destroy", "dg_error_string"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2510_21213_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_and_error_strings():
    from paper_2510_21213_gb300 import build, dgx

    build.build()
    lib = dgx.load()
    assert lib.dg_error_string(0) == b"ok"
    assert lib.dg_error_string(-3) == b"not converged"
    o = dgx.dg_default_opts()
    assert o.rtol == pytest.approx(1e-8) and o.penalty_eps == pytest.approx(0.125) and o.smoother_degree == 4 and o.smoother == 1


def test_options_are_checked_before_any_device_work():
    """dg_poisson_setup refuses out-of-range options on the host (no GPU
    needed): the device-loop switch takes 0, 1 or 2 (2, adaptive, by default)."""
    from paper_2510_21213_gb300 import dgx

    lib = dgx.load()
    C = dgx.C
    assert dgx.dg_default_opts().device_loop == 2
    desc = dgx.dg_mesh_desc((C.c_double * 3)(-1, -1, -1), (C.c_double * 3)(1, 1, 1), (C.c_int32 * 3)(2, 2, 2), 2)
    for bad in (-1, 3):
        o = dgx.dg_default_opts(device_loop=bad)
        h = C.c_void_p()
        assert lib.dg_poisson_setup(C.byref(desc), C.byref(o), C.byref(h)) == dgx.DG_ERR_INVALID_ARG and not h.value
