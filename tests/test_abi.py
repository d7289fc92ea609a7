"""The C-ABI library builds for sm_103a, loads on a machine without a GPU and
exports every entry point include/cmles.h declares (no compute calls)."""
import ctypes

from paper_2110_00853_b300 import build as B
from paper_2110_00853_b300 import cmles


def test_library_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    names = cmles.header_symbols()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_default_params_match_constants_table():
    P = cmles.default_params()
    assert (P.Rd, P.Rv, P.cvd, P.cvv, P.cvl, P.cvi) == (287.0, 462.0, 717.5, 1397.5, 4181.0, 2100.0)
    assert (P.T0, P.Lv0, P.Lf0) == (273.16, 2.5008e6, 0.3336e6)
    assert abs(P.Prt - 1.0 / 3.0) < 1e-16


def test_create_rejects_bad_arguments_without_gpu_work():
    L = cmles.load()
    m = cmles.make_mesh(dict(N=4, nex=0, ney=1, nez=1, Lx=1.0, Ly=1.0, Lz=1.0))
    P = cmles.default_params()
    h = ctypes.c_void_p()
    assert L.cmles_create(ctypes.byref(m), ctypes.byref(P), ctypes.byref(h)) == 6   # CMLES_ERR_MESH
    m = cmles.make_mesh(dict(N=9, nex=1, ney=1, nez=1, Lx=1.0, Ly=1.0, Lz=1.0))
    assert L.cmles_create(ctypes.byref(m), ctypes.byref(P), ctypes.byref(h)) == 1   # CMLES_ERR_ARG
    assert L.cmles_create(None, ctypes.byref(P), ctypes.byref(h)) == 1
