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


def test_create_rejects_unsupported_combinations_without_gpu_work():
    """Argument checks of cmles_create run before any device allocation."""
    L = cmles.load()
    h = ctypes.c_void_p()
    good = dict(N=4, nex=2, ney=2, nez=2, Lx=1000.0, Ly=1000.0, Lz=1000.0)

    def status(mesh=good, precision="fp64", **kw):
        m = cmles.make_mesh(mesh)
        P = cmles.make_params(kw, precision)
        return L.cmles_create(ctypes.byref(m), ctypes.byref(P), ctypes.byref(h))

    ERR_ARG = 1
    assert status(closure="mlp") == ERR_ARG                         # learned closure runs in the FP32 kernels
    assert status(mesh=dict(good, warp=True)) == ERR_ARG             # warped meshes run on the FP32 path
    P = cmles.make_params({}, "fp64")
    P.flux = 7
    m = cmles.make_mesh(good)
    assert L.cmles_create(ctypes.byref(m), ctypes.byref(P), ctypes.byref(h)) == ERR_ARG
    P = cmles.make_params(dict(filter_order=8, filter_vars=0b0001), "fp64")   # density is not filterable
    assert L.cmles_create(ctypes.byref(m), ctypes.byref(P), ctypes.byref(h)) == ERR_ARG
    P = cmles.make_params(dict(filter_order=-1), "fp64")
    assert L.cmles_create(ctypes.byref(m), ctypes.byref(P), ctypes.byref(h)) == ERR_ARG
    # HEVI: flat mesh, walls at the bottom and top; an unknown integrator
    assert status(mesh=dict(good, periodic=(1, 1, 1)), integrator="ark2_hevi") == ERR_ARG
    assert status(mesh=dict(good, warp=True), precision="fp32", integrator="ark2_hevi") == ERR_ARG
    P = cmles.make_params({}, "fp64")
    P.integrator = 3
    assert L.cmles_create(ctypes.byref(m), ctypes.byref(P), ctypes.byref(h)) == ERR_ARG
    P = cmles.make_params({}, "fp64")
    P.precision = 5
    assert L.cmles_create(ctypes.byref(m), ctypes.byref(P), ctypes.byref(h)) == ERR_ARG
    # the drag coefficient of the bottom wall: non-negative and finite
    for cd in (-0.01, float("inf"), float("nan")):
        P = cmles.make_params({"drag_cd": cd}, "fp64")
        assert L.cmles_create(ctypes.byref(m), ctypes.byref(P), ctypes.byref(h)) == ERR_ARG, cd
    # no-slip walls: a mask over the six faces
    P = cmles.make_params({"noslip": 1 << 6}, "fp64")
    assert L.cmles_create(ctypes.byref(m), ctypes.byref(P), ctypes.byref(h)) == ERR_ARG


def test_create_order_limits_without_gpu_work():
    """Both precisions take the orders 1 .. 7 on flat meshes, the FP32 path
    on warped meshes, and HEVI (the instantiated kernels); other orders are
    rejected before any device work."""
    L = cmles.load()
    h = ctypes.c_void_p()

    def status(N, precision="fp64", warp=False, **kw):
        m = cmles.make_mesh(dict(N=N, nex=2, ney=2, nez=2, Lx=1000.0, Ly=1000.0, Lz=1000.0, warp=warp))
        P = cmles.make_params(kw, precision)
        return L.cmles_create(ctypes.byref(m), ctypes.byref(P), ctypes.byref(h))

    for N in (0, 8, 9):
        assert status(N) == 1
    for N in (0, 8):
        assert status(N, "fp32") == 1
    assert status(8, "fp32", closure="mlp") == 1
    assert status(8, integrator="ark2_hevi") == 1
    assert status(8, "fp32", warp=True) == 1


def test_host_download_calls_reject_a_null_handle_without_gpu_work():
    L = cmles.load()
    assert L.cmles_fetch_state_host(None, None) == 1    # CMLES_ERR_ARG
    assert L.cmles_wait_fetch(None) == 1
