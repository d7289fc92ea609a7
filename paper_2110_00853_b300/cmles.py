"""Thin Python binding of the cmles C ABI (include/cmles.h).

Argument marshalling only: every step of the DG right-hand side, the
Runge-Kutta update, the diagnostics and the initial-state evaluation runs in
the library's CUDA kernels.  torch supplies device memory and the stream.
There is no CPU fallback: creating a Solver without the built library or
without a CUDA device raises.
"""
import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcmles.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "cmles.h")

CMLES_FP64, CMLES_FP32_ACC64 = 0, 1
CLOSURE = {"none": 0, "sl": 1, "mlp": 2, "vreman": 3}
FLUX = {"rusanov": 0, "hllc": 1, "roe": 2}
INTEGRATOR = {"lsrk54": 0, "lsrk144": 1, "ark2_hevi": 2}
PRECISION = {"fp64": CMLES_FP64, "fp32": CMLES_FP32_ACC64, "fp32acc64": CMLES_FP32_ACC64}
STATUS = {0: "CMLES_OK", 1: "CMLES_ERR_ARG", 2: "CMLES_ERR_OOM", 3: "CMLES_ERR_CUDA", 4: "CMLES_ERR_SATADJ",
          5: "CMLES_ERR_NONFINITE", 6: "CMLES_ERR_MESH", 7: "CMLES_ERR_STATE", 8: "CMLES_ERR_TIMEOUT"}
MLP_PARAMS = 64 * 13 + 64 + 64 * 64 + 64 + 2 * 64 + 2 + 13 + 2   # 5201
MLP_NET = MLP_PARAMS - 15                                        # trainable part: W1 .. b3


class Mesh(C.Structure):
    _fields_ = [("N", C.c_int), ("nex", C.c_int), ("ney", C.c_int), ("nez", C.c_int),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("Lx", C.c_double), ("Ly", C.c_double), ("Lz", C.c_double), ("periodic", C.c_int * 3),
                ("warp", C.c_int), ("hill_h", C.c_double), ("hill_a", C.c_double), ("hill_xc", C.c_double)]


class Params(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("g", "p0", "Rd", "Rv", "cvd", "cvv", "cvl", "cvi", "T0", "Lv0", "Lf0",
                                          "ptr", "Ttr")] + [
        ("closure", C.c_int), ("Cs", C.c_double), ("Prt", C.c_double), ("richardson", C.c_int),
        ("moist", C.c_int), ("sponge_alpha", C.c_double), ("sponge_zs", C.c_double), ("sponge_gamma", C.c_double),
        ("u_relax", C.c_double * 3), ("lateral_sponge_frac", C.c_double), ("surface_flux", C.c_int),
        ("shf", C.c_double), ("lhf", C.c_double), ("Omega", C.c_double * 3), ("precision", C.c_int),
        ("dt", C.c_double), ("satadj_max_iter", C.c_int), ("flux", C.c_int), ("filter_order", C.c_int),
        ("filter_alpha", C.c_double), ("filter_vars", C.c_int), ("integrator", C.c_int), ("drag_cd", C.c_double),
        ("noslip", C.c_int)]


class Diag(C.Structure):
    _fields_ = [("budget", C.c_double * 6), ("time", C.c_double), ("steps", C.c_longlong),
                ("nonfinite", C.c_int), ("satadj_failures", C.c_int), ("tc_timeouts", C.c_int),
                ("cold_saturated", C.c_int)]


class Case(C.Structure):
    _fields_ = [("id", C.c_int), ("seed", C.c_uint64), ("theta0", C.c_double), ("dtheta", C.c_double),
                ("r0", C.c_double), ("xc", C.c_double), ("yc", C.c_double), ("zc", C.c_double),
                ("noise_theta", C.c_double), ("noise_qt", C.c_double), ("noise_zmax", C.c_double),
                ("NBV", C.c_double), ("u0", C.c_double * 3), ("qt_sfc", C.c_double), ("qt_ml", C.c_double),
                ("z_ml", C.c_double), ("qt_top", C.c_double), ("dthdz_above", C.c_double), ("moist", C.c_int),
                ("nmodes", C.c_int), ("modes", C.POINTER(C.c_double)), ("qt_H", C.c_double)]


_lib = None
_H = C.c_void_p
_VP = C.c_void_p
_DP = C.POINTER(C.c_double)


def header_symbols():
    """Function names declared in include/cmles.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(cmles_[a-z0-9_]+)\s*\(", text)))


def load(path=LIB_PATH):
    """Load libcmles.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"cmles CUDA library not built: {path} is missing (run __graft_entry__.build())")
    L = C.CDLL(path)
    L.cmles_default_params.argtypes = [C.POINTER(Params)]
    L.cmles_default_params.restype = None
    L.cmles_create.argtypes = [C.POINTER(Mesh), C.POINTER(Params), C.POINTER(_H)]
    L.cmles_destroy.argtypes = [_H]
    L.cmles_last_error_message.argtypes = [_H]
    L.cmles_last_error_message.restype = C.c_char_p
    L.cmles_set_stream.argtypes = [_H, _VP]
    L.cmles_set_reference.argtypes = [_H, _DP, _DP, _DP, C.c_size_t]
    L.cmles_init_case.argtypes = [_H, C.POINTER(Case)]
    for n in ("cmles_set_state", "cmles_get_state", "cmles_set_state_host", "cmles_get_state_host"):
        getattr(L, n).argtypes = [_H, _VP]
    L.cmles_tendency.argtypes = [_H, _VP, _VP]
    L.cmles_step.argtypes = [_H, C.c_int]
    L.cmles_filter.argtypes = [_H]
    L.cmles_diagnostics.argtypes = [_H, C.POINTER(Diag)]
    L.cmles_profiles.argtypes = [_H, _DP]
    L.cmles_set_closure_weights.argtypes = [_H, C.POINTER(C.c_float), C.c_size_t]
    L.cmles_enable_timing.argtypes = [_H, C.c_int]
    L.cmles_kernel_times.argtypes = [_H, C.POINTER(C.c_longlong), _DP, C.POINTER(C.c_longlong)]
    L.cmles_budgets_noalloc.argtypes = [_VP, C.c_longlong, C.c_int, C.c_double, _VP, _VP]
    L.cmles_set_closure_weights_device.argtypes = [_H, _VP]
    L.cmles_closure_samples.argtypes = [_H, C.c_int, _VP, _VP, _VP, C.c_longlong, C.POINTER(C.c_longlong)]
    L.cmles_mlp_forward.argtypes = [_VP, _VP, _VP, C.c_longlong, _VP]
    L.cmles_mlp_loss_grad.argtypes = [_VP, _VP, _VP, C.c_longlong, _VP, _VP, _VP]
    L.cmles_mlp_adam.argtypes = [_VP, _VP, _VP, _VP, C.c_int, C.c_float, C.c_float, C.c_float, C.c_float, _VP]
    L.cmles_test_stall_tc.argtypes = [_H, C.c_int]
    L.cmles_stage_state_host.argtypes = [_H, _VP]
    L.cmles_commit_staged_state.argtypes = [_H]
    L.cmles_fetch_state_host.argtypes = [_H, _VP]
    L.cmles_wait_fetch.argtypes = [_H]
    L.cmles_hevi_operator.argtypes = [_H, _VP, _VP]
    L.cmles_hevi_solve.argtypes = [_H, _VP, _VP]
    L.cmles_spectrum.argtypes = [_H, C.c_int, _DP]
    L.cmles_group_create.argtypes = [C.POINTER(Mesh), C.POINTER(Params), C.c_int, C.c_int, C.POINTER(_VP)]
    L.cmles_group_destroy.argtypes = [_VP]
    L.cmles_group_last_error_message.argtypes = [_VP]
    L.cmles_group_last_error_message.restype = C.c_char_p
    L.cmles_group_set_stream.argtypes = [_VP, _VP]
    L.cmles_group_set_reference.argtypes = [_VP, _DP, _DP, _DP, C.c_size_t]
    L.cmles_group_set_closure_weights.argtypes = [_VP, C.POINTER(C.c_float), C.c_size_t]
    for n in ("cmles_group_set_state", "cmles_group_get_state"):
        getattr(L, n).argtypes = [_VP, _VP]
    L.cmles_group_tendency.argtypes = [_VP, _VP, _VP]
    L.cmles_group_step.argtypes = [_VP, C.c_int]
    L.cmles_group_diagnostics.argtypes = [_VP, C.POINTER(Diag)]
    L.cmles_group_halo_bytes.argtypes = [_VP]
    L.cmles_group_halo_bytes.restype = C.c_longlong
    L.cmles_halo_plan.argtypes = [C.POINTER(Mesh), C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int),
                                  C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
    for n in ("cmles_launch_count", "cmles_num_elements", "cmles_num_nodes", "cmles_device_bytes"):
        getattr(L, n).argtypes = [_H]
        getattr(L, n).restype = C.c_longlong
    _lib = L
    return L


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def mlp_forward(params, X):
    """Y[n][2] = closure network(X[n][13]) on BF16 tensor cores (device tensors)."""
    import torch
    Y = torch.empty((X.shape[0], 2), dtype=torch.float32, device=X.device)
    st = load().cmles_mlp_forward(_ptr(params), _ptr(X), _ptr(Y), X.shape[0], _stream())
    if st != 0:
        raise CmlesError(st, "cmles_mlp_forward failed")
    return Y


def mlp_loss_grad(params, X, T):
    """(loss, grad[5186]) of the closure network on a batch (device tensors)."""
    import torch
    grad = torch.empty(MLP_NET, dtype=torch.float32, device=X.device)
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    st = load().cmles_mlp_loss_grad(_ptr(params), _ptr(X), _ptr(T), X.shape[0], _ptr(grad), _ptr(loss), _stream())
    if st != 0:
        raise CmlesError(st, "cmles_mlp_loss_grad failed")
    return loss, grad


def mlp_adam(params, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    st = load().cmles_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(t), lr, beta1, beta2, eps, _stream())
    if st != 0:
        raise CmlesError(st, "cmles_mlp_adam failed")


class CmlesError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def default_params():
    P = Params()
    load().cmles_default_params(C.byref(P))
    return P


def make_mesh(d):
    m = Mesh()
    m.N, m.nex, m.ney, m.nez = d["N"], d["nex"], d["ney"], d["nez"]
    m.x0, m.y0, m.z0 = d.get("x0", 0.0), d.get("y0", 0.0), d.get("z0", 0.0)
    m.Lx, m.Ly, m.Lz = d["Lx"], d["Ly"], d["Lz"]
    m.periodic = (C.c_int * 3)(*d.get("periodic", (1, 1, 0)))
    m.warp = int(d.get("warp", False))
    m.hill_h, m.hill_a, m.hill_xc = d.get("hill_h", 0.0), d.get("hill_a", 1.0), d.get("hill_xc", 0.0)
    return m


def make_params(d, precision="fp64"):
    P = default_params()
    for k, v in d.items():
        if k == "closure":
            P.closure = CLOSURE[v]
        elif k == "flux":
            P.flux = FLUX[v]
        elif k == "integrator":
            P.integrator = INTEGRATOR[v]
        elif k in ("u_relax", "Omega"):
            setattr(P, k, (C.c_double * 3)(*v))
        elif k in ("richardson", "moist", "surface_flux"):
            setattr(P, k, int(v))
        else:
            setattr(P, k, v)
    P.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    return P


class Solver:
    """A cmles handle: one DG-LES problem on the current CUDA device."""

    def __init__(self, mesh, physics, precision="fp64"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("cmles needs a CUDA device; no CPU fallback exists")
        self.torch = torch
        self.L = load()
        self.mesh_d = dict(mesh)
        self.phys_d = dict(physics)
        self._mesh = make_mesh(mesh)
        self._params = make_params(physics, precision)
        h = _H()
        st = self.L.cmles_create(C.byref(self._mesh), C.byref(self._params), C.byref(h))
        if st != 0:
            raise CmlesError(st, "cmles_create failed")
        self.h = h
        self.N = mesh["N"]
        self.Np = (self.N + 1) ** 3
        self.E = mesh["nex"] * mesh["ney"] * mesh["nez"]
        self.nlev = mesh["nez"] * (self.N + 1)
        self.set_stream(torch.cuda.current_stream())

    def _check(self, st):
        if st != 0:
            raise CmlesError(st, self.L.cmles_last_error_message(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.cmles_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self.stream = stream
        self._check(self.L.cmles_set_stream(self.h, C.c_void_p(stream.cuda_stream)))

    def set_reference(self, rho_r, p_r, qt_r=None):
        rho_r = np.ascontiguousarray(rho_r, np.float64)
        p_r = np.ascontiguousarray(p_r, np.float64)
        q = None if qt_r is None else np.ascontiguousarray(qt_r, np.float64)
        self._check(self.L.cmles_set_reference(self.h, rho_r.ctypes.data_as(_DP), p_r.ctypes.data_as(_DP),
                                               None if q is None else q.ctypes.data_as(_DP), rho_r.size))

    def init_case(self, case):
        cs = Case()
        keep = None
        for k, v in case.items():
            if k == "u0":
                cs.u0 = (C.c_double * 3)(*v)
            elif k == "modes":
                if v is not None:
                    keep = np.ascontiguousarray(v, np.float64)
                    cs.nmodes = keep.shape[0]
                    cs.modes = keep.ctypes.data_as(_DP)
            elif k == "moist":
                cs.moist = int(v)
            elif k in dict(Case._fields_):
                setattr(cs, k, v)
        self._check(self.L.cmles_init_case(self.h, C.byref(cs)))
        del keep

    def _dev(self, t):
        torch = self.torch
        assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
        assert t.numel() == self.E * 6 * self.Np
        return C.c_void_p(t.data_ptr())

    def set_state(self, Q):
        self._check(self.L.cmles_set_state(self.h, self._dev(Q)))

    def get_state(self):
        Q = self.torch.empty((self.E, 6, self.Np), dtype=self.torch.float64, device="cuda")
        self._check(self.L.cmles_get_state(self.h, self._dev(Q)))
        return Q

    def set_state_host(self, Q):
        Q = Q.contiguous()
        assert not Q.is_cuda and Q.dtype == self.torch.float64
        self._check(self.L.cmles_set_state_host(self.h, C.c_void_p(Q.data_ptr())))

    def stage_state_host(self, Q):
        """Start copying the pinned host state Q into the staging buffer
        (asynchronous; Q must stay unchanged until committed)."""
        assert not Q.is_cuda and Q.dtype == self.torch.float64 and Q.is_contiguous()
        self._staged_host = Q
        self._check(self.L.cmles_stage_state_host(self.h, C.c_void_p(Q.data_ptr())))

    def commit_staged_state(self):
        """Take the staged state as the state (the handle's stream waits for the copy)."""
        self._check(self.L.cmles_commit_staged_state(self.h))

    def fetch_state_host(self, out):
        """Start copying the state into the pinned host tensor `out`
        (asynchronous; read `out` only after wait_fetch)."""
        assert not out.is_cuda and out.dtype == self.torch.float64 and out.is_contiguous()
        assert out.numel() == self.E * 6 * self.Np
        self._fetch_host = out
        self._check(self.L.cmles_fetch_state_host(self.h, C.c_void_p(out.data_ptr())))

    def wait_fetch(self):
        """Block until the latest fetch_state_host copy has completed."""
        self._check(self.L.cmles_wait_fetch(self.h))

    def get_state_host(self, out=None):
        if out is None:
            out = self.torch.empty((self.E, 6, self.Np), dtype=self.torch.float64, pin_memory=True)
        self._check(self.L.cmles_get_state_host(self.h, C.c_void_p(out.data_ptr())))
        return out

    def tendency(self, Q, out=None):
        if out is None:
            out = self.torch.empty_like(Q)
        self._check(self.L.cmles_tendency(self.h, self._dev(Q), self._dev(out)))
        return out

    def step(self, n=1):
        self._check(self.L.cmles_step(self.h, int(n)))

    def filter(self):
        """one application of the exponential filter to the current state"""
        self._check(self.L.cmles_filter(self.h))

    def diagnostics(self, raise_on_error=True):
        d = Diag()
        st = self.L.cmles_diagnostics(self.h, C.byref(d))
        if raise_on_error and st not in (0,):
            self._check(st)
        return dict(budget=np.array(d.budget[:]), time=d.time, steps=d.steps, nonfinite=bool(d.nonfinite),
                    satadj_failures=d.satadj_failures, tc_timeouts=d.tc_timeouts,
                    cold_saturated=d.cold_saturated, status=st)

    def profiles(self):
        out = np.zeros((self.nlev, 11))
        self._check(self.L.cmles_profiles(self.h, out.ctypes.data_as(_DP)))
        return out

    def spectrum(self, nshell):
        """Kinetic-energy spectrum E[nshell] of the current state (see cmles_spectrum)."""
        out = np.zeros(nshell)
        self._check(self.L.cmles_spectrum(self.h, int(nshell), out.ctypes.data_as(_DP)))
        return out

    def set_closure_weights(self, flat):
        flat = np.ascontiguousarray(flat, np.float32)
        self._check(self.L.cmles_set_closure_weights(self.h, flat.ctypes.data_as(C.POINTER(C.c_float)),
                                                     flat.size))

    def set_closure_weights_device(self, params):
        assert params.is_cuda and params.dtype == self.torch.float32 and params.numel() == MLP_PARAMS
        self._check(self.L.cmles_set_closure_weights_device(self.h, C.c_void_p(params.data_ptr())))

    def closure_samples(self, factor=4, with_thv=False):
        """(X[n][13], T[n][2]) training samples filtered from the current
        state; with_thv also returns the filtered theta_v [n]."""
        torch = self.torch
        m = self.mesh_d
        n = (m["nex"] // factor) * (m["ney"] // factor) * (m["nez"] // factor) * self.Np
        X = torch.empty((n, 13), dtype=torch.float32, device="cuda")
        T = torch.empty((n, 2), dtype=torch.float32, device="cuda")
        th = torch.empty(n, dtype=torch.float32, device="cuda") if with_thv else None
        cnt = C.c_longlong()
        self._check(self.L.cmles_closure_samples(self.h, factor, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()),
                                                 None if th is None else C.c_void_p(th.data_ptr()), n,
                                                 C.byref(cnt)))
        return (X, T, th) if with_thv else (X, T)

    def enable_timing(self, on=True):
        self._check(self.L.cmles_enable_timing(self.h, int(on)))

    def kernel_times(self):
        cnt = (C.c_longlong * 3)()
        ms = (C.c_double * 3)()
        launches = C.c_longlong()
        self._check(self.L.cmles_kernel_times(self.h, cnt, ms, C.byref(launches)))
        return dict(count=list(cnt), ms=list(ms), launches=launches.value)

    def launch_count(self):
        return self.L.cmles_launch_count(self.h)

    def hevi_operator(self, Q):
        """L (Q - Q_ref) of a HEVI handle (device tensors, FP64 state layout)."""
        out = self.torch.empty_like(Q)
        self._check(self.L.cmles_hevi_operator(self.h, C.c_void_p(Q.data_ptr()), C.c_void_p(out.data_ptr())))
        return out

    def hevi_solve(self, B):
        """Q_ref + (I - dt gamma L)^-1 (B - Q_ref) of a HEVI handle."""
        Y = self.torch.empty_like(B)
        self._check(self.L.cmles_hevi_solve(self.h, C.c_void_p(B.data_ptr()), C.c_void_p(Y.data_ptr())))
        return Y

    def test_stall_tc(self, mode):
        """Test hook of the learned-closure kernels' bounded tensor-core waits
        (see cmles_test_stall_tc): 0 off, 1 (or True) an extra wait on a
        barrier nothing arrives on, 2 the first MMA completion wait of each CTA
        gives up at once."""
        self._check(self.L.cmles_test_stall_tc(self.h, int(mode)))

    def device_bytes(self):
        return self.L.cmles_device_bytes(self.h)


def halo_plan(mesh, px, py, rank):
    """The halo plan of partition `rank` of a px x py split (host-only, see
    cmles_halo_plan): (neighbour[4], count[4], send[4], recv[4]) with send[s]
    and recv[s] arrays of storage node indices."""
    L = load()
    m = make_mesh(mesh)
    nb = (C.c_int * 4)()
    cnt = (C.c_longlong * 4)()
    st = L.cmles_halo_plan(C.byref(m), px, py, rank, nb, cnt, None, None)
    if st != 0:
        raise CmlesError(st, "cmles_halo_plan failed")
    tot = sum(cnt)
    send = np.zeros(max(tot, 1), dtype=np.int64)
    recv = np.zeros(max(tot, 1), dtype=np.int64)
    st = L.cmles_halo_plan(C.byref(m), px, py, rank, nb, cnt, send.ctypes.data_as(C.POINTER(C.c_longlong)),
                           recv.ctypes.data_as(C.POINTER(C.c_longlong)))
    if st != 0:
        raise CmlesError(st, "cmles_halo_plan failed")
    off = np.concatenate([[0], np.cumsum(list(cnt))])
    return (list(nb), list(cnt), [send[off[k]:off[k + 1]] for k in range(4)],
            [recv[off[k]:off[k + 1]] for k in range(4)])


class Group:
    """One mesh split into px x py (x, y) partitions that exchange face halos
    every stage (cmles_group, the single-GPU form of the decomposition)."""

    def __init__(self, mesh, physics, px, py, precision="fp64"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("cmles needs a CUDA device; no CPU fallback exists")
        self.torch = torch
        self.L = load()
        self._mesh = make_mesh(mesh)
        self._params = make_params(physics, precision)
        g = _VP()
        st = self.L.cmles_group_create(C.byref(self._mesh), C.byref(self._params), px, py, C.byref(g))
        if st != 0:
            raise CmlesError(st, "cmles_group_create failed")
        self.g = g
        self.N = mesh["N"]
        self.Np = (self.N + 1) ** 3
        self.E = mesh["nex"] * mesh["ney"] * mesh["nez"]
        self._check(self.L.cmles_group_set_stream(self.g, C.c_void_p(torch.cuda.current_stream().cuda_stream)))

    def _check(self, st):
        if st != 0:
            raise CmlesError(st, self.L.cmles_group_last_error_message(self.g).decode())

    def close(self):
        if getattr(self, "g", None):
            self.L.cmles_group_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_reference(self, rho_r, p_r, qt_r=None):
        rho_r = np.ascontiguousarray(rho_r, np.float64)
        p_r = np.ascontiguousarray(p_r, np.float64)
        q = None if qt_r is None else np.ascontiguousarray(qt_r, np.float64)
        self._check(self.L.cmles_group_set_reference(self.g, rho_r.ctypes.data_as(_DP), p_r.ctypes.data_as(_DP),
                                                     None if q is None else q.ctypes.data_as(_DP), rho_r.size))

    def set_closure_weights(self, flat):
        flat = np.ascontiguousarray(flat, np.float32)
        self._check(self.L.cmles_group_set_closure_weights(self.g, flat.ctypes.data_as(C.POINTER(C.c_float)),
                                                           flat.size))

    def _dev(self, t):
        assert t.is_cuda and t.dtype == self.torch.float64 and t.is_contiguous()
        assert t.numel() == self.E * 6 * self.Np
        return C.c_void_p(t.data_ptr())

    def set_state(self, Q):
        self._check(self.L.cmles_group_set_state(self.g, self._dev(Q)))

    def get_state(self):
        Q = self.torch.empty((self.E, 6, self.Np), dtype=self.torch.float64, device="cuda")
        self._check(self.L.cmles_group_get_state(self.g, self._dev(Q)))
        return Q

    def tendency(self, Q, out=None):
        if out is None:
            out = self.torch.empty_like(Q)
        self._check(self.L.cmles_group_tendency(self.g, self._dev(Q), self._dev(out)))
        return out

    def step(self, n=1):
        self._check(self.L.cmles_group_step(self.g, int(n)))

    def diagnostics(self, raise_on_error=True):
        d = Diag()
        st = self.L.cmles_group_diagnostics(self.g, C.byref(d))
        if raise_on_error and st != 0:
            self._check(st)
        return dict(budget=np.array(d.budget[:]), time=d.time, steps=d.steps, nonfinite=bool(d.nonfinite),
                    satadj_failures=d.satadj_failures, tc_timeouts=d.tc_timeouts,
                    cold_saturated=d.cold_saturated, status=st)

    def halo_bytes(self):
        return self.L.cmles_group_halo_bytes(self.g)
