"""ctypes front end of the FP64 CPU oracle (oracle/liboracle.so).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow correctness reference
for the CUDA path of the DG large-eddy-simulation right-hand side (Sridhar et
al., ClimateMachine LES).  Only tests/, the smoke check and the benchmark's
CPU-baseline leg may import this module.  It shares no code with the product
package; the default constants below are the oracle's own copy of the paper's
Table t:constants plus the readings for g, p0, p_tr and T_tr.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
        _declare(_lib)
    return _lib


class Mesh(C.Structure):
    _fields_ = [("N", C.c_int), ("nex", C.c_int), ("ney", C.c_int), ("nez", C.c_int),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("Lx", C.c_double), ("Ly", C.c_double), ("Lz", C.c_double),
                ("periodic_x", C.c_int), ("periodic_y", C.c_int), ("periodic_z", C.c_int),
                ("warp", C.c_int), ("hill_h", C.c_double), ("hill_a", C.c_double), ("hill_xc", C.c_double)]


class Params(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("g", "p0", "Rd", "Rv", "cvd", "cvv", "cvl", "cvi", "T0", "Lv0",
                                          "Lf0", "ptr", "Ttr")] + [
        ("closure", C.c_int), ("Cs", C.c_double), ("Prt", C.c_double), ("richardson", C.c_int),
        ("moist", C.c_int), ("sponge_alpha", C.c_double), ("sponge_zs", C.c_double),
        ("sponge_gamma", C.c_double), ("u_relax", C.c_double * 3), ("lateral_sponge_frac", C.c_double),
        ("surface_flux", C.c_int), ("shf", C.c_double), ("lhf", C.c_double), ("Omega", C.c_double * 3),
        ("flux", C.c_int), ("drag_cd", C.c_double), ("noslip", C.c_int)]


class Case(C.Structure):
    _fields_ = [("id", C.c_int), ("seed", C.c_uint64), ("theta0", C.c_double),
                ("dtheta", C.c_double), ("r0", C.c_double), ("xc", C.c_double), ("yc", C.c_double),
                ("zc", C.c_double), ("noise_theta", C.c_double), ("noise_qt", C.c_double),
                ("noise_zmax", C.c_double), ("NBV", C.c_double), ("u0", C.c_double * 3),
                ("qt_sfc", C.c_double), ("qt_ml", C.c_double), ("z_ml", C.c_double), ("qt_top", C.c_double),
                ("dthdz_above", C.c_double), ("vortex_beta", C.c_double), ("vortex_R", C.c_double),
                ("vortex_U", C.c_double), ("vortex_T", C.c_double), ("vortex_rho", C.c_double),
                ("moist", C.c_int), ("nmodes", C.c_int), ("modes", C.POINTER(C.c_double)),
                ("qt_H", C.c_double)]


class ThermoState(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("rho", "u0", "u1", "u2", "qt", "etot", "I", "T", "ql", "qv", "Rm", "cvm",
                                          "cpm", "p", "c", "htot", "theta", "thetav")] + [("newton", C.c_int)]


CLOSURE = {"none": 0, "sl": 1, "mlp": 2, "vreman": 3}
FLUX = {"rusanov": 0, "hllc": 1, "roe": 2}

# Table t:constants; g, p0, p_tr, T_tr are readings (the table omits them).
CONSTANTS = dict(g=9.81, p0=1.0e5, Rd=287.0, Rv=462.0, cvd=717.5, cvv=1397.5, cvl=4181.0, cvi=2100.0,
                 T0=273.16, Lv0=2.5008e6, Lf0=0.3336e6, ptr=611.657, Ttr=273.16)

_DP = C.POINTER(C.c_double)


def _declare(L):
    L.orc_lgl.argtypes = [C.c_int, _DP, _DP, _DP]
    L.orc_pvsat.argtypes = [C.POINTER(Params), C.c_double]
    L.orc_pvsat.restype = C.c_double
    L.orc_qsat.argtypes = [C.POINTER(Params), C.c_double, C.c_double]
    L.orc_qsat.restype = C.c_double
    L.orc_internal_energy.argtypes = [C.POINTER(Params), C.c_double, C.c_double, C.c_double]
    L.orc_internal_energy.restype = C.c_double
    L.orc_saturation_adjustment.argtypes = [C.POINTER(Params), C.c_double, C.c_double, C.c_double, _DP, _DP]
    L.orc_saturation_adjustment.restype = C.c_int
    L.orc_flux1_normal.argtypes = [C.POINTER(Params), _DP, C.c_double, C.c_double, _DP, _DP]
    L.orc_rusanov.argtypes = [C.POINTER(Params), _DP, _DP, C.c_double, C.c_double, _DP, _DP]
    L.orc_smagorinsky.argtypes = [C.POINTER(Params), _DP, C.c_double, C.c_double, C.c_double]
    L.orc_smagorinsky.restype = C.c_double
    L.orc_filter_matrix.argtypes = [C.c_int, _DP, C.c_int, C.c_double, _DP]
    L.orc_filter_matrix.restype = None
    L.orc_filter.argtypes = [C.c_void_p, _DP, C.c_int, C.c_double, C.c_int]
    L.orc_filter.restype = None
    L.orc_roe.argtypes = [C.POINTER(Params), _DP, _DP, C.c_double, C.c_double, _DP, _DP]
    L.orc_roe.restype = None
    L.orc_hllc.argtypes = [C.POINTER(Params), _DP, _DP, C.c_double, C.c_double, _DP, _DP]
    L.orc_hllc.restype = None
    L.orc_vreman.argtypes = [C.POINTER(Params), _DP, C.c_double, C.c_double, _DP]
    L.orc_vreman.restype = C.c_double
    L.orc_create.argtypes = [C.POINTER(Mesh), C.POINTER(Params)]
    L.orc_create.restype = C.c_void_p
    L.orc_destroy.argtypes = [C.c_void_p]
    L.orc_num_nodes.argtypes = [C.c_void_p]
    L.orc_num_nodes.restype = C.c_int64
    L.orc_num_elements.argtypes = [C.c_void_p]
    L.orc_geometry.argtypes = [C.c_void_p, _DP, _DP, _DP, _DP, _DP]
    L.orc_set_reference.argtypes = [C.c_void_p, _DP, _DP]
    L.orc_set_mlp.argtypes = [C.c_void_p] + [_DP] * 8
    L.orc_rhs.argtypes = [C.c_void_p, _DP, _DP, C.c_int]
    L.orc_rhs.restype = C.c_int
    L.orc_intermediates.argtypes = [C.c_void_p, _DP, _DP, _DP, _DP, _DP]
    L.orc_lsrk54.argtypes = [C.c_void_p, _DP, C.c_int, C.c_double]
    L.orc_lsrk54.restype = C.c_int
    L.orc_lsrk54_coefficients.argtypes = [_DP, _DP, _DP]
    L.orc_lsrk144.argtypes = [C.c_void_p, _DP, C.c_int, C.c_double]
    L.orc_lsrk144.restype = C.c_int
    L.orc_lsrk144_coefficients.argtypes = [_DP, _DP, _DP]
    L.orc_vlin_reference.argtypes = [C.c_void_p, _DP]
    L.orc_set_reference_qt.argtypes = [C.c_void_p, _DP]
    L.orc_vlin_apply.argtypes = [C.c_void_p, _DP, _DP]
    L.orc_budgets.argtypes = [C.c_void_p, _DP, _DP]
    L.orc_budgets.restype = C.c_int
    L.orc_favre_profiles.argtypes = [C.c_void_p, _DP, _DP]
    L.orc_uniform.argtypes = [C.c_uint64, C.c_uint64]
    L.orc_uniform.restype = C.c_double
    L.orc_init_case.argtypes = [C.c_void_p, C.POINTER(Case), _DP, _DP, _DP]
    L.orc_vortex_exact.argtypes = [C.c_void_p, C.POINTER(Case), C.c_double, _DP]
    L.orc_mlp_forward.argtypes = [C.c_int, _DP] + [_DP] * 6 + [_DP]
    L.orc_mlp_forward_bf16.argtypes = [C.c_int, _DP] + [_DP] * 6 + [_DP]
    L.orc_bf16.argtypes = [C.c_double]
    L.orc_bf16.restype = C.c_double
    L.orc_mlp_loss_grad.argtypes = [C.c_int, _DP, _DP] + [_DP] * 6 + [_DP] * 6
    L.orc_mlp_loss_grad.restype = C.c_double
    L.orc_thermo.argtypes = [C.POINTER(Params), _DP, C.c_double, C.POINTER(ThermoState)]
    L.orc_thermo.restype = C.c_int
    L.orc_closure_primitives.argtypes = [C.c_void_p, _DP, _DP]
    L.orc_closure_primitives.restype = None
    L.orc_closure_samples.argtypes = [C.c_void_p, _DP, C.c_int, _DP, _DP, _DP]
    L.orc_closure_samples.restype = C.c_longlong
    L.orc_adam.argtypes = [C.c_int, _DP, _DP, _DP, _DP, C.c_int, C.c_double, C.c_double, C.c_double,
                           C.c_double]


def _p(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def make_params(closure="sl", moist=False, Cs=0.21, Prt=1.0 / 3.0, richardson=True, sponge_alpha=0.0,
                sponge_zs=0.0, sponge_gamma=2.0, u_relax=(0.0, 0.0, 0.0), lateral_sponge_frac=0.0,
                surface_flux=False, shf=0.0, lhf=0.0, Omega=(0.0, 0.0, 0.0), flux="rusanov", drag_cd=0.0,
                noslip=0, **const):
    c = dict(CONSTANTS)
    c.update(const)
    P = Params(**c)
    P.closure = CLOSURE[closure]
    P.Cs, P.Prt, P.richardson, P.moist = Cs, Prt, int(richardson), int(moist)
    P.sponge_alpha, P.sponge_zs, P.sponge_gamma = sponge_alpha, sponge_zs, sponge_gamma
    P.u_relax = (C.c_double * 3)(*u_relax)
    P.lateral_sponge_frac = lateral_sponge_frac
    P.surface_flux, P.shf, P.lhf = int(surface_flux), shf, lhf
    P.Omega = (C.c_double * 3)(*Omega)
    P.flux = FLUX[flux]
    P.drag_cd = drag_cd
    P.noslip = int(noslip)
    return P


def make_mesh(N, nex, ney, nez, Lx, Ly, Lz, x0=0.0, y0=0.0, z0=0.0, periodic=(1, 1, 0), warp=False,
              hill_h=0.0, hill_a=1.0, hill_xc=0.0):
    return Mesh(N=N, nex=nex, ney=ney, nez=nez, x0=x0, y0=y0, z0=z0, Lx=Lx, Ly=Ly, Lz=Lz,
                periodic_x=periodic[0], periodic_y=periodic[1], periodic_z=periodic[2], warp=int(warp),
                hill_h=hill_h, hill_a=hill_a, hill_xc=hill_xc)


def make_case(id, seed=0, modes=None, **kw):
    cs = Case()
    cs.id, cs.seed = id, seed
    for k, v in kw.items():
        if k == "u0":
            cs.u0 = (C.c_double * 3)(*v)
        else:
            setattr(cs, k, v)
    if modes is not None:
        m = np.ascontiguousarray(modes, dtype=np.float64)
        cs.nmodes = m.shape[0]
        cs._modes_keepalive = m
        cs.modes = _p(m)
    return cs


# ---------------------------------------------------------------- pointwise

def lgl(N):
    xi = np.zeros(N + 1)
    w = np.zeros(N + 1)
    D = np.zeros((N + 1) * (N + 1))
    lib().orc_lgl(N, _p(xi), _p(w), _p(D))
    return xi, w, D.reshape(N + 1, N + 1)


def pvsat(P, T):
    return lib().orc_pvsat(C.byref(P), T)


def qsat(P, T, rho):
    return lib().orc_qsat(C.byref(P), T, rho)


def internal_energy(P, T, qt, ql):
    return lib().orc_internal_energy(C.byref(P), T, qt, ql)


def saturation_adjustment(P, rho, qt, I):
    T = C.c_double()
    ql = C.c_double()
    it = lib().orc_saturation_adjustment(C.byref(P), rho, qt, I, C.byref(T), C.byref(ql))
    return T.value, ql.value, it


def flux1_normal(P, Y, z, pr, n):
    out = np.zeros(6)
    lib().orc_flux1_normal(C.byref(P), _p(np.ascontiguousarray(Y, float)), z, pr,
                           _p(np.ascontiguousarray(n, float)), _p(out))
    return out


def rusanov(P, Ym, Yp, z, pr, n):
    out = np.zeros(6)
    lib().orc_rusanov(C.byref(P), _p(np.ascontiguousarray(Ym, float)), _p(np.ascontiguousarray(Yp, float)),
                      z, pr, _p(np.ascontiguousarray(n, float)), _p(out))
    return out


def filter_matrix(N, order, alpha):
    xi, _, _ = lgl(N)
    F = np.zeros((N + 1) * (N + 1))
    lib().orc_filter_matrix(N, _p(np.ascontiguousarray(xi, float)), order, alpha, _p(F))
    return F.reshape(N + 1, N + 1)


def roe(P, Ym, Yp, z, pr, n):
    out = np.zeros(6)
    lib().orc_roe(C.byref(P), _p(np.ascontiguousarray(Ym, float)), _p(np.ascontiguousarray(Yp, float)),
                  z, pr, _p(np.ascontiguousarray(n, float)), _p(out))
    return out


def hllc(P, Ym, Yp, z, pr, n):
    out = np.zeros(6)
    lib().orc_hllc(C.byref(P), _p(np.ascontiguousarray(Ym, float)), _p(np.ascontiguousarray(Yp, float)),
                   z, pr, _p(np.ascontiguousarray(n, float)), _p(out))
    return out


def smagorinsky(P, gu, dthvdz, thv, Delta):
    return lib().orc_smagorinsky(C.byref(P), _p(np.ascontiguousarray(gu, float).ravel()), dthvdz, thv, Delta)


def vreman(P, gu, dthvdz, thv, Dm):
    return lib().orc_vreman(C.byref(P), _p(np.ascontiguousarray(gu, float).ravel()), dthvdz, thv,
                            _p(np.ascontiguousarray(Dm, float).ravel()))


def thermo(P, Y, z):
    """The pointwise thermodynamic state of conserved variables Y at height z
    (Sec. 2): a dict of rho, u, q_t, e_tot, I, T, q_l, q_v, R_m, c_vm, c_pm,
    p, c, h_tot, theta, theta_v and the Newton iteration count."""
    st = ThermoState()
    lib().orc_thermo(C.byref(P), _p(np.ascontiguousarray(Y, float)), z, C.byref(st))
    d = {n: getattr(st, n) for n, _ in ThermoState._fields_}
    d["u"] = np.array([d.pop("u0"), d.pop("u1"), d.pop("u2")])
    return d


def uniform(seed, counter):
    return lib().orc_uniform(seed, counter)


def lsrk54_coefficients():
    A, B, c = np.zeros(5), np.zeros(5), np.zeros(5)
    lib().orc_lsrk54_coefficients(_p(A), _p(B), _p(c))
    return A, B, c


def ark2_tableaux():
    """ARK2 of Giraldo, Kelly & Constantinescu (2013), the 2nd-order additive
    Runge-Kutta IMEX method Sec. 3.2 cites: explicit tableau Ae, implicit
    (singly diagonally implicit, stiffly accurate) tableau Ai, shared
    weights b; gamma = 1 - 1/sqrt 2, delta = 1/(2 sqrt 2),
    alpha = (3 + 2 sqrt 2)/6."""
    g = 1.0 - 1.0 / np.sqrt(2.0)
    d = 1.0 / (2.0 * np.sqrt(2.0))
    a = (3.0 + 2.0 * np.sqrt(2.0)) / 6.0
    Ae = np.array([[0.0, 0.0, 0.0], [2.0 * g, 0.0, 0.0], [1.0 - a, a, 0.0]])
    Ai = np.array([[0.0, 0.0, 0.0], [g, g, 0.0], [d, d, g]])
    b = np.array([d, d, g])
    return Ae, Ai, b


def lsrk144_coefficients():
    A, B, c = np.zeros(14), np.zeros(14), np.zeros(14)
    lib().orc_lsrk144_coefficients(_p(A), _p(B), _p(c))
    return A, B, c


def mlp_forward(X, W):
    X = np.ascontiguousarray(X, float)
    Y = np.zeros((X.shape[0], 2))
    lib().orc_mlp_forward(X.shape[0], _p(X), *[_p(np.ascontiguousarray(W[k], float))
                                                for k in ("W1", "b1", "W2", "b2", "W3", "b3")], _p(Y))
    return Y


def mlp_forward_bf16(X, W):
    X = np.ascontiguousarray(X, float)
    Y = np.zeros((X.shape[0], 2))
    lib().orc_mlp_forward_bf16(X.shape[0], _p(X), *[_p(np.ascontiguousarray(W[k], float))
                                                     for k in ("W1", "b1", "W2", "b2", "W3", "b3")], _p(Y))
    return Y


def bf16(x):
    return lib().orc_bf16(x)


def mlp_loss_grad(X, T, W):
    X = np.ascontiguousarray(X, float)
    T = np.ascontiguousarray(T, float)
    g = {k: np.zeros_like(np.asarray(W[k], float)) for k in ("W1", "b1", "W2", "b2", "W3", "b3")}
    loss = lib().orc_mlp_loss_grad(X.shape[0], _p(X), _p(T),
                                   *[_p(np.ascontiguousarray(W[k], float)) for k in ("W1", "b1", "W2", "b2", "W3", "b3")],
                                   *[_p(g[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])
    return loss, g


def adam(theta, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    lib().orc_adam(theta.size, _p(theta), _p(np.ascontiguousarray(g, float)), _p(m), _p(v), t, lr, beta1,
                   beta2, eps)


# ---------------------------------------------------------------- solver

class Solver:
    """FP64 DG solver on a structured hexahedral mesh (oracle)."""

    def __init__(self, mesh, params):
        self.mesh, self.params = mesh, params
        self.h = lib().orc_create(C.byref(mesh), C.byref(params))
        self.N = mesh.N
        self.Np = (mesh.N + 1) ** 3
        self.E = mesh.nex * mesh.ney * mesh.nez
        self._mlp_keep = None

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def geometry(self):
        shape = (self.E, self.Np)
        x, y, z, J, wJ = (np.zeros(shape) for _ in range(5))
        lib().orc_geometry(self.h, _p(x), _p(y), _p(z), _p(J), _p(wJ))
        return dict(x=x, y=y, z=z, J=J, wJ=wJ)

    def filter(self, Q, order, alpha, mask):
        """exponential filter (Eq. exponential_filter) applied to a copy of Q"""
        Q = np.ascontiguousarray(Q, float).copy()
        lib().orc_filter(self.h, _p(Q), order, alpha, mask)
        return Q

    def set_reference(self, rho_r, p_r):
        lib().orc_set_reference(self.h, _p(np.ascontiguousarray(rho_r, float)),
                                _p(np.ascontiguousarray(p_r, float)))

    def init_case(self, case):
        Q = np.zeros((self.E, 6, self.Np))
        rho_r = np.zeros((self.E, self.Np))
        p_r = np.zeros((self.E, self.Np))
        lib().orc_init_case(self.h, C.byref(case), _p(Q), _p(rho_r), _p(p_r))
        return Q, rho_r, p_r

    def vortex_exact(self, case, t):
        Q = np.zeros((self.E, 6, self.Np))
        lib().orc_vortex_exact(self.h, C.byref(case), t, _p(Q))
        return Q

    def set_mlp(self, W, in_scale, out_scale):
        keep = [np.ascontiguousarray(W[k], float) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]
        keep += [np.ascontiguousarray(in_scale, float), np.ascontiguousarray(out_scale, float)]
        self._mlp_keep = keep
        lib().orc_set_mlp(self.h, *[_p(a) for a in keep])

    def rhs(self, Q, form=0):
        Q = np.ascontiguousarray(Q, float)
        R = np.zeros_like(Q)
        fails = lib().orc_rhs(self.h, _p(Q), _p(R), form)
        return R, fails

    def intermediates(self):
        G = np.zeros((self.E, 6, self.Np))
        gG = np.zeros((self.E, 18, self.Np))
        nut = np.zeros((self.E, self.Np))
        F2 = np.zeros((self.E, 15, self.Np))
        aux = np.zeros((self.E, 4, self.Np))
        lib().orc_intermediates(self.h, _p(G), _p(gG), _p(nut), _p(F2), _p(aux))
        return dict(G=G, gradG=gG.reshape(self.E, 6, 3, self.Np), nut=nut,
                    F2=F2.reshape(self.E, 3, 5, self.Np), aux=aux)

    def lsrk54(self, Q, nsteps, dt):
        Q = np.ascontiguousarray(Q, float).copy()
        fails = lib().orc_lsrk54(self.h, _p(Q), nsteps, dt)
        return Q, fails

    # ------------------------------------------------------------ HEVI (Sec. 3.2)

    def set_reference_qt(self, qt_r):
        """Reference total water [E][Np] of the HEVI linearisation (default 0)."""
        lib().orc_set_reference_qt(self.h, _p(np.ascontiguousarray(qt_r, float)))

    def vlin_reference(self):
        """The state the vertical linear operator is linearised about."""
        Qr = np.zeros((self.E, 6, self.Np))
        lib().orc_vlin_reference(self.h, _p(Qr))
        return Qr

    def vlin(self, Q):
        """L (Q - Q_ref): the vertical acoustic-gravity operator (hevi.c)."""
        out = np.zeros((self.E, 6, self.Np))
        lib().orc_vlin_apply(self.h, _p(np.ascontiguousarray(Q, float)), _p(out))
        return out

    _HEVI_COMP = (0, 1, 2, 3, 4, 5)

    def _line_nodes(self, ex, ey, i, j):
        """(element, node) of the vertical line (ex, ey, i, j), bottom to top."""
        m, Nq = self.mesh, self.N + 1
        return [(ex + m.nex * (ey + m.ney * ez), i + Nq * (j + Nq * k)) for ez in range(m.nez) for k in range(Nq)]

    def hevi_line_matrix(self, ex=0, ey=0, i=0, j=0):
        """L on one vertical line, assembled column by column by applying the
        operator to unit deviations; unknowns ordered (level node, component)."""
        Qr = self.vlin_reference()
        nodes = self._line_nodes(ex, ey, i, j)
        nc = len(self._HEVI_COMP)
        nl = nc * len(nodes)
        Lm = np.zeros((nl, nl))
        for col in range(nl):
            e, n = nodes[col // nc]
            Q = Qr.copy()
            Q[e, self._HEVI_COMP[col % nc], n] += 1.0
            out = self.vlin(Q)
            for row, (er, nr) in enumerate(nodes):
                for c in range(nc):
                    Lm[nc * row + c, col] = out[er, self._HEVI_COMP[c], nr]
        return Lm

    def _hevi_solve(self, M, B, Qr):
        """Y with (I - dt gamma L)(Y - Q_ref) = B - Q_ref on every vertical
        line, all six components."""
        m, Nq = self.mesh, self.N + 1
        Y = B.copy()
        lines = [(ex, ey, i, j) for ex in range(m.nex) for ey in range(m.ney) for i in range(Nq) for j in range(Nq)]
        idx = [self._line_nodes(*ln) for ln in lines]
        nc = len(self._HEVI_COMP)
        R = np.zeros((M.shape[0], len(lines)))
        for L_, nodes in enumerate(idx):
            for r, (e, n) in enumerate(nodes):
                for c, v in enumerate(self._HEVI_COMP):
                    R[nc * r + c, L_] = B[e, v, n] - Qr[e, v, n]
        X = np.linalg.solve(M, R)
        for L_, nodes in enumerate(idx):
            for r, (e, n) in enumerate(nodes):
                for c, v in enumerate(self._HEVI_COMP):
                    Y[e, v, n] = Qr[e, v, n] + X[nc * r + c, L_]
        return Y

    def ark2_hevi(self, Q, nsteps, dt):
        """nsteps steps of ARK2 with the vertical linear operator implicit and
        the rest of the right-hand side explicit: stage s solves
        Y_s - dt Ai[s,s] L(Y_s) = Q + dt sum_{j<s} (Ae[s,j] E_j + Ai[s,j] I_j),
        E_j = f(Y_j) - L(Y_j), I_j = L(Y_j); Q <- Q + dt sum_j b_j f(Y_j)."""
        Ae, Ai, b = ark2_tableaux()
        Qr = self.vlin_reference()
        M = np.eye(len(self._HEVI_COMP) * self.mesh.nez * (self.N + 1)) - dt * Ai[1, 1] * self.hevi_line_matrix()
        Q = np.ascontiguousarray(Q, float).copy()
        fails = 0
        for _ in range(nsteps):
            E, Im, R = [], [], []
            for s_ in range(3):
                if s_ == 0:
                    Y = Q
                else:
                    B = Q + dt * sum(Ae[s_, j] * E[j] + Ai[s_, j] * Im[j] for j in range(s_))
                    Y = self._hevi_solve(M, B, Qr)
                f, fl = self.rhs(Y)
                fails += fl
                Lq = self.vlin(Y)
                R.append(f)
                E.append(f - Lq)
                Im.append(Lq)
            Q = Q + dt * sum(b[j] * R[j] for j in range(3))
        return Q, fails

    def lsrk144(self, Q, nsteps, dt):
        Q = np.ascontiguousarray(Q, float).copy()
        fails = lib().orc_lsrk144(self.h, _p(Q), nsteps, dt)
        return Q, fails

    def budgets(self, Q):
        out = np.zeros(6)
        bad = lib().orc_budgets(self.h, _p(np.ascontiguousarray(Q, float)), _p(out))
        return out, bool(bad)

    def closure_primitives(self, Q):
        """u, v, w, theta_v at every node, [E][4][Np] (closure.c step 1)."""
        prim = np.zeros((self.E, 4, self.Np))
        lib().orc_closure_primitives(self.h, _p(np.ascontiguousarray(Q, float)), _p(prim))
        return prim

    def closure_samples_from_primitives(self, prim, factor=4):
        """(X[n][13], T[n][2], thv_bar[n]) of the top-hat filter onto the mesh
        coarser by `factor` (closure.c steps 2-5)."""
        m = self.mesh
        n = (m.nex // factor) * (m.ney // factor) * (m.nez // factor) * self.Np
        X, T, th = np.zeros((n, 13)), np.zeros((n, 2)), np.zeros(n)
        got = lib().orc_closure_samples(self.h, _p(np.ascontiguousarray(prim, float)), factor, _p(X), _p(T), _p(th))
        if got != n:
            raise ValueError("element counts must be multiples of factor on a flat mesh")
        return X, T, th

    def closure_samples(self, Q, factor=4):
        """Training samples of the learned closure from the state Q."""
        return self.closure_samples_from_primitives(self.closure_primitives(Q), factor)

    def favre_profiles(self, Q):
        nl = self.mesh.nez * (self.N + 1)
        out = np.zeros((nl, 11))
        lib().orc_favre_profiles(self.h, _p(np.ascontiguousarray(Q, float)), _p(out))
        return out


def from_inputs(mesh, physics, case=None):
    """Oracle solver, initial state and reference for plain-dict workload
    descriptions (the seeded input module's format)."""
    mk = {k: v for k, v in mesh.items()}
    M = make_mesh(mk.pop("N"), mk.pop("nex"), mk.pop("ney"), mk.pop("nez"), mk.pop("Lx"), mk.pop("Ly"),
                  mk.pop("Lz"), **mk)
    pk = {k: v for k, v in physics.items() if k != "dt"}
    P = make_params(**pk)
    S = Solver(M, P)
    if case is None:
        return S
    ck = dict(case)
    cid = ck.pop("id")
    seed = ck.pop("seed", 0)
    modes = ck.pop("modes", None)
    cs = make_case(cid, seed=seed, modes=modes, **ck)
    Q, rho_r, p_r = S.init_case(cs)
    return S, Q, rho_r, p_r, cs
