"""Pins of the oracle's learned-closure training samples (oracle/closure.c)
and of the thermodynamic fields they start from, against closed forms and
brute force that share no code with the oracle.

The paper has no learned closure; the samples follow the readings stated in
closure.c: a top-hat filter of width H/N (the coarse node spacing) centred on
every coarse node, fine nodes weighted by their LGL quadrature weights, the
subgrid stress tau_ij = <u_i u_j> - <u_i><u_j> and theta_v flux, and the
least-squares targets nu* = max(0, -tau:S/(2 S:S)), kappa* =
max(0, -tau_th.g/|g|^2).

For a field linear in x the filtered gradient is the gradient itself and,
because the box is a product of one-dimensional node sets with product
weights, the covariance of the node coordinates is diagonal:
tau_ij = sum_k A_ik A_jk V_k, with V_k the weighted variance of the in-box
node coordinates along axis k, counted here by brute force in one dimension
from numpy's own Gauss-Lobatto nodes.  A transposed index, a wrong weight or
a dropped term in the moments changes these numbers.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npl

CONST = dict(g=9.81, p0=1.0e5, Rd=287.0, Rv=462.0, cvd=717.5, cvv=1397.5, cvl=4181.0, T0=273.16)


def _state(rho, u, T, qt, z, P):
    """Conserved variables of an unsaturated state (q_l = 0) from its
    temperature, written from Sec. 2's internal energy
    I = c_vm (T - T0) + q_t (L_v0 - R_v T0) with c_vm = (1-q_t) c_vd + q_t c_vv."""
    c = CONST
    Iv0 = P.Lv0 - c["Rv"] * c["T0"]
    cvm = (1 - qt) * c["cvd"] + qt * c["cvv"]
    I = cvm * (T - c["T0"]) + qt * Iv0
    e = I + 0.5 * float(np.dot(u, u)) + c["g"] * z
    return np.array([rho, rho * u[0], rho * u[1], rho * u[2], rho * e, rho * qt])


# ---------------------------------------------------------------- thermodynamics

@pytest.mark.parametrize("T", [250.0, 288.15, 300.0, 320.0])
def test_sound_speed_of_dry_air(orc, T):
    """Dry air: c = sqrt(gamma R_d T), gamma = c_pd / c_vd = 1004.5 / 717.5 = 1.4,
    whatever the velocity and height (they leave the internal energy)."""
    P = orc.make_params()
    Y = _state(1.1, np.array([7.0, -3.0, 2.0]), T, 0.0, 850.0, P)
    s = orc.thermo(P, Y, 850.0)
    assert abs(s["T"] - T) < 1e-9
    assert abs(s["c"] - math.sqrt(1.4 * 287.0 * T)) < 1e-10 * s["c"]


def test_potential_temperature_dry():
    """theta = T at p = p0, and theta = T (p0/p)^(R_d/c_pd) = T 2^(2/7) at p = p0/2
    (R_d / c_pd = 287 / 1004.5 = 2/7 exactly)."""
    from oracle import oracle as O
    P = O.make_params()
    T = 291.0
    for p, factor in ((1.0e5, 1.0), (0.5e5, 2.0 ** (2.0 / 7.0))):
        rho = p / (287.0 * T)
        s = O.thermo(P, _state(rho, np.zeros(3), T, 0.0, 0.0, P), 0.0)
        assert abs(s["p"] - p) < 1e-9 * p
        assert abs(s["theta"] - T * factor) < 1e-10 * T
        assert abs(s["thetav"] - s["theta"]) < 1e-12 * T


def test_virtual_potential_temperature_moist_unsaturated(orc):
    """Unsaturated moist air (q_l = 0): theta_v = theta (1 + (R_v/R_d - 1) q_v)
    with the dry Exner function, theta = T (p0/p)^(2/7), p = rho R_m T and
    R_m = (1 - q_t) R_d + q_t R_v."""
    P = orc.make_params(moist=True)
    T, qt, rho = 295.0, 0.008, 1.05
    s = orc.thermo(P, _state(rho, np.array([1.0, 2.0, 0.5]), T, qt, 300.0, P), 300.0)
    assert s["ql"] == 0.0 and abs(s["T"] - T) < 1e-9
    Rm = (1 - qt) * 287.0 + qt * 462.0
    p = rho * Rm * T
    theta = T * (1.0e5 / p) ** (2.0 / 7.0)
    assert abs(s["theta"] - theta) < 1e-10 * theta
    assert abs(s["thetav"] - theta * (1.0 + (462.0 / 287.0 - 1.0) * qt)) < 1e-10 * theta


def test_virtual_potential_temperature_saturated(orc):
    """Saturated air: theta_v = theta (1 + (R_v/R_d - 1) q_v - q_l), the
    density-temperature form, with the oracle's own q_v and q_l."""
    P = orc.make_params(moist=True)
    rho, qt = 1.15, 0.02
    s = orc.thermo(P, _state(rho, np.zeros(3), 285.0, qt, 100.0, P), 100.0)
    assert s["ql"] > 1e-4
    assert abs(s["qv"] + s["ql"] - qt) < 1e-15
    theta = s["T"] * (1.0e5 / s["p"]) ** (2.0 / 7.0)
    ref = theta * (1.0 + (462.0 / 287.0 - 1.0) * s["qv"] - s["ql"])
    assert abs(s["thetav"] - ref) < 1e-10 * ref


def test_sound_speed_moist_is_the_isentropic_derivative(orc):
    """For frozen composition the square of the sound speed is dp/drho along an
    isentrope, on which T rho^(-R_m/c_vm) is constant (ds = c_vm dT/T -
    R_m drho/rho = 0).  A central difference of the oracle's own pressure
    along that curve agrees with its c^2."""
    P = orc.make_params(moist=True)
    T, qt, rho, z = 296.0, 0.01, 1.1, 0.0
    s = orc.thermo(P, _state(rho, np.zeros(3), T, qt, z, P), z)
    Rm = (1 - qt) * 287.0 + qt * 462.0
    cvm = (1 - qt) * 717.5 + qt * 1397.5
    eps = 1e-5
    ps = []
    for sg in (-1.0, 1.0):
        r = rho * (1 + sg * eps)
        Ti = T * (1 + sg * eps) ** (Rm / cvm)
        ps.append(orc.thermo(P, _state(r, np.zeros(3), Ti, qt, z, P), z)["p"])
    c2 = (ps[1] - ps[0]) / (2 * rho * eps)
    assert abs(c2 - s["c"] ** 2) < 1e-7 * c2


# ---------------------------------------------------------------- filter and targets

def _lgl(N):
    x = np.concatenate(([-1.0], np.sort(npl.Legendre.basis(N).deriv().roots().real), [1.0]))
    w = 2.0 / (N * (N + 1) * npl.Legendre.basis(N)(x) ** 2)
    return x, w


def _box_moments_1d(N, nel, L, factor, periodic, c_el, c_node, powers):
    """Brute force along one axis: weighted moments sum w x^p / sum w over the
    fine nodes (each element's copy) within H/(2N) of the coarse node, with x
    the node coordinate relative to the coarse node (nearest periodic image)."""
    x, w = _lgl(N)
    h = L / nel
    H = factor * h
    xc = (c_el + 0.5 * (x[c_node] + 1.0)) * H
    b = 0.5 * H / N
    num = np.zeros(len(powers))
    W = 0.0
    for f in range(nel):
        for a in range(N + 1):
            d = (f + 0.5 * (x[a] + 1.0)) * h - xc
            if periodic:
                d -= L * math.floor(d / L + 0.5)
            if abs(d) <= b * (1 + 1e-9):
                W += w[a]
                num += w[a] * np.array([d ** p for p in powers])
    return num / W, xc


def _mesh_and_solver(orc, N, nel, L, periodic):
    M = orc.make_mesh(N, *nel, *L, periodic=periodic)
    return orc.Solver(M, orc.make_params())


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_linear_field_closed_forms(orc, seed):
    """u = a + A x and theta_v = th0 + g.x on an anisotropic box with walls in
    every direction (so the boxes at the boundary are cut off): filtered
    gradient = A and g; tau = A diag(V) A^T; tau_th = A diag(V) g; and the
    targets from those closed forms, at every coarse node."""
    N, factor = 4, 4
    nel, L = (8, 4, 4), (800.0, 300.0, 200.0)
    S = _mesh_and_solver(orc, N, nel, L, (0, 0, 0))
    geo = S.geometry()
    X3 = np.stack([geo["x"], geo["y"], geo["z"]])          # [3][E][Np]
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(3, 3)) * 0.01
    a = rng.normal(size=3)
    g = rng.normal(size=3) * 0.003
    prim = np.zeros((S.E, 4, S.Np))
    for i in range(3):
        prim[:, i] = a[i] + np.einsum("k,ken->en", A[i], X3)
    prim[:, 3] = 300.0 + np.einsum("k,ken->en", g, X3)
    Xs, Ts, thb = S.closure_samples_from_primitives(prim, factor)
    Nq, Np = N + 1, S.Np
    cn = [n // factor for n in nel]
    H = [L[d] / nel[d] * factor for d in range(3)]
    Delta = (H[0] * H[1] * H[2]) ** (1.0 / 3.0) / N
    checked = 0
    for ce in range(cn[0] * cn[1] * cn[2]):
        cidx = (ce % cn[0], (ce // cn[0]) % cn[1], ce // (cn[0] * cn[1]))
        for n in range(Np):
            nidx = (n % Nq, (n // Nq) % Nq, n // (Nq * Nq))
            V, mean = np.zeros(3), np.zeros(3)
            for d in range(3):
                (m1, m2), xc = _box_moments_1d(N, nel[d], L[d], factor, False, cidx[d], nidx[d], (1, 2))
                V[d] = m2 - m1 * m1
                mean[d] = xc + m1
            q = ce * Np + n
            tau = A @ np.diag(V) @ A.T
            tth = A @ (V * g)
            Sm = 0.5 * (A + A.T)
            SS = (Sm * Sm).sum()
            nu = max(0.0, -(tau * Sm).sum() / (2 * SS))
            ka = max(0.0, -(tth @ g) / (g @ g))
            assert np.allclose(Xs[q, :9], A.ravel(), rtol=0, atol=1e-12)
            assert np.allclose(Xs[q, 9:12], g, rtol=0, atol=1e-12)
            assert abs(Xs[q, 12] - Delta) < 1e-12 * Delta
            assert abs(thb[q] - (300.0 + g @ mean)) < 1e-11 * 300.0
            scale_nu = np.abs(tau).max() / math.sqrt(SS)
            assert abs(Ts[q, 0] - nu) <= 1e-9 * scale_nu, (q, Ts[q, 0], nu)
            assert abs(Ts[q, 1] - ka) <= 1e-9 * np.abs(tth).max() / np.linalg.norm(g), (q, Ts[q, 1], ka)
            checked += 1
    assert checked == S.E // factor ** 3 * Np


def test_quadratic_field_moments(orc):
    """u = (x - s)^2 along x only (s a shift), other components zero: the
    filtered gradient <du/dx> = 2 <x - s> (the LGL derivative of a quadratic
    is exact), <u> = <(x - s)^2>, and tau_xx = <(x-s)^4> - <(x-s)^2>^2, each
    from the one-dimensional brute-force moments; theta_v linear in z gives
    kappa* from tau_th = 0 (u and theta_v vary along different axes):
    0 to rounding."""
    N, factor = 4, 4
    nel, L = (8, 4, 4), (800.0, 400.0, 400.0)
    S = _mesh_and_solver(orc, N, nel, L, (0, 0, 0))
    geo = S.geometry()
    s0 = 137.0
    prim = np.zeros((S.E, 4, S.Np))
    prim[:, 0] = (geo["x"] - s0) ** 2 * 1e-4
    prim[:, 3] = 300.0 + 0.003 * geo["z"]
    Xs, Ts, _ = S.closure_samples_from_primitives(prim, factor)
    Nq, Np = N + 1, S.Np
    for ce in range(2):
        for n in range(0, Np, 7):
            i = n % Nq
            (m1, m2, m3, m4), xc = _box_moments_1d(N, nel[0], L[0], factor, False, ce, i, (1, 2, 3, 4))
            c = xc - s0   # x - s0 = c + d, d the node offset
            Ex = c + m1
            Ex2 = c * c + 2 * c * m1 + m2
            Ex4 = c ** 4 + 4 * c ** 3 * m1 + 6 * c * c * m2 + 4 * c * m3 + m4
            q = ce * Np + n
            assert abs(Xs[q, 0] - 2e-4 * Ex) < 1e-12 * max(1.0, abs(2e-4 * Ex))
            tau = 1e-8 * (Ex4 - Ex2 * Ex2)
            # only S_xx is nonzero: nu* = max(0, -tau_xx S_xx / (2 S_xx^2))
            Sxx = 2e-4 * Ex
            nu = max(0.0, -tau * Sxx / (2 * Sxx * Sxx))
            assert abs(Ts[q, 0] - nu) <= 1e-8 * abs(tau / Sxx) + 1e-18, (q, Ts[q, 0], nu)
            assert abs(Ts[q, 1]) < 1e-18


def test_constant_field_has_no_subgrid_stress(orc):
    """A constant field: zero filtered gradients and subgrid moments to
    rounding, and the filtered value equal to the constant."""
    S = _mesh_and_solver(orc, 4, (4, 4, 4), (400.0, 400.0, 400.0), (1, 1, 0))
    prim = np.empty((S.E, 4, S.Np))
    prim[:, 0], prim[:, 1], prim[:, 2], prim[:, 3] = 3.0, -2.0, 0.5, 301.0
    Xs, Ts, thb = S.closure_samples_from_primitives(prim, 4)
    assert np.abs(Xs[:, :12]).max() < 1e-12
    assert np.abs(thb - 301.0).max() < 1e-12


def test_periodic_wrap_is_translation_invariant(orc):
    """On a triply periodic box, a smooth periodic field shifted by one coarse
    element (4 fine elements) along x and along y permutes the samples: the
    boxes that wrap around the domain see the same nodes as the interior ones."""
    N, factor = 4, 4
    nel, L = (12, 8, 8), (1200.0, 800.0, 400.0)
    S = _mesh_and_solver(orc, N, nel, L, (1, 1, 1))
    geo = S.geometry()
    x, y, z = geo["x"], geo["y"], geo["z"]
    k = 2 * np.pi / np.array(L)

    def field(sx, sy):
        xs, ys = x - sx, y - sy
        p = np.empty((S.E, 4, S.Np))
        p[:, 0] = np.sin(k[0] * xs + 0.3) * np.cos(k[1] * ys) + 0.2 * np.sin(2 * k[2] * z)
        p[:, 1] = np.cos(2 * k[0] * xs) * np.sin(k[1] * ys + 1.0)
        p[:, 2] = np.sin(k[0] * xs + k[1] * ys + k[2] * z)
        p[:, 3] = 300.0 + np.cos(k[0] * xs - 2 * k[1] * ys) + 0.5 * np.sin(k[2] * z)
        return p

    X0, T0, t0 = S.closure_samples_from_primitives(field(0.0, 0.0), factor)
    Hx, Hy = L[0] / nel[0] * factor, L[1] / nel[1] * factor
    X1, T1, t1 = S.closure_samples_from_primitives(field(Hx, Hy), factor)
    # the targets are ratios: where the filtered strain or theta_v gradient
    # vanishes by symmetry (to rounding) they are not determined, so they are
    # compared only where the denominator is well above rounding
    gu = X0[:, :9].reshape(-1, 3, 3)
    SS = (0.25 * (gu + gu.transpose(0, 2, 1)) ** 2 * 4).sum(axis=(1, 2))
    gg = (X0[:, 9:12] ** 2).sum(axis=1)
    ok = np.stack([SS > 1e-8 * SS.max(), gg > 1e-8 * gg.max()], axis=1)
    cn = [n // factor for n in nel]
    Np = S.Np
    for ce in range(cn[0] * cn[1] * cn[2]):
        cx, cy, cz = ce % cn[0], (ce // cn[0]) % cn[1], ce // (cn[0] * cn[1])
        ce2 = (cx + 1) % cn[0] + cn[0] * ((cy + 1) % cn[1] + cn[1] * cz)
        sl, sl2 = slice(ce * Np, ce * Np + Np), slice(ce2 * Np, ce2 * Np + Np)
        assert np.allclose(X1[sl2], X0[sl], rtol=0, atol=1e-9 * np.abs(X0).max())
        tmax = np.abs(T0[ok[:, 0], 0]).max(), np.abs(T0[ok[:, 1], 1]).max()
        for c in range(2):
            m = ok[sl, c]
            assert np.allclose(T1[sl2][m, c], T0[sl][m, c], rtol=0, atol=1e-8 * tmax[c])
        assert np.allclose(t1[sl2], t0[sl], rtol=0, atol=1e-10 * 300.0)
    assert ok.mean() > 0.9


def test_closure_primitives_are_the_thermodynamic_state(orc):
    """Step 1 of the samples: u and theta_v of each node's thermodynamic state
    (moist, saturated somewhere)."""
    from paper_2110_00853_b300 import inputs as I
    m = I.sub_mesh("c2", 2, 2, 4)
    S, Q, _, _, _ = orc.from_inputs(m, I.physics("c2"), I.case("c2"))
    prim = S.closure_primitives(Q)
    geo = S.geometry()
    P = S.params
    for e in (0, S.E // 2, S.E - 1):
        for n in (0, 31, 124):
            th = orc.thermo(P, Q[e, :, n], geo["z"][e, n])
            assert np.array_equal(prim[e, :3, n], th["u"])
            assert prim[e, 3, n] == th["thetav"]
