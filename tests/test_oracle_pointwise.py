"""Pins of the oracle's pointwise pieces against what the paper and the
mathematics fix: LGL closed forms and exactness (Sec. 3.1), the constants
table (Table t:constants), the Clausius-Clapeyron closed form and the
saturation-adjustment round trip (Sec. 2), Rusanov consistency and
conservation (Eq. nonviscFlux), Smagorinsky-Lilly and Richardson closed forms
(Sec. 4), the LSRK(5,4) stability polynomial (Sec. 3.2), the MLP gradient and
the SplitMix64 generator."""
import math
import os

import numpy as np
import pytest

from paper_2110_00853_b300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


# ------------------------------------------------------------------ LGL

def test_lgl_closed_form_n4(orc):
    xi, w, D = orc.lgl(4)
    gold = np.array([[float(r[1]), float(r[2])] for r in _read("lgl_n4.txt")])
    assert np.allclose(xi, gold[:, 0], atol=1e-15, rtol=0)
    assert np.allclose(w, gold[:, 1], atol=1e-15, rtol=0)
    assert abs(xi[3] - math.sqrt(3.0 / 7.0)) < 1e-15


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_lgl_derivative_exact_on_polynomials(orc, N):
    xi, w, D = orc.lgl(N)
    for m in range(N + 1):
        f = xi ** m
        df = m * xi ** (m - 1) if m > 0 else np.zeros_like(xi)
        assert np.abs(D @ f - df).max() < 1e-12 * max(1, m * m)
    # quadrature exact to degree 2N-1
    for m in range(2 * N):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs((w * xi ** m).sum() - exact) < 1e-14
    assert np.abs(D.sum(axis=1)).max() < 1e-13


@pytest.mark.parametrize("N", [2, 3, 4, 6])
def test_lgl_summation_by_parts(orc, N):
    xi, w, D = orc.lgl(N)
    Qm = np.diag(w) @ D
    B = np.zeros((N + 1, N + 1))
    B[0, 0], B[N, N] = -1.0, 1.0
    assert np.abs(Qm + Qm.T - B).max() < 1e-13


# ------------------------------------------------------------------ constants

def test_constants_table(orc):
    for name, val, *_unit in _read("constants.txt"):
        assert orc.CONSTANTS[name] == float(val), name


# ------------------------------------------------------------------ thermodynamics

def test_pvsat_triple_point_and_clausius_clapeyron(orc):
    P = orc.make_params(moist=True)
    assert abs(orc.pvsat(P, P.Ttr) - P.ptr) < 1e-12
    for T in (250.0, 273.16, 290.0, 300.0, 310.0):
        h = 1e-3
        dln = (math.log(orc.pvsat(P, T + h)) - math.log(orc.pvsat(P, T - h))) / (2 * h)
        L = P.Lv0 + (P.cvv + P.Rv - P.cvl) * (T - P.T0)
        assert abs(dln - L / (P.Rv * T * T)) < 1e-8 * dln


def test_pvsat_physical_magnitude(orc):
    # Saturation vapour pressure over liquid water near 300 K is about 3.5 kPa
    # and about 2.3 kPa near 293 K (standard psychrometric values); the closed
    # form must land within a few percent of these.
    P = orc.make_params(moist=True)
    assert abs(orc.pvsat(P, 300.0) / 3537.0 - 1.0) < 0.03
    assert abs(orc.pvsat(P, 293.15) / 2339.0 - 1.0) < 0.03


def test_internal_energy_definition(orc):
    P = orc.make_params(moist=True)
    # dry air: I = c_vd (T - T0); vapour carries I_v0 = L_v0 - R_v T0 at T0
    assert abs(orc.internal_energy(P, 300.0, 0.0, 0.0) - 717.5 * (300.0 - 273.16)) < 1e-9
    Iv0 = 2.5008e6 - 462.0 * 273.16
    assert abs(orc.internal_energy(P, 273.16, 1.0, 0.0) - Iv0) < 1e-6
    assert abs(orc.internal_energy(P, 273.16, 1.0, 1.0)) < 1e-9


def test_saturation_adjustment_round_trip(orc):
    P = orc.make_params(moist=True)
    rng = np.random.default_rng(7)
    for _ in range(200):
        T = rng.uniform(275.0, 305.0)
        rho = rng.uniform(0.8, 1.25)
        qs = orc.qsat(P, T, rho)
        if rng.uniform() < 0.5:
            qt = qs * rng.uniform(1.0001, 1.2)       # saturated, with condensate
            ql = qt - qs
        else:
            qt = qs * rng.uniform(0.2, 0.999)        # unsaturated
            ql = 0.0
        I = orc.internal_energy(P, T, qt, ql)
        T2, ql2, it = orc.saturation_adjustment(P, rho, qt, I)
        assert it >= 0
        assert abs(T2 - T) < 1e-9 * T
        assert abs(ql2 - ql) < 1e-12
        if ql == 0.0:
            assert it == 0
            cvm = (1 - qt) * P.cvd + qt * P.cvv
            assert abs(T2 - (P.T0 + (I - qt * (P.Lv0 - P.Rv * P.T0)) / cvm)) < 1e-12 * T


# ------------------------------------------------------------------ fluxes

def _state(orc, P, T, qt, rho, u, z):
    I = orc.internal_energy(P, T, qt, 0.0)
    return np.array([rho, rho * u[0], rho * u[1], rho * u[2], rho * (I + 0.5 * np.dot(u, u) + P.g * z), rho * qt])


def test_inviscid_flux_closed_form(orc):
    P = orc.make_params(moist=True)
    T, qt, rho, z, pr = 290.0, 0.005, 1.1, 300.0, 9.0e4
    u = np.array([3.0, -2.0, 0.5])
    Y = _state(orc, P, T, qt, rho, u, z)
    p = rho * (P.Rd * (1 - qt) + P.Rv * qt) * T     # Eq. eos, unsaturated
    for n in np.eye(3):
        f = orc.flux1_normal(P, Y, z, pr, n)
        un = u @ n
        assert abs(f[0] - rho * un) < 1e-12
        assert np.allclose(f[1:4], rho * u * un + (p - pr) * n, rtol=1e-12, atol=1e-9)
        assert abs(f[4] - (Y[4] + p) * un) < 1e-9 * abs(Y[4] * un)
        assert abs(f[5] - rho * qt * un) < 1e-14


def test_rusanov_consistency_and_conservation(orc):
    P = orc.make_params(moist=True)
    rng = np.random.default_rng(3)
    for _ in range(20):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        Ym = _state(orc, P, rng.uniform(280, 300), rng.uniform(0, 0.01), rng.uniform(0.9, 1.2),
                    rng.normal(size=3) * 5, 500.0)
        Yp = _state(orc, P, rng.uniform(280, 300), rng.uniform(0, 0.01), rng.uniform(0.9, 1.2),
                    rng.normal(size=3) * 5, 500.0)
        # consistency: F*(Y, Y, n) = n.F(Y)
        assert np.allclose(orc.rusanov(P, Ym, Ym, 500.0, 9.5e4, n), orc.flux1_normal(P, Ym, 500.0, 9.5e4, n),
                           rtol=1e-14, atol=1e-10)
        # conservation: F*(Y-, Y+, n) = -F*(Y+, Y-, -n), exactly
        a = orc.rusanov(P, Ym, Yp, 500.0, 9.5e4, n)
        b = orc.rusanov(P, Yp, Ym, 500.0, 9.5e4, -n)
        assert np.array_equal(a, -b)
        # dissipation is upwinding: jump in rho times lambda/2 >= sound speed/2
        f0 = 0.5 * (orc.flux1_normal(P, Ym, 500.0, 9.5e4, n)[0] + orc.flux1_normal(P, Yp, 500.0, 9.5e4, n)[0])
        lam = 2 * (a[0] - f0) / (Ym[0] - Yp[0])
        assert lam > 300.0


def test_hllc_consistency_symmetry_supersonic(orc):
    P = orc.make_params(moist=True)
    rng = np.random.default_rng(7)
    for _ in range(20):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        Ym = _state(orc, P, rng.uniform(280, 300), rng.uniform(0, 0.01), rng.uniform(0.9, 1.2),
                    rng.normal(size=3) * 5, 500.0)
        Yp = _state(orc, P, rng.uniform(280, 300), rng.uniform(0, 0.01), rng.uniform(0.9, 1.2),
                    rng.normal(size=3) * 5, 500.0)
        f = orc.flux1_normal(P, Ym, 500.0, 9.5e4, n)
        assert np.allclose(orc.hllc(P, Ym, Ym, 500.0, 9.5e4, n), f, rtol=1e-13, atol=1e-9)
        a = orc.hllc(P, Ym, Yp, 500.0, 9.5e4, n)
        b = orc.hllc(P, Yp, Ym, 500.0, 9.5e4, -n)
        assert np.allclose(a, -b, rtol=1e-12, atol=1e-8)
    # supersonic to the right on both sides (u.n > c): the left flux, exactly
    n = np.array([1.0, 0.0, 0.0])
    Ym = _state(orc, P, 290.0, 0.005, 1.1, np.array([400.0, 3.0, 0.0]), 500.0)
    Yp = _state(orc, P, 295.0, 0.002, 1.0, np.array([420.0, -2.0, 1.0]), 500.0)
    assert np.array_equal(orc.hllc(P, Ym, Yp, 500.0, 9.5e4, n), orc.flux1_normal(P, Ym, 500.0, 9.5e4, n))
    assert np.array_equal(orc.hllc(P, Yp, Ym, 500.0, 9.5e4, -n), orc.flux1_normal(P, Ym, 500.0, 9.5e4, -n))


def test_hllc_resolves_contact_and_wall(orc):
    """A contact (equal pressure and normal velocity, different density,
    temperature, water and tangential velocity) is an exact solution of the
    Riemann problem moving with u.n: HLLC returns the upwind flux, where
    Rusanov adds dissipation.  Against its mirror image (the wall ghost) HLLC
    carries no mass, water or energy through the face."""
    P = orc.make_params(moist=True)
    n = np.array([0.0, 0.6, 0.8])
    p, z, pr = 9.6e4, 400.0, 9.5e4
    for un in (4.0, -3.0):
        TL, qL, TR, qR = 290.0, 0.006, 300.0, 0.001
        rL = p / ((P.Rd * (1 - qL) + P.Rv * qL) * TL)
        rR = p / ((P.Rd * (1 - qR) + P.Rv * qR) * TR)
        t = np.array([1.0, 0.8, -0.6])          # tangential to n
        YL = _state(orc, P, TL, qL, rL, un * n + 2.0 * t, z)
        YR = _state(orc, P, TR, qR, rR, un * n - 5.0 * t, z)
        up = YL if un > 0 else YR
        want = orc.flux1_normal(P, up, z, pr, n)
        got = orc.hllc(P, YL, YR, z, pr, n)
        assert np.allclose(got, want, rtol=1e-11, atol=1e-7), (got, want)
        assert np.abs(orc.rusanov(P, YL, YR, z, pr, n) - want).max() > 1.0
    Y = _state(orc, P, 288.0, 0.004, 1.15, np.array([3.0, -7.0, 2.0]), z)
    G = Y.copy()
    rn = Y[1:4] @ n
    G[1:4] = Y[1:4] - 2.0 * rn * n
    f = orc.hllc(P, Y, G, z, pr, n)
    assert abs(f[0]) < 1e-12 and abs(f[5]) < 1e-14 and abs(f[4]) < 1e-7


def test_roe_consistency_symmetry_and_dry_roe_property(orc):
    """Roe flux: consistency and antisymmetry on moist states; for dry air the
    averaged Jacobian is Roe's exact linearisation, so a flow supersonic to
    the right gets exactly the left flux (|A| = A there) and a moving contact
    the upwind flux."""
    P = orc.make_params(moist=True)
    rng = np.random.default_rng(9)
    for _ in range(20):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        Ym = _state(orc, P, rng.uniform(280, 300), rng.uniform(0, 0.01), rng.uniform(0.9, 1.2),
                    rng.normal(size=3) * 5, 500.0)
        Yp = _state(orc, P, rng.uniform(280, 300), rng.uniform(0, 0.01), rng.uniform(0.9, 1.2),
                    rng.normal(size=3) * 5, 500.0)
        assert np.allclose(orc.roe(P, Ym, Ym, 500.0, 9.5e4, n), orc.flux1_normal(P, Ym, 500.0, 9.5e4, n),
                           rtol=1e-13, atol=1e-9)
        a = orc.roe(P, Ym, Yp, 500.0, 9.5e4, n)
        b = orc.roe(P, Yp, Ym, 500.0, 9.5e4, -n)
        assert np.allclose(a, -b, rtol=1e-12, atol=1e-8)
    Pd = orc.make_params(moist=False)
    n = np.array([0.6, 0.0, 0.8])
    for _ in range(10):
        Ym = _state(orc, Pd, rng.uniform(250, 320), 0.0, rng.uniform(0.5, 1.3), 500.0 * n + rng.normal(size=3) * 5,
                    800.0)
        Yp = _state(orc, Pd, rng.uniform(250, 320), 0.0, rng.uniform(0.5, 1.3), 520.0 * n + rng.normal(size=3) * 5,
                    800.0)
        f = orc.flux1_normal(Pd, Ym, 800.0, 8.0e4, n)
        assert np.allclose(orc.roe(Pd, Ym, Yp, 800.0, 8.0e4, n), f, rtol=1e-11, atol=1e-6)
    p, z = 9.6e4, 400.0
    t = np.array([0.8, 0.0, -0.6])
    for un in (4.0, -3.0):
        rL, rR = p / (Pd.Rd * 290.0), p / (Pd.Rd * 300.0)
        YL = _state(orc, Pd, 290.0, 0.0, rL, un * n + 2.0 * t, z)
        YR = _state(orc, Pd, 300.0, 0.0, rR, un * n - 5.0 * t, z)
        want = orc.flux1_normal(Pd, YL if un > 0 else YR, z, 9.5e4, n)
        assert np.allclose(orc.roe(Pd, YL, YR, z, 9.5e4, n), want, rtol=1e-11, atol=1e-7)


def test_roe_wall_and_moist_contact(orc):
    P = orc.make_params(moist=True)
    n = np.array([0.0, 0.6, 0.8])
    z, pr = 400.0, 9.5e4
    Y = _state(orc, P, 288.0, 0.004, 1.15, np.array([3.0, -7.0, 2.0]), z)
    G = Y.copy()
    G[1:4] = Y[1:4] - 2.0 * (Y[1:4] @ n) * n
    f = orc.roe(P, Y, G, z, pr, n)
    assert abs(f[0]) < 1e-12 and abs(f[5]) < 1e-14 and abs(f[4]) < 1e-7
    # a moist contact is resolved up to the linearised pressure jump of the
    # averaged state (second order in the jumps): within 1e-6 of the flux
    # scale of the upwind flux, where Rusanov is off by O(1) of it
    p, t = 9.6e4, np.array([1.0, 0.8, -0.6])
    TL, qL, TR, qR = 290.0, 0.006, 300.0, 0.001
    rL = p / ((P.Rd * (1 - qL) + P.Rv * qL) * TL)
    rR = p / ((P.Rd * (1 - qR) + P.Rv * qR) * TR)
    YL = _state(orc, P, TL, qL, rL, 4.0 * n + 2.0 * t, z)
    YR = _state(orc, P, TR, qR, rR, 4.0 * n - 5.0 * t, z)
    want = orc.flux1_normal(P, YL, z, pr, n)
    e_roe = np.abs(orc.roe(P, YL, YR, z, pr, n) - want).max()
    e_rus = np.abs(orc.rusanov(P, YL, YR, z, pr, n) - want).max()
    assert e_roe < 1e-6 * np.abs(want).max() and e_rus > 0.1 * np.abs(want).max()


# ------------------------------------------------------------------ closure

def test_smagorinsky_simple_shear(orc):
    P = orc.make_params(Cs=0.21, richardson=True)
    gamma, Delta = 0.02, 25.0
    gu = np.zeros((3, 3))
    gu[0, 2] = gamma                  # u = gamma z: S_13 = S_31 = gamma/2, |S| = gamma
    assert abs(orc.smagorinsky(P, gu, 0.0, 300.0, Delta) - (0.21 * Delta) ** 2 * gamma) < 1e-15
    # pure rotation has no strain
    rot = np.array([[0, 1.0, 0], [-1.0, 0, 0], [0, 0, 0]])
    assert orc.smagorinsky(P, rot, 0.0, 300.0, Delta) == 0.0


def test_richardson_correction(orc):
    P = orc.make_params(Cs=0.2, richardson=True)
    gamma, Delta, thv = 0.01, 10.0, 300.0
    gu = np.zeros((3, 3))
    gu[0, 2] = gamma
    base = (0.2 * Delta) ** 2 * gamma
    for Ri in (-1.0, 0.0, 0.1, 0.25, 0.33, 0.34, 0.5):
        dthdz = Ri * gamma * gamma * thv / P.g
        fb = 1.0 if Ri <= 0 else max(0.0, 1.0 - 3.0 * Ri) ** 0.25
        assert abs(orc.smagorinsky(P, gu, dthdz, thv, Delta) - base * fb) < 1e-12 * base


def test_vreman_special_cases(orc):
    """Eq. vreman-sgs: zero for a pure shear (the model's design property), a
    closed form for solid-body rotation with isotropic lengths."""
    P = orc.make_params(Cs=0.18, richardson=False)
    Dm = [25.0, 25.0, 25.0]
    gu = np.zeros((3, 3))
    gu[0, 2] = 0.02                  # u = gamma z
    assert orc.vreman(P, gu, 0.0, 300.0, Dm) == 0.0
    Om = 0.03                        # u = (-Om y, Om x, 0): singular values Om, Om, 0
    rot = np.array([[0.0, -Om, 0.0], [Om, 0.0, 0.0], [0.0, 0.0, 0.0]])
    want = 2.5 * 0.18 ** 2 * 25.0 ** 2 * Om / np.sqrt(2.0)
    assert abs(orc.vreman(P, rot, 0.0, 300.0, Dm) - want) < 1e-14 * want
    assert orc.vreman(P, np.zeros((3, 3)), 0.0, 300.0, Dm) == 0.0


def test_vreman_against_singular_values(orc):
    """B_beta is the sum of the 2x2 principal minors of beta = A A^T with
    A = grad(u) diag(Delta_m), i.e. sum_{i<j} s_i^2 s_j^2 over the singular
    values of A; checked on random gradients and anisotropic lengths."""
    P = orc.make_params(Cs=0.21, richardson=False)
    rng = np.random.default_rng(11)
    for _ in range(20):
        gu = rng.normal(size=(3, 3)) * 0.05
        Dm = rng.uniform(10.0, 80.0, size=3)
        s = np.linalg.svd(gu @ np.diag(Dm), compute_uv=False) ** 2
        B = s[0] * s[1] + s[0] * s[2] + s[1] * s[2]
        want = 2.5 * 0.21 ** 2 * np.sqrt(B / (gu ** 2).sum())
        assert abs(orc.vreman(P, gu, 0.0, 300.0, Dm) - want) < 1e-12 * want
        # lengths enter per direction m (columns of grad u), not per component
        gT = gu.T.copy()
        sT = np.linalg.svd(gT @ np.diag(Dm), compute_uv=False) ** 2
        BT = sT[0] * sT[1] + sT[0] * sT[2] + sT[1] * sT[2]
        assert abs(orc.vreman(P, gT, 0.0, 300.0, Dm) - 2.5 * 0.21 ** 2 * np.sqrt(BT / (gu ** 2).sum())) < 1e-12 * want * 10


def test_vreman_richardson_factor_same_as_smagorinsky(orc):
    Pn = orc.make_params(Cs=0.2, richardson=False)
    Pr = orc.make_params(Cs=0.2, richardson=True)
    rng = np.random.default_rng(5)
    for Ri in (-0.5, 0.1, 0.3, 0.4):
        gu = rng.normal(size=(3, 3)) * 0.02
        S = 0.5 * (gu + gu.T)
        thv = 300.0
        dthdz = Ri * 2.0 * (S * S).sum() * thv / Pr.g
        Dm = [20.0, 30.0, 10.0]
        f_sl = orc.smagorinsky(Pr, gu, dthdz, thv, 10.0) / orc.smagorinsky(Pn, gu, dthdz, thv, 10.0)
        v0 = orc.vreman(Pn, gu, dthdz, thv, Dm)
        assert abs(orc.vreman(Pr, gu, dthdz, thv, Dm) - f_sl * v0) <= 1e-13 * v0


# ------------------------------------------------------------------ LSRK(5,4)

def test_lsrk54_stability_polynomial(orc):
    A, B, c = orc.lsrk54_coefficients()
    # stage times are consistent: c_s = sum of the weights reached so far
    assert abs(B[0] - c[1]) < 1e-16
    for z in (-0.3, -1.0 + 0.5j, 0.7j, -2.5, 1.2 - 0.4j):
        y, dy = 1.0 + 0j, 0j
        for s in range(5):
            dy = A[s] * dy + z * y
            y = y + B[s] * dy
        Rz = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24 + z ** 5 / 200
        assert abs(y - Rz) < 1e-10 * max(1, abs(Rz))


# ------------------------------------------------------------------ LSRK order conditions

def _butcher_2n(A, B):
    """Butcher tableau (a, b) of a 2N-storage scheme: with k_j = dt RHS(Y_j),
    the register after stage i is dQ_i = sum_{j<=i} (prod_{m=j+1..i} A_m) k_j
    and Y_{s+1} = Q + sum_{i<=s} B_i dQ_i."""
    S = len(A)
    a = np.zeros((S + 1, S))
    for s in range(1, S + 1):
        for j in range(s):
            a[s, j] = sum(B[i] * np.prod(A[j + 1:i + 1]) for i in range(j, s))
    return a[:S], a[S]


@pytest.mark.parametrize("scheme", ["lsrk54", "lsrk144"])
def test_lsrk_fourth_order_conditions(orc, scheme):
    """The eight order conditions of a fourth-order Runge-Kutta method (Butcher
    trees up to order 4) hold for the 2N-storage tables of Sec. 3.2's
    integrators, Carpenter & Kennedy (1994) with 5 stages and Niegemann, Diehl
    & Busch (2012) with 14; the stage times are the row sums, and neither
    scheme is fifth order."""
    A, B, c = getattr(orc, scheme + "_coefficients")()
    assert len(A) == {"lsrk54": 5, "lsrk144": 14}[scheme] and A[0] == 0.0
    a, b = _butcher_2n(A, B)
    assert np.abs(a.sum(1) - c).max() < 1e-12
    conds = [(b.sum(), 1.0), (b @ c, 1 / 2), (b @ c ** 2, 1 / 3), (b @ (a @ c), 1 / 6), (b @ c ** 3, 1 / 4),
             (b @ (c * (a @ c)), 1 / 8), (b @ (a @ c ** 2), 1 / 12), (b @ (a @ (a @ c)), 1 / 24)]
    for v, t in conds:
        assert abs(v - t) < 1e-12, (scheme, v, t)
    assert abs(b @ c ** 4 - 1 / 5) > 1e-5


def _amplification(A, B, z):
    y, dy = 1.0 + 0j, 0j
    for s in range(len(A)):
        dy = A[s] * dy + z * y
        y = y + B[s] * dy
    return abs(y)


def test_lsrk144_real_axis_stability(orc):
    """The 14-stage scheme is stable on the negative real axis down to about
    -18.5, 1.3 per stage against LSRK(5,4)'s 4.65 / 5 = 0.93: the large
    explicit stability region Sec. 3.2 cites it for."""
    A, B, _ = orc.lsrk144_coefficients()
    assert all(_amplification(A, B, x) <= 1 + 1e-12 for x in np.linspace(-18.4, 0.0, 4001))
    assert _amplification(A, B, -19.0) > 1.0
    A5, B5, _ = orc.lsrk54_coefficients()
    assert all(_amplification(A5, B5, x) <= 1 + 1e-12 for x in np.linspace(-4.6, 0.0, 1001))
    assert _amplification(A5, B5, -4.8) > 1.0


# ------------------------------------------------------------------ MLP

def _rand_w(rng, scale=0.3):
    return dict(W1=rng.normal(size=(64, 13)) * scale, b1=rng.normal(size=64) * 0.1,
                W2=rng.normal(size=(64, 64)) * scale / 2, b2=rng.normal(size=64) * 0.1,
                W3=rng.normal(size=(2, 64)) * scale, b3=rng.normal(size=2) * 0.1)


def test_mlp_forward_silu_closed_form(orc):
    W = dict(W1=np.zeros((64, 13)), b1=np.full(64, 0.7), W2=np.zeros((64, 64)), b2=np.full(64, -1.3),
             W3=np.ones((2, 64)), b3=np.array([0.5, -0.5]))
    silu = lambda a: a / (1 + math.exp(-a))
    Y = orc.mlp_forward(np.zeros((1, 13)), W)
    assert abs(Y[0, 0] - (64 * silu(-1.3) + 0.5)) < 1e-12


def test_mlp_gradient_finite_difference(orc):
    rng = np.random.default_rng(11)
    W = _rand_w(rng)
    X = rng.normal(size=(17, 13))
    T = rng.normal(size=(17, 2))
    loss, g = orc.mlp_loss_grad(X, T, W)
    for key in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = W[key].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            h = 1e-5
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = orc.mlp_loss_grad(X, T, W)
            flat[idx] = old - h
            lm, _ = orc.mlp_loss_grad(X, T, W)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[key].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-7 * max(1e-3, abs(an)), (key, idx, fd, an)


def test_bf16_rounding_definition(orc):
    # BF16 keeps 8 significand bits: spacing 2^-7 at 1.0.  Round to nearest,
    # ties to even.
    assert orc.bf16(1.0 + 2.0 ** -8) == 1.0
    assert orc.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert orc.bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert orc.bf16(-3.0) == -3.0 and orc.bf16(0.0) == 0.0


def test_adam_first_step(orc):
    theta = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 1e-3])
    m, v = np.zeros(3), np.zeros(3)
    orc.adam(theta, g, m, v, 1, lr=0.01, eps=1e-12)
    # bias-corrected first step moves each parameter by lr * sign(g)
    assert np.allclose(theta, [0.99, -1.99, 2.99], atol=1e-9)


# ------------------------------------------------------------------ generator

def test_splitmix64_published_vector(orc):
    # First output of SplitMix64 seeded with 0 is 0xE220A8397B1DCDAF; the
    # uniform double keeps its top 53 bits.
    assert orc.uniform(0, 0) == (0xE220A8397B1DCDAF >> 11) * 2.0 ** -53
    assert orc.uniform(0, 1) == (0x6E789E6AA1B965F4 >> 11) * 2.0 ** -53


# ------------------------------------------------------------------ exponential filter

def test_filter_matrix_modal_definition(orc):
    """F = V diag(exp(-alpha (k/N)^s)) V^-1 against numpy's Legendre
    Vandermonde: mode k is scaled by sigma(k/N), the element mean (LGL
    quadrature) is kept, the top mode is removed (sigma(1) = e^-alpha)."""
    from numpy.polynomial import legendre as npl
    N, s, alpha = 4, 64, -np.log(np.finfo(float).eps)
    xi, w, _ = orc.lgl(N)
    F = orc.filter_matrix(N, s, alpha)
    V = npl.legvander(xi, N)
    sig = np.exp(-alpha * (np.arange(N + 1) / N) ** s)
    assert np.abs(F - V @ np.diag(sig) @ np.linalg.inv(V)).max() < 1e-13
    for k in range(N + 1):
        assert np.abs(F @ V[:, k] - sig[k] * V[:, k]).max() < 1e-13
    assert np.abs(F @ V[:, N]).max() < 1e-13          # e^-36 ~ 2e-16
    rng = np.random.default_rng(2)
    u = rng.normal(size=N + 1)
    assert abs(w @ (F @ u) - w @ u) < 1e-14
    # a gentler filter (s = 2, alpha = 1) to see every mode damped
    F2 = orc.filter_matrix(N, 2, 1.0)
    for k in range(N + 1):
        assert np.abs(F2 @ V[:, k] - np.exp(-(k / N) ** 2) * V[:, k]).max() < 1e-13


def test_filter_on_solver_state(orc):
    """Tensor-product filter on the momentum of a 3D state: a product of
    Legendre modes P_a(xi) P_b(eta) P_c(zeta) is scaled by
    sigma(a/N) sigma(b/N) sigma(c/N); unselected variables are untouched and
    each element's momentum integral is kept."""
    from numpy.polynomial import legendre as npl
    m = I.sub_mesh("c1", 2, 2, 2)
    S = orc.from_inputs(m, I.physics("c1"))
    N = 4
    xi, w, _ = orc.lgl(N)
    E, Np = S.E, S.Np
    g = S.geometry()
    V = npl.legvander(xi, N)
    rng = np.random.default_rng(4)
    Q = rng.normal(size=(E, 6, Np))
    a, b, c = 4, 1, 3
    i, j, k = np.arange(Np) % 5, (np.arange(Np) // 5) % 5, np.arange(Np) // 25
    mode = V[i, a] * V[j, b] * V[k, c]
    Q[:, 2] = 3.0 * mode
    s, alpha = 8, 2.0
    Qf = S.filter(Q, s, alpha, 0b1110)
    sig = lambda q: np.exp(-alpha * (q / N) ** s)
    assert np.abs(Qf[:, 2] - 3.0 * mode * sig(a) * sig(b) * sig(c)).max() < 1e-12
    for v in (0, 4, 5):
        assert np.array_equal(Qf[:, v], Q[:, v])
    wJ = g["wJ"]
    for v in (1, 2, 3):
        assert np.abs((wJ * Qf[:, v]).sum(1) - (wJ * Q[:, v]).sum(1)).max() < 1e-12 * np.abs(wJ * Q[:, v]).sum()
