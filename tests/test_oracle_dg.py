"""Discrete invariants of the oracle's DG right-hand side and time stepper,
each fixed by the paper or by the mathematics of the method rather than by the
oracle itself:
  * a hydrostatic rest state equal to the reference state stays at rest
    (reference-state subtraction, Eq. momentum);
  * mass, total energy and total water are conserved to round-off on periodic
    and free-slip meshes (Sec. 6: O(1e-15) drift), and with prescribed surface
    fluxes the budgets change by exactly the prescribed boundary flux (App. A.1);
  * strong and weak forms agree under LGL collocation (Eqs. weak, weakDG2 and
    matrixProblem, summation by parts);
  * free-stream preservation on the warped mesh (metric identities);
  * a linear shear gives the closed-form Smagorinsky viscosity through the
    whole BR1 gradient pipeline (Sec. 3.1 and Eq. smago);
  * order N+1 convergence on a translating isentropic vortex;
  * fourth-order temporal convergence of LSRK(5,4) (Sec. 3.2).
"""
import numpy as np
import pytest

from paper_2110_00853_b300 import inputs as I


def _fuzz_velocity(S, Q, amp, seed):
    """add a seeded smooth-ish velocity field (momentum and kinetic energy)"""
    g = S.geometry()
    rng = np.random.default_rng(seed)
    k = rng.uniform(0.5, 2.0, size=(3, 3)) * 2 * np.pi / 2000.0
    ph = rng.uniform(0, 2 * np.pi, size=3)
    rho = Q[:, 0]
    Q = Q.copy()
    for c in range(3):
        u = amp * np.sin(k[c, 0] * g["x"] + k[c, 1] * g["y"] + k[c, 2] * g["z"] + ph[c])
        Q[:, 4] += 0.5 * rho * u * u + Q[:, 1 + c] * u
        Q[:, 1 + c] += rho * u
    return Q


def test_rest_state_stays_at_rest(orc):
    # dry neutral c1 background and a moist c2-shaped background (with
    # sponge; total water lowered so that the reference, built with q_l = 0,
    # is unsaturated): Q = reference state -> RHS = 0 to round-off
    for name, sub in (("c1", None), ("c2", (3, 3, 16))):
        m = I.mesh(name) if sub is None else I.sub_mesh(name, *sub)
        c = I.case(name)
        c.update(dtheta=0.0, noise_theta=0.0, noise_qt=0.0)
        if name == "c2":
            c.update(qt_sfc=10e-3, qt_ml=9.5e-3, qt_top=2e-3)
        ph = I.physics(name)
        ph["surface_flux"] = False
        S, Q, rr, pr, _ = orc.from_inputs(m, ph, c)
        R, fails = S.rhs(Q)
        assert fails == 0
        # scale: buoyancy of a 1 K perturbation, rho g / 300
        assert np.abs(R[:, 1:4]).max() < 1e-9 * 1.2 * 9.81 / 300.0
        assert np.abs(R[:, 0]).max() < 1e-12
        assert np.abs(R[:, 4]).max() < 1e-6


@pytest.mark.parametrize("name,sub,flux", [("c1", None, "rusanov"), ("c2", (3, 3, 8), "rusanov"),
                                           ("c2", (3, 3, 8), "hllc"), ("c2", (3, 3, 8), "roe")])
def test_conservation_periodic_free_slip(orc, name, sub, flux):
    m = I.mesh(name) if sub is None else I.sub_mesh(name, *sub)
    ph = I.physics(name)
    ph["surface_flux"] = False
    ph["flux"] = flux
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, I.case(name))
    Q = _fuzz_velocity(S, Q, 2.0, 1)
    R, fails = S.rhs(Q)
    assert fails == 0
    wJ = S.geometry()["wJ"]
    for v in (0, 4, 5):
        tot = (wJ * R[:, v]).sum()
        scale = (wJ * np.abs(R[:, v])).sum() + 1e-300
        assert abs(tot) <= 1e-13 * scale, (v, tot, scale)


@pytest.mark.parametrize("N,flux", [(3, "rusanov"), (5, "hllc")])
def test_conservation_warped_free_slip(orc, N, flux):
    """Mass, energy and water are conserved to rounding on the warped mesh
    (curl-form metric terms, free-slip terrain and lid, periodic sides, no
    sponge): the weighted sums of the tendency vanish at every order."""
    h = 40000.0 / 128
    m = dict(N=N, nex=6, ney=2, nez=5, Lx=6 * h, Ly=2 * h, Lz=5 * h, x0=20000.0 - 3 * h, y0=0.0, z0=0.0,
             periodic=(1, 1, 0), warp=True, hill_h=400.0, hill_a=1000.0, hill_xc=20000.0)
    ph = dict(I.physics("c3"), sponge_alpha=0.0, lateral_sponge_frac=0.0, flux=flux)
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, I.case("c3"))
    assert S.geometry()["J"].std() / S.geometry()["J"].mean() > 1e-2     # genuinely curved
    Q = _fuzz_velocity(S, Q, 2.0, 2)
    R, fails = S.rhs(Q)
    assert fails == 0
    wJ = S.geometry()["wJ"]
    for v in (0, 4, 5):
        tot = (wJ * R[:, v]).sum()
        scale = (wJ * np.abs(R[:, v])).sum() + 1e-300
        assert abs(tot) <= 1e-13 * scale, (v, tot, scale)


def test_surface_flux_budget(orc):
    m = I.sub_mesh("c2", 3, 3, 8)
    ph = I.physics("c2")
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, I.case("c2"))
    Q = _fuzz_velocity(S, Q, 1.0, 2)
    R, _ = S.rhs(Q)
    wJ = S.geometry()["wJ"]
    area = m["Lx"] * m["Ly"]
    # d/dt of total energy = (SHF + LHF) * area; of water and mass = LHF/L_v0 * area
    assert abs((wJ * R[:, 4]).sum() / ((ph["shf"] + ph["lhf"]) * area) - 1.0) < 1e-11
    assert abs((wJ * R[:, 5]).sum() / (ph["lhf"] / 2.5008e6 * area) - 1.0) < 1e-10
    assert abs((wJ * R[:, 0]).sum() / (ph["lhf"] / 2.5008e6 * area) - 1.0) < 1e-10


@pytest.mark.parametrize("name,sub,flux", [("c1", None, "rusanov"), ("c2", (3, 3, 8), "rusanov"),
                                           ("c1", None, "hllc"), ("c1", None, "roe")])
def test_weak_equals_strong_form(orc, name, sub, flux):
    m = I.mesh(name) if sub is None else I.sub_mesh(name, *sub)
    S, Q, rr, pr, _ = orc.from_inputs(m, dict(I.physics(name), flux=flux), I.case(name))
    Q = _fuzz_velocity(S, Q, 2.0, 3)
    Rs, _ = S.rhs(Q, form=0)
    Rw, _ = S.rhs(Q, form=1)
    for v in range(6):
        scale = np.abs(Rs[:, v]).max() + 1e-300
        assert np.abs(Rw[:, v] - Rs[:, v]).max() <= 1e-10 * scale, v


@pytest.mark.parametrize("N", [2, 4, 6])
def test_free_stream_preservation_warped(orc, N):
    """The curl-form metric terms satisfy the discrete metric identities at
    every order, so a uniform flow stays uniform inside the warped mesh (the
    GPU's curvilinear kernels are checked against this oracle at N = 2 .. 7)."""
    P = orc.make_params(closure="sl", g=0.0)
    S = orc.Solver(orc.make_mesh(N, 6, 2, 4, 6000.0, 2000.0, 4000.0, periodic=(1, 1, 0), warp=True, hill_h=600.0,
                                 hill_a=800.0, hill_xc=3000.0), P)
    E, Np = S.E, S.Np
    rho, T = 1.2, 300.0
    u = np.array([10.0, 2.0, 0.0])   # tangential to the flat top only if w = 0
    I0 = orc.internal_energy(P, T, 0.0, 0.0)
    p = rho * 287.0 * T
    Q = np.zeros((E, 6, Np))
    Q[:, 0] = rho
    Q[:, 1:4] = (rho * u)[None, :, None]
    Q[:, 4] = rho * (I0 + 0.5 * u @ u)
    S.set_reference(np.full((E, Np), rho), np.full((E, Np), p))
    R, _ = S.rhs(Q)
    # the walls (hill and lid) reflect the normal velocity, so only test the
    # interior elements, whose faces are all interior
    ez = np.arange(E) // (6 * 2)
    inner = (ez > 0) & (ez < 3)
    scale = rho * np.linalg.norm(u) ** 2 / 100.0     # momentum-flux divergence over 100 m
    assert np.abs(R[inner][:, 0]).max() < 1e-11 * rho * 10 / 100
    assert np.abs(R[inner][:, 1:4]).max() < 1e-9 * scale
    # the same field on a version of the mesh without conservative metrics
    # would not be preserved; check the warp is really non-affine:
    J = S.geometry()["J"]
    assert J.std() / J.mean() > 1e-3


def test_linear_shear_smagorinsky_through_pipeline(orc):
    m = I.mesh("c1")
    c = I.case("c1")
    c.update(dtheta=0.0, noise_theta=0.0)
    ph = I.physics("c1")
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, c)
    g = S.geometry()
    gamma = 0.01
    u = gamma * (g["z"] - 1000.0)
    Q = Q.copy()
    Q[:, 4] += 0.5 * Q[:, 0] * u * u
    Q[:, 1] = Q[:, 0] * u
    S.rhs(Q)
    it = S.intermediates()
    gu = it["gradG"][:, 0]                # d u / d (x, y, z)
    assert np.abs(gu[:, 2] - gamma).max() < 1e-12
    assert np.abs(gu[:, :2]).max() < 1e-12
    Delta = 500.0 / 4                    # (h_x h_y h_z)^(1/3) / N
    nut_exact = (0.21 * Delta) ** 2 * gamma
    assert np.abs(it["nut"] / nut_exact - 1.0).max() < 1e-6


def test_solid_body_rotation_vreman_through_pipeline(orc):
    """u = (-Om (y - yc), Om (x - xc), 0) is linear, so the BR1 gradient is
    exact in elements away from the walls and Vreman's nu_t takes its
    closed form 2.5 C_s^2 Delta^2 Om / sqrt(2) (isotropic Delta = 125 m)."""
    m = dict(I.mesh("c1"), periodic=(0, 0, 0))
    c = I.case("c1")
    c.update(dtheta=0.0, noise_theta=0.0)
    ph = dict(I.physics("c1"), closure="vreman", Cs=0.18, richardson=False)
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, c)
    g = S.geometry()
    Om = 0.01
    u, v = -Om * (g["y"] - 1000.0), Om * (g["x"] - 1000.0)
    Q = Q.copy()
    Q[:, 4] += 0.5 * Q[:, 0] * (u * u + v * v)
    Q[:, 1] = Q[:, 0] * u
    Q[:, 2] = Q[:, 0] * v
    S.rhs(Q)
    it = S.intermediates()
    e = np.arange(S.E)
    ex, ey = e % 4, (e // 4) % 4
    inner = (ex > 0) & (ex < 3) & (ey > 0) & (ey < 3)
    want = 2.5 * 0.18 ** 2 * 125.0 ** 2 * Om / np.sqrt(2.0)
    assert np.abs(it["nut"][inner] / want - 1.0).max() < 1e-8
    # a pure shear gives no Vreman viscosity
    Q2 = Q.copy()
    w = 0.01 * (g["z"] - 1000.0)
    Q2[:, 1] = Q[:, 0] * w
    Q2[:, 2] = 0.0
    Q2[:, 4] = Q[:, 4] - 0.5 * Q[:, 0] * (u * u + v * v) + 0.5 * Q[:, 0] * w * w
    S.rhs(Q2)
    assert np.abs(S.intermediates()["nut"][inner]).max() < 1e-8 * want


def _vortex_error(orc, N, nel, T=0.02, cfl=0.3):
    M = orc.make_mesh(N, nel, nel, 1, 10.0, 10.0, 10.0 / nel, x0=-5.0, y0=-5.0, periodic=(1, 1, 1))
    P = orc.make_params(closure="none", g=0.0)
    S = orc.Solver(M, P)
    c = orc.make_case(10, vortex_beta=5.0, vortex_R=1.0, vortex_U=10.0, vortex_T=300.0, vortex_rho=1.0)
    Q, _, _ = S.init_case(c)
    dt = cfl * 10.0 / nel / N / 360.0
    n = int(np.ceil(T / dt))
    Q1, _ = S.lsrk54(Q, n, T / n)
    Qe = S.vortex_exact(c, T)
    wJ = S.geometry()["wJ"]
    return np.sqrt((wJ * (Q1[:, 0] - Qe[:, 0]) ** 2).sum() / wJ.sum())


def test_isentropic_vortex_convergence_order(orc):
    e8 = _vortex_error(orc, 4, 8)
    e16 = _vortex_error(orc, 4, 16)
    order = np.log2(e8 / e16)
    assert order > 4.5, (e8, e16, order)     # N + 1 = 5


@pytest.mark.parametrize("scheme", ["lsrk54", "lsrk144"])
def test_lsrk_fourth_order_in_time(orc, scheme):
    m = I.mesh("c1")
    S, Q, rr, pr, _ = orc.from_inputs(m, I.physics("c1"), I.case("c1"))
    Q = _fuzz_velocity(S, Q, 3.0, 4)
    T = 0.32 if scheme == "lsrk54" else 0.96
    step = getattr(S, scheme)
    sols = [step(Q, n, T / n)[0] for n in (4, 8, 16)]
    e1 = np.abs(sols[0] - sols[1])[:, 1:4].max()
    e2 = np.abs(sols[1] - sols[2])[:, 1:4].max()
    assert 12.0 < e1 / e2 < 20.0, (e1, e2)
