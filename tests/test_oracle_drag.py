"""Pins of the oracle's bottom-wall drag law (App. A.1, Eq. drag_law):
n.(rho tau) = -rho C_d |u_p| u_p with n the inward normal, rho at the wall
node and u_p the wall-parallel velocity at the node of the first interior
layer above it.

The tendency with the drag law minus the tendency without it is the lifted
wall-stress term alone.  On a flat bottom it has a closed form: at a bottom
face node, -lift rho_w C_d |u_p| u_p in the two horizontal momentum
components, with lift = N (N + 1) / h_z (the LGL end weight 2 / (N (N + 1))
and the face-to-volume Jacobian ratio 2 / h_z), and nothing anywhere else.
The velocity varies with height and has a vertical part at the interior
layer, so reading u_p at the wall node, keeping its normal part, dropping
rho or flipping the sign each fail the pin.  On the warped mesh the term is
tangent to the terrain and opposes u_p.
"""
import numpy as np

from paper_2110_00853_b300 import inputs as I

CD = 0.015


def _states(orc, mesh, phys, case, seed):
    S0, Q, rr, pr, _ = orc.from_inputs(mesh, dict(phys, drag_cd=0.0), case)
    S1 = orc.from_inputs(mesh, dict(phys, drag_cd=CD))
    S1.set_reference(rr, pr)
    g = S0.geometry()
    z = g["z"] - g["z"].min()
    rng = np.random.default_rng(seed)
    a, b, c = rng.uniform(0.5, 2.0, size=3)
    Q = Q.copy()
    rho = Q[:, 0]
    u = np.stack([3.0 + a * z / 100.0, -2.0 + b * z / 100.0, c * z / 300.0], axis=1)
    Q[:, 4] += 0.5 * rho * (u ** 2).sum(1) - 0.5 * (Q[:, 1:4] ** 2).sum(1) / rho
    Q[:, 1:4] = rho[:, None] * u
    return S0, S1, Q, g


def test_drag_on_a_flat_bottom_is_the_closed_form(orc):
    mesh = dict(I.sub_mesh("c2", 3, 2, 2), periodic=(1, 1, 0))
    N, nez = mesh["N"], mesh["nez"]
    Nq = N + 1
    S0, S1, Q, g = _states(orc, mesh, I.physics("c2"), I.case("c2"), seed=1)
    R0, f0 = S0.rhs(Q)
    R1, f1 = S1.rhs(Q)
    assert f0 == 0 and f1 == 0
    dR = R1 - R0
    hz = mesh["Lz"] / nez
    lift = N * (N + 1) / hz
    expect = np.zeros_like(dR)
    E = Q.shape[0]
    nxy = mesh["nex"] * mesh["ney"]
    for e in range(nxy):                                  # bottom layer of elements
        for t2 in range(Nq):
            for t1 in range(Nq):
                n = t1 + Nq * t2                            # face node (k = 0)
                ni = n + Nq * Nq                            # first interior layer (k = 1)
                up = Q[e, 1:3, ni] / Q[e, 0, ni]
                expect[e, 1:3, n] = -lift * Q[e, 0, n] * CD * np.sqrt((up ** 2).sum()) * up
    scale = np.abs(expect).max()
    assert scale > 0
    assert np.abs(dR - expect).max() <= 1e-11 * scale, np.abs(dR - expect).max() / scale
    # nothing but the horizontal momentum of bottom face nodes changes
    for v in (0, 3, 4, 5):
        assert np.array_equal(R1[:, v], R0[:, v]), v
    assert np.array_equal(R1[nxy:E], R0[nxy:E])


def test_drag_on_the_warped_bottom_is_tangent_and_opposes_the_flow(orc):
    h = 40000.0 / 128
    mesh = dict(N=4, nex=6, ney=2, nez=3, Lx=6 * h, Ly=2 * h, Lz=3 * h, x0=20000.0 - 3 * h, y0=0.0, z0=0.0,
                periodic=(1, 1, 0), warp=True, hill_h=400.0, hill_a=1000.0, hill_xc=20000.0)
    phys = dict(I.physics("c3"), sponge_alpha=0.0, lateral_sponge_frac=0.0)
    S0, S1, Q, g = _states(orc, mesh, phys, I.case("c3"), seed=2)
    R0, _ = S0.rhs(Q)
    R1, _ = S1.rhs(Q)
    dR = R1 - R0
    Nq = mesh["N"] + 1
    nxy = mesh["nex"] * mesh["ney"]
    x, z = g["x"], g["z"]
    checked = 0
    for e in range(nxy):
        for t2 in range(Nq):
            for t1 in range(Nq):
                n, ni = t1 + Nq * t2, t1 + Nq * t2 + Nq * Nq
                # the terrain normal at the face node from the surface
                # z_s(x) = h exp(-((x - x_c)/a)^2): n ~ (-z_s'(x), 0, 1)
                xs = x[e, n]
                dzs = -2.0 * (xs - 20000.0) / 1000.0 ** 2 * 400.0 * np.exp(-((xs - 20000.0) / 1000.0) ** 2)
                nrm = np.array([-dzs, 0.0, 1.0]) / np.sqrt(1.0 + dzs ** 2)
                u = Q[e, 1:4, ni] / Q[e, 0, ni]
                up = u - (u @ nrm) * nrm
                d = dR[e, 1:4, n]
                # the oracle's normal is that of the discrete (N = 4) metric
                # terms, within ~1e-4 of the analytic one here; a kept normal
                # velocity part (w ~ 3 % of |u| at the interior layer) would
                # show as 1e-2
                assert abs(d @ nrm) <= 1e-3 * np.linalg.norm(d), (e, n)
                cos = (d @ up) / (np.linalg.norm(d) * np.linalg.norm(up))
                assert cos < -1.0 + 1e-6, (e, n, cos)
                checked += 1
    assert checked == nxy * Nq * Nq
    for v in (0, 4, 5):
        assert np.array_equal(R1[:, v], R0[:, v]), v
    assert np.array_equal(R1[nxy:], R0[nxy:])
