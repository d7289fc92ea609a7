"""Pins of the oracle's no-slip walls (App. A.3: u+ = 2 u_bc - u- with
u_bc = 0, so u+ = -u-, scalars copied), against the free-slip reflection
(u_bc = u- - (n.u-) n), on the flat moist layer with walls at the bottom
and top.

* The BR1 gradient: at a no-slip wall the face average of every velocity
  component is zero, so the lifted term adds n_z lift (-u) to du/dz and
  dv/dz of each face node (lift = N (N + 1) / h_z), where the free-slip
  reflection adds nothing; du/dz of the normal component, the scalars and
  every other node are unchanged.
* The Rusanov face flux (no closure, so no diffusive flux): with the
  outward normal n and u_n = u.n, the tangential momentum flux through the
  wall is rho u_t (lambda + u_n) at a no-slip wall and 0 at a free-slip one,
  lambda = |u_n| + c; the tendency of the tangential momentum of each wall
  node differs by -lift rho u_t (lambda + u_n) and nothing else does.
"""
import numpy as np

from paper_2110_00853_b300 import inputs as I


def _solvers(orc, phys, mask):
    mesh = dict(I.sub_mesh("c2", 3, 2, 2), periodic=(1, 1, 0))
    S0, Q, rr, pr, _ = orc.from_inputs(mesh, dict(phys, noslip=0), I.case("c2"))
    S1 = orc.from_inputs(mesh, dict(phys, noslip=mask))
    S1.set_reference(rr, pr)
    rng = np.random.default_rng(4)
    Q = Q.copy()
    rho = Q[:, 0]
    u = rng.uniform(-3.0, 3.0, size=(Q.shape[0], 3, Q.shape[2])) + np.array([2.0, -1.0, 0.0])[None, :, None]
    Q[:, 4] += 0.5 * rho * (u ** 2).sum(1) + (Q[:, 1:4] * u).sum(1)
    Q[:, 1:4] += rho[:, None] * u
    return mesh, S0, S1, Q


def _wall_nodes(mesh):
    """(elements, face nodes, outward n_z) of the bottom and top walls."""
    Nq = mesh["N"] + 1
    nxy = mesh["nex"] * mesh["ney"]
    E = nxy * mesh["nez"]
    face = np.arange(Nq * Nq)
    return [(np.arange(nxy), face, -1.0), (np.arange(E - nxy, E), face + mesh["N"] * Nq * Nq, 1.0)]


def test_noslip_gradient_lift(orc):
    mesh, S0, S1, Q = _solvers(orc, I.physics("c2"), mask=0b110000)
    S0.rhs(Q)
    g0 = S0.intermediates()["gradG"]                    # [e][v][c][n] = d G_v / d x_c
    S1.rhs(Q)
    g1 = S1.intermediates()["gradG"]
    N = mesh["N"]
    lift = N * (N + 1) / (mesh["Lz"] / mesh["nez"])
    u = Q[:, 1:4] / Q[:, 0:1]
    expect = np.zeros_like(g0)
    for els, nodes, nz in _wall_nodes(mesh):
        for c in (0, 1):                                # du/dz, dv/dz
            expect[np.ix_(els, [c], [2], nodes)] = nz * lift * (-u[np.ix_(els, [c], nodes)])[:, :, None, :]
    d = g1 - g0
    scale = np.abs(expect).max()
    assert np.abs(d - expect).max() <= 1e-11 * scale, np.abs(d - expect).max() / scale


def test_noslip_rusanov_wall_flux(orc):
    phys = dict(I.physics("c2"), closure="none")
    mesh, S0, S1, Q = _solvers(orc, phys, mask=0b110000)
    R0, _ = S0.rhs(Q)
    R1, _ = S1.rhs(Q)
    c = S1.intermediates()["aux"][:, 1]                 # sound speed at every node
    N = mesh["N"]
    lift = N * (N + 1) / (mesh["Lz"] / mesh["nez"])
    expect = np.zeros_like(R0)
    for els, nodes, nz in _wall_nodes(mesh):
        ix = np.ix_(els, nodes)
        rho = Q[:, 0][ix]
        un = nz * Q[:, 3][ix] / rho
        lam = np.abs(un) + c[ix]
        for v in (1, 2):
            expect[:, v][ix] = -lift * Q[:, v][ix] * (lam + un)
    d = R1 - R0
    scale = np.abs(expect).max()
    assert np.abs(d - expect).max() <= 1e-10 * scale, np.abs(d - expect).max() / scale
    for v in (0, 3, 4, 5):
        assert np.abs(d[:, v]).max() <= 1e-12 * np.abs(R0[:, v]).max(), v
