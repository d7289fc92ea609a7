"""HEVI on the GPU (Sec. 3.2; FP64 path): ARK2 of Giraldo, Kelly &
Constantinescu (2013) with the vertical linear acoustic-gravity operator
implicit, its block-tridiagonal line solves and the explicit remainder,
against the oracle's ARK2 (dense solves of the same operator assembled by
applying it to unit vectors): step increments to 1e-11 relative L2 on the
bubble box, and on thin elements at a step beyond the explicit vertical
acoustic limit; the operator, the line solve and steps at N = 2, 3, 5, 7."""
import numpy as np
import pytest

from paper_2110_00853_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _levels(arr, mesh):
    Nq = mesh["N"] + 1
    return np.array([arr[ez * mesh["nex"] * mesh["ney"], k * Nq * Nq] for ez in range(mesh["nez"])
                     for k in range(Nq)])


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _qt_reference(S, Q, m):
    """Reference total water of the linearisation: the initial column's q_t
    per node level (the level shared by two elements taken from the lower
    one, as cmles_set_reference does), as levels and as a per-node field."""
    Nq = m["N"] + 1
    lev = _levels(Q[:, 5] / Q[:, 0], m)
    for ez in range(1, m["nez"]):
        lev[ez * Nq] = lev[ez * Nq - 1]
    nodes = np.zeros((S.E, S.Np))
    slab = m["nex"] * m["ney"]
    for e in range(S.E):
        ez = e // slab
        for n in range(S.Np):
            nodes[e, n] = lev[ez * Nq + n // (Nq * Nq)]
    return lev, nodes


def _run(orc, m, ph, c, nsteps, dt, fuzz=0.0, precision="fp64"):
    from paper_2110_00853_b300 import cmles
    ph = dict(ph, integrator="ark2_hevi", dt=dt)
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, c)
    qlev, qnodes = _qt_reference(S, Q, m)
    S.set_reference_qt(qnodes)
    if fuzz:
        rng = np.random.default_rng(4)
        u = rng.uniform(-fuzz, fuzz, size=(Q.shape[0], 3, Q.shape[2]))
        Q = Q.copy()
        Q[:, 4] += 0.5 * Q[:, 0] * (u ** 2).sum(1) + (Q[:, 1:4] * u).sum(1)
        Q[:, 1:4] += Q[:, 0][:, None] * u
    Qo, fails = S.ark2_hevi(Q, nsteps, dt)
    assert fails == 0
    G = cmles.Solver(m, ph, precision=precision)
    G.set_reference(_levels(rr, m), _levels(pr, m), qlev)
    G.set_state(torch.from_numpy(Q).cuda())
    G.step(nsteps)
    Qg = G.get_state().cpu().numpy()
    d = G.diagnostics()
    assert not d["nonfinite"] and d["steps"] == nsteps
    b_orc, _ = S.budgets(Qo)
    for v in (0, 4):
        tol = 1e-13 if precision == "fp64" else 1e-9
        assert abs(d["budget"][v] - b_orc[v]) <= tol * abs(b_orc[v]), v
    return Q, Qo, Qg


def test_hevi_steps_match_oracle_bubble(orc):
    m, ph, c = I.mesh("c1"), I.physics("c1"), I.case("c1")
    Q, Qo, Qg = _run(orc, m, ph, c, 3, 0.02, fuzz=1.0)
    errs = [_rel(Qg[:, v] - Q[:, v], Qo[:, v] - Q[:, v]) for v in range(6) if np.abs(Qo[:, v] - Q[:, v]).max() > 0]
    print("HEVI bubble 3 steps rel L2", errs)
    assert max(errs) <= 1e-11, errs


def test_hevi_thin_elements_beyond_explicit_limit(orc):
    m, ph, c = I.mesh("c1"), I.physics("c1"), I.case("c1")
    m = dict(m, nex=2, ney=2, nez=8, Lx=2000.0, Ly=2000.0, Lz=160.0)
    c = dict(c, zc=80.0, r0=400.0)
    Q, Qo, Qg = _run(orc, m, ph, c, 20, 0.05)
    errs = [_rel(Qg[:, v] - Q[:, v], Qo[:, v] - Q[:, v]) for v in (0, 3, 4)]
    print("HEVI thin elements, dt 0.05 s, 20 steps rel L2", errs)
    assert max(errs) <= 1e-10, errs
    assert np.isfinite(Qg).all() and np.abs(Qg[:, 3] / Qg[:, 0]).max() < 5.0


@pytest.mark.parametrize("case", ["c1", "c2"])
def test_hevi_operator_and_solve_match_oracle(orc, case):
    """The vertical linear operator L (Q - Q_ref) and the solve of
    (I - dt gamma L) y = b on every vertical line, one call each, against the
    oracle's operator and its dense solve of the operator assembled from unit
    vectors; the dry bubble box and the moist layer's sub-box (linearised
    about its reference total water)."""
    from paper_2110_00853_b300 import cmles
    m = I.mesh("c1") if case == "c1" else I.sub_mesh("c2", 4, 3, 16)
    ph = dict(I.physics(case), integrator="ark2_hevi")
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, I.case(case))
    qlev, qnodes = _qt_reference(S, Q, m)
    S.set_reference_qt(qnodes)
    rng = np.random.default_rng(4)
    u = rng.uniform(-0.5, 0.5, size=(Q.shape[0], 3, Q.shape[2]))
    Q = Q.copy()
    Q[:, 4] += 0.5 * Q[:, 0] * (u ** 2).sum(1) + (Q[:, 1:4] * u).sum(1)
    Q[:, 1:4] += Q[:, 0][:, None] * u
    G = cmles.Solver(m, ph, precision="fp64")
    G.set_reference(_levels(rr, m), _levels(pr, m), qlev)
    Qd = torch.from_numpy(Q).cuda()
    Lg, Lo = G.hevi_operator(Qd).cpu().numpy(), S.vlin(Q)
    errs = [_rel(Lg[:, v], Lo[:, v]) for v in range(6) if np.abs(Lo[:, v]).max() > 0]
    print(case, "operator rel L2", errs)
    assert max(errs) <= 1e-13, errs
    Qr = S.vlin_reference()
    _, Ai, _ = orc.ark2_tableaux()
    M = np.eye(6 * m["nez"] * (m["N"] + 1)) - ph["dt"] * Ai[1, 1] * S.hevi_line_matrix()
    Yo, Yg = S._hevi_solve(M, Q, Qr), G.hevi_solve(Qd).cpu().numpy()
    errs = [_rel(Yg[:, v] - Qr[:, v], Yo[:, v] - Qr[:, v]) for v in range(6)]
    print(case, "solve rel L2", errs)
    # both solvers are accurate relative to the largest coupled unknown; rho'
    # is some 1e4 times smaller than (rho e)' here, hence its looser bound
    assert errs[0] <= 1e-10 and max(errs[1:]) <= 1e-12, errs


def test_hevi_moist_layer_matches_oracle(orc):
    """The moist layer's sub-box (saturation adjustment, sponge, surface
    fluxes in the explicit part; the dry linear operator implicit): two
    steps against the oracle."""
    m, ph, c = I.sub_mesh("c2", 4, 3, 16), I.physics("c2"), I.case("c2")
    Q, Qo, Qg = _run(orc, m, ph, c, 2, ph["dt"], fuzz=0.5)
    errs = [_rel(Qg[:, v] - Q[:, v], Qo[:, v] - Q[:, v]) for v in range(6)]
    print("HEVI moist sub-box 2 steps rel L2", errs)
    assert max(errs) <= 1e-11, errs


@pytest.mark.parametrize("case", ["c1", "c2"])
def test_hevi_fp32_path_tracks_oracle(orc, case):
    """HEVI with the stage tendencies from the FP32 kernels (deviation shadow
    of each FP64 stage state); the operator, the line solves and the stage
    combinations stay FP64.  ARK2's weights sum to 1 in absolute value, so
    the FP32 step bound 1e-5 applies."""
    if case == "c1":
        m, ph, c, dt = I.mesh("c1"), I.physics("c1"), I.case("c1"), 0.02
    else:
        m, ph, c = I.sub_mesh("c2", 4, 3, 16), I.physics("c2"), I.case("c2")
        dt = ph["dt"]
    Q, Qo, Qg = _run(orc, m, ph, c, 3, dt, fuzz=1.0, precision="fp32")
    errs = [_rel(Qg[:, v] - Q[:, v], Qo[:, v] - Q[:, v]) for v in range(6) if np.abs(Qo[:, v] - Q[:, v]).max() > 0]
    print("HEVI FP32", case, "3 steps rel L2", errs)
    assert max(errs) <= 1e-5, errs


@pytest.mark.parametrize("N", [2, 3, 5, 7])
def test_hevi_other_orders_operator_solve_and_steps(orc, N):
    """The line kernels at orders other than 4 (3 (N+1) coupled unknowns per
    element on a line, the per-level table sized by N): the operator and the
    line solve on the bubble box against the oracle's, then three ARK2 steps
    (the step scaled with the smallest node spacing)."""
    from paper_2110_00853_b300 import cmles
    m, c = dict(I.mesh("c1"), N=N), I.case("c1")
    ph = dict(I.physics("c1"), integrator="ark2_hevi")
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, c)
    qlev, qnodes = _qt_reference(S, Q, m)
    S.set_reference_qt(qnodes)
    rng = np.random.default_rng(5)
    u = rng.uniform(-0.5, 0.5, size=(Q.shape[0], 3, Q.shape[2]))
    Q = Q.copy()
    Q[:, 4] += 0.5 * Q[:, 0] * (u ** 2).sum(1) + (Q[:, 1:4] * u).sum(1)
    Q[:, 1:4] += Q[:, 0][:, None] * u
    G = cmles.Solver(m, ph, precision="fp64")
    G.set_reference(_levels(rr, m), _levels(pr, m), qlev)
    Qd = torch.from_numpy(Q).cuda()
    Lg, Lo = G.hevi_operator(Qd).cpu().numpy(), S.vlin(Q)
    errs = [_rel(Lg[:, v], Lo[:, v]) for v in range(6) if np.abs(Lo[:, v]).max() > 0]
    print("N", N, "operator rel L2", errs)
    assert max(errs) <= 1e-13, errs
    Qr = S.vlin_reference()
    _, Ai, _ = orc.ark2_tableaux()
    M = np.eye(6 * m["nez"] * (N + 1)) - ph["dt"] * Ai[1, 1] * S.hevi_line_matrix()
    Yo, Yg = S._hevi_solve(M, Q, Qr), G.hevi_solve(Qd).cpu().numpy()
    errs = [_rel(Yg[:, v] - Qr[:, v], Yo[:, v] - Qr[:, v]) for v in range(6)]
    print("N", N, "solve rel L2", errs)
    assert errs[0] <= 1e-10 and max(errs[1:]) <= 1e-12, errs
    G.close()
    dt = 0.02 * min(1.0, (4.0 / N) ** 2)
    Q0, Qo, Qg = _run(orc, m, I.physics("c1"), c, 3, dt, fuzz=1.0)
    errs = [_rel(Qg[:, v] - Q0[:, v], Qo[:, v] - Q0[:, v]) for v in range(6) if np.abs(Qo[:, v] - Q0[:, v]).max() > 0]
    print("N", N, "HEVI 3 steps rel L2", errs)
    assert max(errs) <= 1e-11, errs
