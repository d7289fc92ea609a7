"""Wall options on the GPU against the oracle, with a mean flow over the
walls: the bottom-wall drag law (App. A.1, Eq. drag_law), and no-slip
velocity ghosts (App. A.3) on the bottom and top walls, alone and together;
FP64 and FP32 on the flat moist layer, FP32 on the warped ridge mesh;
tendencies and one LSRK step.  The drag term itself (tendency with C_d minus
tendency without) decelerates the wall-parallel flow of the bottom face
nodes only."""
import numpy as np
import pytest

from paper_2110_00853_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CD = 0.015


def _levels(arr, mesh):
    Nq = mesh["N"] + 1
    return np.array([arr[ez * mesh["nex"] * mesh["ney"], k * Nq * Nq] for ez in range(mesh["nez"])
                     for k in range(Nq)])


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _flow(Q, seed, mean=(2.0, -1.0, 0.0), amp_u=3.0, amp_e=50.0):
    """The state of the other parity tests (velocity fuzzed by +-3 m/s,
    energy by +-50 J m^-3) with a mean flow, so that the wall-parallel
    velocity of every interior-layer node is well away from zero."""
    rng = np.random.default_rng(seed)
    Q = Q.copy()
    rho = Q[:, 0]
    u = rng.uniform(-amp_u, amp_u, size=(Q.shape[0], 3, Q.shape[2])) + np.array(mean)[None, :, None]
    Q[:, 4] += 0.5 * rho * (u ** 2).sum(axis=1) + (Q[:, 1:4] * u).sum(axis=1)
    Q[:, 1:4] += rho[:, None] * u
    Q[:, 4] += rng.uniform(-amp_e, amp_e, size=rho.shape)
    return Q


def _hill_box():
    h = 40000.0 / 128
    return dict(N=4, nex=8, ney=2, nez=4, Lx=8 * h, Ly=2 * h, Lz=4 * h, x0=20000.0 - 4 * h, y0=0.0, z0=0.0,
                periodic=(1, 1, 0), warp=True, hill_h=400.0, hill_a=1000.0, hill_xc=20000.0)


CASES = [("flat fp64", "c2", "fp64", 1e-12), ("flat fp32", "c2", "fp32", 1e-5), ("warped fp32", "c3", "fp32", 1e-5)]


@pytest.mark.parametrize("label,cfg,precision,tol", CASES, ids=[c[0] for c in CASES])
def test_drag_tendency_and_step_against_oracle(orc, label, cfg, precision, tol):
    from paper_2110_00853_b300 import cmles
    if cfg == "c2":
        m = I.sub_mesh("c2", 5, 4, 3)
        ph = dict(I.physics("c2"), drag_cd=CD)
    else:
        m = _hill_box()
        ph = dict(I.physics("c3"), sponge_zs=0.75 * m["Lz"], drag_cd=CD)
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, I.case(cfg))
    Q = _flow(Q, seed=7)
    S0 = orc.from_inputs(m, dict(ph, drag_cd=0.0))
    S0.set_reference(rr, pr)
    G = cmles.Solver(m, ph, precision=precision)
    G0 = cmles.Solver(m, dict(ph, drag_cd=0.0), precision=precision)
    if cfg == "c2":
        ref = (_levels(rr, m), _levels(pr, m), _levels(Q[:, 5] / Q[:, 0], m))
    else:
        ref = (rr.ravel(), pr.ravel(), None)
    G.set_reference(*ref)
    G0.set_reference(*ref)
    R_orc, fails = S.rhs(Q)
    assert fails == 0
    Qd = torch.from_numpy(Q).cuda()
    R_gpu = G.tendency(Qd).cpu().numpy()
    for v in range(5):
        err = _rel(R_gpu[:, v], R_orc[:, v])
        assert err <= tol, (label, v, err)
        assert np.abs(R_gpu[:, v] - R_orc[:, v]).max() <= 10 * tol * np.abs(R_orc[:, v]).max(), (label, v)
    # the drag term alone (with C_d minus without): against the oracle's, on
    # the bottom face nodes only, wall-parallel and against the flow.  Its
    # bound is the tendency's own: the FP32 tendency's rounding (~1e-7 of
    # |R|, 1e-5 at most) over the drag term's share of |R| (~1e-2 here).
    R0_orc, _ = S0.rhs(Q)
    dR = R_gpu - G0.tendency(Qd).cpu().numpy()
    dR_orc = R_orc - R0_orc
    share = np.linalg.norm(dR_orc[:, 1:4]) / np.linalg.norm(R_orc[:, 1:4])
    print(label, "drag share of |R_momentum|", share)
    for v in (1, 2, 3):
        if np.abs(dR_orc[:, v]).max() > 0:
            err = _rel(dR[:, v], dR_orc[:, v])
            assert err <= (1e-10 if precision == "fp64" else 10 * tol / share), (label, v, err)
    Nq = m["N"] + 1
    nxy = m["nex"] * m["ney"]
    assert np.abs(dR[nxy:]).max() <= 1e-4 * np.abs(dR).max()
    bottom = dR[:nxy, 1:4, :Nq * Nq]
    u_int = Q[:nxy, 1:4, Nq * Nq:2 * Nq * Nq] / Q[:nxy, 0:1, Nq * Nq:2 * Nq * Nq]
    work = (bottom * u_int).sum(1)
    # where the term stands above the tendency's rounding
    big = np.linalg.norm(dR_orc[:nxy, 1:4, :Nq * Nq], axis=1) > 1e-3 * np.abs(dR_orc).max()
    assert big.sum() > 0.9 * big.size
    assert (work[big] < 0).all(), label
    # one LSRK step
    G.set_state(Qd)
    G.step(1)
    Qo, _ = S.lsrk54(Q, 1, ph["dt"])
    Qg = G.get_state().cpu().numpy()
    for v in range(5):
        e = _rel(Qg[:, v] - Q[:, v], Qo[:, v] - Q[:, v])
        assert e <= (1e-11 if precision == "fp64" else 1e-5), (label, v, e)
    G.close()
    G0.close()


def test_wall_options_reject_bad_values():
    from paper_2110_00853_b300 import cmles
    with pytest.raises(cmles.CmlesError):
        cmles.Solver(I.sub_mesh("c2", 2, 2, 2), dict(I.physics("c2"), drag_cd=-1.0), precision="fp64")
    with pytest.raises(cmles.CmlesError):
        cmles.Solver(I.sub_mesh("c2", 2, 2, 2), dict(I.physics("c2"), noslip=1 << 6), precision="fp64")


NOSLIP_CASES = [("flat fp64", "c2", "fp64", 1e-12, 0.0), ("flat fp32", "c2", "fp32", 1e-5, 0.0),
                ("flat fp32 with drag", "c2", "fp32", 1e-5, CD), ("warped fp32 with drag", "c3", "fp32", 1e-5, CD)]


@pytest.mark.parametrize("label,cfg,precision,tol,cd", NOSLIP_CASES, ids=[c[0] for c in NOSLIP_CASES])
def test_noslip_walls_against_oracle(orc, label, cfg, precision, tol, cd):
    from paper_2110_00853_b300 import cmles
    if cfg == "c2":
        m = I.sub_mesh("c2", 5, 4, 3)
        ph = dict(I.physics("c2"), drag_cd=cd, noslip=0b110000)
    else:
        m = _hill_box()
        ph = dict(I.physics("c3"), sponge_zs=0.75 * m["Lz"], drag_cd=cd, noslip=0b010000)
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, I.case(cfg))
    Q = _flow(Q, seed=11)
    G = cmles.Solver(m, ph, precision=precision)
    if cfg == "c2":
        G.set_reference(_levels(rr, m), _levels(pr, m), _levels(Q[:, 5] / Q[:, 0], m))
    else:
        G.set_reference(rr.ravel(), pr.ravel(), None)
    R_orc, fails = S.rhs(Q)
    assert fails == 0
    # the no-slip ghost changes the wall tendency: it must differ from free slip
    S_fs = orc.from_inputs(m, dict(ph, noslip=0))
    S_fs.set_reference(rr, pr)
    R_fs, _ = S_fs.rhs(Q)
    assert _rel(R_orc[:, 1], R_fs[:, 1]) > 1e-3
    Qd = torch.from_numpy(Q).cuda()
    R_gpu = G.tendency(Qd).cpu().numpy()
    for v in range(5):
        err = _rel(R_gpu[:, v], R_orc[:, v])
        assert err <= tol, (label, v, err)
        assert np.abs(R_gpu[:, v] - R_orc[:, v]).max() <= 10 * tol * np.abs(R_orc[:, v]).max(), (label, v)
    G.set_state(Qd)
    G.step(1)
    Qo, _ = S.lsrk54(Q, 1, ph["dt"])
    Qg = G.get_state().cpu().numpy()
    for v in range(5):
        e = _rel(Qg[:, v] - Q[:, v], Qo[:, v] - Q[:, v])
        assert e <= (1e-11 if precision == "fp64" else 1e-5), (label, v, e)
    G.close()
