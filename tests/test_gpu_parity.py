"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
the same seeded inputs, element by element.

Tolerance (FP64 path): relative L2 per tendency variable <= 1e-12, the bar
for the plain FP64 method (a few hundred roundings of 1e-16 each, with the
oracle's different summation order).  Inputs come from the
oracle's own initial-state code (or are seeded fuzz on top of it); no expected
value comes from the CUDA path.
"""
import numpy as np
import pytest

from paper_2110_00853_b300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _levels(S_orc, arr, mesh):
    """per-node oracle array [E][Np] -> per node level (ez, k) values"""
    Nq = mesh["N"] + 1
    out = np.zeros(mesh["nez"] * Nq)
    for ez in range(mesh["nez"]):
        e = ez * mesh["nex"] * mesh["ney"]
        for k in range(Nq):
            out[ez * Nq + k] = arr[e, k * Nq * Nq]
    return out


def _fuzz(Q, seed, amp_u=3.0, amp_rho=1e-3, amp_e=50.0):
    rng = np.random.default_rng(seed)
    Q = Q.copy()
    rho = Q[:, 0]
    u = rng.uniform(-amp_u, amp_u, size=(Q.shape[0], 3, Q.shape[2]))
    Q[:, 4] += 0.5 * rho * (u ** 2).sum(axis=1) + (Q[:, 1:4] * u).sum(axis=1)
    Q[:, 1:4] += rho[:, None] * u
    Q[:, 0] *= 1.0 + rng.uniform(-amp_rho, amp_rho, size=rho.shape)
    Q[:, 4] += rng.uniform(-amp_e, amp_e, size=rho.shape)
    return Q


def _setup(orc, name, mesh, phys=None, case=None, fuzz_seed=None, smooth_u=None):
    from paper_2110_00853_b300 import cmles
    phys = phys or I.physics(name)
    case = case or I.case(name)
    S, Q, rr, pr, _ = orc.from_inputs(mesh, phys, case)
    if fuzz_seed is not None:
        Q = _fuzz(Q, fuzz_seed)
    G = cmles.Solver(mesh, phys, precision="fp64")
    qt_lev = None
    G.set_reference(_levels(S, rr, mesh), _levels(S, pr, mesh), qt_lev)
    return S, Q, G


def _rel_l2(a, b):
    return np.sqrt(((a - b) ** 2).sum()) / max(np.sqrt((b ** 2).sum()), 1e-300)


def _compare_rhs(S, Q, G, tol):
    R_orc, fails = S.rhs(Q)
    assert fails == 0
    Qd = torch.from_numpy(Q).cuda()
    R_gpu = G.tendency(Qd).cpu().numpy()
    torch.cuda.synchronize()
    errs = [_rel_l2(R_gpu[:, v], R_orc[:, v]) for v in range(6)]
    for v in range(6):
        if np.abs(R_orc[:, v]).max() == 0.0:
            assert np.abs(R_gpu[:, v]).max() == 0.0
        else:
            assert errs[v] <= tol, (v, errs)
            # node by node as well: a wrong value on a few nodes (one face)
            # can hide in the norm over the whole field
            node_err = np.abs(R_gpu[:, v] - R_orc[:, v]).max()
            assert node_err <= 10 * tol * np.abs(R_orc[:, v]).max(), (v, node_err, np.abs(R_orc[:, v]).max())
    return errs, R_gpu, R_orc


def test_tendency_c1_dry_bubble(orc):
    S, Q, G = _setup(orc, "c1", I.mesh("c1"), fuzz_seed=1)
    _compare_rhs(S, Q, G, 1e-12)


def test_tendency_c2_moist_ragged(orc):
    # moist layer with saturation adjustment, sponge and surface fluxes on a
    # 5 x 3 x 16 sub-box (odd element counts: ragged grid-stride tail)
    m = I.sub_mesh("c2", 5, 3, 16)
    S, Q, G = _setup(orc, "c2", m, fuzz_seed=2)
    S.rhs(Q)
    assert (S.intermediates()["aux"][:, 3] > 0).mean() > 0.1   # saturated nodes present
    _compare_rhs(S, Q, G, 1e-12)


def test_tendency_walls_all_sides_and_rotation(orc):
    m = I.sub_mesh("c1", 3, 2, 3)
    m["periodic"] = (0, 0, 0)
    ph = I.physics("c1")
    ph.update(Omega=(0.0, 1e-4, 7.29e-5), sponge_alpha=0.2, sponge_zs=900.0, u_relax=(1.0, -0.5, 0.0))
    S, Q, G = _setup(orc, "c1", m, phys=ph, fuzz_seed=3)
    _compare_rhs(S, Q, G, 1e-12)


def test_tendency_closure_none_and_no_richardson(orc):
    for kw in (dict(closure="none"), dict(richardson=False)):
        ph = I.physics("c1")
        ph.update(kw)
        S, Q, G = _setup(orc, "c1", I.mesh("c1"), phys=ph, fuzz_seed=4)
        _compare_rhs(S, Q, G, 1e-12)


@pytest.mark.parametrize("richardson", [True, False])
def test_tendency_vreman(orc, richardson):
    # Vreman closure (Eq. vreman-sgs) on the moist sub-box with anisotropic
    # elements (200 x 200 x 120 m): Delta_m differs per direction
    m = I.sub_mesh("c2", 5, 3, 16)
    m["Lz"] = 16 * 120.0
    ph = I.physics("c2", closure="vreman")
    ph["richardson"] = richardson
    S, Q, G = _setup(orc, "c2", m, phys=ph, fuzz_seed=6)
    S.rhs(Q)
    assert np.abs(S.intermediates()["nut"]).max() > 0.0
    _compare_rhs(S, Q, G, 1e-12)


@pytest.mark.parametrize("flux", ["hllc", "roe"])
@pytest.mark.parametrize("case", ["walls", "moist"])
def test_tendency_hllc_roe(orc, case, flux):
    # HLLC or Roe faces (Sec. 3.1): walls on all sides with rotation, or the
    # ragged moist sub-box with saturation, sponge and surface fluxes
    if case == "walls":
        m = I.sub_mesh("c1", 3, 2, 3)
        m["periodic"] = (0, 0, 0)
        ph = I.physics("c1")
        ph.update(Omega=(0.0, 1e-4, 7.29e-5), sponge_alpha=0.2, sponge_zs=900.0)
        name = "c1"
    else:
        m = I.sub_mesh("c2", 5, 3, 16)
        ph = I.physics("c2")
        name = "c2"
    ph["flux"] = flux
    S, Q, G = _setup(orc, name, m, phys=ph, fuzz_seed=8)
    errs, R_gpu, R_orc = _compare_rhs(S, Q, G, 1e-12)
    # the flux differs from Rusanov on these states
    ph2 = dict(ph, flux="rusanov")
    S2, _, _ = _setup(orc, name, m, phys=ph2, fuzz_seed=8)
    R_rus, _ = S2.rhs(Q)
    assert np.abs(R_rus - R_orc).max() > 1e-6 * np.abs(R_orc).max()


ALPHA = -np.log(2.0 ** -52)


@pytest.mark.parametrize("order,mask", [(64, 0b1110), (4, 0b0100)])
def test_exponential_filter(orc, order, mask):
    # Eq. exponential_filter on the momentum: one application on a fuzzed
    # state, then one LSRK step followed by the filter (as cmles_step does)
    m = I.sub_mesh("c2", 5, 3, 16)
    ph = dict(I.physics("c2"), filter_order=order, filter_alpha=ALPHA, filter_vars=mask)
    S, Q, G = _setup(orc, "c2", m, phys=ph, fuzz_seed=9)
    G.set_state(torch.from_numpy(Q).cuda())
    G.filter()
    got = G.get_state().cpu().numpy()
    want = S.filter(Q, order, ALPHA, mask)
    for v in range(6):
        assert _rel_l2(got[:, v], want[:, v]) <= 1e-14, v
    assert np.abs(want[:, 2] - Q[:, 2]).max() > 1e-3 * np.abs(Q[:, 2]).max()
    Q1, fails = S.lsrk54(Q, 1, ph["dt"])
    assert fails == 0
    want1 = S.filter(Q1, order, ALPHA, mask)
    G.set_state(torch.from_numpy(Q).cuda())
    G.step(1)
    got1 = G.get_state().cpu().numpy()
    for v in range(6):
        d_g, d_o = got1[:, v] - Q[:, v], want1[:, v] - Q[:, v]
        assert _rel_l2(d_g, d_o) <= 1e-12, v


def test_filter_off_by_default(orc):
    from paper_2110_00853_b300 import cmles
    S, Q, G = _setup(orc, "c1", I.mesh("c1"))
    with pytest.raises(cmles.CmlesError):
        G.filter()


def test_single_element_periodic_degenerate(orc):
    # one element periodic in x and y: every neighbour is the element itself
    m = I.sub_mesh("c1", 1, 1, 2)
    S, Q, G = _setup(orc, "c1", m, fuzz_seed=5)
    _compare_rhs(S, Q, G, 1e-12)


def test_single_element_box_walls_everywhere(orc):
    # one element, six walls: every face is a boundary face
    m = I.sub_mesh("c1", 1, 1, 1)
    m["periodic"] = (0, 0, 0)
    S, Q, G = _setup(orc, "c1", m, fuzz_seed=6)
    _compare_rhs(S, Q, G, 1e-12)


def test_lsrk_steps_and_budgets(orc):
    m = I.sub_mesh("c2", 3, 4, 16)
    ph = I.physics("c2")
    S, Q, G = _setup(orc, "c2", m, phys=ph, fuzz_seed=6)
    nsteps = 3
    Q_orc, fails = S.lsrk54(Q, nsteps, ph["dt"])
    assert fails == 0
    G.set_state(torch.from_numpy(Q).cuda())
    G.step(nsteps)
    Q_gpu = G.get_state().cpu().numpy()
    for v in range(6):
        d = Q_gpu[:, v] - Q_orc[:, v]
        assert _rel_l2(Q_gpu[:, v] - Q[:, v], Q_orc[:, v] - Q[:, v]) <= 1e-11, v
    diag = G.diagnostics()
    b_orc, _ = S.budgets(Q_orc)
    assert np.allclose(diag["budget"], b_orc, rtol=1e-13, atol=0)
    assert diag["steps"] == nsteps and not diag["nonfinite"]


def test_lsrk144_steps_and_budgets(orc):
    # the 14-stage integrator of Sec. 3.2 (Niegemann, Diehl & Busch 2012) at
    # twice the 5-stage scheme's step, against the oracle's
    m = I.sub_mesh("c2", 3, 4, 16)
    ph = dict(I.physics("c2"), integrator="lsrk144")
    ph["dt"] *= 2.0
    S, Q, G = _setup(orc, "c2", m, phys=ph, fuzz_seed=7)
    nsteps = 2
    Q_orc, fails = S.lsrk144(Q, nsteps, ph["dt"])
    assert fails == 0
    G.set_state(torch.from_numpy(Q).cuda())
    G.step(nsteps)
    Q_gpu = G.get_state().cpu().numpy()
    for v in range(6):
        assert _rel_l2(Q_gpu[:, v] - Q[:, v], Q_orc[:, v] - Q[:, v]) <= 1e-11, v
    diag = G.diagnostics()
    b_orc, _ = S.budgets(Q_orc)
    # mass, energy and water relative to themselves; the momentum budgets are
    # sums of both signs, relative to the mass times the fuzz speed (a few m/s)
    for v in (0, 4, 5):
        assert abs(diag["budget"][v] - b_orc[v]) <= 1e-13 * abs(b_orc[v]), v
    for v in (1, 2, 3):
        assert abs(diag["budget"][v] - b_orc[v]) <= 1e-13 * 10.0 * abs(b_orc[0]), v
    assert diag["steps"] == nsteps and abs(diag["time"] - nsteps * ph["dt"]) < 1e-12


def test_determinism(orc):
    S, Q, G = _setup(orc, "c1", I.mesh("c1"), fuzz_seed=7)
    Qd = torch.from_numpy(Q).cuda()
    a = G.tendency(Qd).cpu().numpy()
    b = G.tendency(Qd).cpu().numpy()
    assert np.array_equal(a, b)


def test_kernel_timing_and_launch_counters(orc):
    # per-pass CUDA-event timing (the numbers bench.py reports) and the
    # launch counter: two passes per stage, five stages per step
    S, Q, G = _setup(orc, "c1", I.mesh("c1"), fuzz_seed=7)
    G.set_state(torch.from_numpy(Q).cuda())
    G.step(1)
    n0 = G.launch_count()
    G.enable_timing(True)
    G.kernel_times()
    G.step(3)
    kt = G.kernel_times()
    G.enable_timing(False)
    assert G.launch_count() - n0 == 3 * 5 * 2
    assert kt["count"][0] == 15 and kt["count"][1] == 15
    assert kt["ms"][0] > 0.0 and kt["ms"][1] > 0.0


def test_conservation_on_gpu(orc):
    m = I.sub_mesh("c2", 4, 4, 16)
    ph = I.physics("c2")
    ph["surface_flux"] = False
    S, Q, G = _setup(orc, "c2", m, phys=ph, fuzz_seed=8)
    G.set_state(torch.from_numpy(Q).cuda())
    b0 = G.diagnostics()["budget"]
    G.step(10)
    b1 = G.diagnostics()["budget"]
    for v in (0, 4, 5):
        assert abs(b1[v] - b0[v]) <= 1e-14 * abs(b0[v]) * 10, (v, b0[v], b1[v])


def test_initial_state_builder_matches_oracle(orc):
    from paper_2110_00853_b300 import cmles
    for name, m in (("c1", I.mesh("c1")), ("c2", I.sub_mesh("c2", 4, 3, 16)), ("c5", I.sub_mesh("c5", 3, 3, 8))):
        ph = I.physics(name)
        c = I.case(name)
        S, Q, rr, pr, _ = orc.from_inputs(m, ph, c)
        G = cmles.Solver(m, ph, precision="fp64")
        G.init_case(c)
        Qg = G.get_state().cpu().numpy()
        for v in range(6):
            scale = np.abs(Q[:, v]).max() + 1e-300
            tol = 1e-12 if (name != "c5" or v in (0, 5)) else 1e-6
            if name == "c5" and v in (1, 2, 3, 4):
                # the builder evaluates the 1000 velocity-mode cosines in FP32
                # (FP64 sums): absolute error well below 1e-6 of rho * u_rms
                scale = max(scale, np.abs(Q[:, 0]).max() * 1.0)
                tol = 2e-6 if v != 4 else 1e-9
            assert np.abs(Qg[:, v] - Q[:, v]).max() <= tol * scale, (name, v)


def test_profiles_match_oracle(orc):
    m = I.sub_mesh("c2", 4, 4, 8)
    S, Q, G = _setup(orc, "c2", m, fuzz_seed=9)
    G.set_state(torch.from_numpy(Q).cuda())
    pg = G.profiles()
    po = orc.Solver.favre_profiles(S, Q)
    assert np.allclose(pg, po, rtol=1e-10, atol=1e-12)
