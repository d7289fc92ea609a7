"""Physics check of the whole solver: the 2.5D density current of Sec. 5.2
run to t = 900 s at 50 m effective resolution (200 m elements, N = 4) with
Smagorinsky-Lilly or Vreman (C_s = 0.18, no Richardson correction: the case
is neutral) and the Rusanov flux, on the FP32 path.  The paper reports the
front at 14770 m (SL) and 14739 m (Vreman) for this resolution (Appendix B,
Table t:densityCurrentComparisonTAB; stored in
tests/golden/density_current_front.txt).
The front is read as the largest x where the surface potential-temperature
perturbation reaches -1 K (the paper does not define it); other models in the
same table place it between 14535 and 15027 m at 50 m resolution, so the check
allows 3 %.  The initial state is also compared with the oracle's."""
import os

import numpy as np
import pytest

from paper_2110_00853_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLD = os.path.join(os.path.dirname(__file__), "golden", "density_current_front.txt")


def _front_reference(res_m, closure="sl"):
    for line in open(GOLD):
        if line.strip() and not line.startswith("#"):
            r, f_sl, f_vr = line.split()
            if float(r) == res_m:
                return float(f_sl if closure == "sl" else f_vr)
    raise KeyError(res_m)


def _surface_theta(Q, m, xi):
    """theta at the bottom node row (z = 0) of the dry state, with x"""
    cvd, Rd, T0, p0 = 717.5, 287.0, 273.16, 1.0e5
    Nq = m["N"] + 1
    hx = m["Lx"] / m["nex"]
    xs, th = [], []
    for ex in range(m["nex"]):
        e = ex                                   # ey = ez = 0
        for i in range(Nq):
            n = i                               # j = k = 0
            rho = Q[e, 0, n]
            u = Q[e, 1:4, n] / rho
            T = T0 + (Q[e, 4, n] / rho - 0.5 * u @ u) / cvd
            p = rho * Rd * T
            xs.append((ex + 0.5 * (xi[i] + 1.0)) * hx)
            th.append(T * (p0 / p) ** (Rd / (cvd + Rd)))
    order = np.argsort(xs)
    return np.array(xs)[order], np.array(th)[order]


def test_density_current_initial_state_matches_oracle(orc):
    from paper_2110_00853_b300 import cmles
    m, ph, c = I.mesh("dc"), I.physics("dc"), I.case("dc")
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, c)
    G = cmles.Solver(m, ph, precision="fp32")
    G.init_case(c)
    Qg = G.get_state().cpu().numpy()
    for v in range(5):
        assert np.abs(Qg[:, v] - Q[:, v]).max() <= 1e-12 * np.abs(Q[:, v]).max(), v


@pytest.mark.parametrize("res", [50.0, 100.0])
@pytest.mark.parametrize("closure", ["sl", "vreman"])
def test_density_current_front_at_900s(orc, closure, res):
    from paper_2110_00853_b300 import cmles
    m, ph, c = I.mesh("dc"), I.physics("dc", closure=closure), I.case("dc")
    if res != 50.0:
        # same box, element size 4 res (N = 4), time step scaled with it
        h = 4.0 * res
        m.update(nex=int(round(m["Lx"] / h)), nez=int(round(m["Lz"] / h)), Ly=h)
        ph["dt"] = 0.025 * res / 50.0
    G = cmles.Solver(m, ph, precision="fp32")
    G.init_case(c)
    nsteps = int(round(900.0 / ph["dt"]))
    G.step(nsteps)
    d = G.diagnostics()
    assert not d["nonfinite"]
    Q = G.get_state().cpu().numpy()
    xi, _, _ = orc.lgl(4)
    x, th = _surface_theta(Q, m, xi)
    cold = np.where(th - 300.0 <= -1.0)[0]
    i = cold.max()
    # linear interpolation to the -1 K crossing beyond the last cold node
    front = x[i] + (x[i + 1] - x[i]) * ((th[i] - 299.0) / (th[i] - th[i + 1])) if i + 1 < len(x) else x[i]
    ref = _front_reference(res, closure)
    print("density current front at 900 s,", closure, res, "m:", front, "m; paper:", ref, "m; time", d["time"])
    assert abs(front - ref) <= 0.03 * ref


@pytest.mark.parametrize("flux", ["hllc", "roe"])
def test_density_current_hllc_roe_vreman(orc, flux):
    """Fig. dc(c, d) of Sec. 5.2: the same run with Roe or HLLC faces and
    Vreman stays finite to 900 s, and its front is within 3 % of the paper's
    50 m Vreman value (the table gives no Roe or HLLC row)."""
    from paper_2110_00853_b300 import cmles
    m, ph, c = I.mesh("dc"), I.physics("dc", closure="vreman"), I.case("dc")
    ph["flux"] = flux
    G = cmles.Solver(m, ph, precision="fp32")
    G.init_case(c)
    G.step(int(round(900.0 / ph["dt"])))
    assert not G.diagnostics()["nonfinite"]
    Q = G.get_state().cpu().numpy()
    xi, _, _ = orc.lgl(4)
    x, th = _surface_theta(Q, m, xi)
    i = np.where(th - 300.0 <= -1.0)[0].max()
    front = x[i] + (x[i + 1] - x[i]) * ((th[i] - 299.0) / (th[i] - th[i + 1]))
    ref = _front_reference(50.0, "vreman")
    print("density current front at 900 s, vreman +", flux, front, "m; paper (vreman, 50 m):", ref)
    assert abs(front - ref) <= 0.03 * ref


def test_density_current_lsrk144_double_step(orc):
    """The 14-stage integrator (Sec. 3.2) at twice the 5-stage scheme's time
    step (0.05 s, 18000 steps to 900 s) on the 50 m SL case: stays finite and
    puts the front within 3 % of the paper's value."""
    from paper_2110_00853_b300 import cmles
    m, ph, c = I.mesh("dc"), I.physics("dc", closure="sl"), I.case("dc")
    ph["integrator"] = "lsrk144"
    ph["dt"] = 0.05
    G = cmles.Solver(m, ph, precision="fp32")
    G.init_case(c)
    G.step(int(round(900.0 / ph["dt"])))
    d = G.diagnostics()
    assert not d["nonfinite"] and abs(d["time"] - 900.0) < 1e-6
    Q = G.get_state().cpu().numpy()
    xi, _, _ = orc.lgl(4)
    x, th = _surface_theta(Q, m, xi)
    i = np.where(th - 300.0 <= -1.0)[0].max()
    front = x[i] + (x[i + 1] - x[i]) * ((th[i] - 299.0) / (th[i] - th[i + 1]))
    ref = _front_reference(50.0, "sl")
    print("density current front at 900 s, SL, LSRK(14,4), dt 0.05 s:", front, "m; paper:", ref)
    assert abs(front - ref) <= 0.03 * ref
