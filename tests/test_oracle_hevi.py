"""Pins of the oracle's HEVI time stepping (Sec. 3.2): the ARK2 tableaux of
Giraldo, Kelly & Constantinescu (2013) against the order and stability
conditions of additive Runge-Kutta methods, the vertical linear operator
against its structural properties (zero at the reference, conservation of
mass and energy, a dissipative spectrum, one matrix for every vertical line,
the closed-form wall response to a uniform vertical momentum), and the
scheme against second-order convergence in time and stability beyond the
explicit vertical acoustic limit."""
import numpy as np
import pytest

from paper_2110_00853_b300 import inputs as I


def test_ark2_tableaux_order_and_stability(orc):
    Ae, Ai, b = orc.ark2_tableaux()
    c_e, c_i = Ae.sum(1), Ai.sum(1)
    assert np.abs(c_e - c_i).max() < 1e-15                 # shared stage times
    assert abs(b.sum() - 1.0) < 1e-15
    assert abs(b @ c_e - 0.5) < 1e-15                       # second order (both parts, coupled)
    assert np.allclose(np.triu(Ae), 0.0)                    # explicit
    assert Ai[0, 0] == 0.0 and Ai[1, 1] == Ai[2, 2] > 0.0    # explicit first stage, one diagonal value
    assert np.allclose(Ai[2], b)                            # stiffly accurate
    # implicit part's stability function R(z) = 1 + z b^T (I - z Ai)^-1 1:
    # bounded by 1 on the imaginary axis and the negative real axis, -> 0 at infinity
    def R(z):
        return 1.0 + z * (b @ np.linalg.solve(np.eye(3) - z * Ai, np.ones(3)))
    assert all(abs(R(1j * y)) <= 1.0 + 1e-12 for y in np.linspace(0.0, 1e3, 2001))
    assert all(abs(R(-x)) <= 1.0 + 1e-12 for x in np.logspace(-3, 6, 400))
    assert abs(R(-1e9)) < 1e-6


def _bubble(orc, thin=False):
    m, ph, c = I.mesh("c1"), I.physics("c1"), I.case("c1")
    if thin:
        # the bubble box with 20 m thin elements under 1 km wide ones
        m = dict(m, nex=2, ney=2, nez=8, Lx=2000.0, Ly=2000.0, Lz=160.0)
        c = dict(c, zc=80.0, r0=400.0)
    S, Q, rr, pr, _ = orc.from_inputs(m, ph, c)
    return S, Q, m, ph, pr


def test_vertical_operator_structure(orc):
    S, Q, m, ph, pr = _bubble(orc)
    Qr = S.vlin_reference()
    assert np.abs(S.vlin(Qr)).max() == 0.0
    rng = np.random.default_rng(1)
    scale = np.array([1e-3, 1e-1, 1e-1, 1e-1, 1e2, 1e-5])[None, :, None]
    y1, y2 = rng.normal(size=Qr.shape) * scale, rng.normal(size=Qr.shape) * scale
    L1, L2, L12 = S.vlin(Qr + y1), S.vlin(Qr + y2), S.vlin(Qr + 2.0 * y1 - 3.0 * y2)
    assert np.abs(L12 - (2.0 * L1 - 3.0 * L2)).max() <= 1e-12 * np.abs(L12).max()
    # walls top and bottom: mass and energy change only by fluxes, which cancel
    wJ = S.geometry()["wJ"]
    for v in (0, 4, 5, 1, 2):
        tot, mag = (wJ * L1[:, v]).sum(), (wJ * np.abs(L1[:, v])).sum()
        assert abs(tot) <= 1e-13 * mag, v
    # one matrix for every vertical line of the flat mesh, with a dissipative
    # spectrum
    Lm = S.hevi_line_matrix()
    assert np.abs(S.hevi_line_matrix(1, 2, 3, 1) - Lm).max() == 0.0
    ev = np.linalg.eigvals(Lm)
    assert ev.real.max() <= 1e-12 * np.abs(ev).max()
    # uniform vertical momentum m: no interior response in rho; at the walls
    # the mirrored state gives d rho/dt = n_z lift m and d(rho w)/dt = -lift c_r m
    m0 = 2.0
    Lw = S.vlin(Qr + np.array([0, 0, 0, m0, 0, 0.0])[None, :, None])
    g = S.geometry()
    hz = m["Lz"] / m["nez"]
    _, w, _ = orc.lgl(4)
    lift = 2.0 / (hz * w[0])
    zb, zt = g["z"] < 1e-9, g["z"] > m["Lz"] - 1e-9
    inner = ~(zb | zt)
    assert np.abs(Lw[:, 0][inner]).max() <= 1e-12 * lift * m0
    assert np.allclose(Lw[:, 0][zb], -lift * m0, rtol=1e-13) and np.allclose(Lw[:, 0][zt], lift * m0, rtol=1e-13)
    P = orc.CONSTANTS
    c_r = np.sqrt((P["cvd"] + P["Rd"]) / P["cvd"] * pr / Qr[:, 0])
    assert np.allclose(Lw[:, 3][zb], -lift * c_r[zb] * m0, rtol=1e-12)


def test_ark2_hevi_second_order_in_time(orc):
    S, Q, m, ph, _ = _bubble(orc)
    T = 0.2
    sols = [S.ark2_hevi(Q, n, T / n)[0] for n in (8, 16, 32)]
    e1 = np.abs(sols[0] - sols[1])[:, (0, 3, 4)].max()
    e2 = np.abs(sols[1] - sols[2])[:, (0, 3, 4)].max()
    assert 3.0 < e1 / e2 < 5.0, (e1, e2)


def test_ark2_hevi_stable_beyond_the_explicit_vertical_limit(orc):
    """Thin elements (20 m under 1 km): LSRK(5,4) diverges at dt = 0.05 s, the
    vertical acoustic limit being about 0.01 s; ARK2 with the vertical
    operator implicit stays bounded and tracks a small-step LSRK(5,4) run
    (0.002 s) to its own second-order error."""
    S, Q, m, ph, _ = _bubble(orc, thin=True)
    Ql, _ = S.lsrk54(Q, 20, 0.05)
    assert not np.isfinite(Ql).all() or np.abs(Ql[:, 3] / Ql[:, 0]).max() > 100.0
    Qa, fails = S.ark2_hevi(Q, 20, 0.05)
    assert fails == 0 and np.isfinite(Qa).all()
    Qf, _ = S.lsrk54(Q, 500, 0.002)
    for v in (0, 3, 4):
        err = np.linalg.norm(Qa[:, v] - Qf[:, v]) / np.linalg.norm(Qf[:, v] - Q[:, v])
        print("ARK2 HEVI dt 0.05 vs LSRK(5,4) dt 0.002, var", v, err)
        assert err < 0.05, (v, err)
