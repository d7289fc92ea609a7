"""GPU parity of the learned closure's training samples (cmles_closure_samples)
against the oracle (oracle/closure.c), sample by sample.

The fine run is the moist layer with a k^-5/3 random-phase velocity field that
reaches the coarse mesh's subgrid scales, as the closure's training runs use
it.  Both sides start from the same FP64 state; the library's samples are FP32
outputs of FP64 arithmetic, so every input and the filtered theta_v agree to
FP32 rounding.  The targets are ratios (tau:S / S:S and tau_th.g / |g|^2):
they are compared per sample against a bound relative to their column's
largest value, over the samples whose denominator is not degenerate, and must
be non-negative everywhere.

Two sizes: a 16 x 16 x 8-element fine box (4000 samples, all compared) and the
full 128 x 128 x 64-element fine mesh of the training configuration (131M
nodes), where sampled coarse elements (interior, at both walls and across the
periodic seam) are compared with the oracle on a 3 x 3 x 3-coarse-element
window around them, which holds every fine node their filter boxes reach.
"""
import numpy as np
import pytest

from paper_2110_00853_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FACTOR = 4


def _fine_case(m, seed=4):
    c = I.case("c4fine")
    c["modes"] = I.velocity_modes(m["Lx"], m["Ly"], m["Lz"], nmodes=2000, kmax=200, seed=seed)
    return c


def _compare(Xg, Tg, thg, Xo, To, tho, label):
    # inputs: per-sample bound relative to the column's largest magnitude
    scale = np.abs(Xo).max(axis=0)
    err = np.abs(Xg - Xo).max(axis=0)
    assert np.all(err <= 1e-6 * scale), (label, err / scale)
    rel = np.linalg.norm(Xg - Xo, axis=0) / np.maximum(np.linalg.norm(Xo, axis=0), 1e-300)
    assert np.all(rel <= 2e-7), (label, rel)
    assert np.abs(thg - tho).max() <= 2e-7 * np.abs(tho).max(), label
    # targets: non-negative everywhere; per sample where the denominator is
    # not degenerate (S:S or |g|^2 above 1e-8 of its largest value)
    assert np.all(Tg >= 0.0), label
    gu = Xo[:, :9].reshape(-1, 3, 3)
    SS = (0.25 * (gu + gu.transpose(0, 2, 1)) ** 2).sum(axis=(1, 2))
    gg = (Xo[:, 9:12] ** 2).sum(axis=1)
    for c, den in ((0, SS), (1, gg)):
        ok = den > 1e-8 * den.max()
        assert ok.mean() > 0.99, label
        tmax = np.abs(To[ok, c]).max()
        d = np.abs(Tg[ok, c] - To[ok, c])
        assert d.max() <= 1e-5 * tmax, (label, c, d.max(), tmax)
        assert np.linalg.norm(d) <= 1e-6 * np.linalg.norm(To[ok, c]), (label, c)


def test_closure_samples_match_the_oracle(orc):
    from paper_2110_00853_b300 import cmles
    m = I.sub_mesh("c4fine", 16, 16, 8)
    ph = I.physics("c4fine")
    G = cmles.Solver(m, ph, precision="fp64")
    G.init_case(_fine_case(m))
    Q = G.get_state().cpu().numpy()
    Xg, Tg, thg = (a.cpu().numpy().astype(np.float64) for a in G.closure_samples(FACTOR, with_thv=True))
    S = orc.from_inputs(m, ph)
    Xo, To, tho = S.closure_samples(Q, FACTOR)
    assert Xg.shape == Xo.shape == (4 * 4 * 2 * 125, 13)
    assert To[:, 0].max() > 0 and To[:, 1].max() > 0
    _compare(Xg, Tg, thg, Xo, To, tho, "16x16x8")
    G.close()


def test_closure_samples_full_fine_mesh_sampled(orc):
    from paper_2110_00853_b300 import cmles
    m = I.mesh("c4fine")
    ph = I.physics("c4fine")
    G = cmles.Solver(m, ph, precision="fp32")
    G.init_case(_fine_case(m))
    Xg, Tg, thg = G.closure_samples(FACTOR, with_thv=True)
    Qd = G.get_state()
    nex, ney, nez = m["nex"], m["ney"], m["nez"]
    cnx, cny, cnz = nex // FACTOR, ney // FACTOR, nez // FACTOR
    Np = G.Np
    hx, hy, hz = m["Lx"] / nex, m["Ly"] / ney, m["Lz"] / nez
    # coarse elements: interior, bottom wall, top wall, periodic seam in x and y
    picks = [(13, 7, 8), (20, 30, 0), (5, 11, cnz - 1), (0, 17, 4), (cnx - 1, 0, 9), (0, cny - 1, cnz - 1)]
    for cx, cy, cz in picks:
        # window of 3 coarse elements per direction; in z it stays inside the walls
        wz0 = min(max(cz - 1, 0), cnz - 3)
        fx = [(FACTOR * (cx - 1) + a) % nex for a in range(3 * FACTOR)]
        fy = [(FACTOR * (cy - 1) + a) % ney for a in range(3 * FACTOR)]
        fz = [FACTOR * wz0 + a for a in range(3 * FACTOR)]
        idx = torch.tensor([x + nex * (y + ney * z) for z in fz for y in fy for x in fx], device="cuda")
        Qw = Qd.index_select(0, idx).cpu().numpy()
        wm = dict(m, nex=3 * FACTOR, ney=3 * FACTOR, nez=3 * FACTOR, Lx=3 * FACTOR * hx, Ly=3 * FACTOR * hy,
                  Lz=3 * FACTOR * hz, x0=0.0, y0=0.0, z0=FACTOR * wz0 * hz, periodic=(0, 0, 0))
        S = orc.from_inputs(wm, ph)
        Xo, To, tho = S.closure_samples(Qw, FACTOR)
        # the window's coarse element that is (cx, cy, cz)
        wc = 1 + 3 * (1 + 3 * (cz - wz0))
        o = slice(wc * Np, wc * Np + Np)
        ce = cx + cnx * (cy + cny * cz)
        g = slice(ce * Np, ce * Np + Np)
        Xgw, Tgw, thgw = (a[g].cpu().numpy().astype(np.float64) for a in (Xg, Tg, thg))
        # windows have walls in x and y where the full mesh is periodic: only
        # the centre coarse element, whose boxes stay inside the window, is compared
        scale = Xg[:, :12].abs().amax(dim=0).cpu().numpy().astype(np.float64)
        err = np.abs(Xgw[:, :12] - Xo[o, :12]).max(axis=0)
        assert np.all(err <= 1e-6 * scale), ((cx, cy, cz), err / scale)
        assert np.abs(Xgw[:, 12] - Xo[o, 12]).max() <= 1e-6 * Xo[o, 12].max()
        assert np.abs(thgw - tho[o]).max() <= 2e-7 * 310.0
        assert np.all(Tgw >= 0.0)
        gu = Xo[o, :9].reshape(-1, 3, 3)
        SS = (0.25 * (gu + gu.transpose(0, 2, 1)) ** 2).sum(axis=(1, 2))
        gg = (Xo[o, 9:12] ** 2).sum(axis=1)
        for c, den in ((0, SS), (1, gg)):
            ok = den > 1e-8 * den.max()
            tmax = np.abs(To[o][ok, c]).max() + 1e-30
            assert np.abs(Tgw[ok, c] - To[o][ok, c]).max() <= 1e-5 * tmax, ((cx, cy, cz), c)
    G.close()
