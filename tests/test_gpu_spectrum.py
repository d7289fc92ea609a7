"""GPU parity of the kinetic-energy spectrum (cmles_spectrum) against the
oracle's (oracle/spectrum.py: the same resampling and shell definition, with
numpy's FFT), on the moist layer with a k^-5/3 random-phase velocity field:
a ragged sub-box and the full 32 x 32 x 16-element coarse mesh of the closure
configuration.  Both are FP64; the bound is 1e-12 of the total energy per
shell."""
import numpy as np
import pytest

from paper_2110_00853_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("sub", [(6, 5, 3), None])
def test_spectrum_matches_the_oracle(orc, sub):
    from oracle import spectrum as SP
    from paper_2110_00853_b300 import cmles
    m = I.mesh("c2") if sub is None else I.sub_mesh("c2", *sub)
    c = I.case("c2")
    c["modes"] = I.velocity_modes(m["Lx"], m["Ly"], m["Lz"], nmodes=500, kmax=40, seed=9)
    G = cmles.Solver(m, I.physics("c2"), precision="fp64")
    G.init_case(c)
    nshell = int(0.75 * m["nex"] * m["N"]) + 2
    Eg = G.spectrum(nshell)
    Q = G.get_state().cpu().numpy()
    M = orc.make_mesh(m["N"], m["nex"], m["ney"], m["nez"], m["Lx"], m["Ly"], m["Lz"], periodic=m["periodic"])
    Eo = SP.ke_spectrum(M, Q, nshell)
    total = Eo.sum()
    assert total > 0 and Eo[1:6].min() > 0
    assert np.abs(Eg - Eo).max() <= 1e-12 * total, np.abs(Eg - Eo).max() / total
    G.close()
