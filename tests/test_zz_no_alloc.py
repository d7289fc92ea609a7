"""The allocation-free budget entry point (cmles_budgets_noalloc), for callers
that cannot call cudaMalloc, against the handle's own budget reduction
(cmles_diagnostics) on two calls in a row.  Collected last on purpose: its
scratch array is shared process-wide, and it must pass both alone and after
every other test."""
import ctypes

import numpy as np
import pytest

from paper_2110_00853_b300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_budgets_noalloc_matches_diagnostics_twice():
    from paper_2110_00853_b300 import cmles
    L = cmles.load()
    m = I.sub_mesh("c2", 5, 3, 16)
    G = cmles.Solver(m, I.physics("c2"), precision="fp64")
    G.init_case(I.case("c2"))
    J = (m["Lx"] / m["nex"]) * (m["Ly"] / m["ney"]) * (m["Lz"] / m["nez"]) / 8.0
    out = torch.full((7,), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        Q = G.get_state()
        st = L.cmles_budgets_noalloc(ctypes.c_void_p(Q.data_ptr()), G.E, G.N, J, ctypes.c_void_p(out.data_ptr()),
                                     stream)
        assert st == 0
        got = out.cpu().numpy()
        ref = G.diagnostics()["budget"]
        # summation order differs between the two reductions: compare to
        # 1e-13 of the sum of |w J Q_v| (an upper bound is J * sum |Q_v|)
        scale = J * Q.abs().sum(dim=(0, 2)).cpu().numpy()
        assert np.all(np.abs(got[:6] - ref) <= 1e-13 * scale), (call, got, ref)
        assert got[6] == 0.0
        G.step(1)     # the second call sees a different state


@pytest.mark.parametrize("N,nel", [(1, (3, 2, 2)), (3, (4, 3, 2)), (7, (2, 2, 3)), (2, (16, 12, 8))])
def test_budgets_noalloc_other_orders_match_the_oracle(orc, N, nel):
    """Orders other than the handle's: the entry point computes its own LGL
    weights, so each order is checked against the oracle's budgets of the same
    seeded state (1e-13 of the summed magnitudes).  The last case has 1536
    elements, 24 blocks in the final fixed-order reduction."""
    from paper_2110_00853_b300 import cmles
    L = cmles.load()
    nex, ney, nez = nel
    M = orc.make_mesh(N, nex, ney, nez, 300.0 * nex, 200.0 * ney, 100.0 * nez)
    S = orc.Solver(M, orc.make_params())
    rng = np.random.default_rng(10 + N)
    Q = rng.uniform(0.5, 1.5, size=(S.E, 6, S.Np))
    Q[:, 1:4] -= 1.0
    ref, bad = S.budgets(Q)
    assert not bad
    J = 300.0 * 200.0 * 100.0 / 8.0
    Qd = torch.from_numpy(Q).cuda()
    out = torch.full((7,), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        st = L.cmles_budgets_noalloc(ctypes.c_void_p(Qd.data_ptr()), S.E, N, J, ctypes.c_void_p(out.data_ptr()),
                                     stream)
        assert st == 0
        got = out.cpu().numpy()
        scale = J * np.abs(Q).sum(axis=(0, 2))
        assert np.all(np.abs(got[:6] - ref) <= 1e-13 * scale), (N, call, got, ref)
        assert got[6] == 0.0


def test_budgets_noalloc_rejects_sizes_beyond_its_limit():
    from paper_2110_00853_b300 import cmles
    L = cmles.load()
    out = torch.zeros(7, dtype=torch.float64, device="cuda")
    Q = torch.zeros(6 * 125, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p
    assert L.cmles_budgets_noalloc(p(Q.data_ptr()), 2 ** 21 + 1, 4, 1.0, p(out.data_ptr()), None) == 1
    assert L.cmles_budgets_noalloc(p(Q.data_ptr()), 1, 8, 1.0, p(out.data_ptr()), None) == 1
    assert L.cmles_budgets_noalloc(None, 1, 4, 1.0, p(out.data_ptr()), None) == 1
