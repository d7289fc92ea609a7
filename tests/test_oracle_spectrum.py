"""Pins of the oracle's kinetic-energy spectrum (oracle/spectrum.py): the
uniform resampling reproduces polynomials of degree <= N exactly (it is the
element's own interpolant), a single Fourier mode on the grid puts all its
energy, (A/2)^2 per conjugate pair summed, into its own shell, and Parseval's
identity holds for any field.  The expected values are closed forms; the
shell of a mode is computed here from its integer wavenumbers."""
import math

import numpy as np
import pytest

from oracle import spectrum as SP


def _mesh(orc, N, nex, ney, nez, Lx, Ly, Lz):
    return orc.make_mesh(N, nex, ney, nez, Lx, Ly, Lz, periodic=(1, 1, 0))


@pytest.mark.parametrize("N", [2, 4, 5])
def test_resampling_is_exact_on_polynomials(orc, N):
    M = _mesh(orc, N, 3, 2, 2, 600.0, 400.0, 300.0)
    S = orc.Solver(M, orc.make_params())
    g = S.geometry()
    x, y, z = g["x"], g["y"], g["z"]
    Q = np.zeros((S.E, 6, S.Np))
    rho = 1.2
    fields = [lambda x, y, z: 1e-6 * x ** N - 2e-5 * y * z,
              lambda x, y, z: 3.0 + 1e-4 * (x - 100.0) * (y - 50.0),
              lambda x, y, z: 1e-7 * z ** N + 1e-3 * y]
    Q[:, 0] = rho
    for c, f in enumerate(fields):
        Q[:, 1 + c] = rho * f(x, y, z)
    U = SP.resample(M, Q)
    Mx, My, Mz = 3 * N, 2 * N, 2 * N
    xs = (np.arange(Mx) + 0.5) * 600.0 / Mx
    ys = (np.arange(My) + 0.5) * 400.0 / My
    zs = (np.arange(Mz) + 0.5) * 300.0 / Mz
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    for c, f in enumerate(fields):
        ref = f(X, Y, Z)
        assert np.abs(U[c] - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max()), (N, c)


@pytest.mark.parametrize("p0,q0,Lx,Ly", [(3, 0, 1000.0, 1000.0), (2, 5, 1000.0, 1000.0), (4, 1, 2000.0, 1000.0),
                                         (0, 7, 1000.0, 1000.0)])
def test_single_mode_lands_in_one_shell(p0, q0, Lx, Ly):
    Mx, My, Mz = 32, 24, 3
    A = [1.5, -0.7, 0.25]
    i = np.arange(Mx)[None, :]
    j = np.arange(My)[:, None]
    U = np.zeros((3, Mz, My, Mx))
    for c in range(3):
        for lev in range(Mz):
            U[c, lev] = A[c] * np.cos(2 * math.pi * (p0 * i / Mx + q0 * j / My) + 0.3 * c + lev)
    s0 = round(max(Lx, Ly) * math.sqrt((p0 / Lx) ** 2 + (q0 / Ly) ** 2))
    E = SP.spectrum_from_grid(U, Lx, Ly, 40)
    want = sum(a * a for a in A) / 4.0          # (A/2)^2 for each of the two conjugate modes, / 2
    assert abs(E[s0] - want) <= 1e-13 * want
    others = np.delete(E, s0)
    assert np.abs(others).max() <= 1e-13 * want


def test_parseval_random_field():
    rng = np.random.default_rng(4)
    U = rng.normal(size=(3, 4, 20, 30))
    E = SP.spectrum_from_grid(U, 3000.0, 2000.0, 200)
    assert abs(E.sum() - 0.5 * (U ** 2).sum(axis=0).mean()) <= 1e-13 * E.sum()


def test_state_with_one_mode(orc):
    """Through the whole pipeline: a state whose velocity is one smooth mode
    (resolved many times over) keeps all but 1e-6 of its energy in that
    mode's shell, and the total is the mean of |u|^2 / 2 on the grid."""
    N = 4
    M = _mesh(orc, N, 8, 8, 2, 1000.0, 1000.0, 200.0)
    S = orc.Solver(M, orc.make_params())
    g = S.geometry()
    Q = np.zeros((S.E, 6, S.Np))
    Q[:, 0] = 1.1
    Q[:, 1] = 1.1 * 2.0 * np.cos(2 * math.pi * (1 * g["x"] + 2 * g["y"]) / 1000.0)
    E = SP.ke_spectrum(M, Q, 48)
    s0 = round(math.sqrt(5.0))
    assert abs(E[s0] - 1.0) <= 1e-4
    assert (E.sum() - E[s0]) <= 1e-6 * E[s0]
