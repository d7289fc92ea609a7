"""Oracle of the kinetic-energy spectrum (test infrastructure only).

The paper judges its turbulence runs by the kinetic-energy spectrum of the
velocity field, computed by a Fourier transform (Sec. 5.5, Decaying
Taylor-Green Vortex).  On the nodal DG field this needs a uniform grid first.
The readings, stated here and used by the library alike:

  1. Velocity at every node: u_i = (rho u_i) / rho.
  2. Uniform resampling: in each direction N points per element at the cell
     centres xi_s = -1 + (2 s + 1) / N (s = 0 .. N-1) of the element's
     reference interval, so the whole mesh gets M_x = nex N by M_y = ney N
     points per level and M_z = nez N levels, none of them on an element
     face; the value at a point is the element's nodal (Lagrange) polynomial
     of degree N in each direction, evaluated there.
  3. On each level, the discrete Fourier coefficients
       u^(p, q) = 1/(M_x M_y) sum_ij u_ij exp(-2 pi i (p i / M_x + q j / M_y)),
     p in [-M_x/2, M_x/2), q in [-M_y/2, M_y/2) (numpy's FFT ordering).
  4. Shell s = round(L sqrt((p / L_x)^2 + (q / L_y)^2)), L = max(L_x, L_y):
     the horizontal wavenumber magnitude in units of 2 pi / L.
  5. E(s) = the level average of sum over the shell of
     (|u^|^2 + |v^|^2 + |w^|^2) / 2.
     By Parseval, sum_s E(s) = the mean over all grid points of |u|^2 / 2.

The mesh is periodic in x and y (the configurations this is used on); z may
be bounded by walls, which is why the transform is horizontal, per level.
"""
import numpy as np

from . import oracle as O


def lagrange_matrix(xi, pts):
    """L[s][a] = l_a(pts[s]), the Lagrange basis of the nodes xi (product formula)."""
    n = len(xi)
    L = np.ones((len(pts), n))
    for a in range(n):
        for b in range(n):
            if b != a:
                L[:, a] *= (pts - xi[b]) / (xi[a] - xi[b])
    return L


def resample(mesh, Q):
    """Steps 1-2: the velocity on the uniform grid, U[3][M_z][M_y][M_x]."""
    N = mesh.N
    Nq = N + 1
    xi, _, _ = O.lgl(N)
    pts = -1.0 + (2.0 * np.arange(N) + 1.0) / N
    L = lagrange_matrix(xi, pts)                                # [N][Nq]
    nex, ney, nez = mesh.nex, mesh.ney, mesh.nez
    E = nex * ney * nez
    Q = np.asarray(Q, float).reshape(E, 6, Nq, Nq, Nq)          # [e][v][k][j][i]
    U = np.zeros((3, nez * N, ney * N, nex * N))
    for c in range(3):
        u = Q[:, 1 + c] / Q[:, 0]                               # [e][k][j][i]
        # apply L along i, j and k: us[e][kz][jy][ix]
        us = np.einsum("xi,ekji->ekjx", L, u)
        us = np.einsum("yj,ekjx->ekyx", L, us)
        us = np.einsum("zk,ekyx->ezyx", L, us)
        us = us.reshape(nez, ney, nex, N, N, N)                 # [ez][ey][ex][kz][jy][ix]
        U[c] = us.transpose(0, 3, 1, 4, 2, 5).reshape(nez * N, ney * N, nex * N)
    return U


def spectrum_from_grid(U, Lx, Ly, nshell):
    """Steps 3-5 on a uniform grid U[3][M_z][M_y][M_x]: E[nshell] (shells
    beyond nshell - 1 are dropped)."""
    _, Mz, My, Mx = U.shape
    Lref = max(Lx, Ly)
    p = np.fft.fftfreq(Mx, 1.0 / Mx)
    q = np.fft.fftfreq(My, 1.0 / My)
    shell = np.rint(Lref * np.sqrt((p[None, :] / Lx) ** 2 + (q[:, None] / Ly) ** 2)).astype(int)
    E = np.zeros(nshell)
    for lev in range(Mz):
        e = np.zeros((My, Mx))
        for c in range(3):
            F = np.fft.fft2(U[c, lev]) / (Mx * My)
            e += 0.5 * np.abs(F) ** 2
        ok = shell < nshell
        E += np.bincount(shell[ok], weights=e[ok], minlength=nshell)[:nshell]
    return E / Mz


def ke_spectrum(mesh, Q, nshell):
    """The kinetic-energy spectrum E[nshell] of the state Q [E][6][Np] on
    `mesh` (an oracle Mesh)."""
    U = resample(mesh, Q)
    return spectrum_from_grid(U, mesh.Lx, mesh.Ly, nshell)
