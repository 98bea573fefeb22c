"""Charge deposition, finite-volume Poisson solve and E = -grad(phi) (FP64).

Part of the FP64 CPU oracle: test infrastructure only.

Sec. 2.2: the electric field is E = -grad(phi) with laplacian(phi) = -rho_el/eps,
where the charge density of a grid cell is the sum of its particles' charges
divided by the cell volume.  Sec. 3.1: the electrostatic equation is
discretised to second order with finite volumes; the walls are grounded
conductors (phi = 0, Sec. 4.2 discussion of the image-charge attraction).

Readings (the paper states neither the stencil nor the gradient scheme):
* FV operator per cell (i, j, k), 3-point central differences in x and z and
  the flux form in y on the stretched grid,
    (phi[i+1] - 2 phi[i] + phi[i-1]) / dx^2 + (same in z)
    + [ (phi[j+1]-phi[j]) / (yc[j+1]-yc[j]) - (phi[j]-phi[j-1]) / (yc[j]-yc[j-1]) ] / dy[j]
  with phi = 0 on the wall faces, a distance dy[0]/2 (dy[Ny-1]/2) from the
  first (last) centre.
* The operator is diagonalised in x, z by the discrete Fourier transform with
  modified wavenumbers lam(m) = (4/dx^2) sin^2(pi m / Nx); each (m_x, m_z)
  pencil is a tridiagonal system in y, solved by the Thomas algorithm.  This is
  an exact direct solver of the FV system above.
* Gradient (Gauss-linear): E_x, E_z by central differences; E_y from face
  values linearly interpolated between centres, phi = 0 on the wall faces.
  On the wall nodes of the gather lattice E_x = E_z = 0 (tangential field of a
  conductor) and E_y is the one-sided difference to the wall face.
"""
from __future__ import annotations

import numpy as np

from .grid import Grid


def deposit(g: Grid, q, i, j, k) -> np.ndarray:
    """Cell charge density rho[k, j, i] = sum of charges in the cell / volume."""
    rho = np.zeros((g.nz, g.ny, g.nx))
    np.add.at(rho, (np.asarray(k), np.asarray(j), np.asarray(i)), np.asarray(q, np.float64))
    rho /= g.vol_y[None, :, None]
    return rho


def y_coefficients(g: Grid):
    """Off-diagonals (lower a, upper c) and diagonal b of the y FV operator.

    Row j: a[j] phi[j-1] + b[j] phi[j] + c[j] phi[j+1]; a[0] = c[Ny-1] = 0 and
    the wall terms sit in b.
    """
    ny = g.ny
    dyc = np.diff(g.yc)                      # centre spacings, ny-1
    a = np.zeros(ny)
    c = np.zeros(ny)
    a[1:] = 1.0 / (g.dy[1:] * dyc)
    c[:-1] = 1.0 / (g.dy[:-1] * dyc)
    b = -(a + c)
    b[0] -= 1.0 / (g.dy[0] * (g.yc[0] - g.yf[0]))
    b[-1] -= 1.0 / (g.dy[-1] * (g.yf[-1] - g.yc[-1]))
    return a, b, c


def modified_wavenumbers(n: int, h: float) -> np.ndarray:
    m = np.arange(n)
    return (4.0 / h ** 2) * np.sin(np.pi * m / n) ** 2


def thomas(a, b, c, r):
    """Thomas algorithm for a tridiagonal system along axis 0.

    a, b, c have shape (n, ...) broadcastable to r (n, ...).
    """
    n = r.shape[0]
    cp = np.empty(np.broadcast_shapes(np.shape(b), np.shape(r)), dtype=np.float64)
    dp = np.empty(r.shape, dtype=np.result_type(r, np.float64))
    den = b[0]
    cp[0] = c[0] / den
    dp[0] = r[0] / den
    for j in range(1, n):
        den = b[j] - a[j] * cp[j - 1]
        cp[j] = c[j] / den
        dp[j] = (r[j] - a[j] * dp[j - 1]) / den
    x = np.empty_like(dp)
    x[n - 1] = dp[n - 1]
    for j in range(n - 2, -1, -1):
        x[j] = dp[j] - cp[j] * x[j + 1]
    return x


def poisson(g: Grid, rho: np.ndarray, eps: float) -> np.ndarray:
    """Solve the FV system L phi = -rho / eps with grounded walls.

    rho, phi have shape (Nz, Ny, Nx).
    """
    rhs = -np.asarray(rho, np.float64) / eps
    spec = np.fft.fft(np.fft.fft(rhs, axis=2), axis=0)      # (mz, j, mx)
    lam = (modified_wavenumbers(g.nz, g.dz)[:, None]
           + modified_wavenumbers(g.nx, g.dx)[None, :])       # (mz, mx)
    a, b, c = y_coefficients(g)
    # pencils along y: move j to axis 0
    r = np.moveaxis(spec, 1, 0)                              # (j, mz, mx)
    bb = b[:, None, None] - lam[None, :, :]
    sol = thomas(a[:, None, None], bb, c[:, None, None], r)
    sol = np.moveaxis(sol, 0, 1)
    phi = np.fft.ifft(np.fft.ifft(sol, axis=0), axis=2)
    return phi.real.copy()


def fv_apply(g: Grid, phi: np.ndarray) -> np.ndarray:
    """Apply the FV operator (stencil form, walls grounded) to phi."""
    ddx = (np.roll(phi, -1, axis=2) - 2 * phi + np.roll(phi, 1, axis=2)) / g.dx ** 2
    ddz = (np.roll(phi, -1, axis=0) - 2 * phi + np.roll(phi, 1, axis=0)) / g.dz ** 2
    ny = g.ny
    up = np.zeros_like(phi)
    lo = np.zeros_like(phi)
    dyc = np.diff(g.yc)
    # flux through the upper face of cell j (into j+1), and the lower face
    up[:, :-1, :] = (phi[:, 1:, :] - phi[:, :-1, :]) / dyc[None, :, None]
    up[:, -1, :] = (0.0 - phi[:, -1, :]) / (g.yf[-1] - g.yc[-1])
    lo[:, 1:, :] = (phi[:, 1:, :] - phi[:, :-1, :]) / dyc[None, :, None]
    lo[:, 0, :] = (phi[:, 0, :] - 0.0) / (g.yc[0] - g.yf[0])
    ddy = (up - lo) / g.dy[None, :, None]
    assert ddy.shape[1] == ny
    return ddx + ddy + ddz


def dense_poisson(g: Grid, rho: np.ndarray, eps: float) -> np.ndarray:
    """Direct dense solve of the same FV system (tiny grids only)."""
    n = g.ncells
    A = np.zeros((n, n))
    for col in range(n):
        e = np.zeros(n)
        e[col] = 1.0
        A[:, col] = fv_apply(g, e.reshape(g.nz, g.ny, g.nx)).ravel()
    sol = np.linalg.solve(A, (-np.asarray(rho, np.float64) / eps).ravel())
    return sol.reshape(g.nz, g.ny, g.nx)


def efield(g: Grid, phi: np.ndarray) -> np.ndarray:
    """E = -grad(phi) on the wall-extended lattice, shape (Nz, Ny+2, Nx, 3)."""
    nz, ny, nx = phi.shape
    E = np.zeros((nz, ny + 2, nx, 3))
    E[:, 1:-1, :, 0] = -(np.roll(phi, -1, axis=2) - np.roll(phi, 1, axis=2)) / (2 * g.dx)
    E[:, 1:-1, :, 2] = -(np.roll(phi, -1, axis=0) - np.roll(phi, 1, axis=0)) / (2 * g.dz)
    # face values: phi_f[0] = phi_f[ny] = 0, interior by linear interpolation
    phif = np.zeros((nz, ny + 1, nx))
    wgt = (g.yf[1:-1] - g.yc[:-1]) / (g.yc[1:] - g.yc[:-1])          # ny-1
    phif[:, 1:-1, :] = phi[:, :-1, :] + wgt[None, :, None] * (phi[:, 1:, :] - phi[:, :-1, :])
    E[:, 1:-1, :, 1] = -(phif[:, 1:, :] - phif[:, :-1, :]) / g.dy[None, :, None]
    E[:, 0, :, 1] = -(phi[:, 0, :] - 0.0) / (g.yc[0] - g.yf[0])
    E[:, -1, :, 1] = -(0.0 - phi[:, -1, :]) / (g.yf[-1] - g.yc[-1])
    return E
