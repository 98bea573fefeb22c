"""Channel grid, particle location and trilinear gather (FP64 oracle).

Part of the FP64 CPU oracle: test infrastructure only.

The paper's grid (Sec. 3.1) is periodic in x and z with no-slip walls at
y = 0 and y = 2 delta, refined towards the walls; cells are the control volumes
of the finite-volume discretisation (Sec. 2.2, the charge density of a cell is
the sum of its particles' charges over the cell volume).  Readings:

* x and z cells are uniform; cell i covers [i dx, (i+1) dx).  The y faces are
  an input array (tanh-stretched in the workloads).
* a point on a face belongs to the upper cell; x = Lx belongs to cell 0 after
  wrapping, and the cell index is the largest i with x >= i * dx.
* the gas velocity and the electric field are interpolated trilinearly
  (weights linear in physical coordinates) from a lattice whose x, z nodes are
  the cell centres and whose y nodes are [0, cell centres, 2 delta]; the paper
  does not state its interpolation.
"""
from __future__ import annotations

import numpy as np


class Grid:
    def __init__(self, nx: int, nz: int, lx: float, lz: float, y_faces: np.ndarray):
        self.nx, self.nz = int(nx), int(nz)
        self.lx, self.lz = float(lx), float(lz)
        self.yf = np.asarray(y_faces, dtype=np.float64)
        self.ny = self.yf.shape[0] - 1
        self.ly = float(self.yf[-1])
        self.dx = self.lx / self.nx
        self.dz = self.lz / self.nz
        self.xf = np.arange(self.nx + 1, dtype=np.float64) * self.dx
        self.zf = np.arange(self.nz + 1, dtype=np.float64) * self.dz
        self.dy = np.diff(self.yf)
        self.yc = 0.5 * (self.yf[1:] + self.yf[:-1])
        # wall-extended lattice nodes in y
        self.Y = np.concatenate(([self.yf[0]], self.yc, [self.yf[-1]]))
        # cell volumes, shape (ny,)
        self.vol_y = self.dx * self.dy * self.dz

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    def cell_key(self, i, j, k):
        return (np.asarray(k, np.int64) * self.ny + j) * self.nx + i


def _cell_1d(faces: np.ndarray, s: np.ndarray, n: int) -> np.ndarray:
    idx = np.searchsorted(faces, s, side="right") - 1
    return np.clip(idx, 0, n - 1)


def locate(g: Grid, x, y, z):
    """Cell (i, j, k) containing each point: faces[i] <= s < faces[i+1]."""
    i = _cell_1d(g.xf, np.asarray(x, np.float64), g.nx)
    j = _cell_1d(g.yf, np.asarray(y, np.float64), g.ny)
    k = _cell_1d(g.zf, np.asarray(z, np.float64), g.nz)
    return i, j, k


def trilinear(g: Grid, lattice: np.ndarray, x, y, z) -> np.ndarray:
    """Trilinear interpolation of a lattice field (Nz, Ny+2, Nx, C) at points.

    x, z: periodic, nodes at (i + 1/2) dx.  y: nodes g.Y (walls included).
    Returns (n, C).
    """
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    z = np.asarray(z, np.float64)
    sx = x / g.dx - 0.5
    i0 = np.floor(sx)
    wx = sx - i0
    i0 = i0.astype(np.int64) % g.nx
    i1 = (i0 + 1) % g.nx
    sz = z / g.dz - 0.5
    k0 = np.floor(sz)
    wz = sz - k0
    k0 = k0.astype(np.int64) % g.nz
    k1 = (k0 + 1) % g.nz
    j0 = np.clip(np.searchsorted(g.Y, y, side="right") - 1, 0, g.ny)
    j1 = j0 + 1
    wy = (y - g.Y[j0]) / (g.Y[j1] - g.Y[j0])
    out = np.zeros((x.shape[0], lattice.shape[-1]))
    for kk, fz in ((k0, 1.0 - wz), (k1, wz)):
        for jj, fy in ((j0, 1.0 - wy), (j1, wy)):
            for ii, fx in ((i0, 1.0 - wx), (i1, wx)):
                w = fz * fy * fx
                out += w[:, None] * lattice[kk, jj, ii, :]
    return out
