"""Moving a field between two node grids of one rectangle (CPU, float64).

TEST INFRASTRUCTURE: see the package header for who may import this.

The per-frequency grids of the FWI windows (about ten points per wavelength per
window, the full-FWI configuration after Sec. 4.2) carry the model between the
fine grid and each window's grid.  Node (i, j) of an n_x x n_z grid covering
[0, Lx] x [0, Lz] sits at the cell centre ((i + 1/2) Lx / n_x, (j + 1/2) Lz / n_z);
a value at a point is the bilinear interpolation of the four surrounding source
nodes, the point clamped to the outermost source nodes.
"""
from __future__ import annotations

import numpy as np


def resample(src, nx1: int, nz1: int) -> np.ndarray:
    src = np.asarray(src, dtype=np.float64)
    nz0, nx0 = src.shape
    out = np.zeros((nz1, nx1))
    for j in range(nz1):
        z = min(max((j + 0.5) * nz0 / nz1 - 0.5, 0.0), nz0 - 1.0)
        j0 = min(int(z), nz0 - 1)
        j1 = min(j0 + 1, nz0 - 1)
        fz = z - j0
        for i in range(nx1):
            x = min(max((i + 0.5) * nx0 / nx1 - 0.5, 0.0), nx0 - 1.0)
            i0 = min(int(x), nx0 - 1)
            i1 = min(i0 + 1, nx0 - 1)
            fx = x - i0
            out[j, i] = ((1 - fz) * ((1 - fx) * src[j0, i0] + fx * src[j0, i1]) +
                         fz * ((1 - fx) * src[j1, i0] + fx * src[j1, i1]))
    return out
