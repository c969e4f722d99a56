"""Briggs (robust) data weights (oracle).

Section 2 (Eq. 3) applies a density-dependent data weighting, Briggs weighting being the
example it cites, to the data and injects it into the measurement operator.  Briggs'
robust weighting of unit natural weights, written out:

  D_c   = number of visibilities whose (u, v) falls in cell c of the image's Fourier grid
          (n_x x n_y cells of size 1/FoV_x x 1/FoV_y: visibility k is in cell
          (round(u_k FoV_x) mod n_x, round(v_k FoV_y) mod n_y), round = floor(. + 1/2));
  f^2   = (5 * 10^-R)^2 / (sum_c D_c^2 / M);
  w_k   = 1 / (1 + f^2 D_{c(k)}).

R -> +inf gives natural weighting (w = 1), R -> -inf uniform weighting (w proportional to
1 / D_c).  The readings (cell rounding, wrap modulo the grid, no conjugate points) are
listed in the design notes.

This is test infrastructure: only the tests, the smoke check and the
benchmark's CPU-baseline leg use it.
"""
from __future__ import annotations

import numpy as np


def density_cells(uvw: np.ndarray, nx: int, ny: int, fov_x: float, fov_y: float) -> np.ndarray:
    """Flat cell index c(k) = cu * ny + cv of every visibility."""
    uvw = np.asarray(uvw, dtype=np.float64)
    cu = np.floor(uvw[:, 0] * fov_x + 0.5).astype(np.int64) % nx
    cv = np.floor(uvw[:, 1] * fov_y + 0.5).astype(np.int64) % ny
    return cu * ny + cv


def briggs_weights(uvw: np.ndarray, nx: int, ny: int, fov_x: float, fov_y: float,
                   robust: float) -> np.ndarray:
    """w_k of Briggs' robust weighting with parameter R = robust (FP64)."""
    c = density_cells(uvw, nx, ny, fov_x, fov_y)
    M = c.size
    if M == 0:
        return np.zeros(0)
    D = np.bincount(c, minlength=nx * ny).astype(np.float64)
    f2 = (5.0 * 10.0 ** (-robust)) ** 2 / (np.sum(D * D) / M)
    return 1.0 / (1.0 + f2 * D[c])
