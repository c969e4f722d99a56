"""The direct measurement equation, by brute force (oracle pin for Phi).

Eq. 1 and Eq. 2 on the image's pixel grid:
    y_k = sum_{i,j} x[i, j] exp(-2 pi i (u_k l_j + v_k m_i + w_k (sqrt(1 - l_j^2 - m_i^2) - 1)))
          [/ sqrt(1 - l^2 - m^2) when the 1/n factor of Eq. 2 is kept]
with l_j = (j - n_x/2) FoV_x / n_x and m_i = (i - n_y/2) FoV_y / n_y.
O(M N): tiny inputs only.
"""
from __future__ import annotations

import math

import numpy as np

from . import wterm


def direct_phi(x: np.ndarray, uvw: np.ndarray, fov_x: float, fov_y: float,
               div_n: bool = False) -> np.ndarray:
    ny, nx = x.shape
    l = wterm.pixel_lm(nx, fov_x)[None, :]
    m = wterm.pixel_lm(ny, fov_y)[:, None]
    d = wterm.dn(l, m)
    src = np.asarray(x, dtype=np.complex128)
    if div_n:
        src = src / (1.0 + d)
    L = np.broadcast_to(l, (ny, nx)).ravel()
    Mm = np.broadcast_to(m, (ny, nx)).ravel()
    D = d.ravel()
    s = src.ravel()
    y = np.empty(uvw.shape[0], dtype=np.complex128)
    for c0 in range(0, uvw.shape[0], 256):
        u = uvw[c0:c0 + 256]
        ph = np.outer(u[:, 0], L) + np.outer(u[:, 1], Mm) + np.outer(u[:, 2], D)
        y[c0:c0 + 256] = np.exp(-2j * math.pi * ph) @ s
    return y


def direct_phi_adj(y: np.ndarray, uvw: np.ndarray, nx: int, ny: int, fov_x: float,
                   fov_y: float, div_n: bool = False) -> np.ndarray:
    """Adjoint of direct_phi: x[i, j] = sum_k conj(A[k, (i, j)]) y_k."""
    l = wterm.pixel_lm(nx, fov_x)[None, :]
    m = wterm.pixel_lm(ny, fov_y)[:, None]
    d = wterm.dn(l, m)
    L = np.broadcast_to(l, (ny, nx)).ravel()
    Mm = np.broadcast_to(m, (ny, nx)).ravel()
    D = d.ravel()
    out = np.zeros(nx * ny, dtype=np.complex128)
    for c0 in range(0, uvw.shape[0], 256):
        u = uvw[c0:c0 + 256]
        ph = np.outer(u[:, 0], L) + np.outer(u[:, 1], Mm) + np.outer(u[:, 2], D)
        out += np.exp(2j * math.pi * ph).T @ y[c0:c0 + 256]
    out = out.reshape(ny, nx)
    if div_n:
        out = out / (1.0 + d)
    return out
