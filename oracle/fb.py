"""Forward-backward iteration of Eq. 4 with the non-negativity prior (oracle).

Section 2: data fidelity f(x) = 1/2 ||Phi x - y||^2 with gradient Phi^dagger Phi x -
Phi^dagger y; Eq. 4 updates x <- D(x + gamma (x_dirty - Re{Phi^dagger Phi x})) with the
dirty image x_dirty = Re{Phi^dagger y}.  The image model of Eq. 3 is real and
non-negative, so the denoising step used here is the projection onto that set,
D(z) = max(z, 0) (the proximal operator of its indicator), which makes Eq. 4 projected
gradient descent; it converges for 0 < gamma < 2 / L, L = ||Re Phi^dagger Phi||.

This is test infrastructure: only the tests, the smoke check and the
benchmark's CPU-baseline leg use it.
"""
from __future__ import annotations

import numpy as np


def dirty_image(op, y: np.ndarray) -> np.ndarray:
    return op.phi_adj(y).real


def fb_step(op, x: np.ndarray, dirty: np.ndarray, gamma: float) -> np.ndarray:
    """One update of Eq. 4 with D = projection onto x >= 0 (x real)."""
    g = op.phi_adj_phi(x.astype(np.complex128)).real
    return np.maximum(x + gamma * (dirty - g), 0.0)


def objective(op, x: np.ndarray, y: np.ndarray) -> float:
    r = op.phi(x.astype(np.complex128)) - y
    return 0.5 * float(np.vdot(r, r).real)


def lipschitz(op, shape, iters: int = 60, seed: int = 0) -> float:
    """||Re Phi^dagger Phi|| by power iteration on real images."""
    v = np.random.default_rng(seed).standard_normal(shape)
    lam = 0.0
    for _ in range(iters):
        w = op.phi_adj_phi(v.astype(np.complex128)).real
        lam = float(np.vdot(v, w).real / np.vdot(v, v).real)
        v = w / np.linalg.norm(w)
    return lam
