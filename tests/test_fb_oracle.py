"""Pins of the oracle's forward-backward iteration (Eq. 4, non-negativity prior; CPU only).

The iterates must approach the constrained least-squares solution that SciPy's NNLS finds
on the same (real-ified, tiny) problem, decrease the data fidelity monotonically, and the
power-iteration bound must equal the largest eigenvalue of the dense normal matrix.
"""
import math

import numpy as np
import scipy.optimize as so

import synth
from oracle import fb, operator, plan as pl


def tiny():
    n = 8
    uvw = synth.make_uvw(60, 30, 1.28e9, 13) * np.array([0.02, 0.02, 0.002])
    fov = math.radians(6.0)
    pp = pl.PlanParams(nx=n, ny=n, fov_x=fov, fov_y=fov, n_wbins=1, max_wsupport=5, w_norm_frac=1.0)
    op = operator.Operator(uvw, pl.make_plan(uvw, pp))
    # dense Phi by columns
    A = np.zeros((uvw.shape[0], n * n), dtype=np.complex128)
    for j in range(n * n):
        e = np.zeros((n, n))
        e.flat[j] = 1.0
        A[:, j] = op.phi(e.astype(np.complex128))
    rng = np.random.default_rng(4)
    xt = np.maximum(rng.standard_normal((n, n)), 0.0)
    y = A @ xt.ravel() + 0.05 * (rng.standard_normal(uvw.shape[0]) + 1j * rng.standard_normal(uvw.shape[0]))
    return op, A, y, (n, n)


def test_lipschitz_is_the_top_eigenvalue_of_the_normal_matrix():
    op, A, _, shape = tiny()
    N = (A.conj().T @ A).real
    top = float(np.linalg.eigvalsh(N)[-1])
    assert abs(fb.lipschitz(op, shape, iters=200) - top) < 1e-6 * top


def test_fb_descends_and_reaches_the_nnls_solution():
    op, A, y, shape = tiny()
    # min 1/2 ||A x - y||^2 over real x >= 0 == NNLS on [Re A; Im A] x = [Re y; Im y]
    xs, _ = so.nnls(np.vstack([A.real, A.imag]), np.concatenate([y.real, y.imag]), maxiter=10000)
    f_star = 0.5 * float(np.linalg.norm(A @ xs - y) ** 2)
    L = fb.lipschitz(op, shape, iters=200)
    gamma = 1.0 / L
    dirty = fb.dirty_image(op, y)
    x = np.zeros(shape)
    f_prev = fb.objective(op, x, y)
    for _ in range(3000):
        x = fb.fb_step(op, x, dirty, gamma)
        f = fb.objective(op, x, y)
        assert f <= f_prev * (1 + 1e-12) + 1e-12
        f_prev = f
    assert np.all(x >= 0)
    assert f_prev - f_star < 1e-6 * max(1.0, f_star)
    assert np.linalg.norm(x.ravel() - xs) < 1e-2 * max(1.0, np.linalg.norm(xs))
