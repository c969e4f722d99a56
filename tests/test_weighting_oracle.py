"""Pins of the oracle's data weighting (CPU only).

The weighting of Section 2 (Eq. 3) multiplies the data and the model by W = diag(w); the
weights of Briggs' robust scheme follow from the visibility density on the image's Fourier
grid.  These checks use hand-worked values, limits of the scheme, the paper's direct
equation and operator identities.
"""
import math

import numpy as np

import golden_data
import synth
from oracle import direct, operator, plan as pl, weighting


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def small(m=300, n=32, fov_deg=4.0, seed=21):
    uvw = synth.make_uvw(m, 60, 1.28e9, seed) * np.array([0.1, 0.1, 0.01])
    x = synth.make_sky(n, seed + 1).astype(np.complex128)
    return uvw, x, math.radians(fov_deg)


def make_op(uvw, n, fov, weights=None, **kw):
    args = dict(nx=n, ny=n, fov_x=fov, fov_y=fov, n_wbins=2, max_wsupport=9, w_norm_frac=1.0, wkernel_L=64)
    args.update(kw)
    pp = pl.PlanParams(**args)
    return operator.Operator(uvw, pl.make_plan(uvw, pp), weights=weights)


# ---------------------------------------------------------------- Briggs weights
def test_briggs_hand_worked_example():
    g = golden_data.load("briggs_three_visibilities.txt")
    nx, ny = (int(v) for v in g["grid"].split())
    fx, fy = golden_data.numbers(g["fov"])
    uvw = np.array([golden_data.numbers(r) for r in g["uvw"].split("|")])
    for R in (0, 1):
        w = weighting.briggs_weights(uvw, nx, ny, fx, fy, float(R))
        assert np.allclose(w, golden_data.numbers(g[f"weights R={R}"]), rtol=1e-15, atol=0)


def test_briggs_natural_and_uniform_limits():
    uvw = synth.make_uvw(5000, 60, 1.28e9, 5)
    fov = math.radians(1.0)
    wn = weighting.briggs_weights(uvw, 64, 64, fov, fov, 12.0)
    assert np.max(np.abs(wn - 1.0)) < 1e-15 * 1e3
    wu = weighting.briggs_weights(uvw, 64, 64, fov, fov, -12.0)
    c = weighting.density_cells(uvw, 64, 64, fov, fov)
    D = np.bincount(c, minlength=64 * 64)[c]
    # uniform: every occupied cell carries the same total weight D_c w_k
    tot = D * wu
    assert np.max(np.abs(tot / tot[0] - 1.0)) < 1e-12


def test_briggs_cells_wrap_modulo_the_grid():
    # u FoV = 8.1 is the cell of 0.1 on an 8-cell grid; v FoV = -0.4 rounds to cell 0
    uvw = np.array([[0.1, 0.0, 0.0], [8.1, -0.4, 0.0], [4.0, 4.0, 0.0]])
    c = weighting.density_cells(uvw, 8, 8, 1.0, 1.0)
    assert c[0] == c[1] != c[2]
    w = weighting.briggs_weights(uvw, 8, 8, 1.0, 1.0, 0.5)
    assert w[0] == w[1] and w[2] > w[0]


# ---------------------------------------------------------------- weighted operator
def test_weighted_phi_is_w_times_the_direct_equation():
    # coplanar data (w = 0) and J = 9: the discrete model is within 1e-7 of Eq. 1, so the
    # weights must sit on the data side of the direct sum to that precision
    uvw, x, fov = small()
    uvw[:, 2] = 0.0
    w = np.random.default_rng(1).uniform(0.0, 2.0, uvw.shape[0])
    O = make_op(uvw, 32, fov, weights=w, n_wbins=1, kb_support=9)
    yd = w * direct.direct_phi(x, uvw, fov, fov)
    assert rel(O.phi(x), yd) < 1e-7
    y = np.random.default_rng(2).standard_normal(uvw.shape[0]) + 0j
    assert rel(O.phi_adj(y), direct.direct_phi_adj(w * y, uvw, 32, 32, fov, fov)) < 1e-7


def test_weighted_adjoint_normal_operator_and_holographic_identities():
    uvw, x, fov = small(seed=31)
    rng = np.random.default_rng(3)
    w = rng.uniform(0.0, 3.0, uvw.shape[0])
    w[::7] = 0.0
    O = make_op(uvw, 32, fov, weights=w)
    y = rng.standard_normal(uvw.shape[0]) + 1j * rng.standard_normal(uvw.shape[0])
    lhs, rhs = np.vdot(y, O.phi(x)), np.vdot(O.phi_adj(y), x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    assert rel(O.phi_adj_phi(x), O.phi_adj(O.phi(x))) < 1e-12
    # H_p = G_p^dagger W_p^2 G_p: Hermitian, and applied to the grid it is the weighted G^dagger G
    for p in range(O.plan.P):
        H = O.holographic(p)
        assert abs(H - H.conj().T).max() < 1e-12 * abs(H).max()
        z = rng.standard_normal(H.shape[0]) + 1j * rng.standard_normal(H.shape[0])
        wp = w[O.plan.bins == p]
        assert rel(H @ z, O.G[p].conj().T @ (wp ** 2 * (O.G[p] @ z))) < 1e-12


def test_unit_weights_change_nothing():
    uvw, x, fov = small(seed=41)
    O1 = make_op(uvw, 32, fov)
    O2 = make_op(uvw, 32, fov, weights=np.ones(uvw.shape[0]))
    assert np.array_equal(O1.phi(x), O2.phi(x))
    assert np.array_equal(O1.phi_adj_phi(x), O2.phi_adj_phi(x))
