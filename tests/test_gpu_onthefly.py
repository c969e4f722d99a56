"""Exact tiles generated on the fly per w-bin at apply time (no stored G).

The same G-build kernel writes each bin's tiles into a one-bin scratch right before the
gridding step, so the operator equals the stored-G one (up to the fixed-point scales,
which follow the tiles generated so far) and the oracle's.
"""
import math

import numpy as np
import pytest

import synth
from parity_util import TOL, both, rel, to_dev, to_host

pytestmark = pytest.mark.gpu


def test_onthefly_matches_stored_g_and_oracle():
    import paper_2605_26347_gb300 as pkg
    w = synth.make_config(1)
    fov = w.fov_rad
    fly, op = both(w.uvw, 256, 256, fov, fov, n_wbins=4, mode=pkg.MODE_ONTHEFLY)
    stored = pkg.Plan(w.uvw, pkg.default_params(256, 256, fov, fov, n_wbins=4))
    x = to_dev(w.sky)
    rng = np.random.default_rng(8)
    y = (rng.standard_normal(w.uvw.shape[0]) + 1j * rng.standard_normal(w.uvw.shape[0])).astype(np.complex64)
    assert rel(to_host(fly.phi(x)), to_host(stored.phi(x))) < 1e-6
    assert rel(to_host(fly.phi_adj(to_dev(y))), op.phi_adj(y.astype(np.complex128))) < TOL
    assert rel(to_host(fly.phi_adj_phi(x)), op.phi_adj_phi(w.sky.astype(np.complex128))) < TOL
    assert fly.info()["g_bytes"] < 0.05 * stored.info()["g_bytes"]
    # tile read-back generates the bins it needs: the same tiles as the stored ones
    idx = np.random.default_rng(4).choice(w.uvw.shape[0], 300, replace=False)
    a, b = fly.tiles(idx), stored.tiles(idx)
    for q in range(3):
        assert np.array_equal(a[q], b[q])
    assert all(np.array_equal(ta, tb) for ta, tb in zip(a[3], b[3]))


def test_onthefly_rectangular_and_j5():
    import paper_2605_26347_gb300 as pkg
    uvw = synth.make_uvw(3000, 60, 1.28e9, 96)
    fx, fy = math.radians(2.0), math.radians(1.5)
    plan, op = both(uvw, 128, 64, fx, fy, n_wbins=3, kb_support=5, mode=pkg.MODE_ONTHEFLY)
    x = (np.random.default_rng(9).standard_normal((64, 128)) + 0.1j).astype(np.complex64)
    assert rel(to_host(plan.phi_adj_phi(to_dev(x))), op.phi_adj_phi(x.astype(np.complex128))) < TOL


@pytest.mark.parametrize("kw", [
    dict(n_wbins=4),                                   # L = 64, supports up to 9 x 9
    dict(n_wbins=2, max_wsupport=5, kb_support=5),     # L = 32
])
def test_tabulated_wkernels_match_the_chirp_evaluation(kw):
    # K(t; w_r) depends on w_r alone: a per-plan table of 8192 samples with cubic Lagrange
    # interpolation in w_r replaces the per-visibility chirp sums
    import paper_2605_26347_gb300 as pkg
    w = synth.make_config(1)
    fov = w.fov_rad
    exact, op = both(w.uvw, 256, 256, fov, fov, **kw)
    tab = pkg.Plan(w.uvw, pkg.default_params(256, 256, fov, fov, wkernel_table=8192, **kw))
    idx = np.random.default_rng(6).choice(w.uvw.shape[0], 400, replace=False)
    te, tt = exact.tiles(idx)[3], tab.tiles(idx)[3]
    err = max(np.linalg.norm(a - b) / np.linalg.norm(a) for a, b in zip(te, tt))
    assert err < 2e-6, err
    x = to_dev(w.sky)
    assert rel(to_host(tab.phi_adj_phi(x)), op.phi_adj_phi(w.sky.astype(np.complex128))) < TOL
    fly = pkg.Plan(w.uvw, pkg.default_params(256, 256, fov, fov, wkernel_table=8192, mode=pkg.MODE_ONTHEFLY, **kw))
    assert rel(to_host(fly.phi_adj_phi(x)), to_host(tab.phi_adj_phi(x))) < 1e-6


def test_tabulated_wkernels_with_a_single_w():
    # every visibility at one w: all residuals 0, the table collapses to one kernel (a delta)
    import paper_2605_26347_gb300 as pkg
    uvw = synth.make_uvw(3000, 60, 1.28e9, 31)
    uvw[:, 2] = 250.0
    fov = math.radians(1.0)
    plan, op = both(uvw, 64, 64, fov, fov, n_wbins=1)
    tab = pkg.Plan(uvw, pkg.default_params(64, 64, fov, fov, n_wbins=1, wkernel_table=64))
    x = to_dev(synth.make_sky(64, 5))
    assert rel(to_host(tab.phi_adj_phi(x)), to_host(plan.phi_adj_phi(x))) < 1e-6
