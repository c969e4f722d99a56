"""Data weighting injected into the operator (Section 2, Eq. 3) on the device.

The weighted operator W Phi against the oracle's (which applies W to the data side of
its unweighted operator), for stored tiles, tiles built per bin at apply time, surrogate
tiles and a holographic matrix built after the weights; unit weights and removing the
weighting give back the unweighted operator exactly; Briggs weights from the library feed
the weighted PSF.
"""
import math

import numpy as np
import pytest

import synth
from oracle import operator as oop
from oracle import weighting
from parity_util import TOL, both, rel, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    w = synth.make_config(1)
    fov = w.fov_rad
    plan, op = both(w.uvw, 256, 256, fov, fov, n_wbins=4)
    rng = np.random.default_rng(17)
    wt = rng.uniform(0.0, 2.0, w.uvw.shape[0])
    wt[::11] = 0.0
    opw = oop.Operator(w.uvw, op.plan, build_g=False, weights=wt.astype(np.float32).astype(np.float64))
    opw.G = op.G
    return w, plan, op, opw, wt.astype(np.float32)


def test_weighted_stored_g_matches_oracle(case):
    w, plan, op, opw, wt = case
    x = w.sky
    ref0 = to_host(plan.phi_adj_phi(to_dev(x)))
    plan.set_weights(wt)
    try:
        assert plan.info()["weighted"] == 1
        y = np.random.default_rng(3).standard_normal(w.uvw.shape[0]) + 1j * np.random.default_rng(4).standard_normal(
            w.uvw.shape[0])
        assert rel(to_host(plan.phi(to_dev(x))), opw.phi(x)) < TOL
        assert rel(to_host(plan.phi_adj(to_dev(y))), opw.phi_adj(y)) < TOL
        assert rel(to_host(plan.phi_adj_phi(to_dev(x))), opw.phi_adj_phi(x)) < TOL
        # weighted tiles are the unweighted ones times the weight
        idx = np.array([0, 5, 11, 12345 % w.uvw.shape[0]])
        tw = plan.tiles(idx)[3]
    finally:
        plan.set_weights(None)
    assert plan.info()["weighted"] == 0
    t0 = plan.tiles(idx)[3]
    for q, k in enumerate(idx):
        assert np.allclose(tw[q], wt[k] * t0[q], rtol=1e-6, atol=1e-7 * np.abs(t0[q]).max())
    # removing the weighting rebuilds the unweighted tiles exactly
    assert np.array_equal(to_host(plan.phi_adj_phi(to_dev(x))), ref0)


def test_unit_weights_are_exactly_unweighted(case):
    w, plan, _, _, _ = case
    x = to_dev(w.sky)
    ref = to_host(plan.phi_adj_phi(x))
    plan.set_weights(np.ones(w.uvw.shape[0], np.float32))
    try:
        assert np.array_equal(to_host(plan.phi_adj_phi(x)), ref)
    finally:
        plan.set_weights(None)


def test_zero_weights_give_the_zero_operator(case):
    w, plan, _, _, _ = case
    plan.set_weights(np.zeros(w.uvw.shape[0], np.float32))
    try:
        x = to_dev(w.sky)
        assert not np.any(to_host(plan.phi_adj_phi(x)))
        assert not np.any(to_host(plan.phi(x)))
    finally:
        plan.set_weights(None)


def test_generated_tiles_and_holographic_matrix_take_the_weights(case):
    import paper_2605_26347_gb300 as pkg
    w, plan, _, opw, wt = case
    fov = w.fov_rad
    x = w.sky
    want = opw.phi_adj_phi(x)
    fly = pkg.Plan(w.uvw, pkg.default_params(256, 256, fov, fov, n_wbins=4, mode=pkg.MODE_ONTHEFLY))
    fly.set_weights(wt)
    assert rel(to_host(fly.phi_adj_phi(to_dev(x))), want) < TOL
    holo = pkg.Plan(w.uvw, pkg.default_params(256, 256, fov, fov, n_wbins=4))
    holo.set_weights(wt)
    holo.build_holographic()
    assert rel(to_host(holo.phi_adj_phi(to_dev(x))), want) < TOL
    with pytest.raises(pkg.RimoError) as e:
        holo.set_weights(None)
    assert e.value.status == 7


def test_surrogate_tiles_take_the_weights():
    import paper_2605_26347_gb300 as pkg
    w = synth.make_config(1)
    fov = w.fov_rad
    kw = dict(n_wbins=4, w_norm_frac=1.0)
    exact = pkg.Plan(w.uvw, pkg.default_params(256, 256, fov, fov, **kw))
    sur = pkg.Surrogate(seed=3)
    sur.fit(exact, n_samples=20000, steps=50, batch=512, lr=1e-3, seed=2)
    splan = pkg.Plan(w.uvw, pkg.default_params(256, 256, fov, fov, mode=pkg.MODE_SURROGATE, **kw))
    splan.set_surrogate(sur)
    idx = np.array([1, 2, 3, 400, 7000])
    t0 = splan.tiles(idx)[3]
    wt = np.random.default_rng(5).uniform(0.5, 2.0, w.uvw.shape[0]).astype(np.float32)
    splan.set_weights(wt)
    t1 = splan.tiles(idx)[3]
    for q, k in enumerate(idx):
        assert np.array_equal(t1[q], (wt[k] * t0[q]).astype(np.complex64))
    # training wants unweighted exact tiles
    exact.set_weights(wt)
    with pytest.raises(pkg.RimoError) as e:
        sur.fit(exact, n_samples=1000, steps=1, batch=128)
    assert e.value.status == 7


def test_invalid_weights_are_rejected(case):
    import paper_2605_26347_gb300 as pkg
    w, plan, _, _, _ = case
    bad = np.ones(w.uvw.shape[0], np.float32)
    bad[7] = -1.0
    with pytest.raises(pkg.RimoError) as e:
        plan.set_weights(bad)
    assert e.value.status == 1
    bad[7] = np.nan
    with pytest.raises(pkg.RimoError):
        plan.set_weights(bad)
    with pytest.raises(ValueError):
        plan.set_weights(np.ones(3, np.float32))
    assert plan.info()["weighted"] == 0


def test_briggs_weighted_psf_matches_oracle():
    import paper_2605_26347_gb300 as pkg
    uvw = synth.make_uvw(6000, 60, 1.28e9, 77)
    fov = math.radians(1.0)
    plan, op = both(uvw, 128, 128, fov, fov, n_wbins=3)
    wb = pkg.briggs_weights(uvw, 128, 128, fov, fov, 0.0)
    wo = weighting.briggs_weights(uvw, 128, 128, fov, fov, 0.0)
    assert np.max(np.abs(wb - wo) / wo) < 1e-6
    plan.set_weights(wb)
    opw = oop.Operator(uvw, op.plan, build_g=False, weights=wb.astype(np.float64))
    opw.G = op.G
    assert rel(to_host(plan.psf()), opw.psf()) < TOL
