"""GPU: level-2 shard plans (Section 3.5: every w-bin's Fourier blocks dealt over workers).

Shard plans made from the same uvw and parameters share the w-stack; each keeps every
w-bin's uv-tiles whose place in the bin's radial order is its rank modulo the shard count,
stores G for their visibilities only, and its Phi^dagger Phi image is its share: the shard
images must sum to the whole plan's (and to the oracle's) Phi^dagger Phi, each shard must hold
exactly the visibilities the host mirror of the partition deals it, and Phi must give its own
visibilities' y exactly as the whole plan does.
"""
import numpy as np
import pytest

import synth
from parity_util import TOL, assert_same_plan, both, rel, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mono256():
    import paper_2605_26347_gb300 as pkg
    w = synth.make_config(1)
    fov = w.fov_rad
    plan, op = both(w.uvw, 256, 256, fov, fov, n_wbins=4, mode=pkg.MODE_STORED_G)
    assert_same_plan(plan, op)
    return w, plan, op


@pytest.mark.parametrize("count", [2, 3])
def test_shard_plans_sum_to_the_whole_operator(mono256, count):
    import paper_2605_26347_gb300 as pkg
    from paper_2605_26347_gb300 import distributed as rd
    w, plan, op = mono256
    x = to_dev(w.sky)
    whole = to_host(plan.phi_adj_phi(x))
    y_whole = to_host(plan.phi(x))
    oracle = op.phi_adj_phi(w.sky.astype(np.complex128))
    shard = rd.tile_shards(op.plan.bins, op.geo.g0, op.geo.h0, op.gx, op.gy, plan.info()["tile_size"], count)
    S2 = (op.geo.S * op.geo.S).astype(np.int64)
    total = np.zeros_like(whole)
    for r in range(count):
        sp = pkg.Plan(w.uvw, rd.shard_params(plan.params, r, count))
        own = shard == r
        assert own.any()
        # the library deals the tiles as the host mirror does: its taps are exactly those
        assert sp.info()["K"] == int(S2[own].sum())
        img = to_host(sp.phi_adj_phi(x))
        total += img
        y = to_host(sp.phi(x))
        assert np.array_equal(y[own], y_whole[own]) and not np.any(y[~own])
        with pytest.raises(pkg.RimoError):
            sp.tiles(np.array([int(np.flatnonzero(~own)[0])]))
        sp.status()
        sp.close()
    assert rel(total, whole) < 1e-6
    assert rel(total, oracle) < TOL


def test_shard_parameters_are_checked(mono256):
    import paper_2605_26347_gb300 as pkg
    from paper_2605_26347_gb300 import distributed as rd
    w, plan, _ = mono256
    with pytest.raises(pkg.RimoError):   # rank out of range
        pkg.Plan(w.uvw, rd.shard_params(plan.params, 2, 2))
    q = rd.shard_params(plan.params, 0, 2)
    q.mode = pkg.MODE_ONTHEFLY           # a shard stores G
    with pytest.raises(pkg.RimoError):
        pkg.Plan(w.uvw, q)
