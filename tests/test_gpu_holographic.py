"""Holographic matrices H_p = G_p^dagger G_p (Section 3.3) built on the device.

Pins: the stored entries equal the oracle's G_p^H G_p (and H is Hermitian); after the
build, Phi^dagger Phi and the PSF run through H and match the oracle's G^dagger G path
within the complex-FP32 tolerance; a budget below G + H refuses the build.
"""
import math

import numpy as np
import pytest

import synth
from parity_util import TOL, both, rel, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def holo():
    """256^2, FoV 1 deg, 20k visibilities (60 time steps), 4 w-bins; H built."""
    w = synth.make_config(1)
    fov = w.fov_rad
    plan, op = both(w.uvw, 256, 256, fov, fov, n_wbins=4)
    x = w.sky
    before = to_host(plan.phi_adj_phi(to_dev(x)))
    plan.build_holographic()
    return w, plan, op, before


def test_entries_match_oracle_and_are_hermitian(holo):
    w, plan, op, _ = holo
    rng = np.random.default_rng(11)
    for p in range(op.plan.P):
        H = op.holographic(p).tocoo()
        if H.nnz == 0:
            continue
        pick = rng.choice(H.nnz, size=min(400, H.nnz), replace=False)
        r, c, v = H.row[pick], H.col[pick], H.data[pick]
        pairs = np.stack([r // op.gy, r % op.gy, c // op.gy, c % op.gy], axis=1)
        got = plan.holographic_entries(p, pairs)
        assert rel(got, v) < TOL, (p, rel(got, v))
        swapped = plan.holographic_entries(p, pairs[:, [2, 3, 0, 1]])
        assert np.array_equal(swapped, np.conj(got))
    # a pair no footprint covers (cells far apart) is zero
    assert plan.holographic_entries(0, [[0, 0, 100, 100]])[0] == 0


def test_nonzero_count_matches_oracle(holo):
    # the full H_p = G_p^H G_p of the oracle, both triangles: its non-zeros over all bins
    w, plan, op, _ = holo
    nnz = 0
    for p in range(op.plan.P):
        H = op.holographic(p)
        H.eliminate_zeros()
        nnz += H.nnz
    info = plan.info()
    assert info["h_nnz"] == nnz
    assert 0 < info["h_nonzero"] <= info["h_entries"]


def test_phi_adj_phi_and_psf_through_h(holo):
    w, plan, op, before = holo
    out = to_host(plan.phi_adj_phi(to_dev(w.sky)))
    assert rel(out, op.phi_adj_phi(w.sky.astype(np.complex128))) < TOL
    assert rel(out, before) < TOL           # the G^dagger G path: same operator, other rounding order
    assert rel(to_host(plan.psf()), op.psf()) < TOL
    info = plan.info()
    assert info["h_bytes"] > 0
    # deterministic: fixed-point accumulation
    assert np.array_equal(to_host(plan.phi_adj_phi(to_dev(w.sky))), out)


def test_rectangular_grid_and_two_bins():
    uvw = synth.make_uvw(3000, 60, 1.28e9, 91)
    fx, fy = math.radians(2.0), math.radians(1.5)
    plan, op = both(uvw, 128, 64, fx, fy, n_wbins=2, kb_support=5)
    plan.build_holographic()
    x = (np.random.default_rng(5).standard_normal((64, 128)) + 0.2j).astype(np.complex64)
    assert rel(to_host(plan.phi_adj_phi(to_dev(x))), op.phi_adj_phi(x.astype(np.complex128))) < TOL


def test_budget_refuses_the_build():
    import paper_2605_26347_gb300 as pkg
    uvw = synth.make_uvw(3000, 60, 1.28e9, 92)
    fov = math.radians(1.0)
    plan, _ = both(uvw, 64, 64, fov, fov, n_wbins=2, mode=pkg.MODE_STORED_G)
    g = plan.info()["g_bytes"]
    plan2 = pkg.Plan(uvw, pkg.default_params(64, 64, fov, fov, n_wbins=2, mode=pkg.MODE_STORED_G,
                                             mem_budget_bytes=g + 1))
    with pytest.raises(pkg.RimoError) as e:
        plan2.build_holographic()
    assert e.value.status == 3


def test_dense_coverage_parity():
    # many visibilities per grid cell (the regime H is for): 64^2 image, 128^2 grid,
    # 150k visibilities over 2 bins, about 9 per covered cell
    uvw = synth.make_uvw(150_000, 28_800, 1.28e9, 93) * np.array([0.25, 0.25, 1.0])
    fov = math.radians(1.0)
    plan, op = both(uvw, 64, 64, fov, fov, n_wbins=2)
    x = synth.make_sky(64, 94)
    g_path = to_host(plan.phi_adj_phi(to_dev(x)))
    plan.build_holographic()
    h_path = to_host(plan.phi_adj_phi(to_dev(x)))
    ref = op.phi_adj_phi(x.astype(np.complex128))
    assert rel(g_path, ref) < TOL
    assert rel(h_path, ref) < TOL


def test_holographic_plan_without_stored_g():
    # a plan in holographic mode keeps no G: tiles on the fly, then H built bin by bin
    # from freshly generated exact tiles (Fig. 2, regime b)
    import paper_2605_26347_gb300 as pkg
    w = synth.make_config(1)
    fov = w.fov_rad
    plan, op = both(w.uvw, 256, 256, fov, fov, n_wbins=4, mode=pkg.MODE_HOLOGRAPHIC)
    assert plan.info()["g_bytes"] < 0.05 * op.plan.K * 8
    ref = op.phi_adj_phi(w.sky.astype(np.complex128))
    assert rel(to_host(plan.phi_adj_phi(to_dev(w.sky))), ref) < TOL      # on the fly
    assert rel(to_host(plan.phi(to_dev(w.sky))), op.phi(w.sky.astype(np.complex128))) < TOL
    plan.build_holographic()
    assert rel(to_host(plan.phi_adj_phi(to_dev(w.sky))), ref) < TOL      # through H
    H = op.holographic(1).tocoo()
    pick = np.random.default_rng(3).choice(H.nnz, size=200, replace=False)
    r, c = H.row[pick], H.col[pick]
    pairs = np.stack([r // op.gy, r % op.gy, c // op.gy, c % op.gy], axis=1)
    assert rel(plan.holographic_entries(1, pairs), H.data[pick]) < TOL
