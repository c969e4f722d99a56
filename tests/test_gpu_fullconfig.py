"""Element-wise parity of Phi, Phi^dagger and Phi^dagger Phi at the workloads' own geometries.

The FP64 oracle cannot hold the 50M-visibility operator, so each workload keeps its image
size, field of view, grid and w-bin count and takes a subset of its own visibilities:
every visibility within a core radius of the (u, v) origin (there the uv-tiles are as full
as in the whole workload: heavy tiles that the plan splits into several work units, merged
afterwards, and full 20-visibility chunks of the grid step's pipeline) plus a seeded uniform
draw of the rest (long baselines, the whole w range, so every w-bin including the outer
ones is populated).  Every output element is compared with the oracle (relative l2 over
the whole vector or image, tolerance 1e-5 for complex FP32 against FP64):

* 4096^2 image, FoV 3 deg, 8192^2 grid, 32 w-bins, stored G (the benchmark's plan):
  Phi on all visibilities, Phi^dagger of the oracle's y, Phi^dagger Phi (Eq. 6-8);
* 2048^2, FoV 2.5 deg, 16 w-bins, Phi^dagger Phi through H_p = G_p^dagger G_p (Section 3.3)
  and through G^dagger G before H is built;
* 1024^2 wideband: three channels (0.9, 1.29, 1.7 GHz; 4, 18 and 32 w-bins) batched in one
  graph launch, staged (one launch per pass over every channel and bin, the grid step one
  persistent launch over all their work units) and as branches, against the oracle of
  each channel.
"""
import math
import os

import numpy as np
import pytest

import synth
from oracle import operator as oop
from oracle import plan as opl
from parity_util import TOL, assert_same_plan, rel, to_dev, to_host

pytestmark = pytest.mark.gpu

WORKERS = max(1, min(16, os.cpu_count() or 1))


def core_plus_uniform(uvw, r_core, n_uniform, seed):
    """All rows with |(u, v)| < r_core plus n_uniform rows drawn uniformly from the rest."""
    r = np.hypot(uvw[:, 0], uvw[:, 1])
    core = np.nonzero(r < r_core)[0]
    rest = np.nonzero(r >= r_core)[0]
    rng = np.random.default_rng(seed)
    pick = rng.choice(rest, size=min(n_uniform, rest.size), replace=False)
    return np.ascontiguousarray(uvw[np.sort(np.concatenate([core, pick]))]), core.size


def uv_tile_counts(op, bins, ts):
    """Visibilities per (w-bin, uv-tile of ts x ts cells holding the first cell)."""
    tu = (op.geo.g0 % op.gx) // ts
    tv = (op.geo.h0 % op.gy) // ts
    key = (bins.astype(np.int64) * (op.gx // ts) + tu) * (op.gy // ts) + tv
    return np.unique(key, return_counts=True)[1]


@pytest.fixture(scope="module")
def c5sub():
    import paper_2605_26347_gb300 as pkg
    uvw50 = synth.make_uvw(50_000_000, 28_800, 1.28e9, seed=1005)
    uvw, n_core = core_plus_uniform(uvw50, 1000.0, 900_000, seed=31)
    del uvw50
    sky = synth.make_sky(4096, seed=2005)
    fov = math.radians(3.0)
    plan = pkg.Plan(uvw, pkg.default_params(4096, 4096, fov, fov, n_wbins=32, mode=pkg.MODE_STORED_G))
    oplan = opl.make_plan(uvw, opl.PlanParams(nx=4096, ny=4096, fov_x=fov, fov_y=fov, n_wbins=32))
    op = oop.Operator(uvw, oplan, workers=WORKERS)
    x = sky.astype(np.complex128)
    y_o = op.phi(x)
    z_o = op.phi_adj(y_o)  # Phi^dagger Phi x: sum over p of Phi_p^dagger Phi_p x (Eq. 7)
    yield dict(uvw=uvw, n_core=n_core, sky=sky, plan=plan, op=op, y_o=y_o, z_o=z_o)
    plan.close()


def test_c5_subset_exercises_every_bin_split_tiles_and_full_chunks(c5sub):
    plan, op = c5sub["plan"], c5sub["op"]
    assert c5sub["uvw"].shape[0] >= 1_000_000 and c5sub["n_core"] > 100_000
    assert_same_plan(plan, op)
    ws, bins, _ = plan.bins()
    assert np.all(np.bincount(bins, minlength=32) > 0)     # all 32 bins populated
    info = plan.info()
    counts = uv_tile_counts(op, bins, info["tile_size"])
    # units hold at most max(256, visibilities of the bin / (2 x SMs)) visibilities: tiles
    # above 1024 are split in any bin of this subset (the densest holds about 18k); over
    # 300k visibilities sit in tiles that fill the 20-visibility chunks
    assert counts.max() > 1024
    assert counts[counts >= 20].sum() > 300_000


def test_c5_subset_phi_every_visibility(c5sub):
    y = to_host(c5sub["plan"].phi(to_dev(c5sub["sky"])))
    assert rel(y, c5sub["y_o"]) < TOL


def test_c5_subset_phi_adj(c5sub):
    x = to_host(c5sub["plan"].phi_adj(to_dev(c5sub["y_o"])))
    assert rel(x, c5sub["z_o"]) < TOL


def test_c5_subset_phi_adj_phi_every_pixel(c5sub):
    plan = c5sub["plan"]
    z = to_host(plan.phi_adj_phi(to_dev(c5sub["sky"])))
    assert rel(z, c5sub["z_o"]) < TOL
    # the real-part output of the imaging loop (Section 3.5)
    zr = to_host(plan.phi_adj_phi(to_dev(c5sub["sky"]), real_part_only=True))
    assert rel(zr, c5sub["z_o"].real) < TOL
    # the w-stack's outer bins alone (largest |w_stack|, where the w-phase is largest)
    mask = np.zeros(32, dtype=np.uint8)
    mask[[0, 1, 30, 31]] = 1
    zb = to_host(plan.phi_adj_phi_bins(to_dev(c5sub["sky"]), mask))
    ref = c5sub["op"].phi_adj_phi(c5sub["sky"].astype(np.complex128), bins=[0, 1, 30, 31])
    assert rel(zb, ref) < TOL


def test_c5_w_phase_at_the_largest_w_stack(c5sub):
    """Z_p element by element against the oracle's FP64 Z_p at the bin of largest |w_stack|
    (there the w-phase w (sqrt(1 - l^2 - m^2) - 1) spans tens of turns).  An FP32 product
    w (n - 1) before the sincos would be off by up to about |w (n - 1)| 2^-24 turns: the test
    checks that this reading fails the bound the device's double-float phase meets."""
    from oracle import wterm
    plan, op = c5sub["plan"], c5sub["op"]
    ws, _, _ = plan.bins()
    p = int(np.argmax(np.abs(ws)))
    zg = to_host(plan.zlayer(p))
    zo = op.z_layer(p)
    err = np.max(np.abs(zg - zo) / np.abs(zo))
    assert err < 1e-6, err
    # the same factor with the phase argument rounded to FP32 first
    pp = op.pp
    l = wterm.pixel_lm(pp.nx, pp.fov_x)[None, :]
    m = wterm.pixel_lm(pp.ny, pp.fov_y)[:, None]
    arg32 = (np.float32(ws[p]) * wterm.dn(l, m).astype(np.float32)).astype(np.float64)
    z32 = op.gc * np.exp(-2j * math.pi * arg32)
    assert abs(float(np.max(np.abs(op.plan.w_stack))) - abs(ws[p])) < 1e-6 * abs(ws[p])
    assert np.max(np.abs(z32 - zo) / np.abs(zo)) > 3 * err


def test_c3_subset_through_h_and_g():
    import paper_2605_26347_gb300 as pkg
    uvw20 = synth.make_uvw(20_000_000, 28_800, 1.28e9, seed=1003)
    uvw, n_core = core_plus_uniform(uvw20, 1000.0, 4_000, seed=33)
    del uvw20
    assert n_core > 50_000
    sky = synth.make_sky(2048, seed=2003)
    fov = math.radians(2.5)
    plan = pkg.Plan(uvw, pkg.default_params(2048, 2048, fov, fov, n_wbins=16, mode=pkg.MODE_STORED_G))
    oplan = opl.make_plan(uvw, opl.PlanParams(nx=2048, ny=2048, fov_x=fov, fov_y=fov, n_wbins=16))
    op = oop.Operator(uvw, oplan, workers=WORKERS)
    assert_same_plan(plan, op)
    ref = op.phi_adj_phi(sky.astype(np.complex128))
    via_g = to_host(plan.phi_adj_phi(to_dev(sky)))
    assert rel(via_g, ref) < TOL
    plan.build_holographic()
    assert plan.info()["h_bytes"] > 0
    via_h = to_host(plan.phi_adj_phi(to_dev(sky)))
    assert rel(via_h, ref) < TOL
    assert rel(to_host(plan.psf()), op.psf()) < TOL
    plan.close()


def test_c4_three_channels_batched():
    import torch
    import paper_2605_26347_gb300 as pkg
    chans = synth.wideband_channels(n_chan=32)
    fov = math.radians(2.5)
    plans, ops, xs = [], [], []
    for c in (0, 15, 31):
        f, uvw_c = chans[c]
        rng = np.random.default_rng(40 + c)
        uvw = np.ascontiguousarray(uvw_c[np.sort(rng.choice(uvw_c.shape[0], 150_000, replace=False))])
        nb = int(round(4 + 28 * c / 31))
        kw = dict(n_wbins=nb)
        plans.append(pkg.Plan(uvw, pkg.default_params(1024, 1024, fov, fov, tile_size=64, **kw)))
        oplan = opl.make_plan(uvw, opl.PlanParams(nx=1024, ny=1024, fov_x=fov, fov_y=fov, **kw))
        ops.append(oop.Operator(uvw, oplan, workers=WORKERS))
        assert_same_plan(plans[-1], ops[-1])
        xs.append(synth.make_sky(1024, 2004 + c))
    assert [p.info()["P"] for p in plans] == [4, 18, 32]
    x = np.stack(xs)
    refs = [op.phi_adj_phi(x[i].astype(np.complex128)) for i, op in enumerate(ops)]
    for form in (pkg.BATCH_STAGED, pkg.BATCH_BRANCHES):
        batch = pkg.Batch(plans, form=form)
        assert batch.layout()["staged"] == (form == pkg.BATCH_STAGED)
        out = to_host(batch.phi_adj_phi(torch.from_numpy(x).cuda()))
        for i in range(len(ops)):
            assert rel(out[i], refs[i]) < TOL, (form, i)
        batch.close()
    for p in plans:
        p.close()
