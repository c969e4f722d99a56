"""Batched wideband Phi^dagger Phi (one graph launch over per-channel plans) and the
tile-size autotuner.

The batch runs the same kernels as the per-plan applies and the grid step sums in fixed
point, so a channel's batched result equals its own apply bit for bit, in both forms of a
batch: staged (one launch per pass over every (channel, w-bin); the grid step one
persistent launch over a heaviest-first queue of every channel's and bin's work units) and
branches (each channel's apply on its own graph branch).  Each plan is also checked
against the FP64 oracle.
"""
import json
import math

import numpy as np
import pytest

import synth
from parity_util import TOL, both, rel, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def channels():
    """Three 128^2 channels of uneven size: frequencies, visibility counts and w-bins differ."""
    chans = synth.wideband_channels(n_chan=3, m_lo=500, m_hi=4000, seed=31)
    fov = math.radians(2.0)
    out = []
    for c, (f, uvw) in enumerate(chans):
        plan, op = both(uvw, 128, 128, fov, fov, n_wbins=2 + 2 * c)
        out.append((f, uvw, plan, op))
    return out


def test_batch_matches_plans_and_oracle(channels):
    import torch
    import paper_2605_26347_gb300 as pkg
    plans = [c[2] for c in channels]
    batch = pkg.Batch(plans)
    rng = np.random.default_rng(7)
    x = (rng.standard_normal((3, 128, 128)) + 0.3j * rng.standard_normal((3, 128, 128))).astype(np.complex64)
    xd = torch.from_numpy(x).cuda()
    out = batch.phi_adj_phi(xd)
    ref = torch.stack([p.phi_adj_phi(xd[i].contiguous()) for i, p in enumerate(plans)])
    assert torch.equal(out, ref)
    for i, (_, _, _, op) in enumerate(channels):
        assert rel(to_host(out[i]), op.phi_adj_phi(x[i].astype(np.complex128))) < TOL
    assert batch.info() == {"n_plans": 3, "captures": 1}


@pytest.fixture(scope="module")
def mixed():
    """Four 128^2 channels of uneven size and w-bins (1 to 6) with Kaiser-Bessel kernels of
    7 and 5 taps, so that their tile and patch sides differ."""
    chans = synth.wideband_channels(n_chan=4, m_lo=800, m_hi=6000, seed=37)
    fov = math.radians(2.0)
    out = []
    for c, (f, uvw) in enumerate(chans):
        kw = dict(n_wbins=[1, 3, 6, 2][c], kb_support=[7, 7, 5, 7][c])
        plan, op = both(uvw, 128, 128, fov, fov, **kw)
        out.append((f, uvw, plan, op))
    return out


def test_staged_batch_equals_each_plan_and_the_oracle(mixed):
    import torch
    import paper_2605_26347_gb300 as pkg
    plans = [c[2] for c in mixed]
    assert len({p.info()["max_tile"] for p in plans}) > 1     # patch sides differ
    staged = pkg.Batch(plans, form=pkg.BATCH_STAGED)
    lay = staged.layout()
    nonempty = sum(int(np.count_nonzero(np.bincount(p.bins()[1], minlength=p.info()["P"]))) for p in plans)
    assert lay["staged"] and lay["jobs"] == nonempty and lay["units"] > 0 and lay["scratch_bytes"] > 0
    rng = np.random.default_rng(8)
    x = (rng.standard_normal((4, 128, 128)) + 0.3j * rng.standard_normal((4, 128, 128))).astype(np.complex64)
    xd = torch.from_numpy(x).cuda()
    out = staged.phi_adj_phi(xd)
    ref = torch.stack([p.phi_adj_phi(xd[i].contiguous()) for i, p in enumerate(plans)])
    assert torch.equal(out, ref)
    for i, (_, _, plan, op) in enumerate(mixed):
        plan.status()
        assert rel(to_host(out[i]), op.phi_adj_phi(x[i].astype(np.complex128))) < TOL
    branches = pkg.Batch(plans, form=pkg.BATCH_BRANCHES)
    assert not branches.layout()["staged"]
    assert torch.equal(branches.phi_adj_phi(xd), out)
    # replay, a second output buffer (recorded again), the real part
    o2 = torch.empty_like(out)
    staged.phi_adj_phi(xd, o2)
    staged.phi_adj_phi(xd, o2)
    assert torch.equal(o2, out) and staged.info()["captures"] == 2
    o3 = staged.phi_adj_phi(xd, real_part_only=True)
    assert torch.all(o3.imag == 0) and torch.equal(o3.real, out.real)
    staged.close()
    branches.close()


def test_staged_form_refuses_plans_it_cannot_stage(mixed):
    import paper_2605_26347_gb300 as pkg
    uvw = mixed[0][1]
    fov = math.radians(2.0)
    tile64 = pkg.Plan(uvw, pkg.default_params(128, 128, fov, fov, n_wbins=2, tile_size=64))
    with pytest.raises(pkg.RimoError) as e:
        pkg.Batch([mixed[1][2], tile64], form=pkg.BATCH_STAGED)
    assert e.value.status == 6
    auto = pkg.Batch([mixed[1][2], tile64])          # falls back to branches
    assert not auto.layout()["staged"]
    auto.close()
    tile64.close()


def test_batch_replays_and_recaptures(channels):
    import torch
    import paper_2605_26347_gb300 as pkg
    plans = [c[2] for c in channels]
    batch = pkg.Batch(plans)
    x = torch.from_numpy(np.stack([synth.make_sky(128, 40 + i) for i in range(3)])).cuda()
    o1 = batch.phi_adj_phi(x)
    o2 = torch.empty_like(o1)
    batch.phi_adj_phi(x, o2)                     # new output buffer: recorded again
    batch.phi_adj_phi(x, o2)                     # same buffers: graph replay
    assert batch.info()["captures"] == 2
    assert torch.equal(o1, o2)
    o3 = batch.phi_adj_phi(x, real_part_only=True)
    assert torch.all(o3.imag == 0) and torch.equal(o3.real, o1.real)


def test_batch_rejects_bad_groups(channels):
    import paper_2605_26347_gb300 as pkg
    plans = [c[2] for c in channels]
    with pytest.raises(pkg.RimoError):
        pkg.Batch([plans[0], plans[0]])
    other, _ = both(channels[0][1], 64, 64, math.radians(2.0), math.radians(2.0), n_wbins=2)
    with pytest.raises(pkg.RimoError):
        pkg.Batch([plans[0], other])


def test_autotuner_picks_and_caches(tmp_path):
    import paper_2605_26347_gb300 as pkg
    uvw = synth.make_uvw(30000, 600, 1.28e9, 77)
    fov = math.radians(2.0)
    params = pkg.default_params(256, 256, fov, fov, n_wbins=2)
    cache = tmp_path / "tune.json"
    tile, ms = pkg.autotune_tile(uvw, params, str(cache))
    assert tile in (32, 64) and min(ms) > 0
    assert tile == (32 if ms[0] <= ms[1] else 64)
    stored = json.loads(cache.read_text())
    assert list(stored.values()) == [tile]
    tile2, ms2 = pkg.autotune_tile(uvw, params, str(cache))   # cache hit: nothing timed
    assert tile2 == tile and ms2 == [-1.0, -1.0]


def test_tile_and_order_autotuner_picks_and_caches(tmp_path):
    import paper_2605_26347_gb300 as pkg
    uvw = synth.make_uvw(30000, 600, 1.28e9, 78)
    fov = math.radians(2.0)
    params = pkg.default_params(256, 256, fov, fov, n_wbins=2)
    cache = tmp_path / "tune.json"
    r = pkg.autotune(uvw, params, str(cache))
    assert len(r["ms"]) == 6 and min(r["ms"]) > 0
    best = int(np.argmin(r["ms"]))
    assert (r["tile_size"], r["uv_order"]) == ((32, 64)[best // 3], best % 3)
    assert json.loads(cache.read_text()) != {}
    r2 = pkg.autotune(uvw, params, str(cache))               # cache hit: nothing timed
    assert (r2["tile_size"], r2["uv_order"]) == (r["tile_size"], r["uv_order"]) and r2["ms"] == [-1.0] * 6


@pytest.mark.parametrize("order", [1, 2])
def test_visibility_orders_match_the_oracle(order):
    w = synth.make_config(1)
    fov = w.fov_rad
    plan, op = both(w.uvw, 256, 256, fov, fov, n_wbins=4, uv_order=order)
    ref = op.phi_adj_phi(w.sky.astype(np.complex128))
    assert rel(to_host(plan.phi_adj_phi(to_dev(w.sky))), ref) < TOL
    plan.close()


def test_batch_autotuner_times_the_batch_and_caches(tmp_path):
    import paper_2605_26347_gb300 as pkg
    fov = math.radians(2.0)
    uvws = [synth.make_uvw(20000, 600, 1.0e9, 81), synth.make_uvw(30000, 600, 1.5e9, 82)]
    params = [pkg.default_params(256, 256, fov, fov, n_wbins=2), pkg.default_params(256, 256, fov, fov, n_wbins=3)]
    cache = tmp_path / "tune.json"
    r = pkg.autotune_batch(uvws, params, str(cache))
    assert r["workloads"] == 2 and len(r["ms"]) == 6 and min(r["ms"]) > 0
    best = int(np.argmin(r["ms"]))
    assert (r["tile_size"], r["uv_order"]) == ((32, 64)[best // 3], best % 3)
    key = [k for k in json.loads(cache.read_text()) if k.endswith("_batch_tile_order")]
    assert len(key) == 1 and "+" in key[0]
    r2 = pkg.autotune_batch(uvws, params, str(cache))        # cache hit: nothing timed
    assert (r2["tile_size"], r2["uv_order"]) == (r["tile_size"], r["uv_order"]) and r2["ms"] == [-1.0] * 6
    with pytest.raises(ValueError):
        pkg.autotune_batch(uvws, params[:1])
    with pytest.raises(pkg.RimoError):   # the workloads of a batch share one image size
        pkg.autotune_batch(uvws, [params[0], pkg.default_params(128, 128, fov, fov, n_wbins=2)])
