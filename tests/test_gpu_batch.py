"""Batched wideband Phi^dagger Phi (one graph launch over per-channel plans) and the
tile-size autotuner.

The batch runs the same kernels as the per-plan applies and the grid step sums in fixed
point, so a channel's batched result equals its own apply bit for bit; each plan is also
checked against the FP64 oracle.
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
