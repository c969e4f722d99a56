"""Sharding Phi^dagger Phi over ranks by w-bin, on CPU gloo ranks (world size 2 and 3).

Each rank evaluates the oracle's Phi_p^dagger Phi_p terms of its share of the bins (Eq. 7)
and the ranks all-reduce the partial images: every rank must end with the full
Phi^dagger Phi x.  The partition is checked for coverage, determinism and balance.
"""
import math
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

from paper_2605_26347_gb300 import distributed as rd


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    import synth
    from oracle import operator as oop, plan as opl
    uvw = synth.make_uvw(1500, 60, 1.28e9, 41)
    fov = math.radians(1.0)
    pp = opl.PlanParams(nx=64, ny=64, fov_x=fov, fov_y=fov, n_wbins=5)
    op = oop.Operator(uvw, opl.make_plan(uvw, pp))
    x = synth.make_sky(64, 42).astype(np.complex128)
    S = op.plan.s_w + pp.kb_support - 1
    taps = np.bincount(op.plan.bins, weights=(S * S).astype(np.float64), minlength=op.plan.P)
    return op, x, rd.bin_costs(taps, op.gx * op.gy)


def _worker(rank, ws, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for d in (root, os.path.join(root, "tests")):
        if d not in sys.path:
            sys.path.insert(0, d)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        op, x, costs = _case()
        parts = rd.partition_bins(costs, ws)
        t = torch.from_numpy(op.phi_adj_phi(x, bins=parts[rank]))
        dist.all_reduce(t)
        q.put((rank, parts, t.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_bin_sharded_apply_equals_full_apply(ws):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    results = [q.get(timeout=300) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    op, x, costs = _case()
    full = op.phi_adj_phi(x)
    parts = results[0][1]
    assert sorted(b for part in parts for b in part) == list(range(op.plan.P))
    for rank, parts_r, img in results:
        assert parts_r == parts
        assert np.linalg.norm(img - full) <= 1e-12 * np.linalg.norm(full)


def test_partition_is_balanced_and_deterministic():
    costs = np.array([9.0, 1.0, 8.0, 2.0, 7.0, 3.0, 6.0, 4.0, 5.0])
    p = rd.partition_bins(costs, 3)
    assert p == rd.partition_bins(costs, 3)
    loads = [sum(costs[b] for b in part) for part in p]
    # longest-processing-time first: makespan within 4/3 - 1/(3m) of the optimum, which is
    # at least max(mean load, largest bin)
    opt_lb = max(costs.sum() / 3, costs.max())
    assert max(loads) <= (4.0 / 3.0 - 1.0 / 9.0) * opt_lb + 1e-9
    even = rd.partition_bins([4.0] * 6, 3)
    assert [len(part) for part in even] == [2, 2, 2]
    assert rd.partition_bins(costs, 1) == [list(range(9))]
    # more ranks than bins: some ranks get nothing, every bin once
    p = rd.partition_bins([3.0, 1.0], 4)
    assert sorted(b for part in p for b in part) == [0, 1] and sum(1 for part in p if part) == 2
    # empty bins cost nothing
    assert rd.bin_costs([0, 10], 4096)[0] == 0.0


# ----------------------------------------------------------------------------- level 2
# Fourier-block sharding (Section 3.5, level 2): every w-bin's uv-tiles dealt over the ranks
# in radial order; each rank applies the oracle's Phi^dagger Phi to its visibilities only
# and the ranks all-reduce.  G_p^dagger G_p is a sum over visibilities (Eq. 8), so the sum
# must be the whole operator's image.

def _shards(op, ws):
    TS = 32
    return rd.tile_shards(op.plan.bins, op.geo.g0, op.geo.h0, op.gx, op.gy, TS, ws)


def _worker_blocks(rank, ws, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for d in (root, os.path.join(root, "tests")):
        if d not in sys.path:
            sys.path.insert(0, d)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        op, x, _ = _case()
        shard = _shards(op, ws)
        t = torch.from_numpy(op.phi_adj_phi(x, vis=shard == rank))
        dist.all_reduce(t)
        q.put((rank, int(np.sum(shard == rank)), t.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_block_sharded_apply_equals_full_apply(ws):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_blocks, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    results = [q.get(timeout=300) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    op, x, _ = _case()
    full = op.phi_adj_phi(x)
    assert sum(n for _, n, _ in results) == op.plan.bins.size      # every visibility once
    assert all(n > 0 for _, n, _ in results)
    for _, _, img in results:
        assert np.linalg.norm(img - full) <= 1e-12 * np.linalg.norm(full)


def test_tile_shards_deal_every_bins_tiles_in_radial_order():
    import synth
    uvw = synth.make_uvw(3000, 60, 1.28e9, 43)
    bins = np.arange(uvw.shape[0]) % 3
    gx = gy = 256
    g0 = np.floor(uvw[:, 0] * 0.05).astype(np.int64) % gx
    h0 = np.floor(uvw[:, 1] * 0.05).astype(np.int64) % gy
    for count in (1, 2, 3, 5):
        s = rd.tile_shards(bins, g0, h0, gx, gy, 32, count)
        assert np.array_equal(s, rd.tile_shards(bins, g0, h0, gx, gy, 32, count))
        assert s.min() >= 0 and s.max() < count
        for p in range(3):
            sel = bins == p
            tiles = (g0[sel] // 32) * (gy // 32) + h0[sel] // 32
            # a tile's visibilities share a shard, and the shards hold tile counts within one
            per_tile = {}
            for t, sh in zip(tiles, s[sel]):
                assert per_tile.setdefault(t, sh) == sh
            counts = np.bincount(list(per_tile.values()), minlength=count)
            assert counts.max() - counts.min() <= 1
            # the innermost tile (smallest radius) goes to shard 0
            tu, tv = np.array(list(per_tile.keys())) // (gy // 32), np.array(list(per_tile.keys())) % (gy // 32)
            cu = tu * 32 + 16.0
            cv = tv * 32 + 16.0
            cu = np.where(cu >= gx / 2, cu - gx, cu)
            cv = np.where(cv >= gy / 2, cv - gy, cv)
            r = np.hypot(cu, cv)
            inner = list(per_tile.keys())[int(np.lexsort((tv, tu, r))[0])]
            assert per_tile[inner] == 0
