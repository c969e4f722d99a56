"""Sharding Phi^dagger Phi over processes, at both levels of Section 3.5.

Level 1, by w-bin: Phi^dagger Phi = sum_p Phi_p^dagger Phi_p (Eq. 7), the w-bins are
independent, so each rank applies the bins of its share (rimo_apply_phi_adj_phi_bins) and
the partial images are summed with one all-reduce (the paper sums the per-layer images
along a tree of workers; NCCL or gloo does the reduction here).  Bins are shared out by a
longest-processing-time-first greedy on the per-bin terms of the cost model (Eq. 10):
2 (10 N' log2 sqrt(N') + 6 K_p) for a bin with K_p taps on an N'-cell grid.

Level 2, by Fourier block: G_p^dagger G_p is a sum over visibilities, so each rank holds a
shard plan (plan parameters shard_rank, shard_count) with every w-bin's uv-tiles dealt round
robin in radial order, stores G for their visibilities only, applies Phi^dagger Phi over all
bins, and the partial images are summed the same way.
"""
from __future__ import annotations

import math

import numpy as np


def bin_costs(taps_per_bin, grid_cells: int) -> np.ndarray:
    """Eq. 10's terms for each w-bin: FFT pair on the oversampled grid plus 6 K_p.

    Bins without visibilities cost nothing (they are skipped by the applies)."""
    k = np.asarray(taps_per_bin, dtype=np.float64)
    fft = 10.0 * grid_cells * math.log2(math.sqrt(grid_cells))
    return np.where(k > 0, 2.0 * (fft + 6.0 * k), 0.0)


def partition_bins(costs, world_size: int) -> list[list[int]]:
    """Bins per rank: the costliest bin first, each to the least-loaded rank (ties: the
    lower bin index first, the lower rank first).  Deterministic; every bin appears once."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    c = np.asarray(costs, dtype=np.float64)
    order = sorted(range(c.size), key=lambda b: (-c[b], b))
    load = [0.0] * world_size
    parts: list[list[int]] = [[] for _ in range(world_size)]
    for b in order:
        r = min(range(world_size), key=lambda q: (load[q], q))
        parts[r].append(b)
        load[r] += c[b]
    return [sorted(p) for p in parts]


def plan_bin_costs(plan) -> np.ndarray:
    """bin_costs from a plan's per-visibility bins and supports (host data of the plan)."""
    info = plan.info()
    _, bins, sw = plan.bins()
    J = int(plan.params.kb_support)
    S = sw.astype(np.int64) + J - 1
    taps = np.bincount(bins, weights=(S * S).astype(np.float64), minlength=info["P"])
    return bin_costs(taps, 4 * plan.nx * plan.ny)


def sharded_phi_adj_phi(plan, x, out=None, real_part_only: bool = False, group=None, costs=None):
    """This rank's bins of Phi^dagger Phi x, then the sum over the ranks of `group`
    (torch.distributed must be initialised; every rank holds the same plan and x)."""
    import torch.distributed as dist

    ws = dist.get_world_size(group)
    rank = dist.get_rank(group)
    parts = partition_bins(plan_bin_costs(plan) if costs is None else costs, ws)
    mask = np.zeros(plan.info()["P"], dtype=np.uint8)
    mask[parts[rank]] = 1
    out = plan.phi_adj_phi_bins(x, mask, out, real_part_only)
    dist.all_reduce(out, group=group)
    return out


def tile_shards(bins, g0, h0, gx: int, gy: int, TS: int, count: int) -> np.ndarray:
    """The shard of every visibility under level 2, as a shard plan assigns it: per w-bin the
    active uv-tiles (the tile of a visibility's first grid cell (g0, h0), reduced modulo the
    grid) in the order of the distance of their centre from the uv origin (signed
    coordinates; ties by tile row, then column), tile number i to shard i mod count."""
    b = np.asarray(bins, dtype=np.int64)
    tu = (np.asarray(g0, dtype=np.int64) % gx) // TS
    tv = (np.asarray(h0, dtype=np.int64) % gy) // TS
    ntv = gy // TS
    out = np.zeros(b.size, dtype=np.int64)
    for p in np.unique(b):
        sel = np.flatnonzero(b == p)
        tiles = np.unique(tu[sel] * ntv + tv[sel])
        cu = (tiles // ntv) * TS + 0.5 * TS
        cv = (tiles % ntv) * TS + 0.5 * TS
        cu = np.where(cu >= gx / 2, cu - gx, cu)
        cv = np.where(cv >= gy / 2, cv - gy, cv)
        r = np.sqrt(cu * cu + cv * cv)
        order = np.lexsort((tiles % ntv, tiles // ntv, r))   # by r, then row, then column
        shard_of_tile = np.empty(tiles.size, dtype=np.int64)
        shard_of_tile[order] = np.arange(tiles.size) % count
        out[sel] = shard_of_tile[np.searchsorted(tiles, tu[sel] * ntv + tv[sel])]
    return out


def shard_params(params, rank: int, count: int):
    """A copy of plan parameters for level-2 shard `rank` of `count` (stored G)."""
    from . import _lib
    import ctypes as C
    q = _lib.PlanParams()
    C.memmove(C.byref(q), C.byref(params), C.sizeof(q))
    q.shard_count = count
    q.shard_rank = rank
    return q


def block_sharded_phi_adj_phi(plan, x, out=None, real_part_only: bool = False, group=None):
    """Level 2: this rank's shard plan (made with shard_rank = the rank, shard_count = the
    group's size) applies Phi^dagger Phi over all bins, then the images are summed over the
    ranks of `group` (torch.distributed must be initialised; every rank holds the same x)."""
    import torch.distributed as dist

    ws = dist.get_world_size(group)
    rank = dist.get_rank(group)
    if plan.params.shard_count != ws or plan.params.shard_rank != rank:
        raise ValueError("the plan must be this rank's shard (shard_rank = rank, shard_count = world size)")
    out = plan.phi_adj_phi(x, out, real_part_only)
    dist.all_reduce(out, group=group)
    return out
