"""Sharding Phi^dagger Phi over processes by w-bin.

Phi^dagger Phi = sum_p Phi_p^dagger Phi_p (Eq. 7): the w-bins are independent, so each
rank applies the bins of its share (rimo_apply_phi_adj_phi_bins) and the partial images
are summed with one all-reduce (the paper sums the per-layer images along a tree of
workers, Section 3.5; NCCL or gloo does the reduction here).  Bins are shared out by a
longest-processing-time-first greedy on the per-bin terms of the cost model (Eq. 10):
2 (10 N' log2 sqrt(N') + 6 K_p) for a bin with K_p taps on an N'-cell grid.
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
