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
