"""Shared helpers of the GPU parity tests: build a plan on both sides and compare."""
from __future__ import annotations

import math

import numpy as np

from oracle import operator as oop
from oracle import plan as opl

TOL = 1e-5  # relative l2 error of complex FP32 results against the FP64 oracle


def rel(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def oracle_params(nx, ny, fov_x, fov_y, **kw) -> opl.PlanParams:
    names = dict(div_n="n_weight", taper_literal="taper_literal")
    args = dict(nx=nx, ny=ny, fov_x=fov_x, fov_y=fov_y)
    for k, v in kw.items():
        if k == "n_weight":
            args["div_n"] = bool(v)
        elif k in ("tile_size", "block_bytes_max", "uv_order"):
            continue
        elif k == "taper_literal":
            args["taper_literal"] = bool(v)
        else:
            args[k] = v
    del names
    return opl.PlanParams(**args)


def both(uvw, nx, ny, fov_x, fov_y, **kw):
    """(product Plan, oracle Operator) for the same uvw and parameters."""
    import paper_2605_26347_gb300 as pkg
    params = pkg.default_params(nx, ny, fov_x, fov_y, **kw)
    plan = pkg.Plan(uvw, params)
    oplan = opl.make_plan(uvw, oracle_params(nx, ny, fov_x, fov_y, **kw))
    op = oop.Operator(uvw, oplan)
    return plan, op


def assert_same_plan(plan, op):
    ws, b, s = plan.bins()
    assert ws.shape[0] == op.plan.P
    assert np.allclose(ws, op.plan.w_stack, rtol=1e-12, atol=1e-9)
    diff = np.nonzero(b != op.plan.bins)[0]
    # a visibility may only change bin where it is equidistant to two centroids
    for k in diff:
        w = op.uvw[k, 2]
        d1 = abs(w - op.plan.w_stack[b[k]])
        d2 = abs(w - op.plan.w_stack[op.plan.bins[k]])
        assert abs(d1 - d2) <= 1e-9 * max(1.0, abs(w)), k
    assert diff.size == 0, f"{diff.size} visibilities changed bin"
    assert np.array_equal(s, op.plan.s_w)


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a.astype(np.complex64))).cuda()


def to_host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)
