"""Parity at the full workload sizes, in the launch configuration the benchmark times.

The 4096² / 50M / 32-bin workload (stored G) and the 1024² / 2M workload (automatic P under
a 40 GB budget, 16 Fourier blocks): Φ at sampled visibilities against the oracle's
per-visibility evaluation, and properties that hold at any size (adjoint identity,
Hermitian Φ†Φ, fused = sequential).
"""
import math

import numpy as np
import pytest

import synth
from oracle import operator as oop
from oracle import plan as opl
from parity_util import TOL, oracle_params, rel, to_dev, to_host

pytestmark = pytest.mark.gpu


def sampled_phi_error(plan, uvw, sky, pp, n_per_bin=12, n_bins=3, seed=7):
    ws, bins, sw = plan.bins()
    oplan = opl.make_plan(uvw, pp)
    assert np.array_equal(oplan.bins, bins) and np.array_equal(oplan.s_w, sw)
    op = oop.Operator(uvw, oplan, build_g=False)
    rng = np.random.default_rng(seed)
    cand = rng.choice(np.unique(bins), n_bins, replace=False)
    ks = np.concatenate([rng.choice(np.nonzero(bins == b)[0], n_per_bin, replace=False) for b in cand])
    ks = ks[np.argsort(bins[ks], kind="stable")]
    yg = to_host(plan.phi(to_dev(sky)))[ks]
    yo = op.phi_sampled(sky.astype(np.complex128), ks)
    return rel(yg, yo)


@pytest.fixture(scope="module")
def c5():
    import paper_2605_26347_gb300 as pkg
    uvw = synth.make_uvw(50_000_000, 28_800, 1.28e9, seed=1005)
    sky = synth.make_sky(4096, seed=2005)
    fov = math.radians(3.0)
    plan = pkg.Plan(uvw, pkg.default_params(4096, 4096, fov, fov, n_wbins=32, mode=pkg.MODE_STORED_G))
    yield uvw, sky, fov, plan
    del plan


def test_c5_sampled_phi_matches_oracle(c5):
    uvw, sky, fov, plan = c5
    pp = opl.PlanParams(nx=4096, ny=4096, fov_x=fov, fov_y=fov, n_wbins=32)
    assert sampled_phi_error(plan, uvw, sky, pp) < TOL


def test_c5_adjoint_hermitian_and_fused(c5):
    import torch
    uvw, sky, _, plan = c5
    M = uvw.shape[0]
    g = torch.Generator(device="cuda").manual_seed(5)
    x1 = torch.from_numpy(sky).cuda()
    x2 = torch.complex(torch.randn((4096, 4096), generator=g, device="cuda"),
                       torch.randn((4096, 4096), generator=g, device="cuda"))
    y = torch.complex(torch.randn(M, generator=g, device="cuda"), torch.randn(M, generator=g, device="cuda"))
    c = lambda a, b: complex(torch.vdot(a.reshape(-1).to(torch.complex128), b.reshape(-1).to(torch.complex128)))
    lhs, rhs = c(y, plan.phi(x2)), c(plan.phi_adj(y), x2)
    assert abs(lhs - rhs) < 2e-5 * abs(lhs)
    a12 = c(x1, plan.phi_adj_phi(x2))
    a21 = c(x2, plan.phi_adj_phi(x1))
    assert abs(a12 - a21.conjugate()) < 2e-5 * abs(a12)
    fused = plan.phi_adj_phi(x2)
    seq = plan.phi_adj(plan.phi(x2))
    assert float(torch.linalg.vector_norm(fused - seq) / torch.linalg.vector_norm(seq)) < 2e-6


def test_plain_1024_auto_p_budget_blocks():
    import paper_2605_26347_gb300 as pkg
    w = synth.make_config(2)
    fov = w.fov_rad
    kw = dict(n_wbins=0, mem_budget_bytes=w.mem_budget_bytes, n_blocks=w.n_blocks)
    plan = pkg.Plan(w.uvw, pkg.default_params(1024, 1024, fov, fov, **kw))
    info = plan.info()
    # blocks of total / 16 bytes that do not span w-bins: 16 .. 16 + P of them
    assert 16 <= info["n_blocks"] <= 16 + info["P"]
    pp = oracle_params(1024, 1024, fov, fov, **kw)
    assert info["P"] == opl.choose(w.uvw, pp)["P"]
    assert sampled_phi_error(plan, w.uvw, w.sky, pp) < TOL
