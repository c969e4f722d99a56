"""GPU parity: Phi, Phi^dagger, Phi^dagger Phi, PSF and G taps against the FP64 oracle.

Element-by-element comparison through the C ABI on seeded synthetic inputs.  The
bar is a relative l2 error <= 1e-5 (complex FP32 against FP64).
"""
import math

import numpy as np
import pytest

import synth
from parity_util import TOL, assert_same_plan, both, rel, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mono256():
    """Monochromatic 256^2 workload: FoV 1 deg, 20k visibilities, 4 w-bins."""
    w = synth.make_config(1)
    fov = w.fov_rad
    plan, op = both(w.uvw, 256, 256, fov, fov, n_wbins=4)
    return w, plan, op


def test_mono256_plan_agrees(mono256):
    _, plan, op = mono256
    assert_same_plan(plan, op)
    info = plan.info()
    assert info["P"] == 4 and info["K"] == op.plan.K


def test_mono256_taps(mono256):
    w, plan, op = mono256
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(w.uvw.shape[0], 300, replace=False))
    g0, h0, S, taps = plan.tiles(idx)
    ref = op.tiles(idx)
    for q, k in enumerate(idx):
        assert S[q] == op.geo.S[k]
        assert g0[q] == op.geo.g0[k] % op.gx and h0[q] == op.geo.h0[k] % op.gy
        assert rel(taps[q], ref[q]) < TOL, (k, rel(taps[q], ref[q]))


def test_mono256_phi(mono256):
    w, plan, op = mono256
    y = to_host(plan.phi(to_dev(w.sky)))
    assert rel(y, op.phi(w.sky)) < TOL


def test_mono256_phi_adj(mono256):
    w, plan, op = mono256
    rng = np.random.default_rng(1)
    y = (rng.standard_normal(w.uvw.shape[0]) + 1j * rng.standard_normal(w.uvw.shape[0])).astype(np.complex64)
    x = to_host(plan.phi_adj(to_dev(y)))
    assert rel(x, op.phi_adj(y.astype(np.complex128))) < TOL


def test_mono256_phi_adj_phi_and_real_part(mono256):
    w, plan, op = mono256
    ref = op.phi_adj_phi(w.sky)
    out = to_host(plan.phi_adj_phi(to_dev(w.sky)))
    assert rel(out, ref) < TOL
    out_re = to_host(plan.phi_adj_phi(to_dev(w.sky), real_part_only=True))
    assert np.all(out_re.imag == 0)
    assert rel(out_re.real, ref.real) < TOL


def test_device_status_is_clean_after_applies(mono256):
    import torch
    import paper_2605_26347_gb300 as pkg
    w, plan, _ = mono256
    plan.phi_adj_phi(to_dev(w.sky))
    pkg._lib.check(plan._lib.rimo_plan_status(plan._h, torch.cuda.current_stream().cuda_stream))


def test_mono256_psf(mono256):
    _, plan, op = mono256
    psf = to_host(plan.psf())
    ref = op.psf()
    assert rel(psf, ref) < TOL
    assert np.argmax(np.abs(psf)) == 128 * 256 + 128


def test_mono256_fused_equals_sequential_and_adjoint_identity(mono256):
    import torch
    w, plan, _ = mono256
    rng = np.random.default_rng(2)
    x = (rng.standard_normal((256, 256)) + 1j * rng.standard_normal((256, 256))).astype(np.complex64)
    y = (rng.standard_normal(w.uvw.shape[0]) + 1j * rng.standard_normal(w.uvw.shape[0])).astype(np.complex64)
    xd = to_dev(x)
    fused = to_host(plan.phi_adj_phi(xd))
    seq = to_host(plan.phi_adj(plan.phi(xd)))
    assert rel(fused, seq) < 2e-6
    lhs = np.vdot(y.astype(np.complex128), to_host(plan.phi(xd)))
    rhs = np.vdot(to_host(plan.phi_adj(to_dev(y))), x.astype(np.complex128))
    assert abs(lhs - rhs) < 1e-5 * abs(lhs)
    torch.cuda.synchronize()


@pytest.mark.parametrize("case", [
    # rectangular image and field, odd M, 3 bins, J = 5, 1/n weighting
    dict(nx=128, ny=64, fx=2.0, fy=1.5, m=777, kw=dict(n_wbins=3, kb_support=5, n_weight=1)),
    # one visibility, one bin
    dict(nx=64, ny=64, fx=1.0, fy=1.0, m=1, kw=dict(n_wbins=1)),
    # J = 9 with a w-kernel cap of 5, literal taper, L = 32, tile size 32
    dict(nx=256, ny=128, fx=2.0, fy=2.0, m=3000,
         kw=dict(n_wbins=2, kb_support=9, max_wsupport=5, taper_literal=1, wkernel_L=32, tile_size=32)),
    # automatic P, J = 3, energy fraction 0.99, tile size 64
    dict(nx=128, ny=128, fx=3.0, fy=3.0, m=5000, kw=dict(kb_support=3, w_norm_frac=0.99, tile_size=64)),
    # the largest tiles: J = 11 with 9 x 9 w-kernels, S = 19 (two column groups per tap row,
    # taps re-read for the grid step)
    dict(nx=128, ny=128, fx=2.0, fy=2.0, m=2500, kw=dict(n_wbins=2, kb_support=11, max_wsupport=9, w_norm_frac=1.0)),
    # w-kernel grids L = 16 (4 lanes per folded column) and L = 128 (2 columns per lane)
    dict(nx=128, ny=128, fx=2.0, fy=2.0, m=1500, kw=dict(n_wbins=2, max_wsupport=3, wkernel_L=16)),
    dict(nx=128, ny=128, fx=2.5, fy=2.5, m=1500, kw=dict(n_wbins=2, wkernel_L=128)),
])
def test_ragged_and_edge_cases(case):
    uvw = synth.make_uvw(case["m"], 60, 1.28e9, 500 + case["m"])
    fx, fy = math.radians(case["fx"]), math.radians(case["fy"])
    plan, op = both(uvw, case["nx"], case["ny"], fx, fy, **case["kw"])
    assert_same_plan(plan, op)
    rng = np.random.default_rng(3)
    x = (rng.standard_normal((case["ny"], case["nx"])) + 0.1j).astype(np.complex64)
    y = (rng.standard_normal(case["m"]) + 1j * rng.standard_normal(case["m"])).astype(np.complex64)
    assert rel(to_host(plan.phi(to_dev(x))), op.phi(x.astype(np.complex128))) < TOL
    assert rel(to_host(plan.phi_adj(to_dev(y))), op.phi_adj(y.astype(np.complex128))) < TOL
    assert rel(to_host(plan.phi_adj_phi(to_dev(x))), op.phi_adj_phi(x.astype(np.complex128))) < TOL


def test_empty_bins_give_zero_contribution():
    # all visibilities share one w: with 3 requested bins two stay empty
    uvw = synth.make_uvw(400, 60, 1.28e9, 9)
    uvw[:, 2] = 123.0
    fov = math.radians(1.0)
    plan, op = both(uvw, 64, 64, fov, fov, n_wbins=3)
    x = synth.make_sky(64, 4)
    assert rel(to_host(plan.phi_adj_phi(to_dev(x))), op.phi_adj_phi(x.astype(np.complex128))) < TOL


def test_invalid_buffers_are_rejected(mono256):
    import torch
    import paper_2605_26347_gb300 as pkg
    _, plan, _ = mono256
    x = torch.zeros((256, 256), dtype=torch.complex64, device="cuda")
    with pytest.raises(pkg.RimoError) as e:
        pkg._lib.check(plan._lib.rimo_apply_phi_adj_phi(plan._h, x.data_ptr(), x.data_ptr(), 0, None))
    assert e.value.status == 1
    with pytest.raises(ValueError):
        plan.phi(torch.zeros((128, 256), dtype=torch.complex64, device="cuda"))


def test_grid_step_sums_do_not_depend_on_timing(mono256):
    # the grid step adds integers (fixed point), so repeated applies agree bit for bit
    w, plan, _ = mono256
    rng = np.random.default_rng(5)
    y = (rng.standard_normal(w.uvw.shape[0]) + 1j * rng.standard_normal(w.uvw.shape[0])).astype(np.complex64)
    xd, yd = to_dev(w.sky), to_dev(y)
    a, b = to_host(plan.phi_adj_phi(xd)), to_host(plan.phi_adj_phi(xd))
    assert np.array_equal(a, b)
    a, b = to_host(plan.phi_adj(yd)), to_host(plan.phi_adj(yd))
    assert np.array_equal(a, b)


@pytest.mark.parametrize("scale", [1e-20, 1e-6, 1e6, 1e20])
def test_grid_step_follows_input_magnitude(mono256, scale):
    # the fixed-point scales come from bounds on the inputs: any magnitude keeps the accuracy
    w, plan, op = mono256
    rng = np.random.default_rng(6)
    y = (rng.standard_normal(w.uvw.shape[0]) + 1j * rng.standard_normal(w.uvw.shape[0]))
    ref_adj = op.phi_adj(y)
    ref_ata = op.phi_adj_phi(w.sky.astype(np.complex128))
    out_adj = to_host(plan.phi_adj(to_dev((y * scale).astype(np.complex64)))) / scale
    out_ata = to_host(plan.phi_adj_phi(to_dev((w.sky * scale).astype(np.complex64)))) / scale
    assert rel(out_adj, ref_adj) < TOL
    assert rel(out_ata, ref_ata) < TOL


def test_non_finite_input_is_reported(mono256):
    import torch
    import paper_2605_26347_gb300 as pkg
    w, plan, _ = mono256
    stream = torch.cuda.current_stream().cuda_stream
    x = w.sky.copy()
    x[17, 3] = np.nan
    plan.phi_adj_phi(to_dev(x))
    with pytest.raises(pkg.RimoError) as e:
        pkg._lib.check(plan._lib.rimo_plan_status(plan._h, stream))
    assert e.value.status == 1
    y = np.ones(w.uvw.shape[0], dtype=np.complex64)
    y[5] = np.inf
    plan.phi_adj(to_dev(y))
    with pytest.raises(pkg.RimoError):
        pkg._lib.check(plan._lib.rimo_plan_status(plan._h, stream))
    # the flag is cleared and finite inputs work again
    plan.phi_adj_phi(to_dev(w.sky))
    pkg._lib.check(plan._lib.rimo_plan_status(plan._h, stream))


@pytest.mark.parametrize("n", [1024, 4096])
def test_large_image_parity(n):
    # image sizes whose transposed-store passes run as thread-block clusters (2 and 4 CTAs)
    uvw = synth.make_uvw(20000, 28_800, 1.28e9, 700 + n)
    fov = math.radians(3.0)
    plan, op = both(uvw, n, n, fov, fov, n_wbins=2)
    assert_same_plan(plan, op)
    x = synth.make_sky(n, 800 + n)
    rng = np.random.default_rng(n)
    y = (rng.standard_normal(20000) + 1j * rng.standard_normal(20000)).astype(np.complex64)
    assert rel(to_host(plan.phi(to_dev(x))), op.phi(x.astype(np.complex128))) < TOL
    assert rel(to_host(plan.phi_adj(to_dev(y))), op.phi_adj(y.astype(np.complex128))) < TOL
    assert rel(to_host(plan.phi_adj_phi(to_dev(x))), op.phi_adj_phi(x.astype(np.complex128))) < TOL


def test_bin_subsets_sum_to_the_full_apply(mono256):
    # Eq. 7 term by term: disjoint bin subsets add up to Phi^dagger Phi
    import torch
    w, plan, op = mono256
    xd = to_dev(w.sky)
    P = plan.info()["P"]
    m1 = np.zeros(P, np.uint8)
    m1[::2] = 1
    a = to_host(plan.phi_adj_phi_bins(xd, m1))
    b = to_host(plan.phi_adj_phi_bins(xd, 1 - m1))
    full = to_host(plan.phi_adj_phi(xd))
    assert rel(a + b, full) < 1e-6
    assert rel(a, op.phi_adj_phi(w.sky.astype(np.complex128), bins=list(np.nonzero(m1)[0]))) < TOL
    assert not np.any(to_host(plan.phi_adj_phi_bins(xd, np.zeros(P, np.uint8))))
    torch.cuda.synchronize()


def test_sharded_apply_on_one_nccl_rank(mono256):
    import socket
    import torch
    import torch.distributed as dist
    from paper_2605_26347_gb300 import distributed as rd
    w, plan, _ = mono256
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        xd = to_dev(w.sky)
        got = to_host(rd.sharded_phi_adj_phi(plan, xd))
        assert rel(got, to_host(plan.phi_adj_phi(xd))) < 1e-6
    finally:
        dist.destroy_process_group()
