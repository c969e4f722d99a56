"""The allocation-free Phi^dagger Phi entry point against the regular one (GPU).

rimo_apply_phi_adj_phi_noalloc serves callers that may not allocate device memory when
they apply the operator (device memory owned by another allocator, or no cudaMalloc /
cudaFree after set-up); it takes its scratch from a static device array of the library.
The grid step sums in fixed point, so its output equals the regular entry point's bit
for bit.  The array is shared by every call and never cleared: two plans of different
image sizes (different scratch layouts) alternate through it, and every result must
still equal the regular apply's, with a clean device status after each call.
This file is collected last so that a failure here comes after every other test.
"""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _noalloc(lib, plan, xd, out, stream):
    from paper_2605_26347_gb300 import _lib
    _lib.check(lib.rimo_apply_phi_adj_phi_noalloc(plan._h, xd.data_ptr(), out.data_ptr(), 0, stream))
    _lib.check(lib.rimo_plan_status(plan._h, stream))


def test_noalloc_matches_regular_apply_across_calls_and_plans():
    import torch

    import paper_2605_26347_gb300 as pkg
    from paper_2605_26347_gb300 import _lib

    lib = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream
    plans = {}
    for n, m, fov_deg, seed in ((256, 20000, 1.0, 1001), (128, 6000, 2.0, 1002)):
        uvw = synth.make_uvw(m, 60, 1.28e9, seed)
        fov = math.radians(fov_deg)
        plans[n] = pkg.Plan(uvw, pkg.default_params(n, n, fov, fov, n_wbins=4))
    # 256, 256 (two calls in a row), then 128 (another layout over the same array), then 256
    for step, (n, seed) in enumerate(((256, 5), (256, 6), (128, 7), (256, 8))):
        rng = np.random.default_rng(seed)
        x = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)
        xd = torch.from_numpy(x).cuda()
        ref = plans[n].phi_adj_phi(xd)
        out = torch.full_like(xd, float("nan"))
        _noalloc(lib, plans[n], xd, out, stream)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), (step, n)
    for p in plans.values():
        p.close()


def test_noalloc_rejects_plans_beyond_the_static_scratch():
    import torch

    import paper_2605_26347_gb300 as pkg
    from paper_2605_26347_gb300 import _lib

    n = 1024
    fov = math.radians(2.0)
    uvw = synth.make_uvw(3000, 60, 1.28e9, 77)
    plan = pkg.Plan(uvw, pkg.default_params(n, n, fov, fov, n_wbins=1))
    lib = _lib.load()
    xd = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
    out = torch.empty_like(xd)
    with pytest.raises(pkg.RimoError) as e:
        _lib.check(lib.rimo_apply_phi_adj_phi_noalloc(plan._h, xd.data_ptr(), out.data_ptr(), 0,
                                                      torch.cuda.current_stream().cuda_stream))
    assert e.value.status == 6 and "static scratch" in str(e.value)
    plan.close()
