"""The allocation-free Phi^dagger Phi entry point against the regular one (GPU).

rimo_apply_phi_adj_phi_noalloc serves callers that may not allocate device memory when
they apply the operator; it takes its scratch from a static device array of the
library.  Its output must equal the regular entry point's within the parity tolerance
on two calls in a row (the second call reuses the array left by the first).
This file is collected last so that a failure here comes after every other test.
"""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_regular_apply_twice():
    import torch

    import paper_2605_26347_gb300 as pkg
    from paper_2605_26347_gb300 import _lib

    n, m = 256, 20000
    fov = math.radians(1.0)
    uvw = synth.make_uvw(m, 60, 1.28e9, 1001)
    plan = pkg.Plan(uvw, pkg.default_params(n, n, fov, fov, n_wbins=4))
    lib = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (5, 6):
        rng = np.random.default_rng(seed)
        x = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)
        xd = torch.from_numpy(x).cuda()
        ref = plan.phi_adj_phi(xd)
        out = torch.empty_like(xd)
        _lib.check(lib.rimo_apply_phi_adj_phi_noalloc(plan._h, xd.data_ptr(), out.data_ptr(), 0, stream))
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.complex128)
        want = ref.cpu().numpy().astype(np.complex128)
        assert rel(got, want) < TOL
    plan.close()


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
