"""Failure detection on the device without a fault (GPU).

Every wait of the grid step is bounded.  rimo_plan_set_wait_test makes one of them run
out: the consumer warps withhold their release of tap-ring slots (a flag that nothing
sets) and the producer's waits on them give up after a few polls.  The launch must end by
itself, the plan's status must report RIMO_ERR_TIMEOUT (and clear), and the next apply
at the normal limit must be clean and equal, bit for bit, to the apply before the test.
"""
import math
import time

import numpy as np
import pytest

import synth
from parity_util import to_dev, to_host

pytestmark = pytest.mark.gpu

TIMEOUT = 5


@pytest.mark.parametrize("n, m, fov_deg", [
    # 128^2, 20k visibilities, one w-bin: a few dozen uv-tiles of ~300 visibilities, so every
    # block of the grid step streams more tap chunks than its ring holds (two X buffers)
    (128, 20000, 2.0),
    # 512^2, 60k visibilities: units of a few chunks (three X buffers, two units ahead)
    (512, 60000, 2.0),
])
def test_bounded_wait_runs_out_then_the_plan_recovers(n, m, fov_deg):
    import torch

    import paper_2605_26347_gb300 as pkg
    fov = math.radians(fov_deg)
    uvw = synth.make_uvw(m, 60, 1.28e9, 4242)
    plan = pkg.Plan(uvw, pkg.default_params(n, n, fov, fov, n_wbins=1))
    x = to_dev(synth.make_sky(n, 4243))
    before = to_host(plan.phi_adj_phi(x))
    plan.status()
    plan.set_wait_test(True, polls=16)
    t = time.time()
    plan.phi_adj_phi(x)
    torch.cuda.synchronize()
    assert time.time() - t < 2.0          # each block gives up after <= 16 polls of <= 100 us
    with pytest.raises(pkg.RimoError) as e:
        plan.status()
    assert e.value.status == TIMEOUT
    plan.status()                          # the flag was cleared by the report
    plan.set_wait_test(False)
    after = to_host(plan.phi_adj_phi(x))
    plan.status()
    assert np.array_equal(after, before)
    with pytest.raises(pkg.RimoError):
        plan.set_wait_test(True, polls=0)
    plan.close()
