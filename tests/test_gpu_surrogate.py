"""GPU parity of the kernel-surrogate MLP: forward, gradients and training (tcgen05).

The oracle (oracle/mlp.py) rounds to bf16 at the same points as the GPU and accumulates
in FP64, so the comparison isolates the tensor cores' FP32 accumulation order.  The GPU
computes the values it rounds to bf16 in FP32, the oracle in FP64: a value within
~1e-7 of a bf16 rounding boundary can round the other way (one bf16 ulp, 2^-8
relative).  A few such flips among the 10^5 activations of a batch move the outputs by
~1e-4 relative l2, hence the 1e-3 bound; a layout or index error moves them by O(1).
"""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def net():
    import paper_2605_26347_gb300 as pkg
    s = pkg.Surrogate(seed=0)
    p = omlp.init_params(11)
    s.set_params(pkg.pack_params(p))
    p32 = pkg.unpack_params(s.get_params())
    return s, {k: v.astype(np.float64) for k, v in p32.items()}


def batch(B, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, (B, 3)).astype(np.float32)
    t = (0.2 * rng.standard_normal((B, 450))).astype(np.float32)
    return x, t


def test_params_roundtrip(net):
    import paper_2605_26347_gb300 as pkg
    s, p = net
    q = pkg.unpack_params(s.get_params())
    for k in p:
        assert np.array_equal(q[k].astype(np.float64), p[k])


def test_forward_matches_oracle(net):
    s, p = net
    x, _ = batch(512, 1)
    y = s.forward(x).cpu().numpy().astype(np.float64)
    ref = omlp.forward(p, x.astype(np.float64), bf=True)["y"]
    assert rel(y, ref) < 1e-3


@pytest.mark.parametrize("B", [128, 1024])
def test_gradients_match_oracle(net, B):
    import paper_2605_26347_gb300 as pkg
    s, p = net
    x, t = batch(B, 2)
    loss, g = s.gradients(x, t)
    ref_loss, ref = omlp.loss_and_grads(p, x.astype(np.float64), t.astype(np.float64), bf=True)
    assert abs(loss - ref_loss) < 1e-4 * ref_loss
    gd = pkg.unpack_params(g)
    for k in ("W3", "b3", "W2", "b2", "W1", "b1"):
        assert rel(gd[k], ref[k]) < 2e-3, (k, rel(gd[k], ref[k]))


def test_training_reduces_loss():
    import paper_2605_26347_gb300 as pkg
    s = pkg.Surrogate(seed=3)
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, (2048, 3)).astype(np.float32)
    # a smooth target family the network can fit
    k = np.arange(450)[None, :]
    t = (np.sin(np.pi * (x[:, :1] * (1 + k % 3)) + x[:, 2:3] * (k % 5) / 5.0) * 0.3).astype(np.float32)
    first = s.train_step(x, t, 1e-3, want_loss=True)
    for _ in range(300):
        s.train_step(x, t, 1e-3)
    last = s.train_step(x, t, 1e-3, want_loss=True)
    assert last < 0.2 * first, (first, last)
