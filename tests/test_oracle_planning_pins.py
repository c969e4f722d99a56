"""Pins of the oracle's planning rules to hand-worked values (CPU only).

* The support rule of Section 3.1 (smallest centred odd block keeping a fraction eta of the
  w-kernel's l2 norm), on a separable geometric kernel whose block norms have a closed form,
  and on real w-kernels whose block norms the test accumulates ring by ring itself.
* The memory model (Eq. 9 restated for the device layout) and the cost model (Eq. 10) of
  Section 3.4, on tiny planning subsets worked by hand (tests/golden/planning_models.txt).
"""
import math

import numpy as np
import pytest

import golden_data
from oracle import plan as pl, wterm

SUPPORTS = "geometric_kernel_supports.txt"
MODELS = "planning_models.txt"


def geometric_kernel(L=32, r=0.5):
    a = np.abs(np.arange(L) - L // 2).astype(np.float64)
    k1 = r ** a
    return np.outer(k1, k1).astype(np.complex128)


def test_geometric_kernel_block_fractions_match_the_closed_form():
    K = geometric_kernel()
    want = golden_data.numbers(golden_data.load(SUPPORTS)["fractions"])
    c = K.shape[0] // 2
    total = math.sqrt(float(np.sum(np.abs(K) ** 2)))
    for h, f in enumerate(want):
        blk = K[c - h:c + h + 1, c - h:c + h + 1]
        assert abs(math.sqrt(float(np.sum(np.abs(blk) ** 2))) / total - f) < 1e-9


@pytest.mark.parametrize("row", golden_data.entries(SUPPORTS, "case"))
def test_support_of_hand_built_kernel(row):
    eta, cap, want, squared = golden_data.numbers(row)
    K = geometric_kernel()
    assert wterm.support_of(K, eta, int(cap)) == int(want)
    # the same kernel with its phase rotated per tap: only magnitudes enter the rule
    ph = np.exp(2j * math.pi * np.add.outer(np.arange(32) * 0.137, np.arange(32) * 0.291))
    assert wterm.support_of(K * ph, eta, int(cap)) == int(want)
    # the squared-norm reading differs on these rows (the fixture says where)
    if int(squared) != int(want):
        assert wterm.support_of(K, math.sqrt(eta), int(cap)) == int(squared)


def test_support_of_is_centred_on_the_zero_offset_tap():
    # the kernel peaked one tap off the centre keeps less in the centred block: at eta 0.99
    # the support grows from 7 to 9
    K = np.roll(geometric_kernel(), (1, 1), axis=(0, 1))
    assert wterm.support_of(geometric_kernel(), 0.99, 15) == 7
    assert wterm.support_of(K, 0.99, 15) == 9


def _ring_fractions(K):
    """Norm fraction of the centred (2h+1)^2 blocks, accumulated ring by ring."""
    L = K.shape[0]
    c = L // 2
    a = np.abs(np.arange(L) - c)
    ring = np.maximum(a[:, None], a[None, :])          # Chebyshev distance from the centre
    e2 = np.abs(K) ** 2
    per_ring = np.array([e2[ring == h].sum() for h in range(c + 1)])
    return np.sqrt(np.cumsum(per_ring) / e2.sum())


@pytest.mark.parametrize("w_r", [15.0, 60.0, 180.0, 400.0])
@pytest.mark.parametrize("eta", [0.99, 0.9999])
def test_support_of_real_wkernels_keeps_eta_and_the_next_smaller_does_not(w_r, eta):
    fov = math.radians(3.0)
    L = 64
    K = wterm.wkernel_full(w_r, L, fov, fov)
    frac = _ring_fractions(K)
    cap = 31
    s = wterm.support_of(K, eta, cap)
    h = s // 2
    if s < cap:
        assert frac[h] >= eta
    if s > 1:
        assert frac[h - 1] < eta


@pytest.mark.parametrize("name", ["A", "B", "C"])
def test_planning_models_match_hand_worked_values(name):
    head, w_txt, want_txt = golden_data.load(MODELS)[name].split("|")
    P, M, nx, ny = (int(v) for v in golden_data.numbers(head))
    w_sub = np.array(golden_data.numbers(w_txt))
    K, m_G, cost = golden_data.numbers(want_txt)
    fov = 0.1
    pp = pl.PlanParams(nx=nx, ny=ny, fov_x=fov, fov_y=fov, max_wsupport=3, w_norm_frac=1.0)
    d = pl.model_for_P(w_sub, M, P, pp)
    assert d["P"] == P
    assert d["K"] == pytest.approx(K, rel=1e-12)
    assert d["m_G"] == pytest.approx(m_G, rel=1e-12)
    assert d["cost"] == pytest.approx(cost, rel=1e-12)
