"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test checks the oracle against something it does not compute the same
way: a library routine for a special case, numerical quadrature, brute-force
sums of the paper's equations, closed forms and invariants of the operator.
"""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as ss

import golden_data
import synth
from oracle import direct, kb, operator, plan as pl, wterm


def small_case(m=400, n=32, fov_deg=4.0, uv_scale=0.1, w_scale=0.01, seed=11):
    uvw = synth.make_uvw(m, 60, 1.28e9, seed) * np.array([uv_scale, uv_scale, w_scale])
    x = synth.make_sky(n, seed + 1).astype(np.complex128)
    return uvw, x, math.radians(fov_deg)


def make_op(uvw, n, fov, **kw):
    args = dict(nx=n, ny=n, fov_x=fov, fov_y=fov, n_wbins=1, max_wsupport=9, w_norm_frac=1.0,
                wkernel_L=64)
    args.update(kw)
    pp = pl.PlanParams(**args)
    return operator.Operator(uvw, pl.make_plan(uvw, pp))


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ---------------------------------------------------------------- KB kernel
def test_i0_matches_library_bessel():
    x = np.linspace(0.0, 30.0, 301)
    assert np.max(np.abs(kb.i0(x) / ss.i0(x) - 1.0)) < 1e-14


@pytest.mark.parametrize("nu", [0.0, 0.1, 0.23, 0.37, 0.5])
def test_kb_hat_matches_quadrature(nu):
    J, beta = 7, 2.34 * 7
    re, _ = si.quad(lambda t: float(kb.kb(t, J, beta)) * math.cos(2 * math.pi * nu * t),
                    -J / 2, J / 2, epsabs=1e-14, epsrel=1e-13, limit=200)
    assert abs(float(kb.kb_hat(nu, J, beta)) - re) < 1e-11 * max(1.0, abs(re))


def test_kb_taps_sum_tracks_kb_hat_zero():
    # Poisson summation: sum_g KB(u - g) = KB_hat(0) up to aliasing far below 1e-6 for J=7
    J, beta = 7, 2.34 * 7
    phi = np.linspace(0.0, 0.999, 50)
    s = kb.kb_taps(phi, J, beta).sum(axis=1)
    assert np.max(np.abs(s / float(kb.kb_hat(0.0, J, beta)) - 1.0)) < 1e-6


# ---------------------------------------------------------------- oversampled DFT
def test_forward_grid_is_the_oversampled_dft():
    n = 16
    uvw, _, fov = small_case(m=50, n=n)
    O = make_op(uvw, n, fov)
    rng = np.random.default_rng(0)
    z = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    X = O.fwd_grid(z)
    jc = np.arange(n) - n // 2
    g = np.arange(2 * n)
    Eu = np.exp(-2j * math.pi * np.outer(g, jc) / (2 * n))   # [g_u, j]
    ref = np.einsum("ui,vj,ji->uv", Eu, Eu, z)                # X[g_u, g_v] = sum z[i,j] e_u(g_u,j) e_v(g_v,i)
    assert rel(X, ref) < 1e-13


def test_adjoint_grid_is_the_cropped_inverse_dft():
    n = 16
    uvw, _, fov = small_case(m=50, n=n)
    O = make_op(uvw, n, fov)
    rng = np.random.default_rng(1)
    Xh = rng.standard_normal((2 * n, 2 * n)) + 1j * rng.standard_normal((2 * n, 2 * n))
    z = O.adj_grid(Xh)
    jc = np.arange(n) - n // 2
    g = np.arange(2 * n)
    E = np.exp(2j * math.pi * np.outer(jc, g) / (2 * n))     # [j, g]
    ref = np.einsum("ju,iv,uv->ij", E, E, Xh)
    assert rel(z, ref) < 1e-13


# ---------------------------------------------------------------- Phi vs the measurement equation
def test_w_zero_is_kb_nufft_and_error_falls_with_J():
    n = 32
    uvw, x, fov = small_case(m=500, n=n, w_scale=0.0)
    yd = direct.direct_phi(x, uvw, fov, fov)
    errs = []
    for J in (5, 7, 9, 11):
        O = make_op(uvw, n, fov, kb_support=J)
        assert np.all(O.plan.s_w == 1)
        errs.append(rel(O.phi(x), yd))
    assert errs[1] < 2e-6 and errs[3] < 1e-9
    assert all(errs[i + 1] < 0.1 * errs[i] for i in range(3))


def test_w_zero_tiles_are_kb_outer_products():
    n = 32
    uvw, _, fov = small_case(m=20, n=n, w_scale=0.0)
    O = make_op(uvw, n, fov)
    T = O.tiles(np.arange(5))
    for k in range(5):
        wu = kb.kb_taps(O.geo.phi_u[k], 7, 2.34 * 7)
        wv = kb.kb_taps(O.geo.phi_v[k], 7, 2.34 * 7)
        assert np.max(np.abs(T[k] - np.outer(wu, wv))) < 1e-15


def test_widefield_error_falls_with_kernel_support():
    n = 32
    uvw, x, fov = small_case(m=300, n=n, w_scale=0.01)
    yd = direct.direct_phi(x, uvw, fov, fov)
    errs = [rel(make_op(uvw, n, fov, max_wsupport=s, wkernel_L=L).phi(x), yd)
            for s, L in ((9, 64), (15, 64), (31, 64), (63, 128))]
    assert all(errs[i + 1] < 0.7 * errs[i] for i in range(3)), errs
    assert errs[-1] < 1e-4


def test_widefield_error_falls_with_wkernel_sampling_when_support_allows():
    # Section 3.1: the w-kernel is the DFT of the chirp sampled on an L x L grid over twice
    # the FoV; with a support wide enough not to cut it, a finer grid lowers the error
    # until the NUFFT error dominates (with 9 taps the support cut dominates at every L)
    n = 32
    uvw, x, fov = small_case(m=300, n=n, w_scale=0.01)
    yd = direct.direct_phi(x, uvw, fov, fov)
    errs = [rel(make_op(uvw, n, fov, max_wsupport=31, wkernel_L=L).phi(x), yd) for L in (32, 64, 128)]
    assert errs[1] < 0.7 * errs[0] and errs[2] < errs[1], errs


def test_div_n_option_matches_eq2_with_one_over_n():
    n = 32
    uvw, x, fov = small_case(m=200, n=n, w_scale=0.0)
    O = make_op(uvw, n, fov, kb_support=9, div_n=True)
    assert rel(O.phi(x), direct.direct_phi(x, uvw, fov, fov, div_n=True)) < 1e-7


def test_number_of_wbins_does_not_change_phi_beyond_model_error():
    # Section 3.1: P changes cost, not accuracy
    n = 32
    uvw, x, fov = small_case(m=300, n=n, w_scale=0.01)
    yd = direct.direct_phi(x, uvw, fov, fov)
    ys = {P: make_op(uvw, n, fov, n_wbins=P, max_wsupport=31).phi(x) for P in (1, 4, 16)}
    e = {P: rel(ys[P], yd) for P in ys}
    assert max(e.values()) < 2e-4
    for P in (4, 16):
        assert rel(ys[P], ys[1]) < 2.0 * (e[1] + e[P])


def test_wrap_invariance_of_u():
    # the pixel-grid model is periodic in u with period n_x / FoV_x
    n = 32
    uvw, x, fov = small_case(m=200, n=n, w_scale=0.01)
    y0 = make_op(uvw, n, fov).phi(x)
    sh = uvw.copy()
    sh[:, 0] += 3 * n / fov
    sh[:, 1] -= 2 * n / fov
    y1 = make_op(sh, n, fov).phi(x)
    assert rel(y1, y0) < 1e-9


# ---------------------------------------------------------------- adjoint, H, PSF
def test_adjoint_identity():
    n = 32
    uvw, x, fov = small_case(m=400, n=n, w_scale=0.01)
    O = make_op(uvw, n, fov, n_wbins=3)
    rng = np.random.default_rng(5)
    y = rng.standard_normal(uvw.shape[0]) + 1j * rng.standard_normal(uvw.shape[0])
    lhs = np.vdot(y, O.phi(x))
    rhs = np.vdot(O.phi_adj(y), x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_direct_adjoint_identity():
    n = 16
    uvw, x, fov = small_case(m=100, n=n)
    rng = np.random.default_rng(6)
    y = rng.standard_normal(100) + 1j * rng.standard_normal(100)
    lhs = np.vdot(y, direct.direct_phi(x, uvw, fov, fov))
    rhs = np.vdot(direct.direct_phi_adj(y, uvw, n, n, fov, fov), x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_holographic_matrix_is_g_dagger_g_and_hermitian():
    n = 32
    uvw, x, fov = small_case(m=300, n=n, w_scale=0.01)
    O = make_op(uvw, n, fov, n_wbins=2)
    rng = np.random.default_rng(7)
    for p in range(2):
        H = O.holographic(p)
        z = rng.standard_normal(H.shape[0]) + 1j * rng.standard_normal(H.shape[0])
        ref = O.G[p].conj().T @ (O.G[p] @ z)
        assert rel(H @ z, ref) < 1e-13
        assert abs(H - H.conj().T).max() < 1e-14 * abs(H).max()


def test_phi_adj_phi_and_psf():
    n = 32
    uvw, x, fov = small_case(m=300, n=n, w_scale=0.01)
    O = make_op(uvw, n, fov, n_wbins=2)
    assert rel(O.phi_adj_phi(x), O.phi_adj(O.phi(x))) < 1e-13
    psf = O.psf()
    d = np.zeros((n, n), dtype=complex)
    d[n // 2, n // 2] = 1.0
    yd = O.phi(d)
    # PSF peak = <Phi delta, Phi delta> (adjoint relation), real and maximal
    assert abs(psf[n // 2, n // 2] - np.vdot(yd, yd)) < 1e-12 * abs(psf[n // 2, n // 2])
    assert np.argmax(np.abs(psf)) == (n // 2) * n + n // 2
    # Phi^dagger Phi is Hermitian positive semi-definite
    rng = np.random.default_rng(8)
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    q = np.vdot(a, O.phi_adj_phi(a))
    assert abs(q.imag) < 1e-12 * abs(q) and q.real > 0


# ---------------------------------------------------------------- w-kernels and planning
def test_wkernel_zero_offset_is_delta_and_conjugate_symmetry():
    fov, L = math.radians(3.0), 64
    K0 = wterm.wkernel_full(0.0, L, fov, fov)
    d = np.zeros((L, L))
    d[L // 2, L // 2] = 1.0
    assert np.max(np.abs(K0 - d)) < 1e-15
    Kp = wterm.wkernel_full(300.0, L, fov, fov)
    Km = wterm.wkernel_full(-300.0, L, fov, fov)
    # C(.; -w) = conj C(.; w) (Eq. 2) => K_{-w}(t) = conj K_w(-t)
    flip = np.roll(Kp[::-1, ::-1], 1, axis=(0, 1))
    assert np.max(np.abs(Km - np.conj(flip))) < 1e-14


def test_wkernel_reconstructs_chirp_at_samples():
    fov, L = math.radians(3.0), 32
    w = 150.0
    K = wterm.wkernel_full(w, L, fov, fov)
    lam, mu = wterm.kernel_grid(L, fov, fov)
    t = np.arange(-L // 2, L // 2)
    E = np.exp(-2j * math.pi * np.outer(lam, t) / (2 * fov))
    rec = E @ K @ E.T
    assert np.max(np.abs(rec - wterm.tapered_chirp(w, L, fov, fov)[0])) < 1e-13


def test_support_table_monotone_and_eta_one_is_max():
    fov, L = math.radians(3.0), 64
    tab = wterm.support_table(800.0, L, fov, fov, 0.9999, 9)
    assert np.all(np.diff(tab) >= 0) and np.all(tab % 2 == 1) and tab.max() <= 9
    assert np.all(wterm.support_table(800.0, L, fov, fov, 1.0, 9) == 9)


def test_splitmix64_published_sequence():
    g = golden_data.load("splitmix64_seed1234567.txt")
    expect = [int(v) for v in g["outputs"].split()]
    k = np.arange(1, len(expect) + 1, dtype=np.uint64)
    out = pl.splitmix64(np.uint64(int(g["state"])) + k * np.uint64(pl.GOLDEN))
    assert list(map(int, out)) == expect


def test_kmeans_recovers_separated_clusters():
    rng = np.random.default_rng(3)
    centres = np.array([-5000.0, -100.0, 2000.0, 9000.0])
    w = np.concatenate([c + rng.uniform(-50, 50, 500) for c in centres])
    rng.shuffle(w)
    c = pl.kmeans1d(w, 4)
    lab = pl.nearest(w, c)
    for p in range(4):
        assert abs(c[p] - w[lab == p].mean()) < 1e-9
        assert abs(c[p] - centres[p]) < 10.0


def test_wsclean_bound_closed_form():
    w = np.array([-1000.0, 3000.0])
    fov = math.radians(2.0)
    l = fov / 2
    ref = 2 * math.pi * 4000.0 * (1 - math.sqrt(1 - 2 * l * l))
    assert abs(pl.wsclean_bound(w, fov, fov) - ref) < 1e-9 * ref


def test_decision_tree_regimes():
    # Fig. 2: unlimited budget -> stored G at the cost minimiser; tiny budget -> not G
    uvw = synth.make_uvw(20000, 60, 1.28e9, 21)
    base = dict(nx=256, ny=256, fov_x=math.radians(1.0), fov_y=math.radians(1.0))
    big = pl.choose(uvw, pl.PlanParams(**base))
    assert big["mode"] == pl.MODE_STORED_G and big["P"] == big["p_star"]
    # the cost minimiser over the bin counts whose kernels fit the support cap
    ok = [d for d in big["models"] if not d["truncated"]] or [max(big["models"], key=lambda d: d["P"])]
    costs = {d["P"]: d["cost"] for d in ok}
    assert costs[big["P"]] == min(costs.values())
    mG = {d["P"]: d["m_G"] for d in big["models"]}
    mid_budget = int(0.5 * (mG[big["P"]] + min(mG.values())))
    mid = pl.choose(uvw, pl.PlanParams(**base, mem_budget_bytes=mid_budget))
    if mG[big["P"]] > mid_budget:
        if any(m <= mid_budget for m in mG.values()):
            assert mid["mode"] == pl.MODE_STORED_G and mG[mid["P"]] <= mid_budget
        else:
            assert mid["mode"] == pl.MODE_HOLOGRAPHIC
    tiny = pl.choose(uvw, pl.PlanParams(**base, mem_budget_bytes=1000))
    assert tiny["mode"] == pl.MODE_HOLOGRAPHIC and tiny.get("check_h")


def test_rectangular_image_and_field_against_direct_equation():
    # n_x != n_y and FoV_x != FoV_y: catches any swap of the u and v axes
    nx, ny = 32, 16
    fx, fy = math.radians(4.0), math.radians(2.5)
    uvw = synth.make_uvw(300, 60, 1.28e9, 31) * np.array([0.1, 0.12, 0.01])
    rng = np.random.default_rng(4)
    x = rng.standard_normal((ny, nx)) + 0j
    pp = pl.PlanParams(nx=nx, ny=ny, fov_x=fx, fov_y=fy, n_wbins=2, max_wsupport=31,
                       w_norm_frac=1.0, wkernel_L=64)
    O = operator.Operator(uvw, pl.make_plan(uvw, pp))
    yd = direct.direct_phi(x, uvw, fx, fy)
    assert rel(O.phi(x), yd) < 3e-4
    yr = rng.standard_normal(300) + 1j * rng.standard_normal(300)
    xa = direct.direct_phi_adj(yr, uvw, nx, ny, fx, fy)
    assert rel(O.phi_adj(yr), xa) < 3e-4


# ---------------------------------------------------------------- surrogate MLP oracle
def test_mlp_gradients_match_central_differences():
    from oracle import mlp
    p = mlp.init_params(3)
    rng = np.random.default_rng(9)
    x = rng.uniform(-1, 1, (7, 3))
    t = rng.standard_normal((7, mlp.D_OUT)) * 0.1
    _, g = mlp.loss_and_grads(p, x, t)
    h = 1e-6
    for name, picks in (("W1", [(0, 0), (5, 2), (127, 1)]), ("b1", [(3,), (100,)]),
                        ("W2", [(0, 0), (64, 17), (127, 127)]), ("b2", [(9,)]),
                        ("W3", [(0, 0), (200, 64), (449, 127)]), ("b3", [(0,), (449,)])):
        for ij in picks:
            q = {k: v.copy() for k, v in p.items()}
            q[name][ij] += h
            lp, _ = mlp.loss_and_grads(q, x, t)
            q[name][ij] -= 2 * h
            lm, _ = mlp.loss_and_grads(q, x, t)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name][ij]) <= 1e-6 * max(1e-3, abs(fd)), (name, ij, fd, g[name][ij])


def test_bf16_rounding_is_round_to_nearest_even():
    from oracle import mlp
    # 1 + 2^-8 is halfway between bf16 neighbours 1 and 1 + 2^-7: ties go to the even 1
    assert mlp.bf16(np.float32(1.0 + 2.0 ** -8)) == 1.0
    assert mlp.bf16(np.float32(1.0 + 3 * 2.0 ** -8)) == 1.0 + 2.0 ** -6
    assert mlp.bf16(np.float32(-2.5)) == -2.5
    x = np.random.default_rng(1).standard_normal(1000).astype(np.float32)
    y = mlp.bf16(x)
    assert np.max(np.abs(y - x) / np.abs(x)) <= 2.0 ** -8 + 1e-12  # unit roundoff of 8 significant bits


def test_gelu_gradient_matches_difference_quotient():
    from oracle import mlp
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_grad(z))) < 1e-8


@pytest.mark.parametrize("fov_deg", [1.0, 2.5])
def test_truncation_follows_chirp_bandwidth(fov_deg):
    # The residual chirp e^{-2 pi i w_r (n - 1)} has local frequency -w_r l / n over the
    # field, a spread of about w_r FoV cycles per unit l, i.e. 2 w_r FoV^2 grid cells
    # (cell = 1 / (2 FoV)).  Far below one cell the 9-tap cap keeps the 0.9999 norm
    # fraction; far above nine cells it cannot.
    fov = math.radians(fov_deg)
    L = wterm.wkernel_L(9)
    for cells in (0.05, 0.25, 0.5):
        assert not wterm.truncated_at(cells / (2 * fov * fov), L, fov, fov, 0.9999, 9)
    for cells in (12.0, 40.0):
        assert wterm.truncated_at(cells / (2 * fov * fov), L, fov, fov, 0.9999, 9)
    assert not wterm.truncated_at(0.0, L, fov, fov, 0.9999, 9)


def test_automatic_bins_avoid_truncated_kernels():
    # auto P: the chosen bin count keeps every kernel within the cap whenever some
    # candidate does, and any cheaper candidate is one whose kernels the cap truncates
    uvw = synth.make_uvw(20000, 600, 1.28e9, 23)
    pp = pl.PlanParams(nx=256, ny=256, fov_x=math.radians(2.5), fov_y=math.radians(2.5))
    ch = pl.choose(uvw, pp)
    by_p = {d["P"]: d for d in ch["models"]}
    if any(not d["truncated"] for d in ch["models"]):
        assert not by_p[ch["P"]]["truncated"]
        for d in ch["models"]:
            if d["cost"] < by_p[ch["P"]]["cost"]:
                assert d["truncated"]
    else:
        assert ch["P"] == max(by_p)


def test_rational_erf_meets_its_published_bound():
    # the network's GELU on the device uses Abramowitz & Stegun eq. 7.1.26 for erf; its
    # error bound (1.5e-7) checked against SciPy's erf in FP64 and with FP32 arithmetic
    x = np.linspace(-6.0, 6.0, 200001)

    def erf_as(x, dt):
        x = x.astype(dt)
        ax = np.abs(x)
        t = dt(1.0) / (dt(0.3275911) * ax + dt(1.0))
        poly = t * (dt(0.254829592) + t * (dt(-0.284496736) + t * (dt(1.421413741) + t * (dt(-1.453152027)
                                                                                          + t * dt(1.061405429)))))
        return np.copysign(dt(1.0) - poly * np.exp(-ax * ax), x)

    assert np.max(np.abs(erf_as(x, np.float64) - ss.erf(x))) < 1.5e-7
    # FP32 rounding of 1 - poly e near 1 adds a few units of 6e-8
    assert np.max(np.abs(erf_as(x, np.float32).astype(np.float64) - ss.erf(x))) < 1e-6


def test_cubic_interpolation_of_wkernels_in_w():
    # The library's optional kernel table rests on K(t; w_r) being smooth in w_r: the cubic
    # Lagrange interpolant through equispaced samples (8192 intervals over [-w_max, w_max],
    # as the 4096^2 / 3 deg workload uses) reproduces the oracle's kernels between the samples
    fov = math.radians(3.0)
    L, half, w_max, n = 64, 4, 5662.0, 8192
    dw = 2 * w_max / n
    rng = np.random.default_rng(12)
    w = rng.uniform(-w_max, w_max, 40)
    x = (w + w_max) / dw + 1.0                     # sample j at -w_max + (j - 1) dw
    j = np.minimum(np.floor(x).astype(int), n)
    f = x - j
    nodes = np.stack([-w_max + (j - 2 + i) * dw for i in range(4)], axis=1)     # j - 1 .. j + 2
    K = wterm.wkernel(nodes.ravel(), L, half, fov, fov).reshape(40, 4, 2 * half + 1, 2 * half + 1)
    lag = np.stack([-f * (f - 1) * (f - 2) / 6, (f + 1) * (f - 1) * (f - 2) / 2,
                    -(f + 1) * f * (f - 2) / 2, (f + 1) * f * (f - 1) / 6], axis=1)
    Ki = np.einsum("qi,qist->qst", lag, K)
    Ke = wterm.wkernel(w, L, half, fov, fov)
    err = np.linalg.norm(Ki - Ke, axis=(1, 2)) / np.linalg.norm(Ke, axis=(1, 2))
    assert err.max() < 1e-7, err.max()
