"""Planning: w-bins by k-means, residual offsets, supports, P and mode choice (oracle).

Follows Section 3.1 (k-means w-stacking on a random subset, WSClean bound Eq. 5),
Section 3.2 (footnote: supports from kernels over uniformly binned w), and
Section 3.4 (memory model Eq. 9, cost model Eq. 10, decision tree of Fig. 2).

Readings (listed in the design notes):
* the "random subset" is drawn with a counter-based SplitMix64 hash of
  (seed, visibility index), kept when its top 53 bits / 2^53 < fraction, where
  fraction = max(plan_fraction, min(1, 4096 / M));
* k-means starts from the subset quantiles (p + 1/2)/P, runs Lloyd iterations
  (ties to the lower bin, empty clusters keep their centroid) until no point moves
  or 100 iterations; centroids are returned ascending;
* every visibility joins its nearest centroid (ties to the lower index);
* the memory model is restated for the device layout: m_G = 8 sum_k pad2(S_k^2)
  + 16 M (complex64 taps, tiles padded to an even count, 16 B of per-visibility
  metadata); the cost model is Eq. 10 as printed;
* the decision tree of Fig. 2: stored G at P* = argmin c if it fits, else the
  feasible P closest to P*; if none fits, P-bar is the smallest P whose m_G is
  within 5 % of min_P m_G, and H is used there if its footprint fits, else
  kernels are generated on the fly.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import wterm

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
CANDIDATE_P = (1, 2, 3, 4, 5, 6, 8, 10, 12, 16, 20, 24, 32, 40, 48, 64, 80, 96, 128, 160, 192, 256)
MODE_AUTO, MODE_STORED_G, MODE_HOLOGRAPHIC, MODE_SURROGATE, MODE_ONTHEFLY = 0, 1, 2, 3, 4
META_BYTES_PER_VIS = 16


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea & Flood 2014) on uint64 states."""
    with np.errstate(over="ignore"):
        z = x.astype(np.uint64)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def subset_mask(M: int, seed: int, fraction: float) -> np.ndarray:
    """Counter-based selection of the planning subset."""
    frac = max(float(fraction), min(1.0, 4096.0 / max(M, 1)))
    if frac >= 1.0:
        return np.ones(M, dtype=bool)
    with np.errstate(over="ignore"):
        k = np.arange(1, M + 1, dtype=np.uint64)
        state = np.uint64(seed & MASK64) + k * np.uint64(GOLDEN)
    r = splitmix64(state)
    u = (r >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return u < frac


def nearest(w: np.ndarray, centroids: np.ndarray) -> np.ndarray:
    """argmin_p |w - c_p|, ties to the lower p."""
    d = np.abs(w[:, None] - centroids[None, :])
    return np.argmin(d, axis=1)


def nearest_chunked(w: np.ndarray, centroids: np.ndarray, chunk: int = 1 << 20) -> np.ndarray:
    out = np.empty(w.shape[0], dtype=np.int64)
    for s in range(0, w.shape[0], chunk):
        out[s:s + chunk] = nearest(w[s:s + chunk], centroids)
    return out


def kmeans1d(w: np.ndarray, P: int, max_iter: int = 100) -> np.ndarray:
    """Lloyd's k-means in one dimension from quantile initialisation (Section 3.1)."""
    ws = np.sort(w)
    n = ws.shape[0]
    c = np.array([ws[min(n - 1, int((p + 0.5) * n / P))] for p in range(P)], dtype=np.float64)
    lab = nearest_chunked(w, c)
    for _ in range(max_iter):
        for p in range(P):
            sel = w[lab == p]
            if sel.size:
                c[p] = sel.mean()
        new = nearest_chunked(w, c)
        if np.array_equal(new, lab):
            break
        lab = new
    return np.sort(c)


def wsclean_bound(w: np.ndarray, fov_x: float, fov_y: float) -> float:
    """Eq. 5: 2 pi (w_max - w_min) max over the field of (1 - sqrt(1 - l^2 - m^2))."""
    l, m = 0.5 * fov_x, 0.5 * fov_y
    return 2.0 * math.pi * (float(w.max()) - float(w.min())) * (-float(wterm.dn(l, m)))


def pad2(x):
    return x + (x & 1)


@dataclass
class PlanParams:
    nx: int
    ny: int
    fov_x: float
    fov_y: float
    oversampling: int = 2
    kb_support: int = 7
    kb_beta: float = 0.0
    max_wsupport: int = 9
    w_norm_frac: float = 0.9999
    mem_budget_bytes: int = 0
    n_wbins: int = 0
    n_blocks: int = 0
    mode: int = MODE_AUTO
    div_n: bool = False
    plan_fraction: float = 0.01
    seed: int = 12345
    taper_literal: bool = False
    wkernel_L: int = 0

    @property
    def beta(self) -> float:
        return self.kb_beta if self.kb_beta > 0 else 2.34 * self.kb_support

    @property
    def L(self) -> int:
        return self.wkernel_L if self.wkernel_L > 0 else wterm.wkernel_L(self.max_wsupport)


@dataclass
class Plan:
    params: PlanParams
    P: int
    mode: int
    w_stack: np.ndarray          # (P,) ascending
    bins: np.ndarray             # (M,) int
    w_r: np.ndarray              # (M,) float64
    wr_max: float
    support_tab: np.ndarray      # (64,)
    s_w: np.ndarray              # (M,) odd supports
    K: int                       # sum of S_k^2 (S = S_w + J - 1)
    est: dict = field(default_factory=dict)


def supports_for(w_r: np.ndarray, pp: PlanParams):
    wr_max = float(np.max(np.abs(w_r))) if w_r.size else 0.0
    tab = wterm.support_table(wr_max, pp.L, pp.fov_x, pp.fov_y, pp.w_norm_frac,
                              pp.max_wsupport, pp.taper_literal)
    s_w = tab[wterm.support_bin(np.abs(w_r), wr_max)]
    return wr_max, tab, s_w


def model_for_P(w_sub: np.ndarray, M: int, P: int, pp: PlanParams) -> dict:
    """K(P), m_G(P), c(P) estimated on the planning subset and scaled to M (Eq. 9, Eq. 10)."""
    c = kmeans1d(w_sub, P)
    lab = nearest_chunked(w_sub, c)
    w_r = w_sub - c[lab]
    _, _, s_w = supports_for(w_r, pp)
    S = s_w + pp.kb_support - 1
    scale = M / w_sub.shape[0]
    K = float(np.sum(S * S)) * scale
    KP = float(np.sum(pad2(S * S))) * scale
    m_G = 8.0 * KP + META_BYTES_PER_VIS * M
    Np = (pp.oversampling ** 2) * pp.nx * pp.ny
    cost = 2.0 * (10.0 * Np * math.log2(math.sqrt(Np)) * P + 6.0 * K)
    wr_max = float(np.max(np.abs(w_r))) if w_r.size else 0.0
    trunc = wterm.truncated_at(wr_max, pp.L, pp.fov_x, pp.fov_y, pp.w_norm_frac, pp.max_wsupport,
                               pp.taper_literal)
    return dict(P=P, K=K, m_G=m_G, cost=cost, truncated=trunc)


def choose(uvw: np.ndarray, pp: PlanParams) -> dict:
    """Stage 1 of Fig. 3: pick P and the strategy (Fig. 2) from the planning subset."""
    w = uvw[:, 2]
    M = w.shape[0]
    mask = subset_mask(M, pp.seed, pp.plan_fraction)
    w_sub = w[mask]
    if pp.n_wbins > 0:
        cands = [pp.n_wbins]
    else:
        pmax = max(1, int(math.ceil(wsclean_bound(w, pp.fov_x, pp.fov_y))))
        cands = [p for p in CANDIDATE_P if p <= max(pmax, 1)]
        cands = [p for p in cands if p <= max(1, w_sub.shape[0])]
    models = [model_for_P(w_sub, M, p, pp) for p in cands]
    # With an automatic P, only bin counts whose residual kernels fit the support cap keep
    # the eta norm fraction of Section 3.1; if none does, the largest candidate truncates
    # least.  (A capped support makes K(P) flat in P, so the cost model alone would pick
    # the fewest bins however much of the kernels the cap cuts off.)
    pool = [d for d in models if not d["truncated"]] if pp.n_wbins == 0 else models
    if not pool:
        pool = [max(models, key=lambda d: d["P"])]
    best = min(pool, key=lambda d: (d["cost"], d["P"]))
    budget = pp.mem_budget_bytes
    out = dict(models=models, p_star=best["P"], subset=int(w_sub.shape[0]))
    if pp.mode != MODE_AUTO:
        out.update(P=best["P"], mode=pp.mode)
        return out
    if budget <= 0 or best["m_G"] <= budget:
        out.update(P=best["P"], mode=MODE_STORED_G)
        return out
    # under the budget: the nearest P to P* that fits, kernels within the cap preferred
    feas = [d for d in pool if d["m_G"] <= budget] or [d for d in models if d["m_G"] <= budget]
    if feas:
        pick = min(feas, key=lambda d: (abs(d["P"] - best["P"]), d["P"]))
        out.update(P=pick["P"], mode=MODE_STORED_G)
        return out
    mmin = min(d["m_G"] for d in models)
    stable = min((d for d in models if d["m_G"] <= 1.05 * mmin), key=lambda d: d["P"])
    out.update(P=stable["P"], mode=MODE_HOLOGRAPHIC, check_h=True)
    return out


def make_plan(uvw: np.ndarray, pp: PlanParams) -> Plan:
    """Full plan on all visibilities: centroids, bins, residual w, supports."""
    ch = choose(uvw, pp)
    P = ch["P"]
    w = uvw[:, 2]
    mask = subset_mask(w.shape[0], pp.seed, pp.plan_fraction)
    w_stack = kmeans1d(w[mask], P)
    bins = nearest_chunked(w, w_stack)
    w_r = w - w_stack[bins]
    wr_max, tab, s_w = supports_for(w_r, pp)
    S = s_w + pp.kb_support - 1
    return Plan(params=pp, P=P, mode=ch["mode"], w_stack=w_stack, bins=bins, w_r=w_r,
                wr_max=wr_max, support_tab=tab, s_w=s_w, K=int(np.sum(S * S)), est=ch)
