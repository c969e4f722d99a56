"""w-term chirp, w-layers and residual w-kernels, FP64 (oracle).

Section 2, Eq. 2 defines the chirp C(l, m; w) = exp(-2 pi i w (sqrt(1 - l^2 - m^2) - 1))
(optionally divided by sqrt(1 - l^2 - m^2)).  Section 3.1 splits w = w_stack + w_proj:
the w-layer C(.; w_stack) multiplies the image; the residual C(.; w_proj) becomes a
small Fourier-domain kernel (Fig. 1): it is sampled over twice the field of view,
tapered by a Hamming roll-off outside the field of view, transformed by a small
DFT whose frequency spacing equals the NUFFT grid spacing, and truncated to the
smallest centred square that keeps a user fraction of its l2 norm.

Readings where the paper is silent or garbled (listed in the design notes):
* the taper is applied to the chirp's deviation from 1, c = 1 + tau (C - 1), so a
  zero offset gives a delta kernel; the literal product tau * C is option ``literal``;
* the sampling resolution is one L x L grid per plan (the adaptive bandwidth
  formula of Section 3.1 is garbled), L = max(32, next power of two >= 4 S_w,max);
* the support of a kernel is read from a table over 64 uniform bins of |w_proj|,
  evaluated at each bin's upper edge (the "logical kernels" of the Section 3.2
  footnote), made non-decreasing in |w_proj|.
"""
from __future__ import annotations

import math

import numpy as np

HAMMING_A0 = 0.54
HAMMING_A1 = 0.46
N_SUPPORT_BINS = 64


def dn(l, m):
    """sqrt(1 - l^2 - m^2) - 1, written as -s / (1 + sqrt(1 - s)) with s = l^2 + m^2."""
    s = np.asarray(l, dtype=np.float64) ** 2 + np.asarray(m, dtype=np.float64) ** 2
    return -s / (1.0 + np.sqrt(1.0 - s))


def pixel_lm(n: int, fov: float) -> np.ndarray:
    """Direction cosine of pixel j in [0, n): (j - n/2) * fov / n."""
    return (np.arange(n) - n // 2) * (fov / n)


def w_layer(w_stack: float, nx: int, ny: int, fov_x: float, fov_y: float,
            div_n: bool = False) -> np.ndarray:
    """C(l, m; w_stack) on the image pixels, shape (ny, nx) (Eq. 2 at w = w_stack)."""
    l = pixel_lm(nx, fov_x)[None, :]
    m = pixel_lm(ny, fov_y)[:, None]
    d = dn(l, m)
    c = np.exp(-2j * math.pi * w_stack * d)
    if div_n:
        c = c / (1.0 + d)
    return c


def wkernel_L(max_wsupport: int) -> int:
    return max(32, 1 << int(math.ceil(math.log2(4 * max_wsupport))))


def taper(lam, fov: float):
    """1 inside |lam| <= fov/2; Hamming roll-off 0.54 + 0.46 cos(...) outside."""
    a = np.abs(np.asarray(lam, dtype=np.float64))
    half = 0.5 * fov
    roll = HAMMING_A0 + HAMMING_A1 * np.cos(math.pi * (a - half) / half)
    return np.where(a <= half, 1.0, roll)


def kernel_grid(L: int, fov_x: float, fov_y: float, oversampling: int = 2):
    """Sample coordinates (lam_a, mu_b) over o x FoV with L points per axis."""
    lam = (np.arange(L) - L // 2) * (oversampling * fov_x / L)
    mu = (np.arange(L) - L // 2) * (oversampling * fov_y / L)
    return lam, mu


def tapered_chirp(w_r, L: int, fov_x: float, fov_y: float, literal: bool = False,
                  oversampling: int = 2) -> np.ndarray:
    """c[k, a, b] for residual offsets w_r[k] on the L x L kernel grid ([a] along l)."""
    w_r = np.atleast_1d(np.asarray(w_r, dtype=np.float64))
    lam, mu = kernel_grid(L, fov_x, fov_y, oversampling)
    d = dn(lam[:, None], mu[None, :])
    tau = taper(lam, fov_x)[:, None] * taper(mu, fov_y)[None, :]
    ch = np.exp(-2j * math.pi * w_r[:, None, None] * d[None])
    if literal:
        return tau[None] * ch
    return 1.0 + tau[None] * (ch - 1.0)


def dft_matrix(L: int, half: int) -> np.ndarray:
    """E[a, s] = exp(+2 pi i t (a - L/2) / L) for t = s - half, s in [0, 2 half + 1)."""
    a = np.arange(L) - L // 2
    t = np.arange(-half, half + 1)
    return np.exp(2j * math.pi * np.outer(a, t) / L)


def wkernel(w_r, L: int, half: int, fov_x: float, fov_y: float, literal: bool = False):
    """Central (2 half + 1)^2 taps K[k, t_x + half, t_y + half] of the residual kernels.

    K(t) = (1/L^2) sum_{a,b} c[a, b] exp(+2 pi i (t_x a_c + t_y b_c) / L): the Fourier
    series of c sampled at the NUFFT grid spacing 1/(o FoV), so that
    c(l, m) = sum_t K(t) exp(-2 pi i (t_x du l + t_y dv m)) and a visibility at u sees
    the w-free spectrum at u + t du.
    """
    c = tapered_chirp(w_r, L, fov_x, fov_y, literal)
    E = dft_matrix(L, half)
    return np.einsum("kab,as,bt->kst", c, E, E, optimize=True) / (L * L)


def wkernel_full(w_r: float, L: int, fov_x: float, fov_y: float, literal: bool = False):
    """All L x L taps of one kernel, t in [-L/2, L/2) along both axes."""
    return wkernel(np.array([w_r]), L, L // 2, fov_x, fov_y, literal)[0][:L, :L]


def support_of(K_full: np.ndarray, eta: float, max_wsupport: int) -> int:
    """Smallest odd s <= max_wsupport whose centred s x s block keeps >= eta of ||K||_2."""
    L = K_full.shape[0]
    c = L // 2
    total = math.sqrt(float(np.sum(np.abs(K_full) ** 2)))
    for s in range(1, max_wsupport + 1, 2):
        h = s // 2
        blk = K_full[c - h:c + h + 1, c - h:c + h + 1]
        if math.sqrt(float(np.sum(np.abs(blk) ** 2))) >= eta * total:
            return s
    return max_wsupport


def truncated_at(w_r: float, L: int, fov_x: float, fov_y: float, eta: float,
                 max_wsupport: int, literal: bool = False) -> bool:
    """Whether the kernel of residual w_r needs more than max_wsupport taps per axis to keep
    eta of its l2 norm (then the capped support truncates it, Section 3.1)."""
    if w_r == 0.0 or eta >= 1.0:
        return False
    K = wkernel_full(w_r, L, fov_x, fov_y, literal)
    c = L // 2
    h = max_wsupport // 2
    total = math.sqrt(float(np.sum(np.abs(K) ** 2)))
    blk = K[c - h:c + h + 1, c - h:c + h + 1]
    return math.sqrt(float(np.sum(np.abs(blk) ** 2))) < eta * total


def support_table(wr_max: float, L: int, fov_x: float, fov_y: float, eta: float,
                  max_wsupport: int, literal: bool = False) -> np.ndarray:
    """Support S_w for each of 64 uniform |w_r| bins over [0, wr_max], non-decreasing."""
    tab = np.ones(N_SUPPORT_BINS, dtype=np.int64)
    if wr_max <= 0.0:
        return tab
    step = wr_max / N_SUPPORT_BINS
    for q in range(N_SUPPORT_BINS):
        K = wkernel_full((q + 1) * step, L, fov_x, fov_y, literal)
        tab[q] = support_of(K, eta, max_wsupport)
    return np.maximum.accumulate(tab)


def support_bin(abs_wr, wr_max: float) -> np.ndarray:
    """Index of the |w_r| bin: min(floor(|w_r| / (wr_max/64)), 63)."""
    abs_wr = np.asarray(abs_wr, dtype=np.float64)
    if wr_max <= 0.0:
        return np.zeros(abs_wr.shape, dtype=np.int64)
    step = wr_max / N_SUPPORT_BINS
    return np.minimum(np.floor(abs_wr / step), N_SUPPORT_BINS - 1).astype(np.int64)
