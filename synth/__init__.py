"""Seeded synthetic radio-interferometric observations (inputs only).

This module makes the inputs that both the FP64 oracle and the CUDA library
consume: MeerKAT-like uvw coverages and sky images.  It holds none of the
measurement operator's arithmetic (no kernels, no FFTs, no w-terms); it only
simulates an array and a sky, so that both sides of every comparison read the
very same numbers.

Array model (stands in for the MeerKAT layout and SKA SDC1 sky of the paper's
Section 5.1, which are not available here): 64 antennas drawn uniformly in a
disc of 8 km diameter at latitude -30.7 deg, a source at declination -30 deg,
hour angle swept uniformly over 8 h, uvw expressed in wavelengths.  Every
antenna pair at every time step is a candidate row; M rows are drawn without
replacement.  The sky is 2n point sources (log-uniform flux in [1e-3, 1]) at
uniform pixel positions in the inner 90 % of the image plus 5 Gaussian blobs
(sigma uniform in [2, n/32] pixels, peak log-uniform in [1e-3, 1e-1]).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C_LIGHT = 299_792_458.0
N_ANT = 64
ARRAY_DIAMETER_M = 8000.0
LATITUDE_DEG = -30.7
DEC_DEG = -30.0
SYNTH_HOURS = 8.0
ANTENNA_SEED = 7


def antenna_enu(n_ant: int = N_ANT, diameter_m: float = ARRAY_DIAMETER_M,
                seed: int = ANTENNA_SEED) -> np.ndarray:
    """East/north/up positions (m) uniform in a disc; returns (n_ant, 3)."""
    rng = np.random.default_rng(seed)
    r = 0.5 * diameter_m * np.sqrt(rng.random(n_ant))
    th = 2.0 * np.pi * rng.random(n_ant)
    enu = np.zeros((n_ant, 3))
    enu[:, 0] = r * np.cos(th)
    enu[:, 1] = r * np.sin(th)
    return enu


def baselines_xyz(enu: np.ndarray, lat_deg: float = LATITUDE_DEG) -> np.ndarray:
    """All antenna-pair baselines (i<j) rotated from ENU to equatorial XYZ (m)."""
    lat = math.radians(lat_deg)
    i, j = np.triu_indices(enu.shape[0], k=1)
    b = enu[j] - enu[i]
    e, n, u = b[:, 0], b[:, 1], b[:, 2]
    x = -math.sin(lat) * n + math.cos(lat) * u
    y = e
    z = math.cos(lat) * n + math.sin(lat) * u
    return np.stack([x, y, z], axis=1)


def hour_angles(n_steps: int, hours: float = SYNTH_HOURS) -> np.ndarray:
    """Hour angles (rad) at the centres of n_steps equal intervals over [-h/2, h/2]."""
    t = (np.arange(n_steps) + 0.5) / n_steps
    return np.radians((t - 0.5) * hours * 15.0)


def uvw_rows(xyz: np.ndarray, ha: np.ndarray, rows: np.ndarray, freq_hz: float,
             dec_deg: float = DEC_DEG) -> np.ndarray:
    """uvw (wavelengths) of selected rows; row r = time step r // nb, baseline r % nb."""
    nb = xyz.shape[0]
    b = rows % nb
    t = rows // nb
    h = ha[t]
    d = math.radians(dec_deg)
    x, y, z = xyz[b, 0], xyz[b, 1], xyz[b, 2]
    sh, ch = np.sin(h), np.cos(h)
    u = sh * x + ch * y
    v = -math.sin(d) * ch * x + math.sin(d) * sh * y + math.cos(d) * z
    w = math.cos(d) * ch * x - math.cos(d) * sh * y + math.sin(d) * z
    lam = C_LIGHT / freq_hz
    return np.ascontiguousarray(np.stack([u, v, w], axis=1) / lam)


def make_uvw(n_vis: int, n_steps: int, freq_hz: float, seed: int) -> np.ndarray:
    """Draw n_vis of the (n_steps x 2016) candidate rows without replacement."""
    xyz = baselines_xyz(antenna_enu())
    ha = hour_angles(n_steps)
    total = n_steps * xyz.shape[0]
    if n_vis > total:
        raise ValueError(f"n_vis={n_vis} exceeds the {total} available rows")
    rng = np.random.default_rng(seed)
    if n_vis == total:
        rows = np.arange(total)
    else:
        rows = np.sort(rng.choice(total, size=n_vis, replace=False))
    return uvw_rows(xyz, ha, rows, freq_hz)


def make_sky(n: int, seed: int, n_points: int | None = None, n_blobs: int = 5) -> np.ndarray:
    """Point sources + Gaussian blobs on an n x n grid, returned as complex64."""
    rng = np.random.default_rng(seed)
    img = np.zeros((n, n))
    npts = 2 * n if n_points is None else n_points
    lo, hi = int(0.05 * n), int(math.ceil(0.95 * n))
    ii = rng.integers(lo, hi, size=npts)
    jj = rng.integers(lo, hi, size=npts)
    flux = 10.0 ** rng.uniform(-3.0, 0.0, size=npts)
    np.add.at(img, (ii, jj), flux)
    yy, xx = np.mgrid[0:n, 0:n]
    for _ in range(n_blobs):
        ci, cj = rng.uniform(lo, hi, size=2)
        sig = rng.uniform(2.0, max(2.0, n / 32.0))
        peak = 10.0 ** rng.uniform(-3.0, -1.0)
        img += peak * np.exp(-((yy - ci) ** 2 + (xx - cj) ** 2) / (2.0 * sig * sig))
    return img.astype(np.complex64)


@dataclass
class Workload:
    """One synthetic observation plus the plan parameters it is imaged with."""
    name: str
    n: int
    fov_deg: float
    uvw: np.ndarray               # (M, 3) float64, wavelengths
    sky: np.ndarray               # (n, n) complex64
    n_wbins: int = 0              # 0 = automatic
    max_wsupport: int = 9
    kb_support: int = 7
    mem_budget_bytes: int = 0
    n_blocks: int = 0
    freq_hz: float = 1.28e9
    extra: dict = field(default_factory=dict)

    @property
    def fov_rad(self) -> float:
        return math.radians(self.fov_deg)


# The five workloads: (name, n, FoV deg, M, time steps, w-bins, budget, blocks)
CONFIGS = {
    1: dict(name="mono-256", n=256, fov=1.0, m=20_000, steps=60, bins=4, budget=0, blocks=0),
    2: dict(name="plain-1024", n=1024, fov=2.5, m=2_000_000, steps=28_800, bins=0,
            budget=40 * 2**30, blocks=16),
    3: dict(name="holo-2048", n=2048, fov=2.5, m=20_000_000, steps=28_800, bins=16,
            budget=0, blocks=0),
    4: dict(name="wideband-32x1024", n=1024, fov=2.5, m=0, steps=28_800, bins=0,
            budget=0, blocks=0),
    5: dict(name="surrogate-4096", n=4096, fov=3.0, m=50_000_000, steps=28_800, bins=32,
            budget=0, blocks=0),
}


def make_config(i: int, m_override: int | None = None) -> Workload:
    """Workload i (1..3, 5) with its seeded uvw and sky; m_override shrinks M."""
    c = CONFIGS[i]
    m = c["m"] if m_override is None else m_override
    uvw = make_uvw(m, c["steps"], 1.28e9, seed=1000 + i)
    sky = make_sky(c["n"], seed=2000 + i)
    return Workload(name=c["name"], n=c["n"], fov_deg=c["fov"], uvw=uvw, sky=sky,
                    n_wbins=c["bins"], mem_budget_bytes=c["budget"], n_blocks=c["blocks"])


def wideband_channels(n_chan: int = 32, f_lo: float = 0.9e9, f_hi: float = 1.7e9,
                      m_lo: int = 500_000, m_hi: int = 4_000_000, seed: int = 1004,
                      scale: float = 1.0) -> list[tuple[float, np.ndarray]]:
    """Per-channel (frequency, uvw) for the batched wideband workload.

    Each channel draws its own row count uniformly in [m_lo, m_hi] (times
    `scale`, for reduced test sizes) and its own rows, then scales the shared
    baselines by its frequency.
    """
    rng = np.random.default_rng(seed)
    counts = rng.integers(m_lo, m_hi + 1, size=n_chan)
    freqs = np.linspace(f_lo, f_hi, n_chan)
    out = []
    for c in range(n_chan):
        m = max(1, int(counts[c] * scale))
        out.append((float(freqs[c]), make_uvw(m, 28_800, float(freqs[c]), seed=seed * 100 + c)))
    return out
