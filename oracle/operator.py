"""Phi, Phi^dagger, Phi^dagger Phi, PSF and holographic H in FP64 (oracle).

Eq. 6: Phi = [Phi_1 ... Phi_P]^T with Phi_p = G_p F Z_p.
  Z_p  - diagonal: grid correction 1/KB_hat times the w-layer C(.; w_stack[p]).
  F    - oversampled (x2 per axis) 2-D DFT, unnormalised, forward sign -,
         X[g_u, g_v] = sum_{i,j} z[i, j] exp(-2 pi i (g_u j_c / 2n_x + g_v i_c / 2n_y)),
         with j_c = j - n_x/2, i_c = i - n_y/2 (centred pixels).
  G_p  - sparse rows: visibility k reads the S x S cells starting at (g0, h0)
         (indices modulo the grid) with weights T_k = w-kernel (*) KB taps.
Eq. 7 and Eq. 8: Phi^dagger Phi = sum_p Z_p^dagger F^dagger G_p^dagger G_p F Z_p.
Section 3.3: H_p = G_p^dagger G_p (Hermitian).
Section 2 (Eq. 3): a data weighting (e.g. Briggs) is applied to the data and injected
into the model: with weights w the operator is W Phi, W = diag(w), so that Phi^dagger Phi
becomes Phi^dagger W^2 Phi and H_p becomes G_p^dagger W_p^2 G_p.

This is test infrastructure: only the tests, the smoke check and the
benchmark's CPU-baseline leg use it.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft as sfft
import scipy.sparse as sp

from . import kb as kbm
from . import wterm
from .plan import Plan

CHUNK = 256  # visibilities per vectorised step (small arrays stay in cache)


def _workers() -> int:
    import os
    return os.cpu_count() or 1


class Geometry:
    """Per-visibility grid placement: u~ = u * o * FoV_x (one FP64 multiply)."""

    def __init__(self, uvw: np.ndarray, plan: Plan):
        pp = plan.params
        o = pp.oversampling
        self.gx, self.gy = o * pp.nx, o * pp.ny
        J = pp.kb_support
        ut = uvw[:, 0] * (o * pp.fov_x)
        vt = uvw[:, 1] * (o * pp.fov_y)
        tu = ut - J / 2.0
        tv = vt - J / 2.0
        fu = np.floor(tu)
        fv = np.floor(tv)
        self.phi_u = tu - fu
        self.phi_v = tv - fv
        h = (plan.s_w - 1) // 2
        self.g0 = fu.astype(np.int64) + 1 - h
        self.h0 = fv.astype(np.int64) + 1 - h
        self.S = plan.s_w + J - 1


_POOL_OP = None


def _pool_init(op) -> None:
    global _POOL_OP
    _POOL_OP = op


def _pool_tiles(idx: np.ndarray) -> list[np.ndarray]:
    return _POOL_OP.tiles(idx)


class Operator:
    """The discrete hybrid w-stacking / w-projection operator of one plan."""

    def __init__(self, uvw: np.ndarray, plan: Plan, build_g: bool = True, weights=None,
                 workers: int = 1):
        self.uvw = np.asarray(uvw, dtype=np.float64)
        # diagonal data weighting W (None: W = I)
        self.w = None if weights is None else np.asarray(weights, dtype=np.float64)
        self.plan = plan
        pp = plan.params
        self.pp = pp
        self.J = pp.kb_support
        self.beta = pp.beta
        self.geo = Geometry(self.uvw, plan)
        self.gx, self.gy = self.geo.gx, self.geo.gy
        gcx = kbm.grid_correction_1d(pp.nx, self.J, self.beta)
        gcy = kbm.grid_correction_1d(pp.ny, self.J, self.beta)
        self.gc = gcy[:, None] * gcx[None, :]
        self.M = self.uvw.shape[0]
        self.G = None
        if build_g:
            # tiles of every visibility (in caller order), then one sparse G_p per bin
            allt = self.tiles_parallel(np.arange(self.M), workers)
            self.G = [self._build_g(p, allt) for p in range(plan.P)]

    # ---- Z_p ------------------------------------------------------------
    def z_layer(self, p: int) -> np.ndarray:
        pp = self.pp
        return self.gc * wterm.w_layer(self.plan.w_stack[p], pp.nx, pp.ny, pp.fov_x,
                                       pp.fov_y, pp.div_n)

    # ---- tiles ----------------------------------------------------------
    def tiles(self, idx: np.ndarray) -> list[np.ndarray]:
        """T_k[a, b] (a along u, b along v) for visibilities idx, FP64."""
        idx = np.asarray(idx, dtype=np.int64)
        pp = self.pp
        out: list[np.ndarray | None] = [None] * idx.size
        sw = self.plan.s_w[idx]
        for s in np.unique(sw):
            sel = np.nonzero(sw == s)[0]
            h = int(s) // 2
            S = int(s) + self.J - 1
            for c0 in range(0, sel.size, CHUNK):
                part = sel[c0:c0 + CHUNK]
                k = idx[part]
                Kw = wterm.wkernel(self.plan.w_r[k], pp.L, h, pp.fov_x, pp.fov_y,
                                   pp.taper_literal)
                wu = kbm.kb_taps(self.geo.phi_u[k], self.J, self.beta)
                wv = kbm.kb_taps(self.geo.phi_v[k], self.J, self.beta)
                Wu = np.zeros((k.size, S, int(s)))
                Wv = np.zeros((k.size, S, int(s)))
                for su in range(int(s)):
                    Wu[:, su:su + self.J, su] = wu
                    Wv[:, su:su + self.J, su] = wv
                T = np.einsum("kas,kst,kbt->kab", Wu, Kw, Wv, optimize=True)
                for q, j in enumerate(part):
                    out[j] = T[q]
        return out  # type: ignore[return-value]

    def tiles_parallel(self, idx: np.ndarray, workers: int = 1) -> list[np.ndarray]:
        """tiles(idx) computed by `workers` processes over contiguous slices of idx (the
        same arithmetic per visibility; a spawned pool, safe after CUDA was initialised)."""
        idx = np.asarray(idx, dtype=np.int64)
        if workers <= 1 or idx.size < 8 * CHUNK:
            return self.tiles(idx)
        import multiprocessing as mp
        light = object.__new__(Operator)
        light.__dict__.update({k: v for k, v in self.__dict__.items() if k not in ("G", "gc")})
        parts = np.array_split(idx, 4 * workers)
        with mp.get_context("spawn").Pool(workers, initializer=_pool_init, initargs=(light,)) as pool:
            res = pool.map(_pool_tiles, parts)
        return [t for r in res for t in r]

    def tile_cells(self, k: int):
        """Grid cells (g_u, g_v) touched by visibility k, each (S,) modulo the grid."""
        S = int(self.geo.S[k])
        a = np.arange(S)
        return (self.geo.g0[k] + a) % self.gx, (self.geo.h0[k] + a) % self.gy

    def _build_g(self, p: int, all_tiles=None) -> sp.csr_matrix:
        rows_k = np.nonzero(self.plan.bins == p)[0]
        Ts = self.tiles(rows_k) if all_tiles is None else [all_tiles[k] for k in rows_k]
        r, c, v = [], [], []
        for q, k in enumerate(rows_k):
            cu, cv = self.tile_cells(int(k))
            S = cu.size
            r.append(np.full(S * S, q))
            c.append((cu[:, None] * self.gy + cv[None, :]).ravel())
            v.append(Ts[q].ravel())
        if rows_k.size == 0:
            return sp.csr_matrix((0, self.gx * self.gy), dtype=np.complex128)
        G = sp.coo_matrix((np.concatenate(v), (np.concatenate(r), np.concatenate(c))),
                          shape=(rows_k.size, self.gx * self.gy)).tocsr()
        G.sum_duplicates()
        return G

    # ---- F and F^dagger ---------------------------------------------------
    def fwd_grid(self, z: np.ndarray) -> np.ndarray:
        """X[g_u, g_v] of the centred image z[i, j] (oversampled DFT)."""
        ny, nx = z.shape
        P = np.zeros((self.gy, self.gx), dtype=np.complex128)
        ii = (np.arange(ny) - ny // 2) % self.gy
        jj = (np.arange(nx) - nx // 2) % self.gx
        P[np.ix_(ii, jj)] = z
        return sfft.fft2(P, workers=_workers()).T

    def adj_grid(self, Xh: np.ndarray) -> np.ndarray:
        """z[i, j] = sum_g Xh[g_u, g_v] exp(+2 pi i (...)), cropped to the image."""
        pp = self.pp
        R = sfft.ifft2(Xh.T, workers=_workers()) * (self.gx * self.gy)
        ii = (np.arange(pp.ny) - pp.ny // 2) % self.gy
        jj = (np.arange(pp.nx) - pp.nx // 2) % self.gx
        return R[np.ix_(ii, jj)]

    # ---- operators ------------------------------------------------------
    def phi(self, x: np.ndarray) -> np.ndarray:
        x = np.asarray(x, dtype=np.complex128)
        y = np.zeros(self.M, dtype=np.complex128)
        for p in range(self.plan.P):
            rows = np.nonzero(self.plan.bins == p)[0]
            if rows.size == 0:
                continue
            X = self.fwd_grid(self.z_layer(p) * x)
            y[rows] = self.G[p] @ X.ravel()
        return y if self.w is None else self.w * y

    def phi_adj(self, y: np.ndarray) -> np.ndarray:
        y = np.asarray(y, dtype=np.complex128)
        if self.w is not None:
            y = self.w * y
        pp = self.pp
        out = np.zeros((pp.ny, pp.nx), dtype=np.complex128)
        for p in range(self.plan.P):
            rows = np.nonzero(self.plan.bins == p)[0]
            if rows.size == 0:
                continue
            Xh = (self.G[p].conj().T @ y[rows]).reshape(self.gx, self.gy)
            out += np.conj(self.z_layer(p)) * self.adj_grid(Xh)
        return out

    def phi_adj_phi(self, x: np.ndarray, real_part_only: bool = False, bins=None, vis=None) -> np.ndarray:
        """sum_p Phi_p^dagger Phi_p x (Eq. 7), over all w-bins or the listed ones; with `vis`
        (boolean, one entry per visibility) only the selected visibilities' rows of each G_p
        (G_p^dagger G_p of Eq. 8 is a sum over the bin's visibilities)."""
        pp = self.pp
        x = np.asarray(x, dtype=np.complex128)
        out = np.zeros((pp.ny, pp.nx), dtype=np.complex128)
        for p in (range(self.plan.P) if bins is None else bins):
            G = self.G[p]
            if vis is not None:
                G = G[np.flatnonzero(np.asarray(vis, dtype=bool)[self.plan.bins == p])]
            if G.shape[0] == 0:
                continue
            Zp = self.z_layer(p)
            X = self.fwd_grid(Zp * x).ravel()
            yp = G @ X
            if self.w is not None:
                wp = self.w[self.plan.bins == p]
                if vis is not None:
                    wp = wp[np.asarray(vis, dtype=bool)[self.plan.bins == p]]
                yp = wp ** 2 * yp
            Xh = (G.conj().T @ yp).reshape(self.gx, self.gy)
            out += np.conj(Zp) * self.adj_grid(Xh)
        return out.real.astype(np.complex128) if real_part_only else out

    def psf(self) -> np.ndarray:
        pp = self.pp
        d = np.zeros((pp.ny, pp.nx), dtype=np.complex128)
        d[pp.ny // 2, pp.nx // 2] = 1.0
        return self.phi_adj_phi(d)

    def holographic(self, p: int) -> sp.csr_matrix:
        """H_p = G_p^dagger G_p as an N' x N' sparse matrix (Section 3.3)."""
        G = self.G[p]
        if self.w is not None:
            G = sp.diags(self.w[self.plan.bins == p]) @ G
        return (G.conj().T @ G).tocsr()

    # ---- full-size sampled evaluation --------------------------------------
    def phi_sampled(self, x: np.ndarray, ks: np.ndarray) -> np.ndarray:
        """y_k for selected visibilities without forming G or full grids.

        X_p is evaluated only on the S x S cells of each sampled visibility by the
        separable DFT sum X[g_u, g_v] = sum_i e_v(g_v, i) sum_j z[i, j] e_u(g_u, j).
        """
        pp = self.pp
        ks = np.asarray(ks, dtype=np.int64)
        x = np.asarray(x, dtype=np.complex128)
        jc = np.arange(pp.nx) - pp.nx // 2
        ic = np.arange(pp.ny) - pp.ny // 2
        Ts = self.tiles(ks)
        y = np.zeros(ks.size, dtype=np.complex128)
        zc: dict[int, np.ndarray] = {}
        for q, k in enumerate(ks):
            p = int(self.plan.bins[k])
            if p not in zc:
                zc.clear()
                zc[p] = self.z_layer(p) * x
            cu, cv = self.tile_cells(int(k))
            Eu = np.exp(-2j * math.pi * np.outer(jc, cu) / self.gx)   # (nx, S)
            Ev = np.exp(-2j * math.pi * np.outer(cv, ic) / self.gy)   # (S, ny)
            Xs = (Ev @ (zc[p] @ Eu)).T                                 # (S_u, S_v)
            y[q] = np.sum(Ts[q] * Xs)
        return y if self.w is None else self.w[ks] * y
