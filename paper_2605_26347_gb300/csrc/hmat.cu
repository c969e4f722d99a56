// Holographic matrices H_p = G_p^dagger G_p (Section 3.3): device build and apply.
//
// H_p[c1][c2] = sum_k conj(G_p[k][c1]) G_p[k][c2] couples two grid cells when some
// visibility's S x S footprint covers both, so |c2 - c1| <= D = S_max - 1 per axis.  H_p is
// Hermitian; each unordered pair is stored once, at its owner: the top-left corner of the
// pair's bounding box.  Owner o stores
//   type A: (a, b) in [0, D]^2                 H[o][o + (a, b)]
//   type B: a in [1, D], b in [1, D]           H[o + (0, b)][o + (a, 0)]
// ((D+1)^2 + D^2 entries; pairs with du = 0 > dv are type A of the swapped pair).  Every
// cell an owner's entries touch lies in o + [0, D]^2, so the apply writes the same patch
// geometry as the gridding step ([tile origin, + TS + D) per axis), and the same fold
// sums the patches into the grid.
//
// Only owners that some footprint covers get a row: a coverage pass marks the covered
// cells of each needed tile (bitmap), the host turns the counts into row offsets, and the
// build pass writes the rows.  Where cells see one or a few visibilities most pairs are
// never covered together, so a bin's rows keep only their non-zero entries (value and entry
// number, rows found by offsets) when that is smaller than the dense rows: the build writes
// the bin's rows densely to a temporary, a count pass decides, and a compaction pass keeps
// each row's non-zero values; a bin of dense coverage keeps the dense rows as they are.  Build: one CTA per 4 x 4 block of owners, one warp per
// owner keeping its entries in shared memory (no atomics); the candidate visibilities
// (anchor within D before the block) come from an anchor index sorted by (g0, h0) that the
// host prepares.  Apply: one CTA per needed tile, one warp per owner; the gathered sum
// of the type-A row and the scattered conjugate terms are accumulated in the two-word
// fixed-point patch of the gridding step.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "internal.h"
#include "planner.h"

using namespace rimo;

namespace rimo {

namespace {

constexpr int HB_OWN = 4;                 // owner block edge of the build
constexpr int HB_WARPS = HB_OWN * HB_OWN;  // one warp per owner
constexpr int HB_CHUNK = 16;              // candidate visibilities staged at a time
constexpr int HA_WARPS = 16;              // apply: consumer warps per CTA
constexpr float HX_MAGIC = 12582912.0f;   // 1.5 x 2^23 (rint by the shift)
constexpr int HX_MAGIC_BITS = 0x4B400000;

// entry e of an owner row -> (type, a, b), packed type << 16 | a << 8 | b
std::vector<int32_t> entry_table(int D) {
    std::vector<int32_t> t;
    for (int a = 0; a <= D; ++a)
        for (int b = 0; b <= D; ++b) t.push_back((0 << 16) | (a << 8) | b);
    for (int a = 1; a <= D; ++a)
        for (int b = 1; b <= D; ++b) t.push_back((1 << 16) | (a << 8) | b);
    return t;
}

struct AnchorIndex {
    int32_t* pos = nullptr;      // sorted position of each visibility, ordered by (g0, h0) per bin
    uint16_t* h0 = nullptr;      // its anchor column (grid cells < 65536)
    int64_t* row = nullptr;      // [bin][g0 + 1]: first index of anchor row g0 (bin ranges [vb, ve))
    ~AnchorIndex() {
        cudaFree(pos);
        cudaFree(h0);
        cudaFree(row);
    }
};

__device__ __forceinline__ int wrap(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

// candidate ranges: anchors in rows [r0, r0 + nr) and columns [c0, c0 + nc) (mod grid); a
// column window that wraps splits in two.  Writes up to 2 nr ranges [lo, hi) into rng.
__device__ int candidate_ranges(const int64_t* __restrict__ row, const uint16_t* __restrict__ h0, int gx, int gy,
                                int r0, int nr, int c0, int nc, int64_t* rng_lo, int64_t* rng_hi, int* rng_row,
                                int tid, int nthreads) {
    // windows along v: [c0, c0 + nc) possibly wrapping
    int wlo[2], whi[2], nw = 0;
    const int cs = wrap(c0, gy);
    if (cs + nc <= gy) {
        wlo[0] = cs, whi[0] = cs + nc, nw = 1;
    } else {
        wlo[0] = cs, whi[0] = gy, wlo[1] = 0, whi[1] = cs + nc - gy, nw = 2;
    }
    for (int q = tid; q < nr * nw; q += nthreads) {
        const int r = wrap(r0 + q / nw, gx), w = q % nw;
        int64_t lo = row[r], hi = row[r + 1];
        // first index with h0 >= wlo, first with h0 >= whi (h0 ascending within a row)
        int64_t a = lo, b = hi;
        while (a < b) {
            const int64_t m = (a + b) >> 1;
            if ((int)h0[m] < wlo[w]) a = m + 1;
            else b = m;
        }
        const int64_t first = a;
        b = hi;
        while (a < b) {
            const int64_t m = (a + b) >> 1;
            if ((int)h0[m] < whi[w]) a = m + 1;
            else b = m;
        }
        rng_lo[q] = first;
        rng_hi[q] = a;
        rng_row[q] = r;
    }
    return nr * nw;
}

struct HArgs {
    const VisMeta* meta;
    float2* const* gblk;
    const int32_t* apos;     // anchor index (this bin's slice starts at 0 of row[])
    const uint16_t* ah0;
    const int64_t* arow;     // [gx + 1]
    const int32_t* need;     // needed tiles of the bin
    uint32_t* bits;          // [needed tile][TS*TS/32]
    int64_t* count;          // [needed tile] covered cells (coverage pass)
    const int64_t* hoff;     // [needed tile + 1]
    float2* rows;            // [owner][ne]
    uint32_t* tmax;          // [needed tile] max |h.x| + |h.y| over the tile's rows (float bits)
    const int32_t* ent;      // entry table
    uint32_t* fx;
    int gx, gy, ntv, TS, D, ne;
};

// Coverage pass: one CTA per needed tile marks the cells that some footprint covers.
__global__ void __launch_bounds__(256) hcover_kernel(HArgs A) {
    extern __shared__ __align__(16) unsigned char csm[];
    const int words = A.TS * A.TS / 32;
    const int nrmax = 2 * (A.TS + A.D);
    int64_t* rlo = reinterpret_cast<int64_t*>(csm);
    int64_t* rhi = rlo + nrmax;
    int* rrow = reinterpret_cast<int*>(rhi + nrmax);
    uint32_t* bm = reinterpret_cast<uint32_t*>(rrow + nrmax);
    const int tile = A.need[blockIdx.x];
    const int tu = tile / A.ntv, tv = tile - tu * A.ntv;
    const int u0 = tu * A.TS, v0 = tv * A.TS;
    for (int e = threadIdx.x; e < words; e += blockDim.x) bm[e] = 0u;
    // anchors whose footprint (at most D + 1 cells from the anchor) can reach the tile
    const int nrng = candidate_ranges(A.arow, A.ah0, A.gx, A.gy, u0 - A.D, A.TS + A.D, v0 - A.D, A.TS + A.D, rlo,
                                      rhi, rrow, threadIdx.x, blockDim.x);
    __syncthreads();
    for (int q = 0; q < nrng; ++q) {
        const int g0 = rrow[q];
        for (int64_t j = rlo[q] + threadIdx.x; j < rhi[q]; j += blockDim.x) {
            const VisMeta mt = A.meta[A.apos[j]];
            const int S = (mt.pos >> 16) & 255;
            const int h0 = A.ah0[j];
            for (int a = 0; a < S; ++a) {
                const int rr = wrap(g0 + a - u0, A.gx);  // row of the footprint relative to the tile
                if (rr >= A.TS) continue;
                for (int b = 0; b < S; ++b) {
                    const int cc = wrap(h0 + b - v0, A.gy);
                    if (cc >= A.TS) continue;
                    const int cell = rr * A.TS + cc;
                    atomicOr(&bm[cell >> 5], 1u << (cell & 31));
                }
            }
        }
    }
    __syncthreads();
    int cnt = 0;
    for (int e = threadIdx.x; e < words; e += blockDim.x) {
        A.bits[(size_t)blockIdx.x * words + e] = bm[e];
        cnt += __popc(bm[e]);
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    __shared__ int wsum[8];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
        A.count[blockIdx.x] = t;
    }
}

// Rank of cell `cell` among the covered cells of a tile (row-major) from its bitmap.
__device__ __forceinline__ int64_t owner_rank(const uint32_t* bm, int cell) {
    int r = 0;
    for (int w = 0; w < (cell >> 5); ++w) r += __popc(bm[w]);
    return r + __popc(bm[cell >> 5] & ((1u << (cell & 31)) - 1u));
}

// Build pass: one CTA per HB_OWN x HB_OWN owners of a needed tile.
__global__ void __launch_bounds__(HB_WARPS * 32, 1) hbuild_kernel(HArgs A, int S_max) {
    extern __shared__ __align__(16) unsigned char hsm[];
    const int ne = A.ne;
    float2* acc = reinterpret_cast<float2*>(hsm);                       // [HB_WARPS][ne]
    float2* taps = acc + (size_t)HB_WARPS * ne;                          // [HB_CHUNK][S_max^2]
    int4* cmeta = reinterpret_cast<int4*>(taps + (size_t)HB_CHUNK * S_max * S_max);  // g0, h0, S, -
    int* sent = reinterpret_cast<int*>(cmeta + HB_CHUNK);               // [ne]
    int64_t* rlo = reinterpret_cast<int64_t*>(sent + ne + (ne & 1));
    const int nrmax = 2 * (HB_OWN + A.D);
    int64_t* rhi = rlo + nrmax;
    int* rrow = reinterpret_cast<int*>(rhi + nrmax);
    __shared__ uint32_t tbits[128];

    const int per_side = A.TS / HB_OWN;
    const int t_idx = blockIdx.x / (per_side * per_side);
    const int sub = blockIdx.x - t_idx * per_side * per_side;
    const int tile = A.need[t_idx];
    const int tu = tile / A.ntv, tv = tile - tu * A.ntv;
    const int su0 = tu * A.TS + (sub / per_side) * HB_OWN, sv0 = tv * A.TS + (sub % per_side) * HB_OWN;
    const int words = A.TS * A.TS / 32;
    for (int e = threadIdx.x; e < words; e += blockDim.x) tbits[e] = A.bits[(size_t)t_idx * words + e];
    for (int e = threadIdx.x; e < ne; e += blockDim.x) sent[e] = A.ent[e];
    for (int e = threadIdx.x; e < HB_WARPS * ne; e += blockDim.x) acc[e] = make_float2(0.f, 0.f);
    const int nrng = candidate_ranges(A.arow, A.ah0, A.gx, A.gy, su0 - A.D, HB_OWN + A.D, sv0 - A.D, HB_OWN + A.D,
                                      rlo, rhi, rrow, threadIdx.x, blockDim.x);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ou = su0 + warp / HB_OWN, ov = sv0 + warp % HB_OWN;  // this warp's owner (grid cell)
    const int lcell = (ou - tu * A.TS) * A.TS + (ov - tv * A.TS);
    const bool covered = (tbits[lcell >> 5] >> (lcell & 31)) & 1u;
    float2* my = acc + (size_t)warp * ne;

    // walk the candidates in chunks
    int q = 0;
    int64_t j = nrng > 0 ? rlo[0] : 0;
    while (true) {
        // gather the next chunk's indices (same on every thread)
        int64_t idx[HB_CHUNK];
        int irow[HB_CHUNK];
        int nvis = 0;
        while (nvis < HB_CHUNK && q < nrng) {
            if (j >= rhi[q]) {
                ++q;
                if (q < nrng) j = rlo[q];
                continue;
            }
            irow[nvis] = rrow[q];
            idx[nvis++] = j++;
        }
        if (nvis == 0) break;
        __syncthreads();  // previous chunk consumed
        if (threadIdx.x < nvis) {
            int64_t jj = 0;
            int g0 = 0;
#pragma unroll
            for (int t = 0; t < HB_CHUNK; ++t)
                if (t == (int)threadIdx.x) jj = idx[t], g0 = irow[t];
            const VisMeta mt = A.meta[A.apos[jj]];
            cmeta[threadIdx.x] = make_int4(g0, (int)A.ah0[jj], (mt.pos >> 16) & 255, 0);
        }
        __syncthreads();
        for (int v = 0; v < nvis; ++v) {
            const int64_t jj = idx[v];
            const VisMeta mt = A.meta[A.apos[jj]];
            const int S = cmeta[v].z;
            const float2* src = A.gblk[mt.pos >> 24] + mt.off;
            for (int e = threadIdx.x; e < S * S; e += blockDim.x) taps[(size_t)v * S_max * S_max + e] = src[e];
        }
        __syncthreads();
        if (covered) {
            for (int v = 0; v < nvis; ++v) {
                const int4 cm = cmeta[v];
                const int S = cm.z;
                const int pu = wrap(ou - cm.x, A.gx), pv = wrap(ov - cm.y, A.gy);
                if (pu >= S || pv >= S) continue;  // the footprint misses this owner
                const float2* T = taps + (size_t)v * S_max * S_max;
                for (int e = lane; e < ne; e += 32) {
                    const int en = sent[e];
                    const int a = (en >> 8) & 255, b = en & 255;
                    int u1, v1, u2, v2;
                    if ((en >> 16) == 0) {
                        u1 = pu, v1 = pv, u2 = pu + a, v2 = pv + b;
                    } else {
                        u1 = pu, v1 = pv + b, u2 = pu + a, v2 = pv;
                    }
                    if (u2 >= S || v1 >= S || v2 >= S) continue;
                    const float2 t1 = T[u1 * S + v1], t2 = T[u2 * S + v2];
                    // conj(t1) t2; the diagonal (e = 0) is |t1|^2, real by construction
                    my[e].x = fmaf(t1.x, t2.x, fmaf(t1.y, t2.y, my[e].x));
                    if (e != 0) my[e].y = fmaf(t1.x, t2.y, fmaf(-t1.y, t2.x, my[e].y));
                }
            }
        }
    }
    __syncthreads();
    if (!covered) return;
    const int64_t row = A.hoff[t_idx] + owner_rank(tbits, lcell);
    float2* dst = A.rows + (size_t)row * ne;
    float m = 0.f;
    for (int e = lane; e < ne; e += 32) {
        const float2 h = my[e];
        dst[e] = h;
        m = fmaxf(m, fabsf(h.x) + fabsf(h.y));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) {
        atomicMax(A.fx + FX_HMAX, __float_as_uint(m));
        atomicMax(A.tmax + t_idx, __float_as_uint(m));
    }
}

// ---- apply
struct HApplyArgs {
    const float2* X;          // forward grid [gx][gy] (valid on needed tiles)
    const uint8_t* need_mask; // [tile] of this bin
    const int32_t* need;      // needed tiles of the bin
    const uint32_t* bits;
    const int64_t* hoff;
    const float2* val;        // the owner rows: dense [owner][ne], or their non-zero entries
    const uint16_t* idx;      // compressed: the entry numbers
    const int64_t* roff;      // compressed: [owner + 1] first entry of each owner row (null: dense)
    const uint32_t* tmax;     // [needed tile] max |h|_1 of the tile's rows
    const int32_t* ent;
    float2* patch;            // [needed tile][PW * PW]
    int gx, gy, ntv, TS, D, PW, ne, shift;
};

__device__ __forceinline__ void fx_add(int* hi, int* lo, int ci, float d) {
    const float tq = __fadd_rn(d, HX_MAGIC);
    const int q1 = __float_as_int(tq) - HX_MAGIC_BITS;
    const float rf = __fsub_rn(d, __fsub_rn(tq, HX_MAGIC));
    const int q2 = __float_as_int(__fmaf_rn(rf, 65536.f, HX_MAGIC)) - HX_MAGIC_BITS;
    atomicAdd(hi + ci, q1);
    atomicAdd(lo + ci, q2);
}

__global__ void __launch_bounds__(HA_WARPS * 32, 1) happly_kernel(HApplyArgs A) {
    extern __shared__ __align__(16) unsigned char hsm[];
    const int PW = A.PW, np = PW * PW, ne = A.ne;
    float2* Z = reinterpret_cast<float2*>(hsm);          // input patch
    int* Ohi = reinterpret_cast<int*>(Z + np);            // [cell][re, im]
    int* Olo = Ohi + 2 * np;
    int* sent = Olo + 2 * np;
    __shared__ uint32_t tbits[128];
    __shared__ float s_scale[2];
    __shared__ float s_zmax[HA_WARPS];
    const int t_idx = blockIdx.x;
    const int tile = A.need[t_idx];
    const int tu = tile / A.ntv, tv = tile - tu * A.ntv;
    const int u0 = tu * A.TS, v0 = tv * A.TS;
    const int words = A.TS * A.TS / 32;
    const int ntu = A.gx / A.TS;
    for (int e = threadIdx.x; e < words; e += blockDim.x) tbits[e] = A.bits[(size_t)t_idx * words + e];
    for (int e = threadIdx.x; e < ne; e += blockDim.x) sent[e] = A.ent[e];
    float zm = 0.f;
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
        const int a = e / PW, b = e - a * PW;
        const int gu = wrap(u0 + a, A.gx), gv = wrap(v0 + b, A.gy);
        const int tt = (gu >> A.shift) * A.ntv + (gv >> A.shift);
        const float2 z = A.need_mask[tt] ? A.X[(size_t)gu * A.gy + gv] : make_float2(0.f, 0.f);
        Z[e] = z;
        zm = fmaxf(zm, fabsf(z.x) + fabsf(z.y));
        Ohi[2 * e] = Ohi[2 * e + 1] = 0;
        Olo[2 * e] = Olo[2 * e + 1] = 0;
    }
    (void)ntu;
    for (int o = 16; o > 0; o >>= 1) zm = fmaxf(zm, __shfl_xor_sync(0xffffffffu, zm, o));
    if ((threadIdx.x & 31) == 0) s_zmax[threadIdx.x >> 5] = zm;
    __syncthreads();
    if (threadIdx.x == 0) {
        // bound on one accumulated term of this tile: the gathered type-A sum, (D+1)^2
        // entries of |h|_1 <= the tile's max times |z|_1 <= the patch's max (margin 2);
        // at most 2 ne terms per cell.  Per-tile bounds keep the fixed-point resolution
        // relative to the tile's own values where H spans orders of magnitude.
        float zmax = 0.f;
        for (int w = 0; w < HA_WARPS; ++w) zmax = fmaxf(zmax, s_zmax[w]);
        const float hmax = __uint_as_float(__ldg(A.tmax + t_idx));
        const float mt = 2.f * (float)((A.D + 1) * (A.D + 1)) * hmax * zmax;
        float s1 = 1.f, inv = 1.f;
        if (mt > 0.f) {
            const float lim = fminf(2097152.f, 1073741824.f / (float)(2 * ne));
            int ex = (int)((__float_as_uint(lim / mt) >> 23) & 255u) - 127;
            ex = ex < -120 ? -120 : (ex > 120 ? 120 : ex);
            s1 = __uint_as_float((uint32_t)(ex + 127) << 23);
            inv = __uint_as_float((uint32_t)(127 - ex) << 23);
        }
        s_scale[0] = s1;
        s_scale[1] = inv;
    }
    __syncthreads();
    const float s1 = s_scale[0];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t base = A.hoff[t_idx];
    const int nown = (int)(A.hoff[t_idx + 1] - base);
    // owners of this warp: covered cells w, w + HA_WARPS, ... in row-major rank order
    int cell = -1, rank = -1;
    for (int k = warp; k < nown; k += HA_WARPS) {
        // advance (cell, rank) to the k-th covered cell
        while (rank < k) {
            ++cell;
            if ((tbits[cell >> 5] >> (cell & 31)) & 1u) ++rank;
        }
        const int lu = cell / A.TS, lv = cell - lu * A.TS;
        const bool dense = A.roff == nullptr;
        const int64_t q0 = dense ? (base + k) * ne : __ldg(&A.roff[base + k]);
        const int64_t q1 = dense ? q0 + ne : __ldg(&A.roff[base + k + 1]);
        const float2 zo = Z[lu * PW + lv];
        float gx = 0.f, gy = 0.f;
        for (int64_t q = q0 + lane; q < q1; q += 32) {
            const float2 h = __ldg(&A.val[q]);
            const int e = dense ? (int)(q - q0) : __ldg(&A.idx[q]);
            const int en = sent[e];
            const int a = (en >> 8) & 255, b = en & 255;
            if ((en >> 16) == 0) {
                const int c2 = (lu + a) * PW + lv + b;
                const float2 z2 = Z[c2];
                gx = fmaf(h.x, z2.x, fmaf(-h.y, z2.y, gx));  // h z2
                gy = fmaf(h.x, z2.y, fmaf(h.y, z2.x, gy));
                if (a | b) {  // conj(h) z_owner into c2
                    fx_add(Ohi, Olo, 2 * c2, s1 * fmaf(h.x, zo.x, h.y * zo.y));
                    fx_add(Ohi, Olo, 2 * c2 + 1, s1 * fmaf(h.x, zo.y, -h.y * zo.x));
                }
            } else {
                const int c1 = lu * PW + lv + b, c2 = (lu + a) * PW + lv;
                const float2 z1 = Z[c1], z2 = Z[c2];
                fx_add(Ohi, Olo, 2 * c1, s1 * fmaf(h.x, z2.x, -h.y * z2.y));      // h z2 into c1
                fx_add(Ohi, Olo, 2 * c1 + 1, s1 * fmaf(h.x, z2.y, h.y * z2.x));
                fx_add(Ohi, Olo, 2 * c2, s1 * fmaf(h.x, z1.x, h.y * z1.y));       // conj(h) z1 into c2
                fx_add(Ohi, Olo, 2 * c2 + 1, s1 * fmaf(h.x, z1.y, -h.y * z1.x));
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            gx += __shfl_xor_sync(0xffffffffu, gx, o);
            gy += __shfl_xor_sync(0xffffffffu, gy, o);
        }
        if (lane == 0) {
            const int co = lu * PW + lv;
            fx_add(Ohi, Olo, 2 * co, s1 * gx);
            fx_add(Ohi, Olo, 2 * co + 1, s1 * gy);
        }
    }
    __syncthreads();
    const float inv = s_scale[1], inv_lo = inv * (1.f / 65536.f);
    float2* dst = A.patch + (size_t)t_idx * np;
    for (int e = threadIdx.x; e < np; e += blockDim.x)
        dst[e] = make_float2(fmaf((float)Olo[2 * e], inv_lo, (float)Ohi[2 * e] * inv),
                             fmaf((float)Olo[2 * e + 1], inv_lo, (float)Ohi[2 * e + 1] * inv));
}

size_t hbuild_smem(int ne, int S_max, int D) {
    return (size_t)HB_WARPS * ne * sizeof(float2) + (size_t)HB_CHUNK * S_max * S_max * sizeof(float2) +
           HB_CHUNK * sizeof(int4) + (size_t)(ne + 2) * sizeof(int) +
           (size_t)2 * (HB_OWN + D) * (2 * sizeof(int64_t) + sizeof(int)) + 64;
}

size_t happly_smem(int PW, int ne) {
    const size_t np = (size_t)PW * PW;
    return np * sizeof(float2) + 4 * np * sizeof(int) + (size_t)ne * sizeof(int);
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { cudaFree(p); }
};

// Non-zero entries of each dense owner row (one warp per row); diag[0] += the rows whose
// entry 0 (H[o][o]) is non-zero.
__global__ void __launch_bounds__(256) hrowcount_kernel(const float2* __restrict__ rows, int64_t nown, int ne,
                                                        int32_t* __restrict__ counts, unsigned long long* diag) {
    const int lane = threadIdx.x & 31;
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= nown) return;
    const float2* row = rows + (size_t)r * ne;
    int n = 0;
    for (int e = lane; e < ne; e += 32) {
        const float2 h = row[e];
        n += (h.x != 0.f || h.y != 0.f) ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if (lane == 0) {
        counts[r] = n;
        const float2 h0 = row[0];
        if (h0.x != 0.f || h0.y != 0.f) atomicAdd(diag, 1ull);
    }
}

// Keeps the non-zero entries of each dense owner row at roff[row] (one warp per row,
// entries in row order).
__global__ void __launch_bounds__(256) hcompact_kernel(const float2* __restrict__ rows, int64_t nown, int ne,
                                                       const int64_t* __restrict__ roff, float2* __restrict__ val,
                                                       uint16_t* __restrict__ idx) {
    const int lane = threadIdx.x & 31;
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= nown) return;
    const float2* row = rows + (size_t)r * ne;
    int64_t q = roff[r];
    for (int e0 = 0; e0 < ne; e0 += 32) {
        const int e = e0 + lane;
        const float2 h = e < ne ? row[e] : make_float2(0.f, 0.f);
        const bool on = h.x != 0.f || h.y != 0.f;
        const uint32_t m = __ballot_sync(0xffffffffu, on);
        if (on) {
            const int64_t at = q + __popc(m & ((1u << lane) - 1u));
            val[at] = h;
            idx[at] = (uint16_t)e;
        }
        q += __popc(m);
    }
}

}  // namespace

void launch_happly(const rimo_plan* p, int bin, cudaStream_t s) {
    const auto& br = p->bins[bin];
    const int nneed = br.n1 - br.n0;
    if (nneed <= 0) return;
    const int ntu = p->gx / p->TS, ntv = p->gy / p->TS;
    const size_t ntile = (size_t)ntu * ntv;
    HApplyArgs A;
    A.X = p->d_X;
    A.need_mask = p->d_need + (size_t)bin * ntile;
    A.need = p->d_need_list + br.n0;
    A.bits = p->d_hbits[bin];
    A.hoff = p->d_hoff[bin];
    A.val = p->d_hval[bin];
    A.idx = p->h_dense[bin] ? nullptr : p->d_hidx[bin];
    A.roff = p->h_dense[bin] ? nullptr : p->d_hroff[bin];
    A.tmax = p->d_htmax[bin];
    A.ent = p->d_hent;
    A.patch = p->d_hpatch;
    A.gx = p->gx;
    A.gy = p->gy;
    A.ntv = ntv;
    A.TS = p->TS;
    A.D = p->H;
    A.PW = p->PW;
    A.ne = p->h_ne;
    A.shift = p->TS == 64 ? 6 : 5;
    const size_t sm = happly_smem(p->PW, p->h_ne);
    RIMO_CUDA(cudaFuncSetAttribute(happly_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    happly_kernel<<<nneed, HA_WARPS * 32, sm, s>>>(A);
}

// Builds H for every bin; see the file comment.  Synchronises s.
static void build_holographic(rimo_plan* p, cudaStream_t s) {
    const int P = p->P, TS = p->TS, D = p->H, gx = p->gx, gy = p->gy;
    const int ntu = gx / TS, ntv = gy / TS;
    const size_t ntile = (size_t)ntu * ntv;
    if (gy > 65536) fail(RIMO_ERR_UNSUPPORTED, "holographic build needs grid columns < 65536");
    if (TS * TS / 32 > 128) fail(RIMO_ERR_UNSUPPORTED, "tile too large for the coverage bitmap");
    const int ne = (D + 1) * (D + 1) + D * D;
    const int words = TS * TS / 32;

    // ---- anchor index on the host: per bin, sorted positions ordered by (g0, h0)
    std::vector<VisMeta> meta((size_t)p->M);
    RIMO_CUDA(cudaMemcpyAsync(meta.data(), p->d_meta, meta.size() * sizeof(VisMeta), cudaMemcpyDeviceToHost, s));
    RIMO_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> g0((size_t)p->M), h0((size_t)p->M);
    for (const auto& u : p->tiles_host)
        for (int64_t i = u.vb; i < u.ve; ++i) {
            g0[i] = u.tu * TS + (int)(meta[i].pos & 255u);
            h0[i] = u.tv * TS + (int)((meta[i].pos >> 8) & 255u);
        }
    std::vector<int32_t> apos((size_t)p->M);
    std::vector<uint16_t> ah0((size_t)p->M);
    std::vector<int64_t> arow((size_t)P * (gx + 1), 0);
    planner::parallel_for(P, [&](int64_t b0, int64_t b1) {
        std::vector<int64_t> ccount;
        for (int64_t b = b0; b < b1; ++b) {
            const int64_t vb = p->bins[b].vb, ve = p->bins[b].ve;
            const int64_t n = ve - vb;
            if (n == 0) continue;
            // stable counting sort by h0, then by g0
            std::vector<int32_t> t1((size_t)n), t2((size_t)n);
            ccount.assign((size_t)gy + 1, 0);
            for (int64_t i = vb; i < ve; ++i) ccount[h0[i] + 1]++;
            for (int c = 0; c < gy; ++c) ccount[c + 1] += ccount[c];
            for (int64_t i = vb; i < ve; ++i) t1[ccount[h0[i]]++] = (int32_t)i;
            int64_t* row = &arow[(size_t)b * (gx + 1)];
            std::vector<int64_t> rc((size_t)gx + 1, 0);
            for (int64_t k = 0; k < n; ++k) rc[g0[t1[k]] + 1]++;
            for (int g = 0; g < gx; ++g) rc[g + 1] += rc[g];
            for (int g = 0; g <= gx; ++g) row[g] = vb + rc[g];  // absolute indices into pos / h0
            for (int64_t k = 0; k < n; ++k) t2[rc[g0[t1[k]]]++] = t1[k];
            for (int64_t k = 0; k < n; ++k) {
                apos[vb + k] = t2[k];
                ah0[vb + k] = (uint16_t)h0[t2[k]];
            }
        }
    }, 1);
    AnchorIndex ai;
    RIMO_CUDA(cudaMalloc(&ai.pos, apos.size() * sizeof(int32_t)));
    RIMO_CUDA(cudaMalloc(&ai.h0, ah0.size() * sizeof(uint16_t)));
    RIMO_CUDA(cudaMalloc(&ai.row, arow.size() * sizeof(int64_t)));
    RIMO_CUDA(cudaMemcpyAsync(ai.pos, apos.data(), apos.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    RIMO_CUDA(cudaMemcpyAsync(ai.h0, ah0.data(), ah0.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, s));
    RIMO_CUDA(cudaMemcpyAsync(ai.row, arow.data(), arow.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));

    // ---- entry table, slots, coverage
    p->d_hent = upload_vec(p, entry_table(D), s);
    std::vector<int32_t> hslot((size_t)P * ntile, -1);
    for (int b = 0; b < P; ++b)
        for (int k = p->bins[b].n0; k < p->bins[b].n1; ++k) hslot[(size_t)b * ntile + p->need_host[k]] = k - p->bins[b].n0;
    p->d_hslot = upload_vec(p, hslot, s);
    p->d_hbits.assign(P, nullptr);
    p->d_hoff.assign(P, nullptr);
    p->d_hval.assign(P, nullptr);
    p->d_hidx.assign(P, nullptr);
    p->d_hroff.assign(P, nullptr);
    p->h_dense.assign(P, 0);
    p->d_htmax.assign(P, nullptr);
    p->hoff_host.assign(P, {});
    int max_need = 1;
    for (int b = 0; b < P; ++b) max_need = std::max(max_need, p->bins[b].n1 - p->bins[b].n0);
    DevBuf counts;
    RIMO_CUDA(cudaMalloc(&counts.p, (size_t)max_need * sizeof(int64_t)));
    HArgs A;
    std::memset(&A, 0, sizeof(A));
    A.meta = p->d_meta;
    A.gblk = p->d_gblock_ptrs;
    A.apos = ai.pos;
    A.ah0 = ai.h0;
    A.ent = p->d_hent;
    A.fx = p->d_fx;
    A.gx = gx;
    A.gy = gy;
    A.ntv = ntv;
    A.TS = TS;
    A.D = D;
    A.ne = ne;
    int64_t total = 0;
    const size_t cover_sm = (size_t)2 * (TS + D) * (2 * sizeof(int64_t) + sizeof(int)) + (size_t)words * sizeof(uint32_t) + 64;
    for (int b = 0; b < P; ++b) {
        const int nneed = p->bins[b].n1 - p->bins[b].n0;
        p->d_hbits[b] = (uint32_t*)dev_alloc(p, (size_t)std::max(1, nneed) * words * sizeof(uint32_t));
        p->hoff_host[b].assign((size_t)nneed + 1, 0);
        if (nneed == 0) {
            p->d_hoff[b] = upload_vec(p, p->hoff_host[b], s);
            continue;
        }
        A.arow = ai.row + (size_t)b * (gx + 1);
        A.need = p->d_need_list + p->bins[b].n0;
        A.bits = p->d_hbits[b];
        A.count = (int64_t*)counts.p;
        hcover_kernel<<<nneed, 256, cover_sm, s>>>(A);
        RIMO_CUDA(cudaGetLastError());
        std::vector<int64_t> c((size_t)nneed);
        RIMO_CUDA(cudaMemcpyAsync(c.data(), counts.p, c.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        RIMO_CUDA(cudaStreamSynchronize(s));
        for (int k = 0; k < nneed; ++k) p->hoff_host[b][k + 1] = p->hoff_host[b][k] + c[k];
        total += p->hoff_host[b][nneed];
        p->d_hoff[b] = upload_vec(p, p->hoff_host[b], s);
    }
    const size_t patch_bytes = (size_t)max_need * p->PW * p->PW * sizeof(float2);
    p->d_hpatch = (float2*)dev_alloc(p, patch_bytes);
    const size_t sm = hbuild_smem(ne, p->max_S, D);
    if (sm > 227 * 1024) fail(RIMO_ERR_UNSUPPORTED, "holographic build: owner rows exceed shared memory");
    RIMO_CUDA(cudaFuncSetAttribute(hbuild_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int per_tile = (TS / HB_OWN) * (TS / HB_OWN);
    // bin by bin: dense rows into a temporary, then only their non-zero entries kept
    std::vector<void*> made;  // the compressed arrays, released again if the budget refuses
    auto keep = [&](size_t bytes) {
        void* q = dev_alloc(p, std::max<size_t>(bytes, 16));
        made.push_back(q);
        return q;
    };
    auto release_made = [&]() {
        for (void* q : made) {
            if (!q) continue;
            auto it = std::find(p->owned.begin(), p->owned.end(), q);
            if (it != p->owned.end()) p->owned.erase(it);
            cudaFree(q);
        }
        made.clear();
    };
    int64_t nnz = 0, h_bytes = 0;
    unsigned long long diag = 0;
    DevBuf dcount, ddiag;
    RIMO_CUDA(cudaMalloc(&ddiag.p, sizeof(unsigned long long)));
    RIMO_CUDA(cudaMemsetAsync(ddiag.p, 0, sizeof(unsigned long long), s));
    try {
        for (int b = 0; b < P; ++b) {
            const int nneed = p->bins[b].n1 - p->bins[b].n0;
            const int64_t nown = p->hoff_host[b][(size_t)nneed];
            p->d_htmax[b] = (uint32_t*)keep((size_t)std::max(1, nneed) * sizeof(uint32_t));
            RIMO_CUDA(cudaMemsetAsync(p->d_htmax[b], 0, (size_t)std::max(1, nneed) * sizeof(uint32_t), s));
            std::vector<int64_t> roff((size_t)nown + 1, 0);
            if (nown > 0) {
                DevBuf dense;
                if (cudaMalloc(&dense.p, (size_t)nown * ne * sizeof(float2)) != cudaSuccess) {
                    cudaGetLastError();
                    fail(RIMO_ERR_OOM, "holographic build: dense rows of one bin");
                }
                made.push_back(nullptr);  // placeholder: the dense rows may be kept
                A.arow = ai.row + (size_t)b * (gx + 1);
                A.need = p->d_need_list + p->bins[b].n0;
                A.bits = p->d_hbits[b];
                A.hoff = p->d_hoff[b];
                A.rows = (float2*)dense.p;
                A.tmax = p->d_htmax[b];
                // without stored G, the bin's exact tiles are generated into the tap scratch first
                if (p->mode != RIMO_MODE_STORED_G)
                    launch_gbuild_range(p, p->bins[b].vb, p->bins[b].ve - p->bins[b].vb, s);
                hbuild_kernel<<<nneed * per_tile, HB_WARPS * 32, sm, s>>>(A, p->max_S);
                RIMO_CUDA(cudaGetLastError());
                cudaFree(dcount.p);
                dcount.p = nullptr;
                RIMO_CUDA(cudaMalloc(&dcount.p, (size_t)nown * sizeof(int32_t)));
                const int64_t blocks = (nown * 32 + 255) / 256;
                hrowcount_kernel<<<(unsigned)blocks, 256, 0, s>>>((const float2*)dense.p, nown, ne, (int32_t*)dcount.p,
                                                                  (unsigned long long*)ddiag.p);
                RIMO_CUDA(cudaGetLastError());
                std::vector<int32_t> c((size_t)nown);
                RIMO_CUDA(cudaMemcpyAsync(c.data(), dcount.p, c.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
                RIMO_CUDA(cudaStreamSynchronize(s));
                for (int64_t k = 0; k < nown; ++k) roff[(size_t)k + 1] = roff[(size_t)k] + c[(size_t)k];
                const int64_t nb = roff[(size_t)nown];
                const int64_t dense_bytes = nown * ne * (int64_t)sizeof(float2);
                const int64_t packed_bytes =
                    nb * (int64_t)(sizeof(float2) + sizeof(uint16_t)) + (nown + 1) * (int64_t)sizeof(int64_t);
                const bool keep_dense = dense_bytes <= packed_bytes;
                h_bytes += keep_dense ? dense_bytes : packed_bytes;
                nnz += nb;
                if (p->prm.mem_budget_bytes > 0 && p->info.g_bytes + h_bytes > p->prm.mem_budget_bytes)
                    fail(RIMO_ERR_BUDGET, "holographic matrices need more than the " +
                                              std::to_string(p->prm.mem_budget_bytes - p->info.g_bytes) +
                                              " bytes the budget leaves beyond G");
                if (keep_dense) {
                    // the bin's coverage is dense: the temporary becomes the stored rows
                    p->owned.push_back(dense.p);
                    made.back() = dense.p;
                    p->d_hval[b] = (float2*)dense.p;
                    dense.p = nullptr;
                    p->h_dense[b] = 1;
                    continue;
                }
                made.pop_back();
                p->d_hroff[b] = (int64_t*)keep(roff.size() * sizeof(int64_t));
                RIMO_CUDA(cudaMemcpyAsync(p->d_hroff[b], roff.data(), roff.size() * sizeof(int64_t),
                                          cudaMemcpyHostToDevice, s));
                p->d_hval[b] = (float2*)keep((size_t)nb * sizeof(float2));
                p->d_hidx[b] = (uint16_t*)keep((size_t)nb * sizeof(uint16_t));
                hcompact_kernel<<<(unsigned)blocks, 256, 0, s>>>((const float2*)dense.p, nown, ne, p->d_hroff[b],
                                                                 p->d_hval[b], p->d_hidx[b]);
                RIMO_CUDA(cudaGetLastError());
                RIMO_CUDA(cudaStreamSynchronize(s));  // the dense rows are freed next
            } else {
                p->d_hroff[b] = (int64_t*)keep(roff.size() * sizeof(int64_t));
                RIMO_CUDA(cudaMemcpyAsync(p->d_hroff[b], roff.data(), roff.size() * sizeof(int64_t),
                                          cudaMemcpyHostToDevice, s));
                p->d_hval[b] = (float2*)keep(16);
                p->d_hidx[b] = (uint16_t*)keep(16);
            }
        }
        RIMO_CUDA(cudaMemcpyAsync(&diag, ddiag.p, sizeof(diag), cudaMemcpyDeviceToHost, s));
        RIMO_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
        cudaStreamSynchronize(s);
        release_made();
        throw;
    }
    p->info.h_entries = total * ne;              // a dense stencil per covered cell
    p->info.h_nonzero = nnz;                      // what the rows keep
    p->info.h_nnz = 2 * (nnz - (int64_t)diag) + (int64_t)diag;
    p->h_ne = ne;
    p->info.h_bytes = h_bytes + (int64_t)patch_bytes;
    p->h_built = true;
}

}  // namespace rimo

extern "C" {

rimo_status rimo_build_holographic(rimo_plan_t p, void* stream) {
    RIMO_API_BEGIN
    if (!p) fail(RIMO_ERR_INVALID_ARG, "null plan");
    if (p->mode == RIMO_MODE_SURROGATE) fail(RIMO_ERR_UNSUPPORTED, "H is built from exact tiles");
    if (p->prm.shard_count >= 2)
        fail(RIMO_ERR_UNSUPPORTED, "H of a shard plan: not provided (shard plans apply G^dagger G)");
    if (!p->h_built) build_holographic(p, (cudaStream_t)stream);
    RIMO_API_END
}

rimo_status rimo_plan_get_holographic(rimo_plan_t p, int32_t bin, const int32_t* pairs, int64_t n,
                                      rimo_cfloat* out, void* stream) {
    RIMO_API_BEGIN
    if (!p || !pairs || !out || n < 0) fail(RIMO_ERR_INVALID_ARG, "null argument");
    if (!p->h_built) fail(RIMO_ERR_STATE, "rimo_build_holographic has not run");
    if (bin < 0 || bin >= p->P) fail(RIMO_ERR_INVALID_ARG, "bin out of range");
    cudaStream_t s = (cudaStream_t)stream;
    const int TS = p->TS, D = p->H, gx = p->gx, gy = p->gy, ntv = gy / TS;
    const int words = TS * TS / 32;
    auto wrapd = [](int d, int n) {  // signed offset of the shorter way round
        d %= n;
        if (d < 0) d += n;
        return d > n / 2 ? d - n : d;
    };
    for (int64_t q = 0; q < n; ++q) {
        int u1 = pairs[4 * q], v1 = pairs[4 * q + 1], u2 = pairs[4 * q + 2], v2 = pairs[4 * q + 3];
        int du = wrapd(u2 - u1, gx), dv = wrapd(v2 - v1, gy);
        bool conj = false;
        if (du < 0 || (du == 0 && dv < 0)) {  // H[c2][c1] = conj(H[c1][c2])
            std::swap(u1, u2);
            std::swap(v1, v2);
            du = -du;
            dv = -dv;
            conj = true;
        }
        out[q] = rimo_cfloat{0.f, 0.f};
        if (du > D || dv > D || dv < -D) continue;
        int ou, ov, e;
        if (dv >= 0) {
            ou = u1, ov = v1, e = du * (D + 1) + dv;
        } else {
            ou = u1, ov = (v2 % gy + gy) % gy, e = (D + 1) * (D + 1) + (du - 1) * D + (-dv - 1);
        }
        ou = (ou % gx + gx) % gx;
        ov = (ov % gy + gy) % gy;
        const int tile = (ou / TS) * ntv + ov / TS;
        int k = -1;
        for (int i = p->bins[bin].n0; i < p->bins[bin].n1; ++i)
            if (p->need_host[i] == tile) k = i - p->bins[bin].n0;
        if (k < 0) continue;
        std::vector<uint32_t> bm((size_t)words);
        RIMO_CUDA(cudaMemcpyAsync(bm.data(), p->d_hbits[bin] + (size_t)k * words, words * sizeof(uint32_t),
                                  cudaMemcpyDeviceToHost, s));
        RIMO_CUDA(cudaStreamSynchronize(s));
        const int cell = (ou % TS) * TS + ov % TS;
        if (!((bm[cell >> 5] >> (cell & 31)) & 1u)) continue;
        int64_t rank = 0;
        for (int w = 0; w < (cell >> 5); ++w) rank += __builtin_popcount(bm[w]);
        rank += __builtin_popcount(bm[cell >> 5] & ((1u << (cell & 31)) - 1u));
        const int64_t row = p->hoff_host[bin][(size_t)k] + rank;
        if (p->h_dense[bin]) {
            float2 h;
            RIMO_CUDA(cudaMemcpyAsync(&h, p->d_hval[bin] + (size_t)row * p->h_ne + e, sizeof(h),
                                      cudaMemcpyDeviceToHost, s));
            RIMO_CUDA(cudaStreamSynchronize(s));
            out[q] = rimo_cfloat{h.x, conj ? -h.y : h.y};
            continue;
        }
        // the row keeps its non-zero entries, in entry order: find entry e among them
        int64_t span[2];
        RIMO_CUDA(cudaMemcpyAsync(span, p->d_hroff[bin] + row, sizeof(span), cudaMemcpyDeviceToHost, s));
        RIMO_CUDA(cudaStreamSynchronize(s));
        std::vector<uint16_t> ids((size_t)(span[1] - span[0]));
        if (!ids.empty()) {
            RIMO_CUDA(cudaMemcpyAsync(ids.data(), p->d_hidx[bin] + span[0], ids.size() * sizeof(uint16_t),
                                      cudaMemcpyDeviceToHost, s));
            RIMO_CUDA(cudaStreamSynchronize(s));
        }
        const auto it = std::lower_bound(ids.begin(), ids.end(), (uint16_t)e);
        if (it == ids.end() || *it != (uint16_t)e) continue;  // a zero entry
        float2 h;
        RIMO_CUDA(cudaMemcpyAsync(&h, p->d_hval[bin] + span[0] + (it - ids.begin()), sizeof(h), cudaMemcpyDeviceToHost, s));
        RIMO_CUDA(cudaStreamSynchronize(s));
        out[q] = rimo_cfloat{h.x, conj ? -h.y : h.y};
    }
    RIMO_API_END
}

}  // extern "C"
