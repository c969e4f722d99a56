// Build of the de-gridding tiles of G (Section 3.2, Eq. 6; stage 3 of Fig. 3): per
// visibility the residual w-kernel (Section 3.1, Fig. 1) convolved with the Kaiser-Bessel
// taps, into the stored blocks of G or into a bin's tap scratch at apply time; and the
// optional per-plan table of sampled w-kernels.
#include <algorithm>
#include <cstring>

#include "internal.h"

namespace rimo {

// ---------------------------------------------------------------------------
// Build of G (stage 3 of Fig. 3): one warp per visibility.
//   1. residual w-kernel (Section 3.1, Fig. 1): K(t) = (1/L^2) sum c[a][b] e^{+2 pi i
//      (t_x a_c + t_y b_c)/L} over the L x L grid (a_c, b_c in [-L/2, L/2)) of the tapered
//      chirp c.  c depends on lam and mu only through lam^2, mu^2, |lam| and |mu|, so it is
//      even in a_c and in b_c (the edge a_c = -L/2 has no partner).  Summing each pair of
//      signs first gives K(t) = (1/L^2) sum over a', b' in [0, L/2] of c(a', b') w(a', t_x)
//      w(b', t_y) with real weights w(0, t) = 1, w(a', t) = 2 cos(2 pi a' t / L) and
//      w(L/2, t) = cos(pi t): (L/2 + 1)^2 chirp samples instead of L^2, and K even in t_x
//      and t_y, so only t in [0, h]^2 is summed: a row pass over a' (chirp in registers),
//      then a column pass over b'; or, with a per-plan table of sampled kernels, cubic
//      Lagrange interpolation in w_r;
//   2. Kaiser-Bessel taps w_u[i] = KB(phi_u + J/2 - 1 - i), KB by Horner in
//      rho = 1 - (2t/J)^2 of its normalised power series;
//   3. T = w_u (*) K (*) w_v  (separable two-step convolution), S = S_w + J - 1.
struct BuildArgs {
    const VisMeta* meta;
    const float* wr;
    const float* phiu;
    const float* phiv;
    float2* const* gblk;
    const float* wk_dn;  // folded dn, Q x Q (Q = L/2 + 1)
    const float* tau_x;  // folded tapers, Q
    const float* tau_y;
    const float* wc;     // folded weights w(a', t), Q x 8 (t < 5 used)
    const float* kb_coef;
    int kb_nterm;
    int L, hmax, J, literal;
    int64_t v0, nvis;        // sorted visibilities [v0, v0 + nvis)
    uint32_t* fx;
    const float* wt;         // data weights (sorted order) multiplying the tiles, or null
    // tabulated kernels: K(t; w_j) at w_j = tab_w0 + j tab_dw, j = 0 .. tab_n + 2, 25 entries
    // [t_x][t_y] each (t in [0, 4]); used when kwtab is set, written by the table build
    const float2* kwtab;
    float2* kwtab_out;
    int tab_n;
    float tab_inv_dw, tab_x0;  // x = w tab_inv_dw + tab_x0: sample coordinate of w
    double tab_w0, tab_dw;
};

__device__ __forceinline__ float kb_eval(float t, float invhalf, const float* coef, int nterm) {
    const float q = t * invhalf;
    const float rho = 1.f - q * q;
    if (rho < 0.f) return 0.f;
    float acc = coef[nterm - 1];
    for (int k = nterm - 2; k >= 0; --k) acc = fmaf(acc, rho, coef[k]);
    return acc;
}

constexpr int BUILD_TQ = 5;     // folded tap offsets t in [0, hmax], hmax <= 4
constexpr int BUILD_WS = 8;     // row stride of the weight table (32 bytes: aligned float4 reads)
constexpr int BUILD_WARPS = 8;

// Chirp sample c(a', b') of the folded grid (a', b' in [0, L/2]) for residual w
__device__ __forceinline__ float2 chirp_at(const float* s_dn, const float* s_tx, const float* s_ty, int Q,
                                          int a, int b, float w, int literal) {
    float sn, cs;
    sincospif(2.f * w * s_dn[a * Q + b], &sn, &cs);
    const float tt = s_tx[a] * s_ty[b];
    return literal ? make_float2(tt * cs, -tt * sn) : make_float2(1.f + tt * (cs - 1.f), -tt * sn);
}

// The folded residual w-kernel K(t_x, t_y; w) for t in [0, hq)^2 into Kq[t_x][t_y] (row
// stride BUILD_TQ), by one warp (Section 3.1, Fig. 1; folding as described above).
// L: the w-kernel grid side (16, 32, 64 or 128).  Row pass: the L/2 columns b' < L/2 are
// spread over the lanes (F lanes per column when L/2 < 32, each summing a slice of a';
// CPL columns per lane when L/2 > 32), with the chirp evaluated in registers; the edge
// row a' = L/2 is added by every lane for its columns; the edge column b' = L/2 is a
// warp reduction (a' over the lanes) plus the corner.  Then the column pass over b'.
template <int L>
__device__ __forceinline__ void folded_wkernel(const float* s_dn, const float* s_tx, const float* s_ty,
                                               const float* s_wc, float w, int literal, int hq, float2* R,
                                               float2* Kq, int lane, float invL2) {
    constexpr int NC = L / 2, Q = NC + 1;
    constexpr int LW = NC < 32 ? NC : 32;
    constexpr int F = 32 / LW;
    constexpr int CPL = NC < 32 ? 1 : NC / 32;
    constexpr int APL = NC / F;
    constexpr int EPL = (NC + 31) / 32;
    const int col0 = lane % LW, a_begin = (lane / LW) * APL;
    // 1a. row pass over a' < L/2 for this lane's columns, chirp in registers
    float2 acc[CPL][BUILD_TQ];
#pragma unroll
    for (int j = 0; j < CPL; ++j)
#pragma unroll
        for (int t = 0; t < BUILD_TQ; ++t) acc[j][t] = make_float2(0.f, 0.f);
#pragma unroll 2
    for (int a = a_begin; a < a_begin + APL; ++a) {
        const float4 w03 = *reinterpret_cast<const float4*>(s_wc + a * BUILD_WS);
        const float w4 = s_wc[a * BUILD_WS + 4];
        const float wt[BUILD_TQ] = {w03.x, w03.y, w03.z, w03.w, w4};
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
            const float2 c = chirp_at(s_dn, s_tx, s_ty, Q, a, col0 + 32 * j, w, literal);
#pragma unroll
            for (int t = 0; t < BUILD_TQ; ++t) {
                acc[j][t].x = fmaf(wt[t], c.x, acc[j][t].x);
                acc[j][t].y = fmaf(wt[t], c.y, acc[j][t].y);
            }
        }
    }
    // the F slices of a column meet in every one of their lanes
#pragma unroll
    for (int o = LW; o < 32; o <<= 1)
#pragma unroll
        for (int j = 0; j < CPL; ++j)
#pragma unroll
            for (int t = 0; t < BUILD_TQ; ++t) {
                acc[j][t].x += __shfl_xor_sync(0xffffffffu, acc[j][t].x, o);
                acc[j][t].y += __shfl_xor_sync(0xffffffffu, acc[j][t].y, o);
            }
    // edge row a' = L/2 (weight (-1)^t), then the columns to shared memory
    if (lane < LW) {
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
            const int b = col0 + 32 * j;
            const float2 c = chirp_at(s_dn, s_tx, s_ty, Q, NC, b, w, literal);
#pragma unroll
            for (int t = 0; t < BUILD_TQ; ++t) {
                const float sg = (t & 1) ? -1.f : 1.f;
                R[b * BUILD_TQ + t] = make_float2(fmaf(sg, c.x, acc[j][t].x), fmaf(sg, c.y, acc[j][t].y));
            }
        }
    }
    // edge column b' = L/2: sum over a' < L/2 across the lanes, plus the corner
    {
        float2 e[BUILD_TQ];
#pragma unroll
        for (int t = 0; t < BUILD_TQ; ++t) e[t] = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < EPL; ++i) {
            const int a = lane + 32 * i;
            if (a < NC) {
                const float2 c = chirp_at(s_dn, s_tx, s_ty, Q, a, NC, w, literal);
#pragma unroll
                for (int t = 0; t < BUILD_TQ; ++t) {
                    const float wt = s_wc[a * BUILD_WS + t];
                    e[t].x = fmaf(wt, c.x, e[t].x);
                    e[t].y = fmaf(wt, c.y, e[t].y);
                }
            }
        }
        if (lane == 0) {
            const float2 c = chirp_at(s_dn, s_tx, s_ty, Q, NC, NC, w, literal);
#pragma unroll
            for (int t = 0; t < BUILD_TQ; ++t) {
                const float sg = (t & 1) ? -1.f : 1.f;
                e[t].x = fmaf(sg, c.x, e[t].x);
                e[t].y = fmaf(sg, c.y, e[t].y);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int t = 0; t < BUILD_TQ; ++t) {
                e[t].x += __shfl_xor_sync(0xffffffffu, e[t].x, o);
                e[t].y += __shfl_xor_sync(0xffffffffu, e[t].y, o);
            }
        if (lane == 0)
#pragma unroll
            for (int t = 0; t < BUILD_TQ; ++t) R[NC * BUILD_TQ + t] = e[t];
    }
    __syncwarp();
    // 1b. column pass: K(t_x, t_y) = (1/L^2) sum_b' R[b'][t_x] w(b', t_y)
    if (lane < hq * hq) {
        const int tx = lane / hq, ty = lane - tx * hq;
        float ar = 0.f, ai = 0.f;
#pragma unroll 4
        for (int b = 0; b < Q; ++b) {
            const float wt = s_wc[b * BUILD_WS + ty];
            const float2 r = R[b * BUILD_TQ + tx];
            ar = fmaf(wt, r.x, ar);
            ai = fmaf(wt, r.y, ai);
        }
        Kq[tx * BUILD_TQ + ty] = make_float2(ar * invL2, ai * invL2);
    }
    __syncwarp();
}

// Shared-memory tables of the folded w-kernel (both kernels below): weights, dn, tapers,
// KB coefficients, then one scratch per warp (row pass Q x 5, kernel 5 x 5, convolution
// 9 x 19, KB taps).
template <int L>
__device__ __forceinline__ void load_wk_tables(const BuildArgs& A, float* smb) {
    constexpr int Q = L / 2 + 1;
    float* s_wc = smb;
    float* s_dn = s_wc + Q * BUILD_WS;
    float* s_tx = s_dn + Q * Q;
    float* s_ty = s_tx + Q;
    float* s_coef = s_ty + Q;
    for (int e = threadIdx.x; e < Q * Q; e += blockDim.x) s_dn[e] = A.wk_dn[e];
    for (int e = threadIdx.x; e < Q; e += blockDim.x) {
        s_tx[e] = A.tau_x[e];
        s_ty[e] = A.tau_y[e];
    }
    for (int e = threadIdx.x; e < A.kb_nterm; e += blockDim.x) s_coef[e] = A.kb_coef[e];
    for (int e = threadIdx.x; e < Q * BUILD_WS; e += blockDim.x) s_wc[e] = A.wc[e];
    __syncthreads();
}

// Table of the folded kernels K(t; w_j), t in [0, 4]^2, at w_j = tab_w0 + j tab_dw for
// j = 0 .. tab_n + 2: one warp per sample, the same evaluation as the per-visibility build.
template <int L>
__global__ void __launch_bounds__(BUILD_WARPS * 32) kwtab_kernel(BuildArgs A) {
    constexpr int NC = L / 2, Q = NC + 1;
    extern __shared__ __align__(16) float smb[];
    load_wk_tables<L>(A, smb);
    const float* s_wc = smb;
    const float* s_dn = s_wc + Q * BUILD_WS;
    const float* s_tx = s_dn + Q * Q;
    const float* s_ty = s_tx + Q;
    constexpr int TABF = (Q * BUILD_WS + Q * Q + 2 * Q + 96 + 1) & ~1;
    constexpr int PER_WARP = Q * BUILD_TQ + BUILD_TQ * BUILD_TQ + 9 * 19 + 16;  // float2
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2* R = reinterpret_cast<float2*>(smb + TABF) + warp * PER_WARP;
    float2* Kq = R + Q * BUILD_TQ;
    const float invL2 = 1.f / ((float)L * (float)L);
    for (int j = blockIdx.x * BUILD_WARPS + warp; j < A.tab_n + 3; j += gridDim.x * BUILD_WARPS) {
        const float w = (float)(A.tab_w0 + (double)j * A.tab_dw);
        if (lane < BUILD_TQ * BUILD_TQ) Kq[lane] = make_float2(0.f, 0.f);
        __syncwarp();
        folded_wkernel<L>(s_dn, s_tx, s_ty, s_wc, w, A.literal, A.hmax + 1, R, Kq, lane, invL2);
        if (lane < BUILD_TQ * BUILD_TQ) A.kwtab_out[(size_t)j * (BUILD_TQ * BUILD_TQ) + lane] = Kq[lane];
        __syncwarp();
    }
}

// 3a. A[su][b] = sum_sv K(su - h, sv - h) w_v[b - sv]   (su < S_w, b < S)
// 3b. T[a][b]  = sum_su w_u[a - su] A[su][b]            (a, b < S), times the weight wk,
// stored to G (and the pad entry of an odd count), with the running tap bounds.
// Lane b < S owns column b: its S_w values of A stay in registers, the folded kernel is
// read by broadcast, and with S_w and J known every tap condition resolves at compile time.
template <int J, int SW>
__device__ __forceinline__ void conv_tile(const float2* Kq, const float* taps, float2* G, float wk, int lane,
                                          float& tmax, float& tsum) {
    constexpr int S = SW + J - 1, h = SW / 2, N = S * S;
    if (lane < S) {
        const int b = lane;
        float wvb[SW];  // w_v[b - sv], zero outside [0, J)
#pragma unroll
        for (int sv = 0; sv < SW; ++sv) {
            const int i = b - sv;
            wvb[sv] = (i >= 0 && i < J) ? taps[16 + (i >= 0 && i < J ? i : 0)] : 0.f;
        }
        float2 acol[SW];
#pragma unroll
        for (int su = 0; su < SW; ++su) {
            float ar = 0.f, ai = 0.f;
#pragma unroll
            for (int sv = 0; sv < SW; ++sv) {
                const float2 kv = Kq[(su > h ? su - h : h - su) * BUILD_TQ + (sv > h ? sv - h : h - sv)];
                ar = fmaf(kv.x, wvb[sv], ar);
                ai = fmaf(kv.y, wvb[sv], ai);
            }
            acol[su] = make_float2(ar, ai);
        }
        float wu[J];
#pragma unroll
        for (int i = 0; i < J; ++i) wu[i] = taps[i];
#pragma unroll
        for (int a = 0; a < S; ++a) {
            float2 out = make_float2(0.f, 0.f);
#pragma unroll
            for (int su = 0; su < SW; ++su) {
                if (a - su >= 0 && a - su < J) {
                    out.x = fmaf(wu[a - su], acol[su].x, out.x);
                    out.y = fmaf(wu[a - su], acol[su].y, out.y);
                }
            }
            out.x *= wk;
            out.y *= wk;
            G[a * S + b] = out;
            const float m = fabsf(out.x) + fabsf(out.y);
            tmax = fmaxf(tmax, m);
            tsum += m;
        }
    }
    if ((N & 1) && lane == 0) G[N] = make_float2(0.f, 0.f);  // the even-count pad
}

// the same for any J and S_w (sizes at run time)
__device__ __forceinline__ void conv_tile_any(const float2* Kq, const float* taps, float2* Ab, float2* G, float wk,
                                              int lane, int J, int Sw, float& tmax, float& tsum) {
    const int S = Sw + J - 1, h = Sw >> 1, n = S * S;
    for (int e = lane; e < Sw * S; e += 32) {
        const int su = e / S, b = e - su * S;
        const float2* Kr = Kq + abs(su - h) * BUILD_TQ;
        float ar = 0.f, ai = 0.f;
        for (int sv = 0; sv < Sw; ++sv) {
            const int i = b - sv;
            if (i >= 0 && i < J) {
                const float wv = taps[16 + i];
                const float2 kv = Kr[abs(sv - h)];
                ar = fmaf(kv.x, wv, ar);
                ai = fmaf(kv.y, wv, ai);
            }
        }
        Ab[su * 19 + b] = make_float2(ar, ai);
    }
    __syncwarp();
    for (int e = lane; e < n + (n & 1); e += 32) {
        float2 out = make_float2(0.f, 0.f);
        if (e < n) {
            const int a = e / S, b = e - a * S;
            for (int su = 0; su < Sw; ++su) {
                const int i = a - su;
                if (i >= 0 && i < J) {
                    const float wu = taps[i];
                    out.x = fmaf(wu, Ab[su * 19 + b].x, out.x);
                    out.y = fmaf(wu, Ab[su * 19 + b].y, out.y);
                }
            }
        }
        out.x *= wk;
        out.y *= wk;
        G[e] = out;
        const float m = fabsf(out.x) + fabsf(out.y);
        tmax = fmaxf(tmax, m);
        tsum += m;
    }
}

template <int L>
__global__ void __launch_bounds__(BUILD_WARPS * 32) gbuild_kernel(BuildArgs A) {
    constexpr int NC = L / 2, Q = NC + 1;
    extern __shared__ __align__(16) float smb[];
    float* s_wc = smb;                 // Q * BUILD_WS (first: 16-byte aligned rows)
    float* s_dn = s_wc + Q * BUILD_WS; // Q * Q
    float* s_tx = s_dn + Q * Q;        // Q
    float* s_ty = s_tx + Q;            // Q
    float* s_coef = s_ty + Q;          // 96
    constexpr int TABF = (Q * BUILD_WS + Q * Q + 2 * Q + 96 + 1) & ~1;
    constexpr int PER_WARP = Q * BUILD_TQ + BUILD_TQ * BUILD_TQ + 9 * 19 + 16;  // float2
    float2* s_w = reinterpret_cast<float2*>(smb + TABF);
    (void)NC;
    load_wk_tables<L>(A, smb);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2* R = s_w + warp * PER_WARP;      // [b'][t_x] Q x 5
    float2* Kq = R + Q * BUILD_TQ;          // [t_x][t_y] 5 x 5
    float2* Ab = Kq + BUILD_TQ * BUILD_TQ;  // [su][b]  9 x 19
    float* taps = reinterpret_cast<float*>(Ab + 9 * 19);  // wu[0..15], wv[16..31]
    const float invL2 = 1.f / ((float)L * (float)L);
    const float invhalf = 2.f / (float)A.J;
    float tmax = 0.f, t1max = 0.f;
    if (A.kwtab && A.J == 7) {
        // tabulated kernels and J = 7: a tile has at most 15 columns, so each half warp takes
        // one visibility (taps and kernel of half 1 in the otherwise unused row-pass scratch)
        const int hw = lane >> 4, hl = lane & 15;
        float2* Kh = hw ? R : Kq;
        float* th = hw ? reinterpret_cast<float*>(R + BUILD_TQ * BUILD_TQ) : taps;
        for (int64_t k0 = A.v0 + 2 * ((int64_t)blockIdx.x * BUILD_WARPS + warp); k0 < A.v0 + A.nvis;
             k0 += 2 * (int64_t)gridDim.x * BUILD_WARPS) {
            const int64_t k = k0 + hw;
            VisMeta mt{};
            if (k < A.v0 + A.nvis) mt = A.meta[k];
            // (visibilities of other shards have no taps)
            const bool act = k < A.v0 + A.nvis && (mt.pos >> 24) != SHARD_SKIP;
            int Sw = 1, h = 0;
            float w = 0.f;
            if (act) {
                Sw = (int)((mt.pos >> 16) & 255) - 6;
                h = Sw >> 1;
                w = A.wr[k];
                // KB taps: lanes 0 .. 6 along u, 8 .. 14 along v
                if (hl < 7) th[hl] = kb_eval(A.phiu[k] + 2.5f - (float)hl, invhalf, s_coef, A.kb_nterm);
                else if (hl >= 8 && hl < 15)
                    th[16 + hl - 8] = kb_eval(A.phiv[k] + 2.5f - (float)(hl - 8), invhalf, s_coef, A.kb_nterm);
                // the folded kernel by cubic Lagrange interpolation in w_r
                const int hq = h + 1;
                const float x = fminf(fmaxf(fmaf(w, A.tab_inv_dw, A.tab_x0), 1.f), (float)(A.tab_n + 1));
                const int j = min((int)x, A.tab_n);
                const float f = x - (float)j;
                const float l0 = -f * (f - 1.f) * (f - 2.f) * (1.f / 6.f);
                const float l1 = (f + 1.f) * (f - 1.f) * (f - 2.f) * 0.5f;
                const float l2 = -(f + 1.f) * f * (f - 2.f) * 0.5f;
                const float l3 = (f + 1.f) * f * (f - 1.f) * (1.f / 6.f);
                for (int e2 = hl; e2 < hq * hq; e2 += 16) {
                    const int tx = e2 / hq, ty = e2 - tx * hq, e = tx * BUILD_TQ + ty;
                    const float2* T = A.kwtab + (size_t)(j - 1) * (BUILD_TQ * BUILD_TQ) + e;
                    const float2 a0 = __ldg(T), a1 = __ldg(T + 25), a2 = __ldg(T + 50), a3 = __ldg(T + 75);
                    Kh[e] = make_float2(fmaf(l0, a0.x, fmaf(l1, a1.x, fmaf(l2, a2.x, l3 * a3.x))),
                                        fmaf(l0, a0.y, fmaf(l1, a1.y, fmaf(l2, a2.y, l3 * a3.y))));
                }
            }
            __syncwarp();
            float tsum = 0.f;
            if (act) {
                float2* G = A.gblk[mt.pos >> 24] + mt.off;
                const float wk = A.wt ? A.wt[k] : 1.f;
                switch (Sw) {
                    case 1: conv_tile<7, 1>(Kh, th, G, wk, hl, tmax, tsum); break;
                    case 3: conv_tile<7, 3>(Kh, th, G, wk, hl, tmax, tsum); break;
                    case 5: conv_tile<7, 5>(Kh, th, G, wk, hl, tmax, tsum); break;
                    case 7: conv_tile<7, 7>(Kh, th, G, wk, hl, tmax, tsum); break;
                    case 9: conv_tile<7, 9>(Kh, th, G, wk, hl, tmax, tsum); break;
                    default: break;  // supports are odd and at most 9
                }
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) tsum += __shfl_xor_sync(0xffffffffu, tsum, o);  // within the half
            t1max = fmaxf(t1max, tsum);
            __syncwarp();
        }
    } else
    for (int64_t k = A.v0 + (int64_t)blockIdx.x * BUILD_WARPS + warp; k < A.v0 + A.nvis;
         k += (int64_t)gridDim.x * BUILD_WARPS) {
        float tsum = 0.f;
        const VisMeta mt = A.meta[k];
        if ((mt.pos >> 24) == SHARD_SKIP) continue;  // another shard's visibility: no taps (warp-uniform)
        const int S = (mt.pos >> 16) & 255;
        const int Sw = S - A.J + 1, h = Sw >> 1, hq = h + 1;
        const float w = A.wr[k];
        // 2. KB taps
        if (lane < A.J) taps[lane] = kb_eval(A.phiu[k] + 0.5f * A.J - 1.f - lane, invhalf, s_coef, A.kb_nterm);
        else if (lane >= 16 && lane < 16 + A.J)
            taps[lane] = kb_eval(A.phiv[k] + 0.5f * A.J - 1.f - (lane - 16), invhalf, s_coef, A.kb_nterm);
        // 1. the folded w-kernel K(t; w), t in [0, h]^2: from the chirp, or interpolated in w
        if (!A.kwtab) {
            folded_wkernel<L>(s_dn, s_tx, s_ty, s_wc, w, A.literal, hq, R, Kq, lane, invL2);
        } else {
            if (lane < hq * hq) {
                // cubic Lagrange through the samples j - 1 .. j + 2 (nodes -1, 0, 1, 2)
                const int tx = lane / hq, ty = lane - tx * hq, e = tx * BUILD_TQ + ty;
                const float x = fminf(fmaxf(fmaf(w, A.tab_inv_dw, A.tab_x0), 1.f), (float)(A.tab_n + 1));
                const int j = min((int)x, A.tab_n);
                const float f = x - (float)j;
                const float l0 = -f * (f - 1.f) * (f - 2.f) * (1.f / 6.f);
                const float l1 = (f + 1.f) * (f - 1.f) * (f - 2.f) * 0.5f;
                const float l2 = -(f + 1.f) * f * (f - 2.f) * 0.5f;
                const float l3 = (f + 1.f) * f * (f - 1.f) * (1.f / 6.f);
                const float2* T = A.kwtab + (size_t)(j - 1) * (BUILD_TQ * BUILD_TQ) + e;
                const float2 a0 = __ldg(T), a1 = __ldg(T + 25), a2 = __ldg(T + 50), a3 = __ldg(T + 75);
                Kq[e] = make_float2(fmaf(l0, a0.x, fmaf(l1, a1.x, fmaf(l2, a2.x, l3 * a3.x))),
                                    fmaf(l0, a0.y, fmaf(l1, a1.y, fmaf(l2, a2.y, l3 * a3.y))));
            }
            __syncwarp();
        }
        // 3. the S x S tile (times the data weight) into G, and its tap bounds
        float2* G = A.gblk[mt.pos >> 24] + mt.off;
        const float wk = A.wt ? A.wt[k] : 1.f;
        bool done = false;
        if (A.J == 7) {  // the common support: sizes known at compile time
            switch (Sw) {
                case 1: conv_tile<7, 1>(Kq, taps, G, wk, lane, tmax, tsum); done = true; break;
                case 3: conv_tile<7, 3>(Kq, taps, G, wk, lane, tmax, tsum); done = true; break;
                case 5: conv_tile<7, 5>(Kq, taps, G, wk, lane, tmax, tsum); done = true; break;
                case 7: conv_tile<7, 7>(Kq, taps, G, wk, lane, tmax, tsum); done = true; break;
                case 9: conv_tile<7, 9>(Kq, taps, G, wk, lane, tmax, tsum); done = true; break;
                default: break;
            }
        }
        if (!done) conv_tile_any(Kq, taps, Ab, G, wk, lane, A.J, Sw, tmax, tsum);
        // bounds for the fixed-point grid step: max |t.x| + |t.y| over all taps, max over
        // visibilities of the tap sum (non-negative floats order like their bit patterns)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tsum += __shfl_xor_sync(0xffffffffu, tsum, o);
        t1max = fmaxf(t1max, tsum);  // one atomic per warp at the end, not per visibility
        __syncwarp();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
        t1max = fmaxf(t1max, __shfl_xor_sync(0xffffffffu, t1max, o));  // the two halves' visibilities
    }
    if (lane == 0) {
        atomicMax(A.fx + FX_TMAX, __float_as_uint(tmax));
        atomicMax(A.fx + FX_T1, __float_as_uint(t1max));
    }
}

size_t gbuild_smem(int L, int /*hmax*/) {
    const int Q = L / 2 + 1;
    const int tabf = (Q * BUILD_WS + Q * Q + 2 * Q + 96 + 1) & ~1;
    const int per_warp = Q * BUILD_TQ + BUILD_TQ * BUILD_TQ + 9 * 19 + 16;
    return (size_t)tabf * sizeof(float) + (size_t)BUILD_WARPS * per_warp * sizeof(float2);
}

void launch_gbuild(const rimo_plan* p, cudaStream_t s) { launch_gbuild_range(p, 0, p->M, s); }

static BuildArgs build_args(const rimo_plan* p) {
    BuildArgs A;
    std::memset(&A, 0, sizeof(A));
    A.meta = p->d_meta;
    A.wr = p->d_wr;
    A.phiu = p->d_phiu;
    A.phiv = p->d_phiv;
    A.gblk = p->d_gblock_ptrs;
    A.wk_dn = p->tab.wk_dn;
    A.tau_x = p->tab.wk_tau_x;
    A.tau_y = p->tab.wk_tau_y;
    A.wc = p->tab.wk_wc;
    A.kb_coef = p->tab.kb_coef;
    A.kb_nterm = p->tab.kb_nterm;
    A.L = p->L;
    A.hmax = p->hmax;
    A.J = p->J;
    A.literal = p->prm.taper_literal != 0;
    A.fx = p->d_fx;
    A.wt = p->d_wt;
    A.kwtab = p->d_kwtab;
    A.tab_n = p->kw_n;
    A.tab_w0 = p->kw_w0;
    A.tab_dw = p->kw_dw;
    A.tab_inv_dw = p->kw_dw > 0.0 ? (float)(1.0 / p->kw_dw) : 0.f;
    A.tab_x0 = p->kw_dw > 0.0 ? (float)(-p->kw_w0 / p->kw_dw) : 1.f;  // x = (w - w0) / dw
    return A;
}

// The table of folded kernels over the plan's residual w (into p->d_kwtab, allocated)
void launch_kwtab(const rimo_plan* p, cudaStream_t s) {
    BuildArgs A = build_args(p);
    A.kwtab = nullptr;
    A.kwtab_out = p->d_kwtab;
    const size_t sm = gbuild_smem(p->L, p->hmax);
    void (*kern)(BuildArgs) = p->L == 16 ? kwtab_kernel<16> : p->L == 32 ? kwtab_kernel<32>
                            : p->L == 64 ? kwtab_kernel<64> : kwtab_kernel<128>;
    RIMO_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int blocks = (p->kw_n + 3 + BUILD_WARPS - 1) / BUILD_WARPS;
    kern<<<blocks, BUILD_WARPS * 32, sm, s>>>(A);
    RIMO_CUDA(cudaGetLastError());
}

void launch_gbuild_range(const rimo_plan* p, int64_t v0, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    BuildArgs A = build_args(p);
    A.v0 = v0;
    A.nvis = n;
    const size_t sm = gbuild_smem(p->L, p->hmax);
    void (*kern)(BuildArgs) = p->L == 16 ? gbuild_kernel<16> : p->L == 32 ? gbuild_kernel<32>
                            : p->L == 64 ? gbuild_kernel<64> : gbuild_kernel<128>;
    RIMO_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int dev = 0, nsm = 0;
    RIMO_CUDA(cudaGetDevice(&dev));
    RIMO_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int64_t blocks = (n + BUILD_WARPS - 1) / BUILD_WARPS;
    blocks = std::min<int64_t>(blocks, (int64_t)nsm * 16);
    kern<<<(int)blocks, BUILD_WARPS * 32, sm, s>>>(A);
}

}  // namespace rimo
