// The sparse de-gridding matrix G_p (Section 3.2, Eq. 6): build, de-grid (G_p), grid
// (G_p^dagger, Eq. 8) and the fused G_p^dagger G_p of Phi^dagger Phi.
//
// Layout.  Visibilities of a w-bin are sorted by the uv-tile (TS x TS grid cells)
// holding their first grid cell.  One thread block owns one uv-tile: it stages the
// (TS + H)^2 patch of the grid that the tile's visibilities can touch (H = largest
// tile side - 1) in shared memory, one warp per visibility reads the visibility's
// S x S taps once (coalesced), gathers the patch (de-gridding, warp-shuffle reduction)
// and scatters conj(taps) * y into a privatised shared-memory accumulator.  The
// accumulator is added to the global grid once per cell.  Patches of neighbouring
// tiles overlap by H cells, so the gridding launches run the four tile colourings
// (even/odd tile index along u and v) one after another; within a colouring no two
// patches overlap and no global atomics are needed.
#include "internal.h"

namespace rimo {

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int MAX_TAPS_PER_LANE = 12;  // ceil(19 * 19 / 32)

// e / S for e < 361, S <= 19 by multiply-shift with ceil(2^16 / S)
__device__ __forceinline__ int div_small(int e, int magic) { return (e * magic) >> 16; }

template <int MODE>  // 0: de-grid (y_out), 1: grid (y_in), 2: fused G^dagger G
__global__ void __launch_bounds__(256) gtg_kernel(const TileDesc* __restrict__ tiles,
                                                  const VisMeta* __restrict__ meta,
                                                  const float2* const* __restrict__ gblk,
                                                  const float2* __restrict__ X, float2* __restrict__ Xh,
                                                  const float2* __restrict__ y_in, float2* __restrict__ y_out,
                                                  int gx, int gy, int TS, int PW) {
    extern __shared__ float2 sm[];
    constexpr bool GATHER = MODE != 1, SCATTER = MODE != 0;
    float2* Xs = sm;
    float2* As = sm + (GATHER ? PW * PW : 0);
    const TileDesc td = tiles[blockIdx.x];
    const int u0 = td.tu * TS, v0 = td.tv * TS;
    const int npatch = PW * PW;
    for (int e = threadIdx.x; e < npatch; e += blockDim.x) {
        const int a = e / PW, b = e - a * PW;
        int gu = u0 + a, gv = v0 + b;
        if (gu >= gx) gu -= gx;
        if (gv >= gy) gv -= gy;
        if (GATHER) Xs[e] = X[(size_t)gu * gy + gv];
        if (SCATTER) As[e] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t k = td.vb + warp; k < td.ve; k += nw) {
        const VisMeta mt = meta[k];
        const int du = mt.pos & 255, dv = (mt.pos >> 8) & 255, S = (mt.pos >> 16) & 255;
        const float2* T = gblk[mt.pos >> 24] + mt.off;
        const int n = S * S;
        const int magic = (65536 + S - 1) / S;
        const int base = du * PW + dv;
        float2 tv[MAX_TAPS_PER_LANE];
        int sidx[MAX_TAPS_PER_LANE];
        float ar = 0.f, ai = 0.f;
#pragma unroll
        for (int it = 0; it < MAX_TAPS_PER_LANE; ++it) {
            const int e = lane + 32 * it;
            if (e < n) {
                const int a = div_small(e, magic), b = e - a * S;
                tv[it] = __ldg(&T[e]);
                sidx[it] = base + a * PW + b;
                if (GATHER) {
                    const float2 x = Xs[sidx[it]];
                    ar = fmaf(tv[it].x, x.x, fmaf(-tv[it].y, x.y, ar));
                    ai = fmaf(tv[it].x, x.y, fmaf(tv[it].y, x.x, ai));
                }
            }
        }
        float2 y;
        if (GATHER) {
            y.x = warp_sum(ar);
            y.y = warp_sum(ai);
            if (MODE == 0 && lane == 0) y_out[mt.orig] = y;
        } else {
            y = __ldg(&y_in[mt.orig]);
        }
        if (SCATTER) {
#pragma unroll
            for (int it = 0; it < MAX_TAPS_PER_LANE; ++it) {
                const int e = lane + 32 * it;
                if (e < n) {
                    // conj(t) * y
                    atomicAdd(&As[sidx[it]].x, fmaf(tv[it].x, y.x, tv[it].y * y.y));
                    atomicAdd(&As[sidx[it]].y, fmaf(tv[it].x, y.y, -tv[it].y * y.x));
                }
            }
        }
    }
    if (SCATTER) {
        __syncthreads();
        for (int e = threadIdx.x; e < npatch; e += blockDim.x) {
            const float2 acc = As[e];
            if (acc.x == 0.f && acc.y == 0.f) continue;
            const int a = e / PW, b = e - a * PW;
            int gu = u0 + a, gv = v0 + b;
            if (gu >= gx) gu -= gx;
            if (gv >= gy) gv -= gy;
            float2* dst = &Xh[(size_t)gu * gy + gv];
            const float2 o = *dst;
            *dst = make_float2(o.x + acc.x, o.y + acc.y);
        }
    }
}

template <int MODE>
static void gtg_launch(const rimo_plan* p, int t0, int t1, const float2* X, float2* Xh,
                       const float2* y_in, float2* y_out, cudaStream_t s) {
    if (t1 <= t0) return;
    const size_t sm = (size_t)p->PW * p->PW * sizeof(float2) * (MODE == 2 ? 2 : 1);
    static bool done = false;
    if (!done) {
        RIMO_CUDA(cudaFuncSetAttribute(gtg_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       2 * 96 * 96 * (int)sizeof(float2)));
        done = true;
    }
    gtg_kernel<MODE><<<t1 - t0, 256, sm, s>>>(p->d_tiles + t0, p->d_meta, p->d_gblock_ptrs, X, Xh, y_in,
                                              y_out, p->gx, p->gy, p->TS, p->PW);
}

void launch_gtg(const rimo_plan* p, int bin, int mode, const float2* X, float2* Xh,
                const float2* y_in, float2* y_out, cudaStream_t s) {
    const auto& br = p->bins[bin];
    if (mode == 0) {  // read-only on the grid: all colourings in one launch
        gtg_launch<0>(p, br.tile_off[0], br.tile_off[4], X, Xh, y_in, y_out, s);
        return;
    }
    for (int ph = 0; ph < 4; ++ph) {
        if (mode == 1) gtg_launch<1>(p, br.tile_off[ph], br.tile_off[ph + 1], X, Xh, y_in, y_out, s);
        else gtg_launch<2>(p, br.tile_off[ph], br.tile_off[ph + 1], X, Xh, y_in, y_out, s);
    }
}

// ---------------------------------------------------------------------------
// Build of G (stage 3 of Fig. 3): one warp per visibility.
//   1. residual w-kernel (Section 3.1, Fig. 1): tapered chirp c[a][b] on the L x L grid
//      over twice the field of view, K(t) = (1/L^2) sum c e^{+2 pi i (t_x a_c + t_y b_c)/L}
//      for the S_w x S_w central taps (row pass over a, then column pass over b);
//   2. Kaiser-Bessel taps w_u[i] = KB(phi_u + J/2 - 1 - i), KB by Horner in
//      rho = 1 - (2t/J)^2 of its normalised power series;
//   3. T = w_u (*) K (*) w_v  (separable two-step convolution), S = S_w + J - 1.
struct BuildArgs {
    const VisMeta* meta;
    const float* wr;
    const float* phiu;
    const float* phiv;
    float2* const* gblk;
    const float* wk_dn;
    const float* tau_x;
    const float* tau_y;
    const float2* E;
    const float* kb_coef;
    int kb_nterm;
    int L, hmax, J, literal;
    int64_t nvis;
};

__device__ __forceinline__ float kb_eval(float t, float invhalf, const float* coef, int nterm) {
    const float q = t * invhalf;
    const float rho = 1.f - q * q;
    if (rho < 0.f) return 0.f;
    float acc = coef[nterm - 1];
    for (int k = nterm - 2; k >= 0; --k) acc = fmaf(acc, rho, coef[k]);
    return acc;
}

constexpr int BUILD_WARPS = 8;

__global__ void __launch_bounds__(BUILD_WARPS * 32) gbuild_kernel(BuildArgs A) {
    extern __shared__ float smb[];
    const int L = A.L, ns = 2 * A.hmax + 1;
    float* s_dn = smb;                                // L * L
    float* s_tx = s_dn + L * L;                       // L
    float* s_ty = s_tx + L;                           // L
    float* s_coef = s_ty + L;                         // 96
    float2* s_E = reinterpret_cast<float2*>(s_coef + 96);  // L * ns
    float2* s_w = s_E + L * ns;                       // per warp scratch
    const int per_warp = L * 9 + 81 + 9 * 19 + 16;    // R, K, A, taps (float2 units)
    for (int e = threadIdx.x; e < L * L; e += blockDim.x) s_dn[e] = A.wk_dn[e];
    for (int e = threadIdx.x; e < L; e += blockDim.x) {
        s_tx[e] = A.tau_x[e];
        s_ty[e] = A.tau_y[e];
    }
    for (int e = threadIdx.x; e < A.kb_nterm; e += blockDim.x) s_coef[e] = A.kb_coef[e];
    for (int e = threadIdx.x; e < L * ns; e += blockDim.x) s_E[e] = A.E[e];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2* R = s_w + warp * per_warp;   // [b][s]  L x 9
    float2* Kw = R + L * 9;              // [su][sv] 9 x 9
    float2* Ab = Kw + 81;                // [su][b]  9 x 19
    float* taps = reinterpret_cast<float*>(Ab + 9 * 19);  // wu[0..15], wv[16..31]
    const float invL2 = 1.f / ((float)L * (float)L);
    const float invhalf = 2.f / (float)A.J;
    for (int64_t k = (int64_t)blockIdx.x * BUILD_WARPS + warp; k < A.nvis; k += (int64_t)gridDim.x * BUILD_WARPS) {
        const VisMeta mt = A.meta[k];
        const int S = (mt.pos >> 16) & 255;
        const int Sw = S - A.J + 1, h = Sw >> 1, t0 = A.hmax - h;
        const float w = A.wr[k];
        // 1a. row pass: R[b][s] = sum_a c[a][b] E[a][s + t0]
        for (int b = lane; b < L; b += 32) {
            float2 acc[9];
#pragma unroll
            for (int s = 0; s < 9; ++s) acc[s] = make_float2(0.f, 0.f);
            const float tb = s_ty[b];
            for (int a = 0; a < L; ++a) {
                float sn, cs;
                sincospif(2.f * w * s_dn[a * L + b], &sn, &cs);
                const float tt = s_tx[a] * tb;
                float2 c;
                if (A.literal) c = make_float2(tt * cs, -tt * sn);
                else c = make_float2(1.f + tt * (cs - 1.f), -tt * sn);
                const float2* Ea = s_E + a * ns + t0;
#pragma unroll
                for (int s = 0; s < 9; ++s) {
                    if (s < Sw) {
                        const float2 e = Ea[s];
                        acc[s].x = fmaf(c.x, e.x, fmaf(-c.y, e.y, acc[s].x));
                        acc[s].y = fmaf(c.x, e.y, fmaf(c.y, e.x, acc[s].y));
                    }
                }
            }
#pragma unroll
            for (int s = 0; s < 9; ++s)
                if (s < Sw) R[b * 9 + s] = acc[s];
        }
        // 2. KB taps
        if (lane < A.J) taps[lane] = kb_eval(A.phiu[k] + 0.5f * A.J - 1.f - lane, invhalf, s_coef, A.kb_nterm);
        else if (lane >= 16 && lane < 16 + A.J)
            taps[lane] = kb_eval(A.phiv[k] + 0.5f * A.J - 1.f - (lane - 16), invhalf, s_coef, A.kb_nterm);
        __syncwarp();
        // 1b. column pass: K[su][sv] = (1/L^2) sum_b R[b][su] E[b][sv + t0]
        for (int e = lane; e < Sw * Sw; e += 32) {
            const int su = e / Sw, sv = e - su * Sw;
            float ar = 0.f, ai = 0.f;
            for (int b = 0; b < L; ++b) {
                const float2 r = R[b * 9 + su], q = s_E[b * ns + sv + t0];
                ar = fmaf(r.x, q.x, fmaf(-r.y, q.y, ar));
                ai = fmaf(r.x, q.y, fmaf(r.y, q.x, ai));
            }
            Kw[su * 9 + sv] = make_float2(ar * invL2, ai * invL2);
        }
        __syncwarp();
        // 3a. A[su][b] = sum_sv K[su][sv] w_v[b - sv]
        for (int e = lane; e < Sw * S; e += 32) {
            const int su = e / S, b = e - su * S;
            float ar = 0.f, ai = 0.f;
            for (int sv = 0; sv < Sw; ++sv) {
                const int i = b - sv;
                if (i >= 0 && i < A.J) {
                    const float wv = taps[16 + i];
                    ar = fmaf(Kw[su * 9 + sv].x, wv, ar);
                    ai = fmaf(Kw[su * 9 + sv].y, wv, ai);
                }
            }
            Ab[su * 19 + b] = make_float2(ar, ai);
        }
        __syncwarp();
        // 3b. T[a][b] = sum_su w_u[a - su] A[su][b]
        float2* G = A.gblk[mt.pos >> 24] + mt.off;
        const int n = S * S;
        for (int e = lane; e < n + (n & 1); e += 32) {
            float2 out = make_float2(0.f, 0.f);
            if (e < n) {
                const int a = e / S, b = e - a * S;
                for (int su = 0; su < Sw; ++su) {
                    const int i = a - su;
                    if (i >= 0 && i < A.J) {
                        const float wu = taps[i];
                        out.x = fmaf(wu, Ab[su * 19 + b].x, out.x);
                        out.y = fmaf(wu, Ab[su * 19 + b].y, out.y);
                    }
                }
            }
            G[e] = out;
        }
        __syncwarp();
    }
}

size_t gbuild_smem(int L, int hmax) {
    const int ns = 2 * hmax + 1;
    const int per_warp = L * 9 + 81 + 9 * 19 + 16;
    return (size_t)(L * L + 2 * L + 96) * sizeof(float) + (size_t)L * ns * sizeof(float2) +
           (size_t)BUILD_WARPS * per_warp * sizeof(float2);
}

void launch_gbuild(const rimo_plan* p, cudaStream_t s) {
    if (p->M == 0) return;
    BuildArgs A;
    A.meta = p->d_meta;
    A.wr = p->d_wr;
    A.phiu = p->d_phiu;
    A.phiv = p->d_phiv;
    A.gblk = p->d_gblock_ptrs;
    A.wk_dn = p->tab.wk_dn;
    A.tau_x = p->tab.wk_tau_x;
    A.tau_y = p->tab.wk_tau_y;
    A.E = p->tab.wk_E;
    A.kb_coef = p->tab.kb_coef;
    A.kb_nterm = p->tab.kb_nterm;
    A.L = p->L;
    A.hmax = p->hmax;
    A.J = p->J;
    A.literal = p->prm.taper_literal != 0;
    A.nvis = p->M;
    const size_t sm = gbuild_smem(p->L, p->hmax);
    RIMO_CUDA(cudaFuncSetAttribute(gbuild_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int dev = 0, nsm = 0;
    RIMO_CUDA(cudaGetDevice(&dev));
    RIMO_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int64_t blocks = (p->M + BUILD_WARPS - 1) / BUILD_WARPS;
    blocks = std::min<int64_t>(blocks, (int64_t)nsm * 8);
    gbuild_kernel<<<(int)blocks, BUILD_WARPS * 32, sm, s>>>(A);
}

}  // namespace rimo
