// Kernel-surrogate MLP: (phi_u, phi_v, w_r) -> 128 -> GELU -> 128 -> GELU -> 450 reals
// (the 15 x 15 complex de-gridding tile of a visibility), trained on tiles of the exact
// method.  bf16 weights and activations feed tcgen05 tensor-core GEMMs with FP32
// accumulation in tensor memory; the elementwise steps (bias, GELU, loss, derivatives)
// run on the CUDA cores in FP32; Adam keeps FP32 master weights.
//
// Training step on a batch of B samples (B a multiple of 128):
//   Z1 = X W1^T + b1, H1 = bf16(gelu(Z1))              (CUDA cores, K = 3)
//   Z2 = H1 W2^T + b2, H2 = bf16(gelu(Z2))              (tcgen05)
//   Y  = H2 W3^T + b3, dY = 2 (Y - T) / (450 B)          (tcgen05, loss on CUDA cores)
//   dW3 = bf16(dY)^T H2, dH2 = bf16(dY) W3               (tcgen05, split-K over the batch)
//   dZ2 = dH2 gelu'(Z2); dW2 = bf16(dZ2)^T H1, dH1 = bf16(dZ2) W2
//   dZ1 = dH1 gelu'(Z1); dW1 = dZ1^T X                   (CUDA cores)
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>

#include "internal.h"
#include "mlp.h"
#include "tc.cuh"

namespace rimo {

typedef __nv_bfloat16 bf16;

// erf by the rational approximation of Abramowitz & Stegun (1964), eq. 7.1.26:
// erf(x) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) e^{-x^2}, t = 1 / (1 + p x), x >= 0,
// |error| <= 1.5e-7 (odd extension to x < 0); one reciprocal and one exponential.
__device__ __forceinline__ float erf_as(float x) {
    const float ax = fabsf(x);
    const float t = __fdividef(1.f, fmaf(0.3275911f, ax, 1.f));
    const float poly =
        t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f), 0.254829592f);
    return copysignf(fmaf(-poly, __expf(-ax * ax), 1.f), x);
}
// GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2 (the network's activation everywhere it
// runs forward: training, batched forward, tile generation)
__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erf_as(z * 0.70710678118654752f)); }
// derivative of that same function (training follows the gradient of the GELU the network
// evaluates): with x = z / sqrt 2, E = erf_as and t, poly as in erf_as,
// dE/dx = e^{-x^2} (2 |x| poly(t) + p t^2 poly'(t)) (even in x), so
// GELU'(z) = (1 + E(x)) / 2 + z dE/dx / (2 sqrt 2).
__device__ __forceinline__ float gelu_grad_f(float z) {
    const float x = z * 0.70710678118654752f;
    const float ax = fabsf(x);
    const float t = __fdividef(1.f, fmaf(0.3275911f, ax, 1.f));
    const float poly =
        t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f), 0.254829592f);
    // d poly / dt = a1 + 2 a2 t + 3 a3 t^2 + 4 a4 t^3 + 5 a5 t^4
    const float dpoly =
        fmaf(t, fmaf(t, fmaf(t, fmaf(t, 5.f * 1.061405429f, 4.f * -1.453152027f), 3.f * 1.421413741f),
                     2.f * -0.284496736f),
             0.254829592f);
    const float e = __expf(-ax * ax);
    const float E = copysignf(fmaf(-poly, e, 1.f), x);
    const float dE = e * fmaf(2.f * ax, poly, 0.3275911f * t * t * dpoly);
    return fmaf(0.5f, 1.f + E, z * dE * 0.35355339059327376f);
}

__device__ __forceinline__ void mbar_init_(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc::smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(tc::smem_addr(bar)), "r"(parity), "r"(100000u)
        : "memory");
    return ok != 0;
}
// bounded: at most 2^15 polls of <= 100 us each
__device__ __forceinline__ bool mbar_wait_(uint64_t* bar, uint32_t parity) {
    for (uint32_t it = 0; it < (1u << 15); ++it)
        if (mbar_try_wait_(bar, parity)) return true;
    return false;
}

// --------------------------------------------------------------------------------------
// C[m][n] (+)= sum_k A[m][k] B[n][k]: A (M x K) and B (N x K) bf16 row-major with K
// contiguous, C fp32.  Block: 128 threads, tile 128 (m) x up to 256 (n), K staged in
// chunks of 64 into shared memory in the canonical K-major layout; one thread issues
// the tcgen05.mma (K = 16 each), the accumulator lives in tensor memory.
constexpr int GEMM_NT = 256;
constexpr int GEMM_KC = 64;
constexpr size_t GEMM_SMEM = 100 * 1024;  // also caps residency at two blocks per SM

struct GemmArgs {
    const bf16* A;
    const bf16* B;
    float* C;
    int lda, ldb, ldc;
    int M, N, K;
    int kspan;   // K range of one split (grid.z)
    int atomic;  // add into C (split-K) instead of storing
    int* status;
};

__global__ void __launch_bounds__(128) gemm_tc_kernel(GemmArgs g) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* sA = sm;                          // 128 x 64 bf16 = 16 KB
    unsigned char* sB = sm + 16384;                  // 256 x 64 bf16 = 32 KB
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n0 = blockIdx.x * GEMM_NT, m0 = blockIdx.y * 128;
    const int nt = min(GEMM_NT, g.N - n0);
    const int k_begin = blockIdx.z * g.kspan, k_end = min(g.K, k_begin + g.kspan);
    if (warp == 0) tc::tmem_alloc(&tslot, GEMM_NT);
    if (tid == 0) {
        mbar_init_(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t idesc = tc::idesc_bf16_f32(128, nt);
    uint32_t phase = 0;
    bool ok = true;
    for (int k0 = k_begin; k0 < k_end; k0 += GEMM_KC) {
        const int kc = min(GEMM_KC, k_end - k0);   // multiple of 16
        const int nv = kc / 8;                      // 16-byte vectors per row
        for (int e = tid; e < 128 * nv; e += 128) {
            const int r = e / nv, v = e - r * nv;
            const uint4 val = *reinterpret_cast<const uint4*>(g.A + (size_t)(m0 + r) * g.lda + k0 + v * 8);
            *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(r, v * 8, 128)) = val;
        }
        for (int e = tid; e < nt * nv; e += 128) {
            const int r = e / nv, v = e - r * nv;
            const uint4 val = *reinterpret_cast<const uint4*>(g.B + (size_t)(n0 + r) * g.ldb + k0 + v * 8);
            *reinterpret_cast<uint4*>(sB + tc::kmajor_offset(r, v * 8, nt)) = val;
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            for (int s = 0; s < kc / 16; ++s) {
                const uint64_t ad = tc::smem_desc(tc::smem_addr(sA) + s * 128 * 32, 128, 256);
                const uint64_t bd = tc::smem_desc(tc::smem_addr(sB) + s * nt * 32, 128, 256);
                tc::mma_bf16(tmem, ad, bd, idesc, (k0 > k_begin || s > 0) ? 1u : 0u);
            }
            tc::mma_commit(&bar);
        }
        ok = mbar_wait_(&bar, phase);
        phase ^= 1;
        if (__syncthreads_or(!ok)) break;
    }
    if (!ok) {
        if (tid == 0) atomicExch(g.status, 2);
    } else if (k_end > k_begin) {
        tc::fence_after_sync();
        const int row = m0 + 32 * warp + lane;
        for (int c = 0; c < nt; c += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + c, v);
            float* dst = g.C + (size_t)row * g.ldc + n0 + c;
            if (g.atomic) {
#pragma unroll
                for (int i = 0; i < 16; ++i) atomicAdd(dst + i, v[i]);
            } else {
#pragma unroll
                for (int i = 0; i < 16; i += 4)
                    *reinterpret_cast<float4*>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) {
        tc::tmem_dealloc(tmem, GEMM_NT);
        tc::tmem_relinquish();
    }
}

static void gemm(const bf16* A, int lda, const bf16* B, int ldb, float* C, int ldc, int M, int N, int K,
                 int splits, bool atomic, int* status, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        RIMO_CUDA(cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GEMM_SMEM));
        attr = true;
    }
    GemmArgs g;
    g.A = A;
    g.B = B;
    g.C = C;
    g.lda = lda;
    g.ldb = ldb;
    g.ldc = ldc;
    g.M = M;
    g.N = N;
    g.K = K;
    g.kspan = ((K / splits + 15) / 16) * 16;
    g.atomic = atomic ? 1 : 0;
    g.status = status;
    dim3 grid((N + GEMM_NT - 1) / GEMM_NT, M / 128, (K + g.kspan - 1) / g.kspan);
    gemm_tc_kernel<<<grid, 128, GEMM_SMEM, s>>>(g);
}

// --------------------------------------------------------------------------------------
// elementwise steps
__global__ void l1_fwd_kernel(const float* __restrict__ X, const float* __restrict__ W1, const float* __restrict__ b1,
                              float* __restrict__ Z1, bf16* __restrict__ H1, int B) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)B * MLP_H) return;
    const int b = (int)(e / MLP_H), j = (int)(e % MLP_H);
    const float w0 = __bfloat162float(__float2bfloat16(W1[j * 3 + 0]));
    const float w1 = __bfloat162float(__float2bfloat16(W1[j * 3 + 1]));
    const float w2 = __bfloat162float(__float2bfloat16(W1[j * 3 + 2]));
    const float z = fmaf(X[b * 3 + 0], w0, fmaf(X[b * 3 + 1], w1, fmaf(X[b * 3 + 2], w2, b1[j])));
    Z1[e] = z;
    H1[e] = __float2bfloat16(gelu_f(z));
}

// Z (in place) += bias; H = bf16(gelu(Z))
__global__ void act_fwd_kernel(float* __restrict__ Z, const float* __restrict__ bias, bf16* __restrict__ H, int B,
                               int n, int ld) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)B * n) return;
    const int b = (int)(e / n), j = (int)(e % n);
    const float z = Z[(size_t)b * ld + j] + bias[j];
    Z[(size_t)b * ld + j] = z;
    H[(size_t)b * n + j] = __float2bfloat16(gelu_f(z));
}

// Y += b3; r = Y - T; loss += r^2; dY = 2 r / (450 B) as bf16 (cols >= 450 zero); db3 += dY
__global__ void loss_bwd_kernel(float* __restrict__ Y, int ldy, const float* __restrict__ b3,
                                const float* __restrict__ T, bf16* __restrict__ dY, int ld_dy, float* __restrict__ db3,
                                float* __restrict__ loss, int B) {
    __shared__ float red[256];
    const int j = blockIdx.x % MLP_OUT_PAD;  // one output column per block x slice of the batch
    const int part = blockIdx.x / MLP_OUT_PAD, nparts = gridDim.x / MLP_OUT_PAD;
    float sq = 0.f, db = 0.f;
    const float scale = 2.f / ((float)MLP_OUT * (float)B);
    for (int b = part * blockDim.x + threadIdx.x; b < B; b += nparts * blockDim.x) {
        float d = 0.f;
        if (j < MLP_OUT) {
            const float y = Y[(size_t)b * ldy + j] + b3[j];
            Y[(size_t)b * ldy + j] = y;
            const float r = y - T[(size_t)b * MLP_OUT + j];
            sq += r * r;
            d = scale * r;
            db += d;
        }
        dY[(size_t)b * ld_dy + j] = __float2bfloat16(d);
    }
    red[threadIdx.x] = sq;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && j < MLP_OUT) atomicAdd(loss, red[0]);
    __syncthreads();
    red[threadIdx.x] = db;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && j < MLP_OUT) atomicAdd(&db3[j], red[0]);
}

// dZ = dH * gelu'(Z) -> bf16; db += dZ (fp32)
__global__ void act_bwd_kernel(const float* __restrict__ dH, const float* __restrict__ Z, bf16* __restrict__ dZ,
                               float* __restrict__ db, int B) {
    __shared__ float red[256];
    const int j = blockIdx.x % MLP_H, part = blockIdx.x / MLP_H, nparts = gridDim.x / MLP_H;
    float acc = 0.f;
    for (int b = part * blockDim.x + threadIdx.x; b < B; b += nparts * blockDim.x) {
        const float d = dH[(size_t)b * MLP_H + j] * gelu_grad_f(Z[(size_t)b * MLP_H + j]);
        dZ[(size_t)b * MLP_H + j] = __float2bfloat16(d);
        acc += d;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&db[j], red[0]);
}

// dZ1 = dH1 * gelu'(Z1); dW1[j][i] += dZ1[b][j] X[b][i]; db1[j] += dZ1[b][j]
__global__ void l1_bwd_kernel(const float* __restrict__ dH1, const float* __restrict__ Z1, const float* __restrict__ X,
                              float* __restrict__ dW1, float* __restrict__ db1, int B) {
    __shared__ float red[4][256];
    const int j = blockIdx.x % MLP_H, part = blockIdx.x / MLP_H, nparts = gridDim.x / MLP_H;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int b = part * blockDim.x + threadIdx.x; b < B; b += nparts * blockDim.x) {
        const float d = dH1[(size_t)b * MLP_H + j] * gelu_grad_f(Z1[(size_t)b * MLP_H + j]);
        a0 += d * X[b * 3 + 0];
        a1 += d * X[b * 3 + 1];
        a2 += d * X[b * 3 + 2];
        a3 += d;
    }
    red[0][threadIdx.x] = a0;
    red[1][threadIdx.x] = a1;
    red[2][threadIdx.x] = a2;
    red[3][threadIdx.x] = a3;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(&dW1[j * 3 + 0], red[0][0]);
        atomicAdd(&dW1[j * 3 + 1], red[1][0]);
        atomicAdd(&dW1[j * 3 + 2], red[2][0]);
        atomicAdd(&db1[j], red[3][0]);
    }
}

// dst[c][r] = src[r][c], bf16, 32 x 32 tiles through shared memory
__global__ void transpose_bf16_kernel(const bf16* __restrict__ src, bf16* __restrict__ dst, int R, int Cn) {
    __shared__ bf16 t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        t[i][threadIdx.x] = (r < R && c < Cn) ? src[(size_t)r * Cn + c] : __float2bfloat16(0.f);
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (c < Cn && r < R) dst[(size_t)c * R + r] = t[threadIdx.x][i];
    }
}

static void transpose(const bf16* src, bf16* dst, int R, int Cn, cudaStream_t s) {
    dim3 grid((Cn + 31) / 32, (R + 31) / 32), block(32, 8);
    transpose_bf16_kernel<<<grid, block, 0, s>>>(src, dst, R, Cn);
}

// Adam on the FP32 masters, then the bf16 operand copies: W2 [128][128], W2^T, W3 [464][128]
// (rows >= 450 zero) and W3^T [128][512] (columns >= 450 zero).
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void pack_weights_kernel(const float* __restrict__ P, bf16* __restrict__ W2b, bf16* __restrict__ W2Tb,
                                    bf16* __restrict__ W3b, bf16* __restrict__ W3Tb) {
    const float* W2 = P + MLP_OFF_W2;
    const float* W3 = P + MLP_OFF_W3;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < MLP_H * MLP_H) {
        const int r = i / MLP_H, c = i % MLP_H;
        const bf16 w = __float2bfloat16(W2[i]);
        W2b[i] = w;
        W2Tb[c * MLP_H + r] = w;
    }
    if (i < MLP_OUT_PAD * MLP_H) {
        const int r = i / MLP_H, c = i % MLP_H;
        const bf16 w = __float2bfloat16(r < MLP_OUT ? W3[r * MLP_H + c] : 0.f);
        W3b[i] = w;
        W3Tb[c * MLP_K3 + r] = w;
    }
    if (i < MLP_H * (MLP_K3 - MLP_OUT_PAD)) {
        const int c = i / (MLP_K3 - MLP_OUT_PAD), r = MLP_OUT_PAD + i % (MLP_K3 - MLP_OUT_PAD);
        W3Tb[c * MLP_K3 + r] = __float2bfloat16(0.f);
    }
}

// --------------------------------------------------------------------------------------
Mlp::~Mlp() {
    for (void* p : owned) cudaFree(p);
}

void* Mlp::alloc(size_t bytes) {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        fail(RIMO_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes for the surrogate failed");
    }
    owned.push_back(p);
    return p;
}

void Mlp::init(uint64_t seed) {
    P = (float*)alloc(MLP_NPARAM * sizeof(float));
    G = (float*)alloc(MLP_NPARAM * sizeof(float));
    Mom = (float*)alloc(MLP_NPARAM * sizeof(float));
    Vel = (float*)alloc(MLP_NPARAM * sizeof(float));
    W2b = (bf16*)alloc(MLP_H * MLP_H * sizeof(bf16));
    W2Tb = (bf16*)alloc(MLP_H * MLP_H * sizeof(bf16));
    W3b = (bf16*)alloc(MLP_OUT_PAD * MLP_H * sizeof(bf16));
    W3Tb = (bf16*)alloc(MLP_H * MLP_K3 * sizeof(bf16));
    loss = (float*)alloc(sizeof(float));
    status = (int*)alloc(sizeof(int));
    RIMO_CUDA(cudaMemset(status, 0, sizeof(int)));
    // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) from a seeded host generator
    std::vector<float> h(MLP_NPARAM);
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    auto fill = [&](int off, int n, int fan_in) {
        const double a = 1.0 / std::sqrt((double)fan_in);
        for (int i = 0; i < n; ++i) h[off + i] = (float)(a * U(rng));
    };
    fill(MLP_OFF_W1, MLP_H * MLP_IN, MLP_IN);
    fill(MLP_OFF_B1, MLP_H, MLP_IN);
    fill(MLP_OFF_W2, MLP_H * MLP_H, MLP_H);
    fill(MLP_OFF_B2, MLP_H, MLP_H);
    fill(MLP_OFF_W3, MLP_OUT * MLP_H, MLP_H);
    fill(MLP_OFF_B3, MLP_OUT, MLP_H);
    set_params(h.data(), 0);
}

void Mlp::set_params(const float* host, cudaStream_t s) {
    RIMO_CUDA(cudaMemcpyAsync(P, host, MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice, s));
    RIMO_CUDA(cudaMemsetAsync(Mom, 0, MLP_NPARAM * sizeof(float), s));
    RIMO_CUDA(cudaMemsetAsync(Vel, 0, MLP_NPARAM * sizeof(float), s));
    t = 0;
    pack(s);
}

void Mlp::pack(cudaStream_t s) {
    const int n = MLP_OUT_PAD * MLP_H;
    pack_weights_kernel<<<(n + 255) / 256, 256, 0, s>>>(P, W2b, W2Tb, W3b, W3Tb);
}

void Mlp::reserve(int B) {
    if (B <= cap) return;
    cap = B;
    Z1 = (float*)alloc((size_t)B * MLP_H * sizeof(float));
    Z2 = (float*)alloc((size_t)B * MLP_H * sizeof(float));
    Y = (float*)alloc((size_t)B * MLP_OUT_PAD * sizeof(float));
    dH = (float*)alloc((size_t)B * MLP_H * sizeof(float));
    H1 = (bf16*)alloc((size_t)B * MLP_H * sizeof(bf16));
    H1T = (bf16*)alloc((size_t)B * MLP_H * sizeof(bf16));
    H2 = (bf16*)alloc((size_t)B * MLP_H * sizeof(bf16));
    H2T = (bf16*)alloc((size_t)B * MLP_H * sizeof(bf16));
    dY = (bf16*)alloc((size_t)B * MLP_K3 * sizeof(bf16));
    dYT = (bf16*)alloc((size_t)B * MLP_K3 * sizeof(bf16));
    dZ = (bf16*)alloc((size_t)B * MLP_H * sizeof(bf16));
    dZT = (bf16*)alloc((size_t)B * MLP_H * sizeof(bf16));
}

void Mlp::forward(const float* X, int B, cudaStream_t s) {
    reserve(B);
    const int n1 = B * MLP_H;
    l1_fwd_kernel<<<(n1 + 255) / 256, 256, 0, s>>>(X, P + MLP_OFF_W1, P + MLP_OFF_B1, Z1, H1, B);
    gemm(H1, MLP_H, W2b, MLP_H, Z2, MLP_H, B, MLP_H, MLP_H, 1, false, status, s);
    act_fwd_kernel<<<(n1 + 255) / 256, 256, 0, s>>>(Z2, P + MLP_OFF_B2, H2, B, MLP_H, MLP_H);
    gemm(H2, MLP_H, W3b, MLP_H, Y, MLP_OUT_PAD, B, MLP_OUT_PAD, MLP_H, 1, false, status, s);
}

void Mlp::grads(const float* X, const float* T, int B, cudaStream_t s) {
    forward(X, B, s);
    RIMO_CUDA(cudaMemsetAsync(G, 0, MLP_NPARAM * sizeof(float), s));
    RIMO_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), s));
    RIMO_CUDA(cudaMemsetAsync(dY, 0, (size_t)B * MLP_K3 * sizeof(bf16), s));
    const int parts = std::max(1, std::min(16, B / 256));
    loss_bwd_kernel<<<MLP_OUT_PAD * parts, 256, 0, s>>>(Y, MLP_OUT_PAD, P + MLP_OFF_B3, T, dY, MLP_K3,
                                                       G + MLP_OFF_B3, loss, B);
    transpose(H2, H2T, B, MLP_H, s);
    transpose(dY, dYT, B, MLP_K3, s);
    const int splits = std::max(1, B / 512);
    // dH2 = dY W3 (K = 464 padded output dimension)
    gemm(dY, MLP_K3, W3Tb, MLP_K3, dH, MLP_H, B, MLP_H, MLP_OUT_PAD, 1, false, status, s);
    // dW3 = dY^T H2 (M = 464 -> rows >= 450 land in a scratch tail of G3)
    RIMO_CUDA(cudaMemsetAsync(Y, 0, (size_t)512 * MLP_H * sizeof(float), s));
    gemm(dYT, B, H2T, B, Y, MLP_H, 512, MLP_H, B, splits, true, status, s);
    RIMO_CUDA(cudaMemcpyAsync(G + MLP_OFF_W3, Y, (size_t)MLP_OUT * MLP_H * sizeof(float), cudaMemcpyDeviceToDevice, s));
    act_bwd_kernel<<<MLP_H * parts, 256, 0, s>>>(dH, Z2, dZ, G + MLP_OFF_B2, B);
    transpose(dZ, dZT, B, MLP_H, s);
    transpose(H1, H1T, B, MLP_H, s);
    gemm(dZT, B, H1T, B, G + MLP_OFF_W2, MLP_H, MLP_H, MLP_H, B, splits, true, status, s);
    gemm(dZ, MLP_H, W2Tb, MLP_H, dH, MLP_H, B, MLP_H, MLP_H, 1, false, status, s);
    l1_bwd_kernel<<<MLP_H * parts, 256, 0, s>>>(dH, Z1, X, G + MLP_OFF_W1, G + MLP_OFF_B1, B);
}

void Mlp::step(const float* X, const float* T, int B, float lr, cudaStream_t s) {
    grads(X, T, B, s);
    ++t;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)t), c2 = 1.f - std::pow(b2, (float)t);
    adam_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(P, G, Mom, Vel, MLP_NPARAM, lr, b1, b2, 1e-8f, c1, c2);
    pack(s);
}

}  // namespace rimo

// --------------------------------------------------------------------------------------
// C ABI
struct rimo_surrogate {
    rimo::Mlp mlp;
    float w_scale = 0.f;          // input normalisation of w_r (set by rimo_surrogate_fit)
    __nv_bfloat16* W3g = nullptr;  // layer 3 for the tile generator: [480][128], see sur_gen_kernel
};

namespace rimo {

__global__ void add_bias_out_kernel(const float* __restrict__ Y, const float* __restrict__ b3, float* __restrict__ out,
                                    int B) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)B * MLP_OUT) return;
    const int b = (int)(e / MLP_OUT), j = (int)(e % MLP_OUT);
    out[e] = Y[(size_t)b * MLP_OUT_PAD + j] + b3[j];
}

static void check_batch(int64_t B) {
    if (B <= 0 || B % 128 != 0 || B > (1 << 24)) fail(RIMO_ERR_INVALID_ARG, "batch must be a positive multiple of 128");
}

static void check_status(Mlp& m, cudaStream_t s) {
    int st = 0;
    RIMO_CUDA(cudaMemcpyAsync(&st, m.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    RIMO_CUDA(cudaStreamSynchronize(s));
    if (st) {
        RIMO_CUDA(cudaMemsetAsync(m.status, 0, sizeof(int), s));
        fail(RIMO_ERR_TIMEOUT, "a bounded tensor-core wait ran out");
    }
}

}  // namespace rimo

using namespace rimo;

#define SUR_BEGIN try {
#define SUR_END                       \
    return RIMO_OK;                   \
    }                                 \
    catch (const Error& e) {          \
        set_last_error(e.msg);        \
        return e.status;              \
    }                                 \
    catch (const std::exception& e) { \
        set_last_error(e.what());     \
        return RIMO_ERR_OOM;          \
    }

namespace rimo {

constexpr int SUR_S = 15;         // tile side the network outputs
constexpr int SUR_TAPS = SUR_S * SUR_S;

// SplitMix64 (Steele, Lea, Flood 2014): counter-based draws for the training samples.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ---- tile generator: the whole network per 128 visibilities in one persistent CTA per SM
// Layer 1 (3 -> 128) on CUDA cores into shared memory (bf16, canonical K-major); layer 2 as
// 8 MMAs (M 128, N 128, K 16) into TMEM columns [0, 128); GELU read-out back into the same
// shared buffer; layer 3 as 2 x 8 MMAs (N 256 + 224) into TMEM columns [0, 480); the read-out
// adds b3 and writes each visibility's 15 x 15 complex tile (plus its even-count pad) to
// the tap scratch at the visibility's offset.  W2 and W3 stay in shared memory (bf16).
// Layer 3's rows are packed so that real and imaginary outputs start at 16-aligned TMEM
// columns: rows [0, 225) the real parts, [240, 465) the imaginary parts, the rest zero.
constexpr int GEN_THREADS = 256;
constexpr int GEN_WG = GEN_THREADS / 128;  // warp groups: each covers the 128 TMEM lanes once
constexpr int GEN_HW = MLP_H / GEN_WG;      // hidden units (columns) per warp group
constexpr int GEN_N3 = 480, GEN_IM = 240;
constexpr size_t GEN_SW2 = (size_t)MLP_H * MLP_H * 2, GEN_SW3 = (size_t)GEN_N3 * MLP_H * 2, GEN_SA = 128 * MLP_H * 2;
constexpr size_t GEN_SMEM = GEN_SW2 + GEN_SW3 + GEN_SA + (384 + 128 + 128 + GEN_N3 + 384) * 4 + 128 * 8;

__global__ void pack_w3g_kernel(const float* __restrict__ P, bf16* __restrict__ W3g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= GEN_N3 * MLP_H) return;
    const int r = i / MLP_H, c = i % MLP_H;
    int src = -1;
    if (r < SUR_TAPS) src = r;
    else if (r >= GEN_IM && r < GEN_IM + SUR_TAPS) src = SUR_TAPS + (r - GEN_IM);
    W3g[i] = __float2bfloat16(src >= 0 ? P[MLP_OFF_W3 + src * MLP_H + c] : 0.f);
}

struct GenArgs {
    const VisMeta* meta;
    float2* taps;
    const float* phiu;
    const float* phiv;
    const float* wr;
    int64_t v0;
    int n;
    float inv_w;
    const float* P;    // FP32 parameters (W1, b1, b2, b3)
    const bf16* W2b;   // [128][128]
    const bf16* W3g;   // [480][128]
    uint32_t* fx;
    int* status;
    const float* wt;   // data weights (sorted order) multiplying the tiles, or null
};

__device__ __forceinline__ uint32_t pack_bf2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

__global__ void __launch_bounds__(GEN_THREADS, 1) sur_gen_kernel(GenArgs A) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* sW2 = sm;
    unsigned char* sW3 = sm + GEN_SW2;
    unsigned char* sA = sW3 + GEN_SW3;
    float* sW1 = reinterpret_cast<float*>(sA + GEN_SA);
    float* sb1 = sW1 + 384;
    float* sb2 = sb1 + 128;
    float* sb3 = sb2 + 128;
    float* sx = sb3 + GEN_N3;
    int64_t* soff = reinterpret_cast<int64_t*>(sx + 384);
    __shared__ float swt[128];  // data weight of each row
    __shared__ float s_tsum[GEN_WG][128];  // per warp group: partial tap sums of each row
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int e = tid; e < MLP_H * 16; e += GEN_THREADS) {
        const int r = e >> 4, v = e & 15;
        *reinterpret_cast<uint4*>(sW2 + tc::kmajor_offset(r, v * 8, MLP_H)) =
            *reinterpret_cast<const uint4*>(A.W2b + (size_t)r * MLP_H + v * 8);
    }
    for (int e = tid; e < GEN_N3 * 16; e += GEN_THREADS) {
        const int r = e >> 4, v = e & 15;
        *reinterpret_cast<uint4*>(sW3 + tc::kmajor_offset(r, v * 8, GEN_N3)) =
            *reinterpret_cast<const uint4*>(A.W3g + (size_t)r * MLP_H + v * 8);
    }
    for (int e = tid; e < 384; e += GEN_THREADS) sW1[e] = __bfloat162float(__float2bfloat16(A.P[MLP_OFF_W1 + e]));
    for (int e = tid; e < 128; e += GEN_THREADS) {
        sb1[e] = A.P[MLP_OFF_B1 + e];
        sb2[e] = A.P[MLP_OFF_B2 + e];
    }
    for (int e = tid; e < GEN_N3; e += GEN_THREADS) {
        int src = -1;
        if (e < SUR_TAPS) src = e;
        else if (e >= GEN_IM && e < GEN_IM + SUR_TAPS) src = SUR_TAPS + (e - GEN_IM);
        sb3[e] = src >= 0 ? A.P[MLP_OFF_B3 + src] : 0.f;
    }
    if (warp == 0) tc::tmem_alloc(&tslot, 512);
    if (tid == 0) {
        mbar_init_(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;  // this warp's TMEM lanes
    uint32_t phase = 0;
    bool ok = true;
    float run_tmax = 0.f, run_t1 = 0.f;  // running bounds over this thread's tiles
    const int ntile = (A.n + 127) / 128;
    // the next tile's inputs are loaded (raw) while this tile computes
    float in_u = 0.f, in_v = 0.f, in_w = 0.f, in_wt = 1.f;
    int64_t in_off = 0;
    auto load_inputs = [&](int t) {
        if (tid < 128 && t < ntile) {
            const int j = t * 128 + tid < A.n ? t * 128 + tid : A.n - 1;
            const int64_t k = A.v0 + j;
            in_u = __ldg(A.phiu + k);
            in_v = __ldg(A.phiv + k);
            in_w = __ldg(A.wr + k);
            in_off = A.meta[k].off;
            in_wt = A.wt ? __ldg(A.wt + k) : 1.f;
        }
    };
    load_inputs(blockIdx.x);
    for (int tile = blockIdx.x; tile < ntile && ok; tile += gridDim.x) {
        const int base = tile * 128;
        if (tid < 128) {
            sx[3 * tid + 0] = 2.f * in_u - 1.f;
            sx[3 * tid + 1] = 2.f * in_v - 1.f;
            sx[3 * tid + 2] = in_w * A.inv_w;
            soff[tid] = in_off;
            swt[tid] = in_wt;
        }
        load_inputs(tile + gridDim.x);
        __syncthreads();
        {   // layer 1: row r, hidden units [GEN_HW h, GEN_HW (h + 1))
            const int r = tid & 127, h = tid >> 7;
            const float x0 = sx[3 * r], x1 = sx[3 * r + 1], x2 = sx[3 * r + 2];
#pragma unroll 1
            for (int g = 0; g < GEN_HW / 8; ++g) {
                uint32_t w[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float z[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int j = GEN_HW * h + 8 * g + 2 * q + u;
                        z[u] = gelu_f(fmaf(x0, sW1[3 * j], fmaf(x1, sW1[3 * j + 1], fmaf(x2, sW1[3 * j + 2], sb1[j]))));
                    }
                    w[q] = pack_bf2(z[0], z[1]);
                }
                *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(r, GEN_HW * h + 8 * g, 128)) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {  // layer 2
            for (int s = 0; s < MLP_H / 16; ++s)
                tc::mma_bf16(tmem, tc::smem_desc(tc::smem_addr(sA) + s * 128 * 32, 128, 256),
                             tc::smem_desc(tc::smem_addr(sW2) + s * MLP_H * 32, 128, 256), tc::idesc_bf16_f32(128, 128),
                             s > 0 ? 1u : 0u);
            tc::mma_commit(&bar);
        }
        ok = mbar_wait_(&bar, phase);
        phase ^= 1;
        if (__syncthreads_or(!ok)) break;
        tc::fence_after_sync();
        {   // layer-2 read-out: row 32 (warp % 4) + lane, columns [GEN_HW (warp / 4), + GEN_HW)
            const int r = 32 * (warp & 3) + lane;
#pragma unroll 1
            for (int c0 = 0; c0 < GEN_HW; c0 += 32) {  // two 16-column loads in flight per wait
                const int col = GEN_HW * (warp >> 2) + c0;
                uint32_t va[16], vb[16];
                tc::tmem_ld16_async(tmem + lane_base + (uint32_t)col, va);
                tc::tmem_ld16_async(tmem + lane_base + (uint32_t)(col + 16), vb);
                tc::tmem_wait_ld_tied(va);
                tc::reg_tie(vb);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t* v = h ? vb : va;
                    const int cc = col + 16 * h;
                    uint32_t w[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        w[i] = pack_bf2(gelu_f(__uint_as_float(v[2 * i]) + sb2[cc + 2 * i]),
                                        gelu_f(__uint_as_float(v[2 * i + 1]) + sb2[cc + 2 * i + 1]));
                    *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(r, cc, 128)) = make_uint4(w[0], w[1], w[2], w[3]);
                    *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(r, cc + 8, 128)) = make_uint4(w[4], w[5], w[6], w[7]);
                }
            }
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {  // layer 3: rows [0, 256) and [256, 480) of W3g
            for (int s = 0; s < MLP_H / 16; ++s) {
                const uint64_t ad = tc::smem_desc(tc::smem_addr(sA) + s * 128 * 32, 128, 256);
                const uint32_t b0 = tc::smem_addr(sW3) + s * GEN_N3 * 32;
                tc::mma_bf16(tmem, ad, tc::smem_desc(b0, 128, 256), tc::idesc_bf16_f32(128, 256), s > 0 ? 1u : 0u);
                tc::mma_bf16(tmem + 256, ad, tc::smem_desc(b0 + (256 / 8) * 256, 128, 256),
                             tc::idesc_bf16_f32(128, GEN_N3 - 256), s > 0 ? 1u : 0u);
            }
            tc::mma_commit(&bar);
        }
        ok = mbar_wait_(&bar, phase);
        phase ^= 1;
        if (__syncthreads_or(!ok)) break;
        tc::fence_after_sync();
        {   // layer-3 read-out: chunks of 16 taps (warp groups take every GEN_WG-th chunk).  The
            // chunk's 32 rows pass through a warp-private 4 KB of the A buffer (free once the
            // layer-3 MMAs completed) so that the warp writes 128-byte row segments, not
            // scattered 16-byte pieces; pieces are XOR-swizzled by row against bank conflicts.
            const int r = 32 * (warp & 3) + lane;
            const bool valid = base + r < A.n;
            const float wk = swt[r];
            float4* stage = reinterpret_cast<float4*>(sA) + warp * 256;  // [32 rows][8 pieces]
            float tmax = 0.f, tsum = 0.f;
#pragma unroll 1
            for (int c = warp >> 2; c < (SUR_TAPS + 15) / 16; c += GEN_WG) {
                const int q0 = 16 * c;
                uint32_t rr[16], ri[16];
                tc::tmem_ld16_async(tmem + lane_base + (uint32_t)q0, rr);
                tc::tmem_ld16_async(tmem + lane_base + (uint32_t)(GEN_IM + q0), ri);
                tc::tmem_wait_ld_tied(rr);
                tc::reg_tie(ri);
#pragma unroll
                for (int j = 0; j < 8; ++j) {  // piece j: taps q0 + 2j, q0 + 2j + 1 (zero past the tile)
                    const int q = q0 + 2 * j;
                    const float2 t0 = q < SUR_TAPS ? make_float2(wk * (__uint_as_float(rr[2 * j]) + sb3[q]),
                                                                 wk * (__uint_as_float(ri[2 * j]) + sb3[GEN_IM + q]))
                                                   : make_float2(0.f, 0.f);
                    const float2 t1 = q + 1 < SUR_TAPS
                                          ? make_float2(wk * (__uint_as_float(rr[2 * j + 1]) + sb3[q + 1]),
                                                        wk * (__uint_as_float(ri[2 * j + 1]) + sb3[GEN_IM + q + 1]))
                                          : make_float2(0.f, 0.f);
                    const float m0 = fabsf(t0.x) + fabsf(t0.y), m1 = fabsf(t1.x) + fabsf(t1.y);
                    tmax = fmaxf(tmax, fmaxf(m0, m1));
                    tsum += m0 + m1;
                    stage[lane * 8 + (j ^ (lane & 7))] = make_float4(t0.x, t0.y, t1.x, t1.y);
                }
                __syncwarp();
                // a tile holds 226 taps (225 and the pad): the last chunk has one piece
                const int npc = q0 + 16 <= SUR_TAPS + 1 ? 8 : (SUR_TAPS + 1 - q0) / 2;
#pragma unroll
                for (int it = 0; it < 8; ++it) {
                    const int row = 4 * it + (lane >> 3), pc = lane & 7;
                    const int rg = 32 * (warp & 3) + row;
                    if (pc < npc && base + rg < A.n)
                        *reinterpret_cast<float4*>(A.taps + soff[rg] + q0 + 2 * pc) = stage[row * 8 + (pc ^ (row & 7))];
                }
                __syncwarp();
            }
            if (valid) run_tmax = fmaxf(run_tmax, tmax);
            s_tsum[warp >> 2][r] = valid ? tsum : 0.f;  // each warp group holds a share of the row
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid < 128 && base + tid < A.n) {
            float t = 0.f;
#pragma unroll
            for (int q = 0; q < GEN_WG; ++q) t += s_tsum[q][tid];
            run_t1 = fmaxf(run_t1, t);
        }
    }
    // the bounds: one atomic per warp for the whole launch (not one per visibility)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        run_tmax = fmaxf(run_tmax, __shfl_xor_sync(0xffffffffu, run_tmax, o));
        run_t1 = fmaxf(run_t1, __shfl_xor_sync(0xffffffffu, run_t1, o));
    }
    if (lane == 0) {
        atomicMax(A.fx + FX_TMAX, __float_as_uint(run_tmax));
        atomicMax(A.fx + FX_T1, __float_as_uint(run_t1));
    }
    if (!ok && tid == 0) atomicExch(A.status, 2);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) {
        tc::tmem_dealloc(tmem, 512);
        tc::tmem_relinquish();
    }
}

void reset_surrogate_bounds(rimo_plan* p, cudaStream_t s) {
    RIMO_CUDA(cudaMemsetAsync(p->d_fx + FX_TMAX, 0, 2 * sizeof(uint32_t), s));  // FX_TMAX, FX_T1
    if (p->mode == RIMO_MODE_SURROGATE)  // this apply's network (it may have trained since)
        pack_w3g_kernel<<<(GEN_N3 * MLP_H + 255) / 256, 256, 0, s>>>(p->sur->mlp.P, p->sur->W3g);
}

int surrogate_generate(rimo_plan* p, int bin, cudaStream_t s) {
    rimo_surrogate* sur = p->sur;
    const float ws = sur->w_scale > 0.f ? sur->w_scale : (p->info.wr_max > 0 ? (float)p->info.wr_max : 1.f);
    const int64_t vb = p->bins[bin].vb, n = p->bins[bin].ve - vb;
    if (n <= 0) return 0;
    GenArgs A;
    A.meta = p->d_meta;
    A.taps = p->d_sur_taps;
    A.phiu = p->d_phiu;
    A.phiv = p->d_phiv;
    A.wr = p->d_wr;
    A.v0 = vb;
    A.n = (int)n;
    A.inv_w = 1.f / ws;
    A.P = sur->mlp.P;
    A.W2b = sur->mlp.W2b;
    A.W3g = sur->W3g;
    A.fx = p->d_fx;
    A.status = p->d_status;
    A.wt = p->d_wt;
    RIMO_CUDA(cudaFuncSetAttribute(sur_gen_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GEN_SMEM));
    const int64_t ntile = (n + 127) / 128;
    const int grid = (int)std::min<int64_t>(ntile, (int64_t)p->n_sm);
    sur_gen_kernel<<<grid, GEN_THREADS, GEN_SMEM, s>>>(A);
    return 1;
}

// training sample i: a visibility k drawn uniformly, its inputs, and its exact tile embedded
// at the centre of 15 x 15 (a smaller support S sits at offset (15 - S) / 2)
__global__ void sur_dataset_kernel(const VisMeta* __restrict__ meta, float2* const* __restrict__ gblk,
                                   const float* __restrict__ phiu, const float* __restrict__ phiv,
                                   const float* __restrict__ wr, int64_t M, uint64_t seed, int64_t n, float inv_w,
                                   float* X, float* T) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int64_t k = (int64_t)(splitmix64(seed + (uint64_t)i) % (uint64_t)M);
    const VisMeta mt = meta[k];
    const int S = (mt.pos >> 16) & 255, off = (SUR_S - S) / 2;
    const float2* G = gblk[mt.pos >> 24] + mt.off;
    if (lane == 0) {
        X[3 * i + 0] = 2.f * phiu[k] - 1.f;
        X[3 * i + 1] = 2.f * phiv[k] - 1.f;
        X[3 * i + 2] = wr[k] * inv_w;
    }
    float* t = T + (size_t)i * MLP_OUT;
    for (int q = lane; q < SUR_TAPS; q += 32) {
        const int a = q / SUR_S - off, b = q % SUR_S - off;
        const float2 v = (a >= 0 && a < S && b >= 0 && b < S) ? G[a * S + b] : make_float2(0.f, 0.f);
        t[q] = v.x;
        t[SUR_TAPS + q] = v.y;
    }
}

__global__ void sur_batch_kernel(const float* __restrict__ X, const float* __restrict__ T, int64_t n, uint64_t seed,
                                 int B, float* Xb, float* Tb) {
    const int j = blockIdx.x;
    const int64_t i = (int64_t)(splitmix64(seed + (uint64_t)j) % (uint64_t)n);
    for (int e = threadIdx.x; e < MLP_OUT; e += blockDim.x) Tb[(size_t)j * MLP_OUT + e] = T[(size_t)i * MLP_OUT + e];
    if (threadIdx.x < 3) Xb[3 * j + threadIdx.x] = X[3 * i + threadIdx.x];
}

struct DevScratch {
    std::vector<void*> v;
    void* get(size_t bytes) {
        void* ptr = nullptr;
        if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
            cudaGetLastError();
            fail(RIMO_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes for the training set failed");
        }
        v.push_back(ptr);
        return ptr;
    }
    ~DevScratch() {
        for (void* ptr : v) cudaFree(ptr);
    }
};

}  // namespace rimo

extern "C" {

rimo_status rimo_surrogate_create(uint64_t seed, rimo_surrogate_t* out) {
    if (out) *out = nullptr;
    rimo_surrogate* s = nullptr;
    try {
        if (!out) fail(RIMO_ERR_INVALID_ARG, "null output");
        s = new rimo_surrogate();
        s->mlp.init(seed);
        RIMO_CUDA(cudaDeviceSynchronize());
        *out = s;
        return RIMO_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        delete s;
        return e.status;
    }
}

rimo_status rimo_surrogate_destroy(rimo_surrogate_t s) {
    delete s;
    return RIMO_OK;
}

rimo_status rimo_surrogate_get_params(rimo_surrogate_t s, float* params) {
    SUR_BEGIN
    if (!s || !params) fail(RIMO_ERR_INVALID_ARG, "null argument");
    RIMO_CUDA(cudaMemcpy(params, s->mlp.P, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    SUR_END
}

rimo_status rimo_surrogate_set_params(rimo_surrogate_t s, const float* params) {
    SUR_BEGIN
    if (!s || !params) fail(RIMO_ERR_INVALID_ARG, "null argument");
    s->mlp.set_params(params, 0);
    RIMO_CUDA(cudaDeviceSynchronize());
    SUR_END
}

rimo_status rimo_surrogate_forward(rimo_surrogate_t s, const float* x, int64_t B, float* y, void* stream) {
    SUR_BEGIN
    if (!s || !x || !y) fail(RIMO_ERR_INVALID_ARG, "null argument");
    check_batch(B);
    cudaStream_t st = (cudaStream_t)stream;
    s->mlp.forward(x, (int)B, st);
    const int64_t n = B * MLP_OUT;
    add_bias_out_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s->mlp.Y, s->mlp.P + MLP_OFF_B3, y, (int)B);
    RIMO_CUDA(cudaGetLastError());
    SUR_END
}

rimo_status rimo_surrogate_gradients(rimo_surrogate_t s, const float* x, const float* t, int64_t B, float* grads,
                                     float* loss, void* stream) {
    SUR_BEGIN
    if (!s || !x || !t) fail(RIMO_ERR_INVALID_ARG, "null argument");
    check_batch(B);
    cudaStream_t st = (cudaStream_t)stream;
    s->mlp.grads(x, t, (int)B, st);
    RIMO_CUDA(cudaGetLastError());
    check_status(s->mlp, st);
    if (grads) RIMO_CUDA(cudaMemcpy(grads, s->mlp.G, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    if (loss) {
        float l = 0.f;
        RIMO_CUDA(cudaMemcpy(&l, s->mlp.loss, sizeof(float), cudaMemcpyDeviceToHost));
        *loss = l / ((float)B * MLP_OUT);
    }
    SUR_END
}

rimo_status rimo_surrogate_train_step(rimo_surrogate_t s, const float* x, const float* t, int64_t B, float lr,
                                      float* loss, void* stream) {
    SUR_BEGIN
    if (!s || !x || !t) fail(RIMO_ERR_INVALID_ARG, "null argument");
    check_batch(B);
    cudaStream_t st = (cudaStream_t)stream;
    s->mlp.step(x, t, (int)B, lr, st);
    RIMO_CUDA(cudaGetLastError());
    if (loss) {
        float l = 0.f;
        RIMO_CUDA(cudaMemcpyAsync(&l, s->mlp.loss, sizeof(float), cudaMemcpyDeviceToHost, st));
        RIMO_CUDA(cudaStreamSynchronize(st));
        *loss = l / ((float)B * MLP_OUT);
    }
    SUR_END
}


rimo_status rimo_plan_set_surrogate(rimo_plan_t p, rimo_surrogate_t s) {
    SUR_BEGIN
    if (!p || !s) fail(RIMO_ERR_INVALID_ARG, "null argument");
    if (p->mode != RIMO_MODE_SURROGATE) fail(RIMO_ERR_INVALID_ARG, "the plan was not created in surrogate mode");
    int dev = 0;
    RIMO_CUDA(cudaGetDevice(&dev));
    if (dev != p->device) fail(RIMO_ERR_INVALID_ARG, "plan and surrogate on different devices");
    // everything the generation needs is allocated here, not during an apply
    if (!s->W3g) s->W3g = (bf16*)s->mlp.alloc((size_t)GEN_N3 * MLP_H * sizeof(bf16));
    p->sur = s;
    SUR_END
}

rimo_status rimo_surrogate_fit(rimo_surrogate_t s, rimo_plan_t exact, int64_t n_samples, int32_t steps,
                               int32_t batch, float lr, uint64_t seed, float* losses, void* stream) {
    SUR_BEGIN
    if (!s || !exact) fail(RIMO_ERR_INVALID_ARG, "null argument");
    if (exact->mode == RIMO_MODE_SURROGATE || exact->d_gblocks.empty())
        fail(RIMO_ERR_INVALID_ARG, "training needs a plan with stored exact tiles");
    if (exact->d_wt) fail(RIMO_ERR_STATE, "training needs unweighted tiles (remove the plan's weighting first)");
    if (exact->J + exact->prm.max_wsupport - 1 != SUR_S)
        fail(RIMO_ERR_INVALID_ARG, "training tiles must be 15 x 15 (kb_support + max_wsupport - 1 = 15)");
    if (n_samples <= 0 || steps <= 0 || !(lr > 0.f)) fail(RIMO_ERR_INVALID_ARG, "n_samples, steps, lr must be > 0");
    check_batch(batch);
    cudaStream_t st = (cudaStream_t)stream;
    const float ws = exact->info.wr_max > 0 ? (float)exact->info.wr_max : 1.f;
    DevScratch tmp;
    float* X = (float*)tmp.get((size_t)n_samples * 3 * sizeof(float));
    float* T = (float*)tmp.get((size_t)n_samples * MLP_OUT * sizeof(float));
    float* Xb = (float*)tmp.get((size_t)batch * 3 * sizeof(float));
    float* Tb = (float*)tmp.get((size_t)batch * MLP_OUT * sizeof(float));
    float* L = (float*)tmp.get((size_t)steps * sizeof(float));
    const uint64_t sample_seed = splitmix64(seed ^ 0x5EEDull);
    sur_dataset_kernel<<<(unsigned)((n_samples * 32 + 255) / 256), 256, 0, st>>>(
        exact->d_meta, exact->d_gblock_ptrs, exact->d_phiu, exact->d_phiv, exact->d_wr, exact->M, sample_seed,
        n_samples, 1.f / ws, X, T);
    RIMO_CUDA(cudaGetLastError());
    s->mlp.reserve(batch);
    for (int k = 0; k < steps; ++k) {
        // cosine decay from lr to lr / 100
        const float lr_k = lr * (0.01f + 0.99f * 0.5f * (1.f + std::cos(3.14159265358979f * (float)k / (float)steps)));
        sur_batch_kernel<<<batch, 128, 0, st>>>(X, T, n_samples, splitmix64(seed + 0x9E37ull * (uint64_t)(k + 1)),
                                                 batch, Xb, Tb);
        s->mlp.step(Xb, Tb, batch, lr_k, st);
        RIMO_CUDA(cudaMemcpyAsync(L + k, s->mlp.loss, sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    RIMO_CUDA(cudaGetLastError());
    check_status(s->mlp, st);
    if (losses) {
        RIMO_CUDA(cudaMemcpyAsync(losses, L, (size_t)steps * sizeof(float), cudaMemcpyDeviceToHost, st));
        RIMO_CUDA(cudaStreamSynchronize(st));
        for (int k = 0; k < steps; ++k) losses[k] /= (float)batch * MLP_OUT;
    }
    RIMO_CUDA(cudaStreamSynchronize(st));
    s->w_scale = ws;
    SUR_END
}

rimo_status rimo_surrogate_get_w_scale(rimo_surrogate_t s, float* w_scale) {
    SUR_BEGIN
    if (!s || !w_scale) fail(RIMO_ERR_INVALID_ARG, "null argument");
    *w_scale = s->w_scale;
    SUR_END
}

rimo_status rimo_surrogate_set_w_scale(rimo_surrogate_t s, float w_scale) {
    SUR_BEGIN
    if (!s || !(w_scale > 0.f)) fail(RIMO_ERR_INVALID_ARG, "null surrogate or w_scale <= 0");
    s->w_scale = w_scale;
    SUR_END
}

}  // extern "C"
