// The forward-backward update of Eq. 4 with the non-negativity prior of Eq. 3, and the
// real inner product of two images (for the data fidelity and the step-size bound).
#include <mutex>

#include "internal.h"

namespace rimo {

// out = (max(Re x + gamma (Re dirty - Re g), 0), 0): Eq. 4 with the projection onto the
// non-negative real images as the denoising step (g = Phi^dagger Phi x)
__global__ void fb_step_kernel(const float2* __restrict__ x, const float2* __restrict__ g,
                               const float2* __restrict__ dirty, float gamma, float2* __restrict__ out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = fmaf(gamma, dirty[i].x - g[i].x, x[i].x);
        out[i] = make_float2(fmaxf(v, 0.f), 0.f);
    }
}

// Re sum conj(a_i) b_i in FP64: fixed partition into DOT_BLOCKS block partials (fixed
// order within each), the last block to finish adds the partials in index order
constexpr int DOT_BLOCKS = 512;
__device__ double g_dot_part[DOT_BLOCKS];
__device__ unsigned int g_dot_count;
__device__ double g_dot_result;

__global__ void __launch_bounds__(256) dot_kernel(const float2* __restrict__ a, const float2* __restrict__ b,
                                                  int64_t n) {
    __shared__ double red[256];
    __shared__ bool last;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 u = a[i], v = b[i];
        s += (double)u.x * (double)v.x + (double)u.y * (double)v.y;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        g_dot_part[blockIdx.x] = red[0];
        __threadfence();
        last = atomicAdd(&g_dot_count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double t = 0.0;
        for (unsigned int q = 0; q < gridDim.x; ++q) t += *((volatile double*)&g_dot_part[q]);
        g_dot_result = t;
        g_dot_count = 0u;
    }
}

}  // namespace rimo

using namespace rimo;

extern "C" {

rimo_status rimo_fb_step(const rimo_cfloat* x, const rimo_cfloat* g, const rimo_cfloat* dirty, float gamma,
                         rimo_cfloat* out, int64_t n, void* stream) {
    RIMO_API_BEGIN
    if (n < 0 || (n > 0 && (!x || !g || !dirty || !out))) fail(RIMO_ERR_INVALID_ARG, "null pointer or n < 0");
    if (!(gamma >= 0.f) || !std::isfinite(gamma)) fail(RIMO_ERR_INVALID_ARG, "gamma must be finite and >= 0");
    if (n == 0) return RIMO_OK;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
    fb_step_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>((const float2*)x, (const float2*)g,
                                                                  (const float2*)dirty, gamma, (float2*)out, n);
    RIMO_CUDA(cudaGetLastError());
    RIMO_API_END
}

rimo_status rimo_image_dot(const rimo_cfloat* a, const rimo_cfloat* b, int64_t n, double* result, void* stream) {
    RIMO_API_BEGIN
    if (n < 0 || !result || (n > 0 && (!a || !b))) fail(RIMO_ERR_INVALID_ARG, "null pointer or n < 0");
    static std::mutex mu;  // one reduction scratch per device: calls take turns
    std::lock_guard<std::mutex> lock(mu);
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, DOT_BLOCKS));
    dot_kernel<<<blocks, 256, 0, s>>>((const float2*)a, (const float2*)b, n);
    RIMO_CUDA(cudaGetLastError());
    RIMO_CUDA(cudaMemcpyFromSymbolAsync(result, g_dot_result, sizeof(double), 0, cudaMemcpyDeviceToHost, s));
    RIMO_CUDA(cudaStreamSynchronize(s));
    RIMO_API_END
}

}  // extern "C"
