// Data weighting injected into the measurement operator (Section 2, Eq. 3) and Briggs'
// robust weights of the Fourier-sampling density (the scheme Section 2 cites).
//
// The weights multiply the tiles: the weighted operator W Phi = (W G) F Z, so a stored-G
// plan rebuilds its tiles with the weights and a plan that generates tiles multiplies them
// as they are made; the gridding, its fixed-point bounds (taken from the tiles) and H
// (built from the tiles) follow without further change.
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "internal.h"
#include "planner.h"

namespace rimo {
void launch_gbuild(const rimo_plan* p, cudaStream_t s);
}

using namespace rimo;

extern "C" {

rimo_status rimo_plan_set_weights(rimo_plan_t p, const float* w, void* stream) {
    RIMO_API_BEGIN
    if (!p) fail(RIMO_ERR_INVALID_ARG, "null plan");
    if (p->h_built) fail(RIMO_ERR_STATE, "the tiles were folded into H: set weights before rimo_build_holographic");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t M = p->M;
    if (w) {
        for (int64_t k = 0; k < M; ++k)
            if (!(w[k] >= 0.f) || !std::isfinite(w[k])) fail(RIMO_ERR_INVALID_ARG, "weights must be finite and >= 0");
        std::vector<float> ws((size_t)M);
        for (int64_t k = 0; k < M; ++k) ws[(size_t)p->inv_perm[k]] = w[k];  // sorted order
        if (!p->d_wt_buf) p->d_wt_buf = (float*)dev_alloc(p, (size_t)std::max<int64_t>(M, 1) * sizeof(float));
        if (M > 0)
            RIMO_CUDA(cudaMemcpyAsync(p->d_wt_buf, ws.data(), (size_t)M * sizeof(float), cudaMemcpyHostToDevice, s));
        p->d_wt = p->d_wt_buf;
        p->info.weighted = 1;
    } else {
        p->d_wt = nullptr;
        p->info.weighted = 0;
    }
    if (p->mode == RIMO_MODE_STORED_G && M > 0) {
        // rebuild the stored tiles (and their bounds) with the new weights
        RIMO_CUDA(cudaMemsetAsync(p->d_fx + FX_TMAX, 0, 2 * sizeof(uint32_t), s));  // FX_TMAX, FX_T1
        launch_gbuild(p, s);
    }
    RIMO_CUDA(cudaGetLastError());
    RIMO_CUDA(cudaStreamSynchronize(s));
    RIMO_API_END
}

rimo_status rimo_briggs_weights(const double* uvw, int64_t M, int32_t nx, int32_t ny, double fov_x, double fov_y,
                                double robust, float* w_out) {
    RIMO_API_BEGIN
    if (M < 0 || (M > 0 && (!uvw || !w_out))) fail(RIMO_ERR_INVALID_ARG, "null pointer or M < 0");
    if (nx < 1 || ny < 1 || !(fov_x > 0.0) || !(fov_y > 0.0) || !std::isfinite(robust))
        fail(RIMO_ERR_INVALID_ARG, "grid, field of view or robustness out of range");
    if (M == 0) return RIMO_OK;
    // cell of each visibility on the image's Fourier grid (spacing 1 / FoV), wrapped; the
    // visibilities are split over host threads and the per-cell counts are integers, so the
    // result does not depend on the split
    const size_t ncell = (size_t)nx * (size_t)ny;
    std::vector<int64_t> cell((size_t)M);
    std::unique_ptr<std::atomic<uint64_t>[]> D(new std::atomic<uint64_t>[ncell]());
    std::atomic<bool> bad{false};
    planner::parallel_for(M, [&](int64_t b, int64_t e) {
        bool ok = true;
        for (int64_t k = b; k < e; ++k) {
            const double fu = std::floor(uvw[3 * k + 0] * fov_x + 0.5), fv = std::floor(uvw[3 * k + 1] * fov_y + 0.5);
            if (!std::isfinite(fu) || !std::isfinite(fv)) {
                ok = false;
                cell[(size_t)k] = 0;
                continue;
            }
            int64_t cu = (int64_t)std::fmod(fu, (double)nx), cv = (int64_t)std::fmod(fv, (double)ny);
            if (cu < 0) cu += nx;
            if (cv < 0) cv += ny;
            cell[(size_t)k] = cu * ny + cv;
            D[(size_t)cell[(size_t)k]].fetch_add(1, std::memory_order_relaxed);
        }
        if (!ok) bad.store(true);
    }, 1 << 16);
    if (bad.load()) fail(RIMO_ERR_INVALID_ARG, "non-finite uvw");
    double sum_d2 = 0.0;
    for (size_t c = 0; c < ncell; ++c) {
        const double d = (double)D[c].load(std::memory_order_relaxed);
        sum_d2 += d * d;
    }
    const double a = 5.0 * std::pow(10.0, -robust);
    const double f2 = a * a / (sum_d2 / (double)M);
    planner::parallel_for(M, [&](int64_t b, int64_t e) {
        for (int64_t k = b; k < e; ++k)
            w_out[k] = (float)(1.0 / (1.0 + f2 * (double)D[(size_t)cell[(size_t)k]].load(std::memory_order_relaxed)));
    }, 1 << 16);
    RIMO_API_END
}

}  // extern "C"
