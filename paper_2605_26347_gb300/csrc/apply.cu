// Application of Phi (Eq. 6), Phi^dagger and Phi^dagger Phi (Eq. 7, Eq. 8) and the PSF.
// Per w-bin p the work is a fixed sequence of launches on the caller's stream:
//   F Z_p        : forward rows pass, forward cols pass          (fft.cu)
//   G_p / G_p^H  : uv-tile de-grid / grid / fused G^H G           (grid.cu)
//   Z_p^H F^H    : inverse cols pass, inverse rows pass (+ accumulate over p)
#include "internal.h"

namespace rimo {

static void check_plan(rimo_plan* p) {
    if (!p) fail(RIMO_ERR_INVALID_ARG, "null plan");
}

static bool bin_empty(const rimo_plan* p, int b) { return p->bins[b].ve == p->bins[b].vb; }

static void zero_image(rimo_plan* p, rimo_cfloat* out, cudaStream_t s) {
    RIMO_CUDA(cudaMemsetAsync(out, 0, (size_t)p->nx * p->ny * sizeof(float2), s));
}

void apply_phi(rimo_plan* p, const float2* x, float2* y, cudaStream_t s) {
    for (int b = 0; b < p->P; ++b) {
        if (bin_empty(p, b)) continue;
        launch_fwd_rows(p, b, x, p->d_AB, s);
        launch_fwd_cols(p, p->d_AB, p->d_X, s);
        launch_gtg(p, b, 0, p->d_X, nullptr, nullptr, y, s);
    }
}

void apply_phi_adj(rimo_plan* p, const float2* y, float2* x, cudaStream_t s) {
    bool first = true;
    for (int b = 0; b < p->P; ++b) {
        if (bin_empty(p, b)) continue;
        RIMO_CUDA(cudaMemsetAsync(p->d_Xh, 0, (size_t)p->gx * p->gy * sizeof(float2), s));
        launch_gtg(p, b, 1, nullptr, p->d_Xh, y, nullptr, s);
        launch_inv_cols(p, p->d_Xh, p->d_AB, s);
        launch_inv_rows(p, b, p->d_AB, x, first ? 0 : 1, 0, s);
        first = false;
    }
    if (first) zero_image(p, (rimo_cfloat*)x, s);
}

void apply_phi_adj_phi(rimo_plan* p, const float2* x, float2* out, int real_only, cudaStream_t s) {
    bool first = true;
    for (int b = 0; b < p->P; ++b) {
        if (bin_empty(p, b)) continue;
        launch_fwd_rows(p, b, x, p->d_AB, s);
        launch_fwd_cols(p, p->d_AB, p->d_X, s);
        RIMO_CUDA(cudaMemsetAsync(p->d_Xh, 0, (size_t)p->gx * p->gy * sizeof(float2), s));
        launch_gtg(p, b, 2, p->d_X, p->d_Xh, nullptr, nullptr, s);
        launch_inv_cols(p, p->d_Xh, p->d_AB, s);
        launch_inv_rows(p, b, p->d_AB, out, first ? 0 : 1, real_only, s);
        first = false;
    }
    if (first) zero_image(p, (rimo_cfloat*)out, s);
}

}  // namespace rimo

using namespace rimo;

#define RIMO_API_BEGIN try {
#define RIMO_API_END                  \
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

extern "C" {

rimo_status rimo_apply_phi(rimo_plan_t p, const rimo_cfloat* x, rimo_cfloat* y, void* stream) {
    RIMO_API_BEGIN
    check_plan(p);
    if (!x || !y) fail(RIMO_ERR_INVALID_ARG, "null buffer");
    apply_phi(p, (const float2*)x, (float2*)y, (cudaStream_t)stream);
    RIMO_CUDA(cudaGetLastError());
    RIMO_API_END
}

rimo_status rimo_apply_phi_adj(rimo_plan_t p, const rimo_cfloat* y, rimo_cfloat* x, void* stream) {
    RIMO_API_BEGIN
    check_plan(p);
    if (!x || !y) fail(RIMO_ERR_INVALID_ARG, "null buffer");
    apply_phi_adj(p, (const float2*)y, (float2*)x, (cudaStream_t)stream);
    RIMO_CUDA(cudaGetLastError());
    RIMO_API_END
}

rimo_status rimo_apply_phi_adj_phi(rimo_plan_t p, const rimo_cfloat* x, rimo_cfloat* out,
                                   int32_t real_part_only, void* stream) {
    RIMO_API_BEGIN
    check_plan(p);
    if (!x || !out) fail(RIMO_ERR_INVALID_ARG, "null buffer");
    if ((const void*)x == (const void*)out) fail(RIMO_ERR_INVALID_ARG, "x and out must be distinct");
    apply_phi_adj_phi(p, (const float2*)x, (float2*)out, real_part_only, (cudaStream_t)stream);
    RIMO_CUDA(cudaGetLastError());
    RIMO_API_END
}

rimo_status rimo_psf(rimo_plan_t p, rimo_cfloat* out, void* stream) {
    RIMO_API_BEGIN
    check_plan(p);
    if (!out) fail(RIMO_ERR_INVALID_ARG, "null buffer");
    apply_phi_adj_phi(p, p->d_delta, (float2*)out, 0, (cudaStream_t)stream);
    RIMO_CUDA(cudaGetLastError());
    RIMO_API_END
}

rimo_status rimo_build_holographic(rimo_plan_t p, void* stream) {
    RIMO_API_BEGIN
    check_plan(p);
    (void)stream;
    fail(RIMO_ERR_UNSUPPORTED, "holographic build not available in this build");
    RIMO_API_END
}

}  // extern "C"
