// Application of Phi (Eq. 6), Phi^dagger and Phi^dagger Phi (Eq. 7, Eq. 8) and the PSF.
// Per w-bin p the work is a fixed sequence of launches on the caller's stream:
//   F Z_p        : forward rows pass, forward cols pass          (fft.cu)
//   G_p / G_p^H  : uv-tile de-grid / grid / fused G^H G           (grid.cu)
//   Z_p^H F^H    : inverse cols pass, inverse rows pass (+ accumulate over p)
#include "internal.h"

namespace rimo {

static cudaEvent_t prof_event(rimo_plan* p) {
    if (!p->prof_pool.empty()) {
        cudaEvent_t e = p->prof_pool.back();
        p->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    RIMO_CUDA(cudaEventCreate(&e));
    return e;
}

void prof_begin(rimo_plan* p, int stage, cudaStream_t s) {
    if (!p->prof_on) return;
    p->prof_open_stage = stage;
    p->prof_open_event = prof_event(p);
    RIMO_CUDA(cudaEventRecord(p->prof_open_event, s));
}

void prof_end(rimo_plan* p, int launches, cudaStream_t s) {
    if (!p->prof_on || p->prof_open_stage < 0) return;
    cudaEvent_t b = prof_event(p);
    RIMO_CUDA(cudaEventRecord(b, s));
    p->prof_pending.push_back({p->prof_open_stage, launches, p->prof_open_event, b});
    p->prof_open_stage = -1;
    p->prof_open_event = nullptr;
}

static void prof_collect(rimo_plan* p) {
    for (auto& m : p->prof_pending) {
        RIMO_CUDA(cudaEventSynchronize(m.b));
        float ms = 0.f;
        RIMO_CUDA(cudaEventElapsedTime(&ms, m.a, m.b));
        p->prof_ms[m.stage] += ms;
        p->prof_launches[m.stage] += m.launches;
        p->prof_pool.push_back(m.a);
        p->prof_pool.push_back(m.b);
    }
    p->prof_pending.clear();
}

static int gtg_launches(const rimo_plan* p, int b, int mode) {
    (void)mode;
    return p->bins[b].t1 > p->bins[b].t0 ? 1 : 0;
}

static void check_plan(rimo_plan* p) {
    if (!p) fail(RIMO_ERR_INVALID_ARG, "null plan");
}

static bool bin_empty(const rimo_plan* p, int b) { return p->bins[b].ve == p->bins[b].vb; }

static void zero_image(rimo_plan* p, rimo_cfloat* out, cudaStream_t s) {
    RIMO_CUDA(cudaMemsetAsync(out, 0, (size_t)p->nx * p->ny * sizeof(float2), s));
}

static void fwd(rimo_plan* p, int b, const float2* x, cudaStream_t s) {
    prof_begin(p, ST_FWD_ROWS, s);
    launch_fwd_rows(p, b, x, p->d_AB, s);
    prof_end(p, 1, s);
    prof_begin(p, ST_FWD_COLS, s);
    launch_fwd_cols(p, b, p->d_AB, p->d_X, s);
    prof_end(p, 1, s);
}

static void reset_schedulers(rimo_plan* p, cudaStream_t s) {
    RIMO_CUDA(cudaMemsetAsync(p->d_counter, 0, (size_t)p->P * sizeof(int32_t), s));
}

static void inv(rimo_plan* p, int b, float2* out, bool first, int real_only, cudaStream_t s, bool holo = false) {
    prof_begin(p, ST_INV_COLS, s);
    launch_inv_cols_from(p, b, holo, p->d_AB, s);
    prof_end(p, p->bins[b].n1 > p->bins[b].n0 ? 2 : 1, s);
    prof_begin(p, ST_INV_ROWS, s);
    launch_inv_rows(p, b, p->d_AB, out, first ? 0 : 1, real_only, s);
    prof_end(p, 1, s);
}

static void gtg(rimo_plan* p, int b, int mode, const float2* y_in, float2* y_out, cudaStream_t s) {
    if (p->mode == RIMO_MODE_SURROGATE) {
        prof_begin(p, ST_MLP, s);
        const int nl = surrogate_generate(p, b, s);  // this bin's tiles into the tap scratch
        prof_end(p, nl, s);
    } else if (p->mode == RIMO_MODE_ONTHEFLY || p->mode == RIMO_MODE_HOLOGRAPHIC) {
        prof_begin(p, ST_GBUILD, s);
        launch_gbuild_range(p, p->bins[b].vb, p->bins[b].ve - p->bins[b].vb, s);  // exact tiles
        prof_end(p, 1, s);
    }
    prof_begin(p, ST_GTG, s);
    launch_gtg(p, b, mode, y_in, y_out, s);
    const bool merge = mode != 0 && p->bins[b].m1 > p->bins[b].m0;
    prof_end(p, gtg_launches(p, b, mode) + (merge ? 1 : 0), s);
}

static void begin_apply(rimo_plan* p, cudaStream_t s) {
    reset_schedulers(p, s);
    if (p->mode == RIMO_MODE_SURROGATE && !p->sur)
        fail(RIMO_ERR_STATE, "surrogate plan without a surrogate (rimo_plan_set_surrogate)");
    if (p->mode != RIMO_MODE_STORED_G) reset_surrogate_bounds(p, s);  // tap bounds of generated tiles
}

void apply_phi(rimo_plan* p, const float2* x, float2* y, cudaStream_t s) {
    begin_apply(p, s);
    for (int b = 0; b < p->P; ++b) {
        if (bin_empty(p, b)) continue;
        fwd(p, b, x, s);
        gtg(p, b, 0, nullptr, y, s);
    }
}

void apply_phi_adj(rimo_plan* p, const float2* y, float2* x, cudaStream_t s) {
    bool first = true;
    begin_apply(p, s);
    prof_begin(p, ST_BOUND, s);
    launch_y_bound(p, y, s);
    prof_end(p, p->M > 0 ? 1 : 0, s);
    for (int b = 0; b < p->P; ++b) {
        if (bin_empty(p, b)) continue;
        gtg(p, b, 1, y, nullptr, s);
        inv(p, b, x, first, 0, s);
        first = false;
    }
    if (first) zero_image(p, (rimo_cfloat*)x, s);
}

void apply_phi_adj_phi(rimo_plan* p, const float2* x, float2* out, int real_only, cudaStream_t s) {
    apply_phi_adj_phi_bins(p, x, out, real_only, nullptr, s);
}

void apply_phi_adj_phi_bins(rimo_plan* p, const float2* x, float2* out, int real_only, const uint8_t* mask,
                            cudaStream_t s) {
    bool first = true;
    begin_apply(p, s);
    prof_begin(p, ST_BOUND, s);
    launch_image_bound(p, x, s);
    prof_end(p, 1, s);
    for (int b = 0; b < p->P; ++b) {
        if (bin_empty(p, b) || (mask && !mask[b])) continue;
        fwd(p, b, x, s);
        if (p->h_built) {
            // H_p in place of G_p^dagger G_p (Section 3.3)
            prof_begin(p, ST_HAPPLY, s);
            launch_happly(p, b, s);
            prof_end(p, p->bins[b].n1 > p->bins[b].n0 ? 1 : 0, s);
        } else {
            gtg(p, b, 2, nullptr, nullptr, s);
        }
        inv(p, b, out, first, real_only, s, p->h_built);
        first = false;
    }
    if (first) zero_image(p, (rimo_cfloat*)out, s);
}

}  // namespace rimo

using namespace rimo;


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

rimo_status rimo_apply_phi_adj_phi_bins(rimo_plan_t p, const rimo_cfloat* x, rimo_cfloat* out,
                                        int32_t real_part_only, const uint8_t* bin_mask, void* stream) {
    RIMO_API_BEGIN
    check_plan(p);
    if (!x || !out) fail(RIMO_ERR_INVALID_ARG, "null buffer");
    if ((const void*)x == (const void*)out) fail(RIMO_ERR_INVALID_ARG, "x and out must be distinct");
    apply_phi_adj_phi_bins(p, (const float2*)x, (float2*)out, real_part_only, bin_mask, (cudaStream_t)stream);
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

rimo_status rimo_profile_enable(rimo_plan_t p, int32_t on) {
    RIMO_API_BEGIN
    check_plan(p);
    p->prof_on = on != 0;
    RIMO_API_END
}

rimo_status rimo_profile_read(rimo_plan_t p, double* ms, int64_t* launches, int32_t n,
                              int32_t reset) {
    RIMO_API_BEGIN
    check_plan(p);
    if (n < 0 || n > RIMO_N_STAGES) fail(RIMO_ERR_INVALID_ARG, "n must be in [0, RIMO_N_STAGES]");
    prof_collect(p);
    for (int i = 0; i < n; ++i) {
        if (ms) ms[i] = p->prof_ms[i];
        if (launches) launches[i] = p->prof_launches[i];
    }
    if (reset)
        for (int i = 0; i < RIMO_N_STAGES; ++i) {
            p->prof_ms[i] = 0.0;
            p->prof_launches[i] = 0;
        }
    RIMO_API_END
}

rimo_status rimo_plan_get_zlayer(rimo_plan_t p, int32_t bin, rimo_cfloat* out, void* stream) {
    RIMO_API_BEGIN
    check_plan(p);
    if (!out) fail(RIMO_ERR_INVALID_ARG, "null buffer");
    if (bin < 0 || bin >= p->P) fail(RIMO_ERR_INVALID_ARG, "bin out of range");
    launch_zlayer(p, bin, (float2*)out, (cudaStream_t)stream);
    RIMO_CUDA(cudaGetLastError());
    RIMO_API_END
}

rimo_status rimo_plan_set_wait_test(rimo_plan_t p, int32_t stall, int32_t polls) {
    RIMO_API_BEGIN
    check_plan(p);
    if (stall != 0 && stall != 1) fail(RIMO_ERR_INVALID_ARG, "stall must be 0 or 1");
    if (stall && (polls < 1 || polls > (1 << 15))) fail(RIMO_ERR_INVALID_ARG, "polls must be in [1, 32768]");
    p->test_stall = stall;
    p->test_polls = stall ? (uint32_t)polls : 0u;
    RIMO_API_END
}

rimo_status rimo_plan_status(rimo_plan_t p, void* stream) {
    RIMO_API_BEGIN
    check_plan(p);
    cudaStream_t s = (cudaStream_t)stream;
    int32_t flag = 0;
    RIMO_CUDA(cudaMemcpyAsync(&flag, p->d_status, sizeof(flag), cudaMemcpyDeviceToHost, s));
    RIMO_CUDA(cudaStreamSynchronize(s));
    if (flag != 0) {
        RIMO_CUDA(cudaMemsetAsync(p->d_status, 0, sizeof(int32_t), s));
        RIMO_CUDA(cudaStreamSynchronize(s));
        if (flag == 3) fail(RIMO_ERR_INVALID_ARG, "non-finite input values (or a fixed-point bound overflowed)");
        fail(RIMO_ERR_TIMEOUT, "a bounded device wait ran out (code " + std::to_string(flag) + ")");
    }
    RIMO_API_END
}



}  // extern "C"
