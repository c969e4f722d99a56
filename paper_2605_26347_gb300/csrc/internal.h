// Internal declarations of the rimo library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "rimo.h"

namespace rimo {

// ---------------------------------------------------------------------------
// Error handling: every public entry point catches rimo::Error and returns its status.
struct Error {
    rimo_status status;
    std::string msg;
};
void set_last_error(const std::string& msg);
[[noreturn]] void fail(rimo_status s, const std::string& msg);
void check_cuda(cudaError_t e, const char* what);
#define RIMO_CUDA(call) ::rimo::check_cuda((call), #call)

// ---------------------------------------------------------------------------
// Per-visibility metadata in sorted (bin, uv-tile) order, 16 bytes.
//   off  : first tap of the visibility's tile inside its Fourier block (complex units)
//   orig : caller-order index
//   pos  : du | dv << 8 | S << 16 | block << 24, where (du, dv) is the tile's first
//          cell relative to its uv-tile origin and S its side.
struct VisMeta {
    int64_t off;
    uint32_t orig;
    uint32_t pos;
};
static_assert(sizeof(VisMeta) == 16, "VisMeta must stay 16 bytes");

// One uv-tile of one w-bin: the visibilities [vb, ve) of the sorted order whose first
// cell falls in the TS x TS cells starting at (tu * TS, tv * TS).
struct TileDesc {
    int32_t tu, tv;
    int64_t vb, ve;
};

struct BinRange {
    int64_t vb = 0, ve = 0;       // visibilities of the bin in sorted order
    int32_t tile_off[5] = {0, 0, 0, 0, 0};  // tiles of phase q: [tile_off[q], tile_off[q+1])
    float w_hi = 0.f, w_lo = 0.f; // w_stack as a float pair (double-float)
    double w = 0.0;
};

// Constant tables the kernels read.
struct DevTables {
    float2* tw_x = nullptr;    // e^{-2 pi i k / (2 nx)}, k in [0, 2 nx)
    float2* tw_y = nullptr;    // e^{-2 pi i k / (2 ny)}
    float* gc_x = nullptr;     // grid correction 1 / KB_hat, per column
    float* gc_y = nullptr;     // per row
    float2* dn = nullptr;      // (sqrt(1-l^2-m^2)-1) as float pairs, [|i_c|][|j_c|], (ny/2+1) x (nx/2+1)
    float* kb_coef = nullptr;  // Horner coefficients of KB(t) in rho = 1 - (2t/J)^2
    int kb_nterm = 0;
    float* wk_dn = nullptr;    // w-kernel grid: (sqrt(1-lam^2-mu^2)-1), L x L (float)
    float* wk_tau_x = nullptr; // taper along lam
    float* wk_tau_y = nullptr; // taper along mu
    float2* wk_E = nullptr;    // E[a][t + hmax] = e^{+2 pi i t (a - L/2) / L}, L x (2 hmax + 1)
};

}  // namespace rimo

// The plan object behind rimo_plan_t.
struct rimo_plan {
    rimo_plan_params prm{};
    rimo_plan_info info{};
    int nx = 0, ny = 0, gx = 0, gy = 0;
    int J = 7, TS = 64, H = 0, PW = 0, L = 32, hmax = 0, max_S = 0;
    double beta = 0.0;
    int64_t M = 0;
    int P = 0, mode = 0;
    std::vector<double> w_stack;
    std::vector<int32_t> bins_user, sw_user;
    std::vector<int32_t> inv_perm;               // caller index -> sorted position
    std::vector<rimo::BinRange> bins;
    std::vector<rimo::TileDesc> tiles_host;      // all bins, grouped by (bin, phase)
    std::vector<int64_t> block_bytes;
    bool holographic = false;

    // device
    rimo::VisMeta* d_meta = nullptr;
    rimo::TileDesc* d_tiles = nullptr;
    std::vector<float2*> d_gblocks;
    float2** d_gblock_ptrs = nullptr;
    float* d_wr = nullptr;     // residual w per visibility (sorted order)
    float* d_phiu = nullptr;   // fractional offsets (sorted order)
    float* d_phiv = nullptr;
    float2* d_X = nullptr;     // forward grid   (gx rows u, gy cols v)
    float2* d_Xh = nullptr;    // gridded grid
    float2* d_AB = nullptr;    // half-transformed intermediates (2 nx ny)
    float2* d_delta = nullptr; // delta image for the PSF
    rimo::DevTables tab;
    std::vector<void*> owned;  // every cudaMalloc of the plan
};

namespace rimo {

void* dev_alloc(rimo_plan* p, size_t bytes);

// Kernel launchers (defined in the .cu files).
void launch_fwd_rows(const rimo_plan* p, int bin, const float2* x, float2* At, cudaStream_t s);
void launch_fwd_cols(const rimo_plan* p, const float2* At, float2* X, cudaStream_t s);
void launch_inv_cols(const rimo_plan* p, const float2* Xh, float2* B, cudaStream_t s);
void launch_inv_rows(const rimo_plan* p, int bin, const float2* B, float2* out, int accumulate,
                     int real_only, cudaStream_t s);
// mode 0: degrid (y_out), 1: grid (y_in), 2: fused degrid + grid
void launch_gtg(const rimo_plan* p, int bin, int mode, const float2* X, float2* Xh,
                const float2* y_in, float2* y_out, cudaStream_t s);
void launch_gbuild(const rimo_plan* p, cudaStream_t s);

}  // namespace rimo
