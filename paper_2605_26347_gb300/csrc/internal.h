// Internal declarations of the rimo library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "rimo.h"

namespace rimo {
// visibilities per tap-ring chunk of the grid step, one per consumer warp
constexpr int GTG_CHUNK = 20;

// ---------------------------------------------------------------------------
// Error handling: every public entry point catches rimo::Error and returns its status.
struct Error {
    rimo_status status;
    std::string msg;
};
void set_last_error(const std::string& msg);

// Body of a C-ABI entry point: errors become status codes and rimo_last_error().
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
[[noreturn]] void fail(rimo_status s, const std::string& msg);
void check_cuda(cudaError_t e, const char* what);
// Parameter and coordinate checks of plan creation (RIMO_ERR_INVALID_ARG on failure).
void validate_params(const rimo_plan_params& q);
void validate_uvw(const double* uvw, int64_t M, const rimo_plan_params& q);
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
// Fourier-block number (pos >> 24) of a visibility that a shard plan does not hold: it has
// no taps, and the G build passes it by
constexpr uint32_t SHARD_SKIP = 255;

// One uv-tile of one w-bin: the visibilities [vb, ve) of the sorted order whose first
// cell falls in the TS x TS cells starting at (tu * TS, tv * TS).
struct TileDesc {
    int32_t tu, tv;
    int64_t vb, ve;
    int64_t cb;   // index of the unit's first chunk descriptor
    // the unit's box within its patch: the cells [a0, a1) x [b0, b1) its footprints reach
    // (a0 | a1 << 8 | b0 << 16 | b1 << 24); the whole patch for the units of a split tile
    uint32_t box;
    uint32_t pad_;
};
__host__ __device__ inline uint32_t box_pack(int a0, int a1, int b0, int b1) {
    return (uint32_t)a0 | ((uint32_t)a1 << 8) | ((uint32_t)b0 << 16) | ((uint32_t)b1 << 24);
}

// One chunk of at most GTG_CHUNK consecutive visibilities of a unit: their taps are the byte
// range [8 off, 8 off + bytes) of Fourier block `block`.
struct ChunkDesc {
    int64_t off;
    uint32_t bytes;
    uint32_t block;
};
static_assert(sizeof(ChunkDesc) == 16, "ChunkDesc must stay 16 bytes");

struct BinRange {
    int64_t vb = 0, ve = 0;       // visibilities of the bin in sorted order
    int32_t t0 = 0, t1 = 0;       // work units of the bin: tiles_host[t0 .. t1) (patch slots 0 ..)
    int32_t m0 = 0, m1 = 0;       // merge groups (split tiles) of the bin: merge_host[m0 .. m1)
    int32_t n0 = 0, n1 = 0;       // needed tiles of the bin: d_need_list[n0 .. n1)
    float w_hi = 0.f, w_lo = 0.f; // w_stack as a float pair (double-float)
    double w = 0.0;
};

// Constant tables the kernels read.
struct DevTables {
    float2* tws_x = nullptr;   // Stockham stage twiddle tables for the 2 nx-point transforms
    float2* tws_y = nullptr;   // ... and the 2 ny-point transforms
    float2* tws32 = nullptr;   // 8192-point transforms with 32 points per thread (radix 32, 16,
                               // 16): W_512^{r j} at [r 32 + j], W_8192^{r j} at [512 + r 512 + j]
    float4* zq = nullptr;      // [|i_c|][|j_c|], (ny/2+1) x (nx/2+1): sqrt(1-l^2-m^2)-1 as a float pair, |Z_p|
    float* kb_coef = nullptr;  // Horner coefficients of KB(t) in rho = 1 - (2t/J)^2
    int kb_nterm = 0;
    // w-kernel grid folded over the signs of (lam, mu): a', b' in [0, L/2], lam = a' 2 fov_x / L
    float* wk_dn = nullptr;    // sqrt(1 - lam^2 - mu^2) - 1, (L/2 + 1)^2
    float* wk_tau_x = nullptr; // taper along lam, L/2 + 1
    float* wk_tau_y = nullptr; // taper along mu, L/2 + 1
    float* wk_wc = nullptr;    // w(a', t) = m(a') cos(2 pi a' t / L), m = 1 at a' = 0, L/2 else 2; (L/2 + 1) x 8 (t in [0, 4])
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
    std::vector<rimo::TileDesc> tiles_host;      // work units (uv-tiles or parts), grouped by bin
    std::vector<int32_t> sched_host;             // per bin: unit indices, heaviest first
    std::vector<int2> merge_host;                // per bin: (first slot, units) of split tiles
    std::vector<int64_t> block_bytes;

    // device
    rimo::VisMeta* d_meta = nullptr;
    rimo::TileDesc* d_tiles = nullptr;
    int32_t* d_sched = nullptr;
    rimo::ChunkDesc* d_chunks = nullptr;
    int2* d_merge = nullptr;
    std::vector<float2*> d_gblocks;
    float2** d_gblock_ptrs = nullptr;
    float* d_wr = nullptr;     // residual w per visibility (sorted order)
    float* d_phiu = nullptr;   // fractional offsets (sorted order)
    float* d_phiv = nullptr;
    float2* d_X = nullptr;     // forward grid   (gx rows u, gy cols v)
    float2* d_patch = nullptr; // gridded accumulator patch of every active tile of one bin
    int2* d_slot = nullptr;    // [bin][tu][tv] -> (index of the tile's patch in d_patch, or -1;
                               //   the box of that patch, TileDesc::box)
    uint8_t* d_need = nullptr; // [bin][tu][tv] != 0: some active patch of the bin reads the tile
    int32_t* d_need_list = nullptr;  // per bin: the needed tiles as tu * ntv + tv
    int32_t* d_counter = nullptr;  // per-bin dynamic tile schedulers (reset at each apply)
    int32_t* d_status = nullptr;   // device-side error flag (bounded waits)
    uint32_t* d_fx = nullptr;      // fixed-point grid-step bounds (layout: rimo::FX_*)
    int max_tiles_bin = 0, chunk_vis = rimo::GTG_CHUNK, chunk_bytes = 0, nbuf = 4, n_sm = 0;
    int device = 0;                // CUDA device the plan lives on
    int test_stall = 0;            // failure-detection test of the grid step's bounded waits
    uint32_t test_polls = 0;       // (rimo_plan_set_wait_test)
    std::vector<int32_t> need_host;  // needed tiles of all bins (host copy of d_need_list)
    std::vector<std::vector<uint16_t>> trows;  // per bin: uv-tile rows (tu) holding a needed tile
    float2* d_kwtab = nullptr;  // tabulated folded w-kernels (wkernel_table > 0), (kw_n + 3) x 25
    int kw_n = 0;
    double kw_w0 = 0.0, kw_dw = 0.0;  // sample j at w = kw_w0 + j kw_dw
    float* d_wt = nullptr;      // data weights in sorted order (null: no weighting)
    float* d_wt_buf = nullptr;  // their buffer (kept when the weighting is removed)

    // kernel surrogate (mode RIMO_MODE_SURROGATE) or exact on-the-fly tiles (mode
    // RIMO_MODE_ONTHEFLY): tiles generated per bin at apply time
    struct rimo_surrogate* sur = nullptr;  // attached by rimo_plan_set_surrogate (not owned)
    float2* d_sur_taps = nullptr;          // one bin's taps, laid out like its G block
    int64_t sur_taps_bytes = 0;

    // holographic matrices (Section 3.3), once rimo_build_holographic has run.  Each pair of
    // cells (c1, c2) of H_p = G_p^dagger G_p with |c2 - c1| <= H per axis is stored once, at
    // its owner: the cell at the top-left corner of the pair's bounding box (see hmat.cu).
    bool h_built = false;
    int h_ne = 0;                         // entries per owner cell: (H+1)^2 + H^2
    // owner rows, per bin either dense (all h_ne entries per row) or keeping their non-zero
    // entries only (Section 3.3: H is sparse), whichever is smaller: per bin
    std::vector<float2*> d_hval;          //   the values, owner row after owner row
    std::vector<uint16_t*> d_hidx;        //   compressed: their entry numbers e < h_ne
    std::vector<int64_t*> d_hroff;        //   compressed: [owner + 1] first value of each row
    std::vector<uint8_t> h_dense;         //   1: the bin's rows are dense
    std::vector<uint32_t*> d_htmax;       // per bin: [needed tile] max |h.x| + |h.y| (float bits)
    std::vector<uint32_t*> d_hbits;       // per bin: [needed tile][TS*TS/32] covered cells
    std::vector<int64_t*> d_hoff;         // per bin: [needed tile + 1] first owner of the tile
    std::vector<std::vector<int64_t>> hoff_host;
    int32_t* d_hslot = nullptr;           // [bin][tile] -> needed-tile index in the bin, or -1
    float2* d_hpatch = nullptr;           // H-apply output patches of one bin [needed tile][PW*PW]
    int32_t* d_hent = nullptr;            // entry table (type << 16 | a << 8 | |b|)
    float2* d_AB = nullptr;    // half-transformed intermediates (2 nx ny)
    float2* d_delta = nullptr; // delta image for the PSF
    rimo::DevTables tab;
    std::vector<void*> owned;  // every cudaMalloc of the plan

    // stage timers
    bool prof_on = false;
    struct Mark { int stage; int launches; cudaEvent_t a, b; };
    std::vector<Mark> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    double prof_ms[RIMO_N_STAGES] = {0};
    int64_t prof_launches[RIMO_N_STAGES] = {0};
    int prof_open_stage = -1;
    cudaEvent_t prof_open_event = nullptr;
};

namespace rimo {

void* dev_alloc(rimo_plan* p, size_t bytes);

// Device copy of a host vector, owned by the plan (freed in rimo_plan_destroy).
template <class T>
T* upload_vec(rimo_plan* p, const std::vector<T>& v, cudaStream_t s) {
    T* d = (T*)dev_alloc(p, v.size() * sizeof(T));
    if (!v.empty()) {
        const cudaError_t e = cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) fail(RIMO_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
    }
    return d;
}

enum Stage { ST_FWD_ROWS = 0, ST_FWD_COLS = 1, ST_CLEAR = 2, ST_GTG = 3, ST_INV_COLS = 4,
             ST_INV_ROWS = 5, ST_GBUILD = 6, ST_HBUILD = 7, ST_HAPPLY = 8, ST_MLP = 9, ST_BOUND = 10 };

constexpr int FX_HMAX = 5;      // max over entries of H of |h.x| + |h.y| (float bits)
constexpr int FX_BX = 6;        // image bound B_x of the current Phi^dagger Phi apply (float)
constexpr int FX_YB = 7;        // max |y.x| + |y.y| of the current Phi^dagger apply (float)

// Fixed-point grid step.  The grid step accumulates each tile patch in two 32-bit integer
// words per real number (hi: the contribution scaled by a power of two s and rounded;
// lo: the rounding residual scaled by 2^16 more), so that the sums are exact integer sums
// (independent of the order of the additions) of the FP32 contributions, to 2^-16 / s.
// s is chosen per work unit from an a-priori bound on every contribution ("maxterm"),
// and the number n of visibilities of the unit: |hi| <= n 2^21 s-scaled terms stay below
// 2^31, |lo| <= n 2^15 likewise for n < 2^16.
// d_fx layout (32-bit words):
constexpr int FX_TMAX = 0;      // max over taps of |t.x| + |t.y| (float bits; plan time)
constexpr int FX_T1 = 1;        // max over visibilities of sum over taps of |t.x| + |t.y|
constexpr int FX_MAXTERM = 2;   // bound on |contribution| of a Phi^dagger Phi apply from the image (float)
constexpr int FX_YMAX = 3;      // running max of |y.x| + |y.y| (float bits)
constexpr int FX_COUNT = 4;     // blocks done (last-block reduction)
constexpr int FX_PART = 64;     // per-block partial sums
constexpr int FX_NPART = 1024;
constexpr int FX_WORDS = FX_PART + FX_NPART;
constexpr int FX_MAX_UNIT = 32768;  // visibilities per work unit (lo word range)
// Bracket a group of `launches` kernel launches of one stage on stream s (no-op when off).
void prof_begin(rimo_plan* p, int stage, cudaStream_t s);
void prof_end(rimo_plan* p, int launches, cudaStream_t s);

// Kernel launchers (defined in the .cu files).
void launch_fwd_rows(const rimo_plan* p, int bin, const float2* x, float2* At, cudaStream_t s);
void launch_fwd_cols(const rimo_plan* p, int bin, const float2* At, float2* X, cudaStream_t s);
// folds the tile patches of bin `bin` into the gridded grid (in d_X, no longer needed by
// then) and runs the inverse cols pass on it
void launch_inv_cols(const rimo_plan* p, int bin, float2* B, cudaStream_t s);
void launch_inv_rows(const rimo_plan* p, int bin, const float2* B, float2* out, int accumulate,
                     int real_only, cudaStream_t s);
// mode 0: degrid (y_out), 1: grid (y_in), 2: fused degrid + grid.  Modes 1 and 2 write the
// accumulator patch of every active tile of the bin to p->d_patch.
void launch_gtg(const rimo_plan* p, int bin, int mode, const float2* y_in, float2* y_out,
                cudaStream_t s);
void launch_gbuild(const rimo_plan* p, cudaStream_t s);
// exact tiles of the sorted visibilities [v0, v0 + n) into their block (the on-the-fly mode's
// scratch), with the tap bounds of the fixed-point grid step
void launch_kwtab(const rimo_plan* p, cudaStream_t s);
void launch_gbuild_range(const rimo_plan* p, int64_t v0, int64_t n, cudaStream_t s);

// ---------------------------------------------------------------------------
// Stage-batched applies (wideband batches): one (plan, w-bin) of the batch and the scratch
// it uses; every pass of Phi^dagger Phi runs as one launch over all jobs.
struct WideJob {
    const rimo_plan* p;
    int bin;
    int group;        // the channel: index of its (x, out) image pair
    float2* AB;       // half-transformed rows, 2 nx ny
    float2* X;        // forward grid, then the folded gridded grid, gx gy
    float2* patch;    // tile patches of the bin's work units, (t1 - t0) PW^2
};
// Job of block b of a launch over a job table: the last job whose first block is <= b
// (first: njobs + 1 non-decreasing block offsets).
__device__ __forceinline__ int job_of(const int* first, int njobs, int b) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(first + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
struct WideFft;   // device job tables of the transform passes (fft.cu)
struct WideGtg;   // device unit queue of the grid step (grid.cu)
WideFft* wide_fft_create(const std::vector<WideJob>& jobs, const std::vector<const float2*>& x,
                         const std::vector<float2*>& out, cudaStream_t s);
void wide_fft_destroy(WideFft* w);
void wide_fwd(const WideFft* w, cudaStream_t s);                 // F Z_p of every job
void wide_inv(const WideFft* w, int real_only, cudaStream_t s);  // fold, Z_p^H F^H, Sigma_p per channel
WideGtg* wide_gtg_create(const std::vector<WideJob>& jobs, cudaStream_t s);
void wide_gtg_destroy(WideGtg* w);
int64_t wide_gtg_units(const WideGtg* w);
void wide_gtg(const WideGtg* w, cudaStream_t s);  // G_p^H G_p of every job: one persistent launch

// The three applies on stream s (defined in apply.cu).
void apply_phi(rimo_plan* p, const float2* x, float2* y, cudaStream_t s);
void apply_phi_adj(rimo_plan* p, const float2* y, float2* x, cudaStream_t s);
void apply_phi_adj_phi(rimo_plan* p, const float2* x, float2* out, int real_only, cudaStream_t s);
// the same over the bins with mask[b] != 0 (mask: host, P entries; NULL: all bins)
void apply_phi_adj_phi_bins(rimo_plan* p, const float2* x, float2* out, int real_only, const uint8_t* mask,
                            cudaStream_t s);
// bound on the grid-step contributions of Phi^dagger Phi x (from the image x) or of
// Phi^dagger y (from y), written to d_fx[FX_MAXTERM]; non-finite input sets status 3
void launch_image_bound(const rimo_plan* p, const float2* x, cudaStream_t s);
// Z_p of bin `bin` at every pixel into out (ny x nx)
void launch_zlayer(const rimo_plan* p, int bin, float2* out, cudaStream_t s);
void launch_y_bound(const rimo_plan* p, const float2* y, cudaStream_t s);
// Kernel surrogate: fill d_sur_taps with the MLP's tiles of bin `bin` (and the tap bounds
// of the fixed-point grid step); reset_surrogate_bounds clears those bounds for an apply.
int surrogate_generate(rimo_plan* p, int bin, cudaStream_t s);  // returns kernel launches
void reset_surrogate_bounds(rimo_plan* p, cudaStream_t s);
// Holographic apply of bin `bin` (forward grid in d_X -> output patches in d_hpatch).
void launch_happly(const rimo_plan* p, int bin, cudaStream_t s);
// Fold of the patches of bin `bin` (GTG's or the holographic ones) into d_X and the
// inverse cols pass.
void launch_inv_cols_from(const rimo_plan* p, int bin, bool holographic, float2* B, cudaStream_t s);

}  // namespace rimo
