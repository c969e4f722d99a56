// The sparse de-gridding matrix G_p (Section 3.2, Eq. 6): de-grid (G_p), grid
// (G_p^dagger, Eq. 8) and the fused G_p^dagger G_p of Phi^dagger Phi (the build of G's
// tiles is in gbuild.cu).
//
// Layout.  Visibilities of a w-bin are sorted by the uv-tile (TS x TS grid cells)
// holding their first grid cell, and their taps are stored tile after tile, so the
// taps of consecutive visibilities of a tile are one contiguous byte range.
//
// Kernel.  Persistent thread blocks (one per SM) take work units (a uv-tile, or a slice
// of a heavy one) from a heaviest-first schedule: for plans of dense units (8 chunks of
// visibilities or more on average, X patches prefetched) the next one through an atomic
// counter (a block that started late or drew light units takes more; 26.31 -> 25.10 ms per
// 4096^2/50M apply against a fixed snake order), else in the snake order.  For a unit,
// the block stages the box of grid cells its visibilities' footprints reach (within the
// (TS + H)^2 patch, H = largest tile side - 1) in shared memory while a producer warp
// streams the taps of GTG_CHUNK visibilities at a time with bulk asynchronous copies
// (cp.async.bulk, completion on an mbarrier) through a shared-memory ring of up to
// GTG_NBUF chunks.
//   de-grid : one warp per visibility reads its S x S taps from shared memory (lanes = two
//             rows of 16 columns), gathers the patch and reduces y_k with warp shuffles;
//   grid    : the same warp adds conj(taps) y_k into the block's shared accumulator patch
//             (shared-memory atomic adds: visibilities of different warps may overlap).
// The finished accumulator box is written once to the unit's slot of the patch buffer
// (slices of a split tile are then added into its first slot); the fold of the inverse
// transform sums the overlapping halos of neighbouring patches tile by tile, so the gridded
// grid is never cleared or written with global atomics.
#include <algorithm>
#include <cstring>

#include "internal.h"

namespace rimo {

// e / S for e < 400, S <= 19 by multiply-shift with ceil(2^16 / S)
__device__ __forceinline__ int div_small(int e, int magic) { return (e * magic) >> 16; }

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) {
    return (uint32_t)__cvta_generic_to_shared(ptr);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// try_wait suspends the thread until the phase completes or about `hint_ns` elapse.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(100000u)
        : "memory");
    return ok != 0;
}

// Bounded wait: at most `polls` suspended polls of <= 100 us (2^15: about 3 s); never spins
// forever.
constexpr uint32_t WAIT_POLLS = 1u << 15;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t polls = WAIT_POLLS) {
    for (uint32_t it = 0; it < polls; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// The consumers' bounded wait, which also gives up once the block has abandoned the launch
// (the producer stops issuing chunks after a failed wait of its own).
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort) {
    for (uint32_t it = 0; it < WAIT_POLLS; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
    }
    return false;
}

// Bulk asynchronous copy global -> shared (16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

constexpr int GTG_CONSUMERS = GTG_CHUNK;                 // consumer warps
constexpr int GTG_THREADS = (GTG_CONSUMERS + 1) * 32;   // + one producer warp
constexpr int GTG_NBUF = 4;   // maximum depth of the tap ring (the plan may use fewer)
constexpr int GTG_NX = 3;     // maximum number of X patch buffers (prefetch NX - 1 units ahead)
constexpr int GTG_HDR = 256;  // shared-memory header: the ring's and the X buffers' mbarriers
constexpr int GTG_CV = GTG_CHUNK;  // visibilities per chunk (one per consumer warp)

// The per-bin side of a grid-step launch: one (plan, w-bin) job.
struct GtgJob {
    const TileDesc* units;  // the bin's work units, in patch-slot order
    const ChunkDesc* chunks;
    const VisMeta* meta;
    const float2* const* gblk;
    const float2* X;        // forward grid [gx][gy]
    float2* patch;          // accumulator patch per unit slot
    const uint32_t* fx;     // fixed-point bounds (tap bounds; maxterm of a Phi^dagger apply)
    const uint8_t* need;    // [tile] of this bin: some footprint reaches the tile
    int* status;            // the plan's device status word
    int PW;                 // the plan's patch side (TS + largest tile side - 1)
};

struct GtgArgs {
    GtgJob one;             // a one-bin launch: the bin
    const int* sched;       //   its unit slots, heaviest first
    const GtgJob* jobs;     // a stage-batched launch: every (plan, bin) of the batch
    const int2* queue;      //   (job, unit slot) of every unit of every job, heaviest first
    int nunits;             // units of the launch (schedule or queue length)
    int* counter;           // dynamic schedule: the next unit to take (zero at launch), or null
    const float2* y_in;
    float2* y_out;
    int gx, gy, TS, PW;
    int chunk_bytes;
    int nbuf;               // ring depth in use, 2..GTG_NBUF
    int ntv, shift;
    int prefetch;           // the producer bulk-copies the X patches of the next units
    int xbufs;              // X patch buffers with prefetch (2 or 3: 1 or 2 units ahead)
    // failure-detection test (rimo_plan_set_wait_test): the consumers withhold their release
    // of ring slots, and the producer's waits on the consumers give up after peer_polls
    int stall;
    uint32_t peer_polls;    // poll limit of the producer's waits on other warps (empty, xfree)
};

// The job and the patch slot of the launch's unit idx.
template <bool TABLE>
__device__ __forceinline__ const GtgJob* unit_job(const GtgArgs& A, int idx, int& slot) {
    if constexpr (TABLE) {
        const int2 q = A.queue[idx];
        slot = q.y;
        return A.jobs + q.x;
    } else {
        slot = A.sched[idx];
        return &A.one;
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void consumers_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(GTG_CONSUMERS * 32) : "memory");
}

// unit processed by block c in round r: snake order over the heaviest-first schedule
__device__ __forceinline__ int unit_of(int r, int c, int G) { return r * G + ((r & 1) ? (G - 1 - c) : c); }

// rint by the 1.5 x 2^23 shift: for |d| < 2^22, d + FX_MAGIC has unit spacing, so its bits
// minus those of FX_MAGIC are rint(d) (round to nearest even)
constexpr float FX_MAGIC = 12582912.0f;
constexpr int FX_MAGIC_BITS = 0x4B400000;

// Scale of one work unit of n visibilities: the largest power of two s with
// s maxterm <= min(2^21, 2^30 / n) (see the fixed-point layout in internal.h).
__device__ __forceinline__ void fx_scale(float maxterm, int64_t n, float& s1, float& inv) {
    s1 = 1.f;
    inv = 1.f;
    if (!(maxterm > 0.f)) return;  // all contributions vanish (or the input was flagged)
    const float lim = fminf(2097152.f, 1073741824.f / (float)(n > 1 ? n : 1));
    int ex = (int)((__float_as_uint(lim / maxterm) >> 23) & 255u) - 127;
    ex = ex < -120 ? -120 : (ex > 120 ? 120 : ex);
    s1 = __uint_as_float((uint32_t)(ex + 127) << 23);
    inv = __uint_as_float((uint32_t)(127 - ex) << 23);
}

// One visibility by one warp, tile side S known at compile time.
// Lane = (cell column, component): lane 2c + k handles column c of a tap row and the real
// (k = 0) or imaginary (k = 1) part, so one instruction covers one row of up to 16 cells
// (two rows of up to 8 cells when S <= 8): the shared-memory loads of a row are 16
// consecutive complex cells and each grid-step reduction 32 consecutive words, both free
// of bank conflicts.  With a = (t.x, t.y)[k], b = (t.y, t.x)[k]:
//   de-grid:  Re(t x) = sum a x.x - sum b x.y  (k = 0),  Im(t x) = sum a x.x + sum b x.y  (k = 1);
//   grid:     component k of conj(t) y = a (+-y.x) + b y.y  (sign + for k = 0, - for k = 1),
//             times the unit's scale s1, added to the fixed-point patch words hi / lo with
//             32-bit integer reductions.
// Both parity classes of lanes reduce with four butterfly steps; one more exchange gives
// every lane y.  Taps stay in registers between the two steps when S <= 16.
template <int S, int MODE, int PWC>  // PWC: the patch side when known at compile time, else 0
__device__ __forceinline__ void vis_tile(const float2* __restrict__ T, const float2* __restrict__ Xs,
                                         int* Ahi, int* Alo, float s1, int pbase, int PWr, int lane, uint32_t orig,
                                         const float2* __restrict__ y_in, float2* __restrict__ y_out) {
    const int PW = PWC > 0 ? PWC : PWr;  // compile-time row strides fold into the address offsets
    constexpr bool GATHER = MODE != 1, SCATTER = MODE != 0;
    constexpr int RPI = S <= 8 ? 2 : 1;         // tap rows per instruction
    constexpr int CW = 16 / RPI;                // cells per row and instruction
    constexpr int NCG = (S + CW - 1) / CW;      // column groups
    constexpr int NI = (S + RPI - 1) / RPI;     // row steps
    constexpr bool KEEP = NI * NCG <= 16;       // keep (a, b) in registers for the grid step
    const int k = lane & 1;
    const int c = (lane % (2 * CW)) >> 1;
    const int roff = lane / (2 * CW);
    // lane k reads its tap as (component k, component 1 - k): no select on the pair
    const float* Tl = reinterpret_cast<const float*>(T + roff * S + c) + k;
    const int tsw = 1 - 2 * k;  // offset of the other component
    const int xl = pbase + roff * PW + c;
    float2 ab[KEEP ? NI : 1][KEEP ? NCG : 1];
    float acc1 = 0.f, acc2 = 0.f;
#pragma unroll
    for (int i = 0; i < NI; ++i)
#pragma unroll
        for (int j = 0; j < NCG; ++j) {
            const bool ok = (i * RPI + roff < S) && (c + j * CW < S);
            const float* tp = Tl + 2 * (i * RPI * S + j * CW);
            const float2 e = ok ? make_float2(tp[0], tp[tsw]) : make_float2(0.f, 0.f);
            if (KEEP) ab[KEEP ? i : 0][KEEP ? j : 0] = e;
            if (GATHER && ok) {
                const float2 x = Xs[xl + i * RPI * PW + j * CW];
                acc1 = fmaf(e.x, x.x, acc1);
                acc2 = fmaf(e.y, x.y, acc2);
            }
        }
    float2 y;
    if (GATHER) {
        float v = k ? acc1 + acc2 : acc1 - acc2;
        v += __shfl_xor_sync(0xffffffffu, v, 16);
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        const float o = __shfl_xor_sync(0xffffffffu, v, 1);
        y = k ? make_float2(o, v) : make_float2(v, o);
        if (MODE == 0 && lane == 0) y_out[orig] = y;
    } else {
        y = y_in[orig];
    }
    if (SCATTER) {
        const float ysx = (k ? -y.x : y.x) * s1, yys = y.y * s1;
#pragma unroll
        for (int i = 0; i < NI; ++i)
#pragma unroll
            for (int j = 0; j < NCG; ++j) {
                const bool ok = (i * RPI + roff < S) && (c + j * CW < S);
                if (ok) {
                    float2 e;
                    if (KEEP) {
                        e = ab[KEEP ? i : 0][KEEP ? j : 0];
                    } else {
                        const float* tp = Tl + 2 * (i * RPI * S + j * CW);
                        e = make_float2(tp[0], tp[tsw]);
                    }
                    // scaled contribution, |d| <= 2^21, split into rint(d) and 2^16 x residual
                    const float d = fmaf(e.x, ysx, e.y * yys);
                    const float tq = __fadd_rn(d, FX_MAGIC);
                    const int q1 = __float_as_int(tq) - FX_MAGIC_BITS;
                    const float rf = __fsub_rn(d, __fsub_rn(tq, FX_MAGIC));
                    const int q2 = __float_as_int(__fmaf_rn(rf, 65536.f, FX_MAGIC)) - FX_MAGIC_BITS;
                    const int ci = 2 * (xl + i * RPI * PW + j * CW) + k;
                    atomicAdd(Ahi + ci, q1);
                    atomicAdd(Alo + ci, q2);
                }
            }
    }
}

template <int MODE, int PWC>
__device__ __forceinline__ void vis_dispatch(int S, const float2* T, const float2* Xs, int* Ahi, int* Alo, float s1,
                                             int pbase, int PW, int lane, uint32_t orig, const float2* y_in,
                                             float2* y_out) {
    switch (S) {
        case 3: vis_tile<3, MODE, PWC>(T, Xs, Ahi, Alo, s1, pbase, PW, lane, orig, y_in, y_out); break;
        case 5: vis_tile<5, MODE, PWC>(T, Xs, Ahi, Alo, s1, pbase, PW, lane, orig, y_in, y_out); break;
        case 7: vis_tile<7, MODE, PWC>(T, Xs, Ahi, Alo, s1, pbase, PW, lane, orig, y_in, y_out); break;
        case 9: vis_tile<9, MODE, PWC>(T, Xs, Ahi, Alo, s1, pbase, PW, lane, orig, y_in, y_out); break;
        case 11: vis_tile<11, MODE, PWC>(T, Xs, Ahi, Alo, s1, pbase, PW, lane, orig, y_in, y_out); break;
        case 13: vis_tile<13, MODE, PWC>(T, Xs, Ahi, Alo, s1, pbase, PW, lane, orig, y_in, y_out); break;
        case 15: vis_tile<15, MODE, PWC>(T, Xs, Ahi, Alo, s1, pbase, PW, lane, orig, y_in, y_out); break;
        case 17: vis_tile<17, MODE, PWC>(T, Xs, Ahi, Alo, s1, pbase, PW, lane, orig, y_in, y_out); break;
        default: vis_tile<19, MODE, PWC>(T, Xs, Ahi, Alo, s1, pbase, PW, lane, orig, y_in, y_out); break;
    }
}

// Warp-specialised pipeline per block:
//   producer warp : for each chunk (GTG_CHUNK consecutive visibilities of a unit) streams their
//                   16-byte metadata and their taps (one contiguous range, from a chunk
//                   descriptor) into ring slot b with cp.async.bulk, once the consumers
//                   released the slot;
//   consumer warps: wait full[b]; each takes one visibility of the chunk, de-grids it
//                   and grids conj(taps) y_k into the block's shared accumulator patch
//                   (shared-memory reductions, one tap row per instruction:
//                   visibilities of different warps may overlap); then arrive on empty[b].
// Only unit boundaries (patch load / store) synchronise all consumers.
// MODE 0: de-grid (y_out), 1: grid (y_in), 2: fused de-grid + grid; PWC: the patch side
// when known at compile time (the common plans), else 0
// TABLE: the units of many (plan, bin) jobs from one queue (a stage-batched wideband apply).
template <int MODE, int PWC, bool TABLE>
__global__ void __launch_bounds__(GTG_THREADS, 1) gtg_kernel(const __grid_constant__ GtgArgs A) {
    constexpr bool GATHER = MODE != 1, SCATTER = MODE != 0;
    extern __shared__ __align__(128) unsigned char smraw[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smraw);
    uint64_t* empty = full + GTG_NBUF;
    uint64_t* xfull = empty + GTG_NBUF;  // [GTG_NX] X patch buffer landed
    uint64_t* xfree = xfull + GTG_NX;    // [GTG_NX] consumers are done with the buffer
    VisMeta* mring = reinterpret_cast<VisMeta*>(smraw + GTG_HDR);      // GTG_NBUF x GTG_CV entries
    float2* taps = reinterpret_cast<float2*>(smraw + GTG_HDR + GTG_NBUF * GTG_CV * sizeof(VisMeta));
    // shared memory laid out for the launch's largest patch (a staged batch's jobs may have
    // different patch sides; every unit uses its own job's)
    const int PWmax = PWC > 0 ? PWC : A.PW, npmax = PWmax * PWmax;
    const int chunk_f2 = A.chunk_bytes / 8;
    const uint32_t NB = (uint32_t)A.nbuf;
    const bool pre = GATHER && A.prefetch;
    const int NX = pre ? A.xbufs : 1;  // X patch buffers
    // dynamic schedule (with prefetch): blocks take units from a counter in heaviest-first
    // order; otherwise the static snake order
    const bool dyn = pre && A.counter != nullptr;
    float2* Xbuf0 = taps + (size_t)NB * chunk_f2;
    int* Ahi = reinterpret_cast<int*>(Xbuf0 + (GATHER ? (size_t)NX * npmax : 0));  // [cell][re, im] words
    int* Alo = Ahi + (SCATTER ? 2 * npmax : 0);
    __shared__ volatile int s_abort;
    __shared__ volatile int s_fail;           // dynamic schedule: a consumer's wait gave up
    __shared__ volatile int s_unit[GTG_NX];   // dynamic schedule: the unit of round q (q % NX)
    __shared__ float s_xmax[GTG_CONSUMERS];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, cb = blockIdx.x;
    if (tid == 0) {
        for (int b = 0; b < GTG_NBUF; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], GTG_CONSUMERS);
        }
        for (int b = 0; b < GTG_NX; ++b) {
            mbar_init(&xfull[b], 1);
            mbar_init(&xfree[b], GTG_CONSUMERS);
        }
        s_abort = 0;
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == GTG_CONSUMERS) {
        // ------------------------------------------------------------ producer
        if (lane != 0) return;
        uint32_t g = 0;
        int xq = 0;         // the next round whose X patch is to be copied
        bool ended = false;  // dynamic schedule: the end of the work was published
        int* const status0 = TABLE ? A.jobs[0].status : A.one.status;
        for (int r = 0;; ++r) {
            int idx = 0;
            if (!dyn) {
                idx = unit_of(r, cb, G);
                if (idx >= A.nunits) break;
            }
            // X patches of rounds r .. r + NX - 2 (buffer q % NX, once the consumers released
            // it after round q - NX); rows wrap along u, a row past the last column splits in
            // two.  Dynamic schedule: round q's unit is the next of the launch's heaviest-first
            // order (one atomic per unit), published in s_unit[q % NX] with the copy's barrier
            // (-1 after the last unit: a plain arrival)
            while (pre && !ended && xq <= r + NX - 2) {
                int iq = 0;
                if (!dyn) {
                    iq = unit_of(xq, cb, G);
                    if (iq >= A.nunits) break;
                }
                const int j = xq % NX;
                if (xq >= NX && !s_abort &&
                    !mbar_wait_bounded(&xfree[j], ((xq / NX) - 1) & 1, A.peer_polls)) {
                    s_abort = 1;
                    atomicExch(status0, 1);
                }
                if (s_abort) break;
                if (dyn) {
                    const int gi = atomicAdd(A.counter, 1);
                    iq = gi < A.nunits ? gi : -1;
                    s_unit[j] = iq;
                    if (iq < 0) {
                        mbar_arrive(&xfull[j]);
                        ended = true;
                        ++xq;
                        break;
                    }
                }
                int sq;
                const GtgJob* Jq = unit_job<TABLE>(A, iq, sq);
                const TileDesc tq = Jq->units[sq];
                const int PW = PWC > 0 ? PWC : (TABLE ? Jq->PW : A.PW);
                float2* dst = Xbuf0 + (size_t)j * npmax;
                const int u0 = tq.tu * A.TS, v0 = tq.tv * A.TS;
                const int n1 = (v0 + PW <= A.gy) ? PW : A.gy - v0;  // cells before the wrap
                // the rows of the unit's box, its columns widened to whole 16-byte pairs
                // (PW, TS, gy and n1 are even)
                const int a0 = (int)(tq.box & 255u), a1 = (int)((tq.box >> 8) & 255u);
                const int c0 = (int)((tq.box >> 16) & 254u), c1 = min(PW, (int)(((tq.box >> 24) + 1u) & 254u));
                const int w1 = max(0, min(c1, n1) - c0), cs = max(c0, n1), w2 = max(0, c1 - cs);
                mbar_arrive_expect_tx(&xfull[j], (uint32_t)((a1 - a0) * (w1 + w2) * (int)sizeof(float2)));
                for (int a = a0; a < a1; ++a) {
                    int gu = u0 + a;
                    if (gu >= A.gx) gu -= A.gx;
                    const float2* row = Jq->X + (size_t)gu * A.gy;
                    if (w1 > 0) bulk_g2s(dst + a * PW + c0, row + v0 + c0, (uint32_t)(w1 * sizeof(float2)), &xfull[j]);
                    if (w2 > 0) bulk_g2s(dst + a * PW + cs, row + (cs - n1), (uint32_t)(w2 * sizeof(float2)), &xfull[j]);
                }
                ++xq;
            }
            if (s_abort) {
                // let the copies already in flight land before the block may exit
                for (uint32_t q = (g > NB ? g - NB : 0); q < g; ++q)
                    (void)mbar_wait_bounded(&full[q % NB], (q / NB) & 1);
                for (int q = (xq > NX ? xq - NX : 0); q < xq; ++q)
                    (void)mbar_wait_bounded(&xfull[q % NX], (q / NX) & 1);
                return;
            }
            if (dyn) {
                idx = s_unit[r % NX];  // written by this thread in the loop above
                if (idx < 0) break;
            }
            int slot;
            const GtgJob* J = unit_job<TABLE>(A, idx, slot);
            const TileDesc td = J->units[slot];
            const int nchunks = (int)((td.ve - td.vb + GTG_CV - 1) / GTG_CV);
            for (int c = 0; c < nchunks; ++c, ++g) {
                const ChunkDesc cd = J->chunks[td.cb + c];
                const int64_t v0 = td.vb + (int64_t)c * GTG_CV;
                const uint32_t nv = (uint32_t)((td.ve - v0) < GTG_CV ? (td.ve - v0) : GTG_CV);
                const uint32_t b = g % NB, use = g / NB;
                if (use > 0 && !s_abort && !mbar_wait_bounded(&empty[b], (use - 1) & 1, A.peer_polls)) {
                    s_abort = 1;
                    atomicExch(J->status, 1);
                }
                if (s_abort) {
                    // let the copies already in flight land before the block may exit
                    for (uint32_t q = (g > NB ? g - NB : 0); q < g; ++q)
                        (void)mbar_wait_bounded(&full[q % NB], (q / NB) & 1);
                    for (int q = (xq > NX ? xq - NX : 0); q < xq; ++q)
                        (void)mbar_wait_bounded(&xfull[q % NX], (q / NX) & 1);
                    return;
                }
                mbar_arrive_expect_tx(&full[b], cd.bytes + nv * (uint32_t)sizeof(VisMeta));
                bulk_g2s(mring + b * GTG_CV, J->meta + v0, nv * (uint32_t)sizeof(VisMeta), &full[b]);
                bulk_g2s(taps + (size_t)b * chunk_f2, J->gblk[cd.block] + cd.off, cd.bytes, &full[b]);
            }
        }
        return;
    }

    // ---------------------------------------------------------------- consumers
    uint32_t g = 0;
    for (int r = 0;; ++r) {
        int idx;
        if (dyn) {
            // the round's unit as the producer published it; a failed wait (abort) records
            // s_fail, and every consumer warp decides to stop from s_fail and the unit after
            // the barrier below, all alike
            const bool ok = !s_abort && mbar_wait_or_abort(&xfull[r % NX], (r / NX) & 1, &s_abort);
            if (!ok) s_fail = 1;
            idx = ok ? s_unit[r % NX] : -1;
        } else {
            idx = unit_of(r, cb, G);
            if (idx >= A.nunits) break;
        }
        const bool have = idx >= 0;
        int slot = 0;
        const GtgJob* J = have ? unit_job<TABLE>(A, idx, slot) : (TABLE ? A.jobs : &A.one);
        TileDesc td;
        if (have) {
            td = J->units[slot];
        } else {  // no unit: nothing to stage or process
            td.tu = td.tv = 0;
            td.vb = td.ve = td.cb = 0;
            td.box = 0u;
        }
        const int nchunks = (int)((td.ve - td.vb + GTG_CV - 1) / GTG_CV);
        const int PW = PWC > 0 ? PWC : (TABLE ? J->PW : A.PW), npatch = PW * PW;
        const int u0 = td.tu * A.TS, v0 = td.tv * A.TS;
        // the unit's box: the only cells its footprints read and write
        const int ba0 = (int)(td.box & 255u), ba1 = (int)((td.box >> 8) & 255u);
        const int bb0 = (int)((td.box >> 16) & 255u), bb1 = (int)(td.box >> 24);
        float xm = 0.f;
        float2* Xs = Xbuf0 + (pre ? (size_t)(r % NX) * npmax : 0);
        if (!dyn && pre && !s_abort && !mbar_wait_or_abort(&xfull[r % NX], (r / NX) & 1, &s_abort)) {
            s_abort = 1;
            atomicExch(J->status, 1);
        }
        for (int a = ba0 + warp; a < ba1; a += GTG_CONSUMERS) {
            int gu = u0 + a;
            if (gu >= A.gx) gu -= A.gx;
            for (int b = bb0 + lane; b < bb1; b += 32) {
                if (GATHER) {
                    float2 x;
                    if (pre) {
                        x = Xs[a * PW + b];  // landed by the producer (cells outside the bin's
                                             // footprints hold finite values of other bins)
                    } else {
                        int gv = v0 + b;
                        if (gv >= A.gy) gv -= A.gy;
                        // cells of tiles no footprint reaches hold no grid values of this bin
                        x = J->need[(gu >> A.shift) * A.ntv + (gv >> A.shift)] ? J->X[(size_t)gu * A.gy + gv]
                                                                              : make_float2(0.f, 0.f);
                        Xs[a * PW + b] = x;
                    }
                    const float m = fabsf(x.x) + fabsf(x.y);
                    if (m <= 3.4028234e38f) xm = fmaxf(xm, m);  // non-finite input is flagged elsewhere
                }
                if (SCATTER) {
                    reinterpret_cast<int2*>(Ahi)[a * PW + b] = make_int2(0, 0);
                    reinterpret_cast<int2*>(Alo)[a * PW + b] = make_int2(0, 0);
                }
            }
        }
        if (MODE == 2) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) xm = fmaxf(xm, __shfl_xor_sync(0xffffffffu, xm, o));
            if (lane == 0) s_xmax[warp] = xm;
        }
        consumers_sync();
        if (dyn && (s_fail || !have)) break;
        float s1 = 1.f, inv_s1 = 1.f;
        if (MODE == 2) {
            // per-unit bound: a de-gridded y of this unit has |y.x| + |y.y| <= 2 T1 max|X|_1
            // over the patch, a contribution component at most tmax times that (margin 2)
            float xmax = 0.f;
#pragma unroll
            for (int w = 0; w < GTG_CONSUMERS; ++w) xmax = fmaxf(xmax, s_xmax[w]);
            const float mt = 4.f * __uint_as_float(__ldg(J->fx + FX_TMAX)) * __uint_as_float(__ldg(J->fx + FX_T1)) * xmax;
            fx_scale(mt, td.ve - td.vb, s1, inv_s1);
        } else if (SCATTER) {
            // twice tmax max|y|_1 (rounding margin); both words final before this launch
            const float mt = 2.f * __uint_as_float(__ldcg(J->fx + FX_TMAX)) * __uint_as_float(__ldcg(J->fx + FX_YB));
            if (!(mt <= 3.4028234e38f)) atomicExch(J->status, 3);
            fx_scale(mt, td.ve - td.vb, s1, inv_s1);
        }
        for (int c = 0; c < nchunks; ++c, ++g) {
            const uint32_t b = g % NB, par = (g / NB) & 1;
            if (!s_abort && !mbar_wait_or_abort(&full[b], par, &s_abort)) {
                s_abort = 1;
                atomicExch(J->status, 1);
            }
            const int64_t cv0 = td.vb + (int64_t)c * GTG_CV;
            const int ncv = (int)((td.ve - cv0) < GTG_CV ? (td.ve - cv0) : GTG_CV);
            if (!s_abort && warp < ncv) {
                const VisMeta mt = mring[b * GTG_CV + warp];
                const int du = mt.pos & 255, dv = (mt.pos >> 8) & 255, S = (mt.pos >> 16) & 255;
                const int loc = (int)(mt.off - mring[b * GTG_CV].off);
                vis_dispatch<MODE, PWC>(S, taps + (size_t)b * chunk_f2 + loc, Xs, Ahi, Alo, s1, du * PW + dv, PW, lane,
                                   mt.orig, A.y_in, A.y_out);
            }
            __syncwarp();
            if (lane == 0 && !A.stall) mbar_arrive(&empty[b]);
        }
        if (pre) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&xfree[r % NX]);
        }
        consumers_sync();
        if (SCATTER && !s_abort) {
            // the box of the patch (the fold and the merge read no cell outside it)
            float2* dst = J->patch + (size_t)slot * npatch;
            const float inv_lo = inv_s1 * (1.f / 65536.f);
            const int bw = bb1 - bb0, nb = (ba1 - ba0) * bw;
            // e / bw = umulhi(e, ceil(2^32 / bw)) while e bw < 2^32 (e < PW^2, bw <= PW)
            const uint32_t mg = 0xffffffffu / (uint32_t)max(bw, 2) + 1u;
            for (int e = tid; e < nb; e += GTG_CONSUMERS * 32) {
                const int da = bw > 1 ? (int)__umulhi((uint32_t)e, mg) : e;
                const int c = (ba0 + da) * PW + bb0 + (e - da * bw);
                const int2 h = reinterpret_cast<const int2*>(Ahi)[c], l = reinterpret_cast<const int2*>(Alo)[c];
                dst[c] = make_float2(fmaf((float)l.x, inv_lo, (float)h.x * inv_s1),
                                     fmaf((float)l.y, inv_lo, (float)h.y * inv_s1));
            }
        }
        consumers_sync();
    }
}

// Adds the patches of the extra units of each split tile into its first unit's slot.
// TABLE: job j (one (plan, bin) of a batch) owns blocks [first[j], first[j + 1]).
struct MergeJob {
    float2* patch;
    const int2* groups;   // (first slot, units) of the bin's split tiles
    int npatch;           // cells of one patch
};

template <bool TABLE>
__global__ void __launch_bounds__(256) merge_patches_kernel(const __grid_constant__ MergeJob one,
                                                            const MergeJob* __restrict__ jobs,
                                                            const int* __restrict__ first, int njobs) {
    int bk = (int)blockIdx.x;
    const MergeJob* J = &one;
    if constexpr (TABLE) {
        const int j = job_of(first, njobs, bk);
        bk -= __ldg(first + j);
        J = jobs + j;
    }
    const int2 gr = J->groups[bk];
    float2* patch = J->patch;
    const int npatch = J->npatch;
    float2* dst = patch + (size_t)gr.x * npatch;
    for (int e = threadIdx.x; e < npatch; e += blockDim.x) {
        float2 acc = dst[e];
        for (int q = 1; q < gr.y; ++q) {
            const float2 v = patch[(size_t)(gr.x + q) * npatch + e];
            acc.x += v.x;
            acc.y += v.y;
        }
        dst[e] = acc;
    }
}

static size_t gtg_smem_dims(int PW, int chunk_bytes, int mode, int nbuf, bool prefetch, int xbufs = 2) {
    const size_t npatch = (size_t)PW * PW * sizeof(float2);
    // X patches (float2; xbufs of them when prefetched) when de-gridding, hi + lo words
    // (2 x int2) when gridding
    const int nx = mode != 1 ? (prefetch ? xbufs : 1) : 0;
    return GTG_HDR + GTG_NBUF * GTG_CV * sizeof(VisMeta) + (size_t)nbuf * chunk_bytes +
           (size_t)(nx + (mode != 0 ? 2 : 0)) * npatch;
}

size_t gtg_smem(const rimo_plan* p, int mode, int nbuf, bool prefetch) {
    return gtg_smem_dims(p->PW, p->chunk_bytes, mode, nbuf, prefetch);
}

// Launch shape of the grid step for a patch side and tap-ring chunk (prefetch, X buffers,
// ring depth, shared memory); `mode` as in launch_gtg.  Units of a few chunks (mean below
// 8 chunks of visibilities) leave too little time between two X patch copies for one copy
// ahead to land: they get a third X buffer, two units ahead, at the price of a ring slot.
static void gtg_shape(const rimo_plan* p, int PW, int chunk_bytes, int mode, double vis_per_unit, GtgArgs& A,
                      size_t& sm) {
    const size_t limit = 227 * 1024 - 2048;  // minus the kernel's static shared memory
    A.xbufs = vis_per_unit < 8.0 * GTG_CV ? GTG_NX : 2;
    // prefetch the X patches when the buffers still leave a 3-deep tap ring (4-deep with two)
    const int ring = A.xbufs == 2 ? GTG_NBUF : GTG_NBUF - 1;
    A.prefetch = mode != 1 && gtg_smem_dims(PW, chunk_bytes, mode, ring, true, A.xbufs) <= limit;
    if (mode != 1 && !A.prefetch && A.xbufs > 2) {
        A.xbufs = 2;
        A.prefetch = gtg_smem_dims(PW, chunk_bytes, mode, GTG_NBUF, true, 2) <= limit;
    }
    A.nbuf = GTG_NBUF;
    while (A.nbuf > 2 && gtg_smem_dims(PW, chunk_bytes, mode, A.nbuf, A.prefetch, A.xbufs) > limit) --A.nbuf;
    sm = gtg_smem_dims(PW, chunk_bytes, mode, A.nbuf, A.prefetch, A.xbufs);
    if (sm > limit) fail(RIMO_ERR_UNSUPPORTED, "tile patch and tap ring exceed shared memory");
    A.gx = p->gx;
    A.gy = p->gy;
    A.TS = p->TS;
    A.PW = PW;
    A.chunk_bytes = chunk_bytes;
    A.ntv = p->gy / p->TS;
    A.shift = p->TS == 64 ? 6 : 5;
    A.stall = p->test_stall;
    A.peer_polls = p->test_stall ? p->test_polls : WAIT_POLLS;
}

static GtgJob gtg_job(const rimo_plan* p, int bin, const float2* X, float2* patch) {
    GtgJob J;
    J.units = p->d_tiles + p->bins[bin].t0;
    J.chunks = p->d_chunks;
    J.meta = p->d_meta;
    J.gblk = p->d_gblock_ptrs;
    J.X = X;
    J.patch = patch;
    J.fx = p->d_fx;
    J.need = p->d_need + (size_t)bin * (size_t)(p->gx / p->TS) * (p->gy / p->TS);
    J.status = p->d_status;
    J.PW = p->PW;
    return J;
}

// the kernel instance: patch sides of the uv-tiles 32 and 64 with 15 x 15 tiles are
// compile-time constants
template <int MODE, bool TABLE>
static void (*gtg_kernel_for(int PW))(GtgArgs) {
    return PW == 46 ? gtg_kernel<MODE, 46, TABLE> : PW == 78 ? gtg_kernel<MODE, 78, TABLE> : gtg_kernel<MODE, 0, TABLE>;
}

template <int MODE>
static void gtg_run(const rimo_plan* p, int bin, const float2* y_in, float2* y_out, cudaStream_t s) {
    const auto& br = p->bins[bin];
    const int nu = br.t1 - br.t0;
    if (nu <= 0) return;
    GtgArgs A;
    std::memset(&A, 0, sizeof(A));
    A.one = gtg_job(p, bin, p->d_X, p->d_patch);
    A.sched = p->d_sched + br.t0;
    A.nunits = nu;
    // dense units take the dynamic schedule (zeroed counter at the start of every apply)
    A.counter = (double)(br.ve - br.vb) / nu >= 8.0 * GTG_CV ? p->d_counter + bin : nullptr;
    A.y_in = y_in;
    A.y_out = y_out;
    size_t sm = 0;
    gtg_shape(p, p->PW, p->chunk_bytes, MODE, (double)(br.ve - br.vb) / nu, A, sm);
    void (*kern)(GtgArgs) = gtg_kernel_for<MODE, false>(p->PW);
    RIMO_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int grid = std::min(nu, p->n_sm);
    kern<<<grid, GTG_THREADS, sm, s>>>(A);
    if (MODE != 0 && br.m1 > br.m0) {
        MergeJob mj;
        mj.patch = p->d_patch;
        mj.groups = p->d_merge + br.m0;
        mj.npatch = p->PW * p->PW;
        merge_patches_kernel<false><<<br.m1 - br.m0, 256, 0, s>>>(mj, nullptr, nullptr, 0);
    }
}

// ---------------------------------------------------------------------------
// The grid step of a stage-batched apply: one persistent launch over the units of every
// (plan, bin) job, taken heaviest first from one queue, then one merge launch.
struct WideGtg {
    GtgArgs A;
    size_t sm = 0;
    int grid = 0, merge_blocks = 0, njobs = 0, PW = 0;
    GtgJob* jobs = nullptr;
    int2* queue = nullptr;
    MergeJob* mjobs = nullptr;
    int* mfirst = nullptr;
    int* counter = nullptr;  // the dynamic schedule's next unit (zeroed before every launch)
    int64_t units = 0;
    ~WideGtg() {
        cudaFree(jobs);
        cudaFree(queue);
        cudaFree(mjobs);
        cudaFree(mfirst);
        cudaFree(counter);
    }
};

WideGtg* wide_gtg_create(const std::vector<WideJob>& jobs, cudaStream_t s) {
    if (jobs.empty()) fail(RIMO_ERR_INVALID_ARG, "no jobs");
    auto* w = new WideGtg();
    try {
        const rimo_plan* p0 = jobs[0].p;
        int pw_max = 0, cb_max = 0;
        bool one_pw = true;
        for (const WideJob& j : jobs) {
            pw_max = std::max(pw_max, j.p->PW);
            cb_max = std::max(cb_max, j.p->chunk_bytes);
            one_pw = one_pw && j.p->PW == p0->PW;
        }
        int64_t nvis = 0, nun = 0;
        for (const WideJob& j : jobs) {
            nvis += j.p->bins[j.bin].ve - j.p->bins[j.bin].vb;
            nun += j.p->bins[j.bin].t1 - j.p->bins[j.bin].t0;
        }
        std::memset(&w->A, 0, sizeof(w->A));
        gtg_shape(p0, pw_max, cb_max, 2, (double)nvis / std::max<int64_t>(1, nun), w->A, w->sm);
        // one patch side: its compile-time kernel; several: the kernel reading each job's
        w->PW = one_pw ? p0->PW : 0;
        std::vector<GtgJob> gj;
        std::vector<MergeJob> mj;
        std::vector<int> mf{0};
        struct Q {
            int64_t n;
            int job, slot;
        };
        std::vector<Q> q;
        for (size_t j = 0; j < jobs.size(); ++j) {
            const rimo_plan* p = jobs[j].p;
            if (p->TS != p0->TS || p->gx != p0->gx || p->gy != p0->gy)
                fail(RIMO_ERR_UNSUPPORTED, "jobs of one grid-step launch need one grid and uv-tile size");
            const auto& br = p->bins[jobs[j].bin];
            gj.push_back(gtg_job(p, jobs[j].bin, jobs[j].X, jobs[j].patch));
            for (int u = 0; u < br.t1 - br.t0; ++u) {
                const TileDesc& td = p->tiles_host[(size_t)br.t0 + u];
                q.push_back(Q{td.ve - td.vb, (int)j, u});
            }
            MergeJob m;
            m.patch = jobs[j].patch;
            m.groups = p->d_merge + br.m0;
            m.npatch = p->PW * p->PW;
            mj.push_back(m);
            mf.push_back(mf.back() + (br.m1 - br.m0));
        }
        // heaviest first over the whole batch (ties: job, then slot), dealt in snake order
        std::stable_sort(q.begin(), q.end(), [](const Q& a, const Q& b) { return a.n > b.n; });
        std::vector<int2> qq(q.size());
        for (size_t i = 0; i < q.size(); ++i) qq[i] = make_int2(q[i].job, q[i].slot);
        w->units = (int64_t)q.size();
        w->njobs = (int)jobs.size();
        w->merge_blocks = mf.back();
        RIMO_CUDA(cudaMalloc(&w->jobs, gj.size() * sizeof(GtgJob)));
        RIMO_CUDA(cudaMalloc(&w->queue, std::max<size_t>(1, qq.size()) * sizeof(int2)));
        RIMO_CUDA(cudaMalloc(&w->mjobs, mj.size() * sizeof(MergeJob)));
        RIMO_CUDA(cudaMalloc(&w->mfirst, mf.size() * sizeof(int)));
        RIMO_CUDA(cudaMalloc(&w->counter, sizeof(int)));
        RIMO_CUDA(cudaMemcpyAsync(w->jobs, gj.data(), gj.size() * sizeof(GtgJob), cudaMemcpyHostToDevice, s));
        if (!qq.empty())
            RIMO_CUDA(cudaMemcpyAsync(w->queue, qq.data(), qq.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
        RIMO_CUDA(cudaMemcpyAsync(w->mjobs, mj.data(), mj.size() * sizeof(MergeJob), cudaMemcpyHostToDevice, s));
        RIMO_CUDA(cudaMemcpyAsync(w->mfirst, mf.data(), mf.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        RIMO_CUDA(cudaStreamSynchronize(s));
        w->A.jobs = w->jobs;
        w->A.queue = w->queue;
        w->A.nunits = (int)q.size();
        w->A.counter = (double)nvis / std::max<int64_t>(1, nun) >= 8.0 * GTG_CV ? w->counter : nullptr;
        if ((int64_t)w->A.nunits != w->units) fail(RIMO_ERR_UNSUPPORTED, "too many work units for one launch");
        w->grid = (int)std::min<int64_t>(w->units, p0->n_sm);
    } catch (...) {
        delete w;
        throw;
    }
    return w;
}

void wide_gtg_destroy(WideGtg* w) { delete w; }

int64_t wide_gtg_units(const WideGtg* w) { return w->units; }

void wide_gtg(const WideGtg* w, cudaStream_t s) {
    if (w->units == 0) return;
    void (*kern)(GtgArgs) = gtg_kernel_for<2, true>(w->PW);
    RIMO_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)w->sm));
    if (w->A.counter) RIMO_CUDA(cudaMemsetAsync(w->counter, 0, sizeof(int), s));
    kern<<<w->grid, GTG_THREADS, w->sm, s>>>(w->A);
    if (w->merge_blocks > 0) {
        MergeJob none;
        none.patch = nullptr;
        none.groups = nullptr;
        none.npatch = 0;
        merge_patches_kernel<true><<<w->merge_blocks, 256, 0, s>>>(none, w->mjobs, w->mfirst, w->njobs);
    }
}

void launch_gtg(const rimo_plan* p, int bin, int mode, const float2* y_in, float2* y_out,
                cudaStream_t s) {
    if (mode == 0) gtg_run<0>(p, bin, y_in, y_out, s);
    else if (mode == 1) gtg_run<1>(p, bin, y_in, y_out, s);
    else gtg_run<2>(p, bin, y_in, y_out, s);
}

// ---------------------------------------------------------------------------
// Bound on the y of Phi^dagger y: max_k(|y_k.x| + |y_k.y|) goes to d_fx[FX_YB] (a grid-step
// contribution component is at most that times max_taps(|t.x| + |t.y|)).  Non-finite y
// sets status 3.  The last block to finish (counter in d_fx[FX_COUNT]) writes the bound and
// resets the running words.
__global__ void __launch_bounds__(256) y_bound_kernel(const float2* __restrict__ y, int64_t M, uint32_t* fx,
                                                      int* status) {
    float mx = 0.f;
    bool bad = false;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < M; k += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = y[k];
        const float m = fabsf(v.x) + fabsf(v.y);
        bad |= !(m <= 3.4028234e38f);
        mx = fmaxf(mx, m);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(fx + FX_YMAX, __float_as_uint(mx));
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(status, 3);
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(fx + FX_COUNT, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        // the gridding step combines it with the tap bound current when it runs (tiles
        // generated per bin at apply time raise the tap bound bin by bin)
        fx[FX_YB] = atomicExch(fx + FX_YMAX, 0u);
        fx[FX_COUNT] = 0u;
    }
}

void launch_y_bound(const rimo_plan* p, const float2* y, cudaStream_t s) {
    if (p->M == 0) return;
    const int64_t want = (p->M + 255) / 256;
    const int blocks = (int)std::min<int64_t>(want, std::min<int64_t>(FX_NPART, 4 * (int64_t)p->n_sm));
    y_bound_kernel<<<blocks, 256, 0, s>>>(y, p->M, p->d_fx, p->d_status);
}

}  // namespace rimo
