/*
 * rimo.h - C ABI of the GB300 widefield radio-interferometric measurement operator.
 *
 * The library applies the widefield measurement operator Phi, its adjoint Phi^dagger
 * and the composite Phi^dagger Phi in hybrid w-stacking / w-projection form
 * (Dabbech & Wiaux, Section 3, Eq. 6 - Eq. 8) on one GPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Complex numbers are rimo_cfloat (two float32, real first): the memory layout of
 * numpy complex64 / torch.complex64.
 *
 * Images are row-major [ny][nx].  Pixel (i, j) sits at direction cosines
 * l = (j - nx/2) * fov_x / nx and m = (i - ny/2) * fov_y / ny.
 *
 * Visibility vectors are in the caller's order: entry k belongs to row k of the uvw
 * array given to rimo_plan_create.  uvw is in wavelengths.
 *
 * Ownership: the caller owns every input and output buffer ("_dev" pointers are
 * device memory the caller allocated, e.g. torch tensors).  A plan owns all the
 * device memory it allocates (de-gridding matrix, holographic blocks, scratch grids)
 * and frees it in rimo_plan_destroy.
 *
 * Streams: work is enqueued on the caller's stream without host synchronisation,
 * except where an entry point says it synchronises.  A plan holds scratch grids,
 * so two applies of one plan must not run concurrently on different streams.
 * Distinct plans are independent.
 *
 * Errors: every call returns a rimo_status; on failure rimo_last_error() gives a
 * thread-local message.  No C++ exception crosses this interface.  Asynchronous
 * CUDA errors of enqueued work surface at a later call that synchronises.
 */
#ifndef RIMO_H
#define RIMO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rimo_cfloat { float re, im; } rimo_cfloat;

typedef enum rimo_status {
    RIMO_OK = 0,
    RIMO_ERR_INVALID_ARG = 1, /* a pointer, size or parameter is out of range        */
    RIMO_ERR_OOM = 2,         /* a device or host allocation failed                   */
    RIMO_ERR_BUDGET = 3,      /* the requested mode does not fit mem_budget_bytes     */
    RIMO_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed          */
    RIMO_ERR_TIMEOUT = 5,     /* a bounded device-side wait ran out                   */
    RIMO_ERR_UNSUPPORTED = 6, /* the plan's mode or sizes do not support this call    */
    RIMO_ERR_STATE = 7        /* the call needs a step that has not been done yet     */
} rimo_status;

typedef enum rimo_mode {
    RIMO_MODE_AUTO = 0,        /* decision tree of Section 3.4 / Fig. 2              */
    RIMO_MODE_STORED_G = 1,    /* precompute and store the de-gridding matrix G      */
    RIMO_MODE_HOLOGRAPHIC = 2, /* H_p = G_p^dagger G_p (Section 3.3) once built; no  */
                               /* stored G: tiles generated on the fly until then    */
    RIMO_MODE_SURROGATE = 3,   /* kernels generated on the fly by the learned MLP    */
    RIMO_MODE_ONTHEFLY = 4     /* exact kernels generated per w-bin at apply time    */
} rimo_mode;

typedef enum rimo_n_weight {
    RIMO_NWEIGHT_NONE = 0,  /* C = exp(-2 pi i w (n - 1))              (default)      */
    RIMO_NWEIGHT_DIV_N = 1  /* C = exp(-2 pi i w (n - 1)) / n, the 1/n of Eq. 2       */
} rimo_n_weight;

/*
 * Plan parameters (Section 3.1 and Section 3.4).  Zero selects the default where
 * one is named.
 *   nx, ny            image size; powers of two in [64, 4096].
 *   fov_x, fov_y      full field of view (radians); (fov/2)^2 * 2 * 4 < 1.
 *   oversampling      must be 2 (the paper's o = 2).
 *   kb_support        Kaiser-Bessel taps J per axis: odd, 3..11 (default 7).
 *   kb_beta           KB shape (0 -> 2.34 J, the Fessler-Sutton choice for o = 2).
 *   max_wsupport      cap on the residual w-kernel support S_w: odd, 1..9 (default 9).
 *                     The per-visibility tile is S x S with S = S_w + J - 1 <= 19.
 *   w_norm_frac       fraction of the w-kernel l2 norm kept by hard-thresholding
 *                     (Section 3.1); in (0, 1], default 0.9999.
 *   mem_budget_bytes  device memory budget m* for the stored matrices (0 = no limit).
 *   n_wbins           number P of w-bins (0 = chosen by the cost model, Eq. 10).
 *   n_blocks          Fourier blocks of G: byte limit total / n_blocks (0 = by block_bytes_max);
 *                     blocks do not span w-bins, so a plan holds n_blocks .. n_blocks + P.
 *   mode              rimo_mode.
 *   n_weight          rimo_n_weight.
 *   plan_fraction     fraction of the data used for planning (default 0.01).
 *   seed              seed of the planning subset.
 *   taper_literal     0: taper the chirp's deviation from 1 (default); 1: taper C.
 *   wkernel_L         w-kernel sampling grid per axis (0 = max(32, 2^ceil(log2(4 S_w,max)))).
 *   tile_size         uv-tile edge in grid cells for sorting/gridding (0 = 32; 32 or 64).
 *   block_bytes_max   upper bound of one Fourier block of G (0 = 8 GiB).
 *   wkernel_table     0: each visibility's residual w-kernel is computed from the chirp
 *                     (Section 3.1); n > 0: the kernels K(t; w_r) (they depend on w_r alone)
 *                     are sampled at n + 3 points spanning [-max|w_r|, max|w_r|] once per
 *                     plan and interpolated by cubic Lagrange polynomials in w_r when tiles
 *                     are built or generated (n >= 16; 8192 keeps the interpolation error
 *                     near 1e-8 relative at the 4096^2 / 50M workload).
 *   uv_order          order of the visibilities within a uv-tile, which sets the groups of
 *                     GTG_CHUNK (20) visibilities the grid step de-grids and grids at once
 *                     (a scheduling choice of this design, no counterpart in the paper):
 *                     0 = time-interleaved (the tile's list in time order read as 20 rows,
 *                     column by column: a group's visibilities come from far-apart instants
 *                     and rarely update the same grid cells; default), 1 = time order,
 *                     2 = shuffled by a counter-based SplitMix64 hash of the visibility
 *                     index.  Results agree within rounding (the grid step sums exactly
 *                     in fixed point; only the split of heavy tiles into units moves).
 *   shard_count,      level-2 distribution of Section 3.5 (G's Fourier blocks of every
 *   shard_rank        w-bin over workers): with shard_count >= 2, shard_count plans made
 *                     from the same uvw and parameters but shard_rank 0 .. shard_count - 1
 *                     share the w-stack and the uv-tiles, and each keeps the tiles of every
 *                     w-bin whose place in the bin's radial order (distance from the uv
 *                     origin; ties by tile row, then column) is shard_rank modulo
 *                     shard_count: it stores G and applies the operator for their
 *                     visibilities only.  Phi writes those visibilities' y (the others are
 *                     left as they are); the Phi^dagger and Phi^dagger Phi images of the
 *                     shard plans sum to the whole operator's (Eq. 7: G_p^dagger G_p is a
 *                     sum over visibilities).  Stored G only (mode STORED_G, or AUTO
 *                     choosing it); 0 or 1: no sharding (the default).
 */
typedef struct rimo_plan_params {
    int32_t nx, ny;
    double fov_x, fov_y;
    int32_t oversampling;
    int32_t kb_support;
    double kb_beta;
    int32_t max_wsupport;
    double w_norm_frac;
    int64_t mem_budget_bytes;
    int32_t n_wbins;
    int32_t n_blocks;
    int32_t mode;
    int32_t n_weight;
    double plan_fraction;
    uint64_t seed;
    int32_t taper_literal;
    int32_t wkernel_L;
    int32_t tile_size;
    int64_t block_bytes_max;
    int32_t wkernel_table;
    int32_t uv_order;
    int32_t shard_count;
    int32_t shard_rank;
} rimo_plan_params;

/* Results of planning (stage 1 of Fig. 3) and the state of a plan. */
typedef struct rimo_plan_info {
    int64_t M;                 /* visibilities                                     */
    int32_t P;                 /* w-bins                                           */
    int32_t mode;              /* rimo_mode actually used                          */
    int32_t p_star;            /* minimiser of the cost model over the candidates  */
    int32_t wkernel_L;
    int32_t max_tile;          /* largest S in the plan                            */
    int32_t n_blocks;          /* Fourier blocks of G                              */
    int32_t n_tiles;           /* active uv-tiles over all bins                    */
    int64_t subset;            /* visibilities used for planning                   */
    int64_t K;                 /* non-zeros of G: sum_k S_k^2                      */
    int64_t g_bytes;           /* device bytes of stored G (taps + metadata)       */
    int64_t h_bytes;           /* device bytes of stored H (0 unless built)        */
    int64_t scratch_bytes;     /* device bytes of scratch grids                    */
    double est_m_g;            /* Eq. 9 analogue at the chosen P, from the subset  */
    double est_cost;           /* Eq. 10 at the chosen P                           */
    double wr_max;             /* max |w - w_stack[bin]|                           */
    double wsclean_p;          /* Eq. 5 bound                                      */
    int32_t support_table[64]; /* S_w per uniform |w_r| bin                        */
    int32_t tile_size;         /* uv-tile edge of the gridding schedule (0: none)  */
    int32_t truncated;         /* 1: at the largest residual w the kernel needs more */
                               /* than max_wsupport taps to keep w_norm_frac         */
    int32_t weighted;          /* 1: a data weighting is injected (set_weights)    */
    /* Holographic matrices (0 until rimo_build_holographic has run; Section 3.3): */
    int64_t h_entries;         /* dense stencil entries: covered owner cells x       */
                               /* entries per owner row (each cell pair once)        */
    int64_t h_nonzero;         /* entries stored: the non-zero ones (cell pairs that */
                               /* some visibility's footprint covers together)       */
    int64_t h_nnz;             /* non-zeros of the full Hermitian H_p = G_p^H G_p,   */
                               /* summed over bins: both triangles and the diagonal  */
    int64_t n_units;           /* grid-step work units over all bins (uv-tiles, or   */
                               /* slices of the heaviest ones)                       */
    int64_t box_cells;         /* sum over the units of their box (the cells their   */
                               /* footprints reach; a split tile's slices: whole     */
                               /* patches): X cells staged and patch cells stored    */
    int64_t n_needed;          /* needed uv-tiles summed over the bins (tiles of X   */
                               /* the forward transform stores and the fold writes)  */
    int64_t sel_rows;          /* grid rows the column passes transform, summed over */
                               /* the bins (the rows of tile rows with a needed tile)*/
} rimo_plan_info;

typedef struct rimo_plan* rimo_plan_t;

/*
 * Default parameters for an nx x ny image over fov_x x fov_y radians.
 * Never fails; writes *p.
 */
void rimo_plan_params_default(rimo_plan_params* p, int32_t nx, int32_t ny, double fov_x,
                              double fov_y);

/*
 * Plan on the host only (Section 3.4, stage 1 of Fig. 3): choose P and the mode from
 * the planning subset without touching a GPU.  uvw: host, M x 3 row-major float64
 * (wavelengths).  Fills *info (per-visibility fields are not computed).
 * Errors: INVALID_ARG (also for a NaN or infinite coordinate, or |u| 2 fov_x, |v| 2 fov_y
 * or |w| of 2^52 or more).
 */
rimo_status rimo_plan_estimate(const double* uvw, int64_t M, const rimo_plan_params* p,
                               rimo_plan_info* info);

/*
 * Create a plan (stages 1 - 3 of Fig. 3): w-bins by k-means (Section 3.1), P and mode
 * (Section 3.4), per-visibility grid coordinates, uv-tile sort and Fourier blocks
 * (Section 3.2), and - in stored-G mode - the de-gridding matrix G on the device.
 * uvw: host, M x 3 row-major float64 (wavelengths); copied, not retained.
 * The plan is built on `stream`; the call synchronises the stream before returning.
 * Errors: INVALID_ARG (also for uvw as in rimo_plan_estimate), OOM, BUDGET (explicit mode
 * beyond the budget), CUDA.
 */
rimo_status rimo_plan_create(const double* uvw, int64_t M, const rimo_plan_params* p,
                             void* stream, rimo_plan_t* out);

/* Free a plan and all device memory it owns.  NULL is accepted. */
rimo_status rimo_plan_destroy(rimo_plan_t plan);

/*
 * Plan files (Section 4: the planning stage may run on its own, and both stages read one
 * parameter file and one observation file of (u, v, w) coordinates).  A plan is fully
 * determined by its coordinates and parameters, so a plan file holds those - and the data
 * weights injected into the operator, if any (Section 2) - and rimo_plan_create_from_file
 * rebuilds the identical plan in another process or later.  Format: an 8-byte magic
 * "RIMOPLAN", format version 1, sizeof(rimo_plan_params), M, a weights flag, the
 * parameters, uvw (M x 3 float64), the weights (M float32) when present, and a 64-bit
 * FNV-1a checksum of every byte before it (per 1 MiB block, then over the block digests);
 * little-endian, the byte order of the machines this library builds for.
 */

/*
 * Write a plan file.  uvw: host, M x 3 row-major float64 (wavelengths); p: the plan
 * parameters; weights: host, M float32 (finite, >= 0) or NULL for none.  Host only (no GPU).
 * The caller's arrays are read, not retained; an existing file is replaced.
 * Errors: INVALID_ARG (null pointer, M out of range, parameters or coordinates that
 * rimo_plan_create would refuse, bad weights, a path that cannot be written).
 */
rimo_status rimo_plan_file_write(const char* path, const double* uvw, int64_t M, const rimo_plan_params* p,
                                 const float* weights);

/*
 * Read and check a whole plan file (magic, version, sizes, checksum, parameters,
 * coordinates, weights) and report its parameters, M and whether it holds weights (any
 * output may be NULL).  Host only.  Errors: INVALID_ARG naming the first check that failed
 * (a corrupted, truncated or foreign file among them).
 */
rimo_status rimo_plan_file_info(const char* path, rimo_plan_params* p, int64_t* M, int32_t* has_weights);

/*
 * Create the plan a plan file describes: the checks of rimo_plan_file_info, then
 * rimo_plan_create on its coordinates and parameters, then rimo_plan_set_weights with its
 * weights when it holds them.  Streams and synchronisation as rimo_plan_create.
 * Errors: those of rimo_plan_file_info, rimo_plan_create and rimo_plan_set_weights; on
 * failure *out is NULL and nothing stays allocated.
 */
rimo_status rimo_plan_create_from_file(const char* path, void* stream, rimo_plan_t* out);

/* Copy the plan summary into *info (host). */
rimo_status rimo_plan_info_get(rimo_plan_t plan, rimo_plan_info* info);

/*
 * Copy plan data to host buffers (any may be NULL): w_stack[P] (ascending w-bin
 * values), bins[M] (w-bin of each visibility, caller order), s_w[M] (residual
 * w-kernel support of each visibility, caller order).
 */
rimo_status rimo_plan_get_bins(rimo_plan_t plan, double* w_stack, int32_t* bins, int32_t* s_w);

/*
 * Copy the de-gridding taps of selected visibilities to the host (Section 3.2, G_p rows).
 * idx[n]: caller-order visibility indices (host).  For visibility idx[q] writes
 * g0[q], h0[q] (first grid cell along u and v, already reduced modulo the grid),
 * S[q] (tile side) and taps[q * 19 * 19 ...]: the S x S tile, row a along u, column b
 * along v, at taps + q * 361 (row stride S).  Synchronises `stream`.
 * Plans without stored G (surrogate, on-the-fly, holographic before H is built) generate
 * the requested visibilities' bins into their tap scratch, as an apply does, and copy
 * from there; such a call must not overlap an apply of the same plan.
 * Errors: INVALID_ARG (also a visibility that a shard plan does not hold), STATE
 * (surrogate plan without a surrogate), UNSUPPORTED (holographic plan whose tiles were
 * folded into H), CUDA.
 */
rimo_status rimo_plan_get_tiles(rimo_plan_t plan, const int64_t* idx, int64_t n, int32_t* g0,
                                int32_t* h0, int32_t* S, rimo_cfloat* taps, void* stream);

/*
 * The image-domain factor Z_p of w-bin `bin` (Eq. 6: grid correction times the w-layer
 * chirp e^{-2 pi i w_stack[bin] (sqrt(1 - l^2 - m^2) - 1)} of Eq. 2, divided by
 * sqrt(1 - l^2 - m^2) with n_weight = DIV_N), exactly as the transform kernels evaluate it
 * (the w-phase argument and its range reduction in double-float arithmetic, then one
 * single-precision sincos).  out_dev: device, ny x nx complex, row-major, pixel (i, j) at
 * l = (j - nx/2) fov_x / nx, m = (i - ny/2) fov_y / ny; enqueued on `stream`.
 * Errors: INVALID_ARG (null plan or buffer, bin out of range), CUDA.
 */
rimo_status rimo_plan_get_zlayer(rimo_plan_t plan, int32_t bin, rimo_cfloat* out_dev, void* stream);

/*
 * y = Phi x (Eq. 6).  x_dev: device, ny x nx image; y_dev: device, M visibilities in
 * caller order.  Errors: INVALID_ARG, UNSUPPORTED (holographic-only plan), CUDA.
 */
rimo_status rimo_apply_phi(rimo_plan_t plan, const rimo_cfloat* x_dev, rimo_cfloat* y_dev,
                           void* stream);

/*
 * x = Phi^dagger y = sum_p Z_p^dagger F^dagger G_p^dagger y_p (adjoint of Eq. 6).
 * y_dev: device, M visibilities (caller order); x_dev: device, ny x nx image (overwritten).
 */
rimo_status rimo_apply_phi_adj(rimo_plan_t plan, const rimo_cfloat* y_dev, rimo_cfloat* x_dev,
                               void* stream);

/*
 * out = Phi^dagger Phi x = sum_p Z_p^dagger F^dagger G_p^dagger G_p F Z_p x (Eq. 7 and Eq. 8),
 * or with H_p in place of G_p^dagger G_p once rimo_build_holographic has run.
 * x_dev, out_dev: device ny x nx images (distinct buffers); real_part_only != 0 writes
 * Re{.} with zero imaginary parts (the Re{} of Eq. 4).
 */
rimo_status rimo_apply_phi_adj_phi(rimo_plan_t plan, const rimo_cfloat* x_dev,
                                   rimo_cfloat* out_dev, int32_t real_part_only, void* stream);

/*
 * Build the holographic matrices H_p = G_p^dagger G_p on the device (Section 3.3) and
 * switch rimo_apply_phi_adj_phi (and rimo_psf) to them; Phi and Phi^dagger keep using the
 * plan's tiles.  A stored-G plan builds H from G; a holographic or on-the-fly plan generates
 * each bin's exact tiles for its build, so all of G is never held (Fig. 2, regime b).
 * H_p is Hermitian and stored once per cell pair: every grid cell that some visibility
 * footprint covers owns a row over the (H+1)^2 + H^2 pairs it can lead (H = S_max - 1: 421
 * for S_max = 15), of which only the non-zero entries are kept (complex value + 16-bit
 * entry number, rows found by offsets), so it pays off where visibilities per covered
 * cell are many.  Built bin by bin through a temporary of the bin's dense rows.  Fails
 * with BUDGET (releasing what it built) when mem_budget_bytes is set and G plus H would
 * exceed it.  A second call does nothing.  info.h_bytes reports the rows and patches.
 * Synchronises `stream`.  Errors: INVALID_ARG, UNSUPPORTED (surrogate plans; shard
 * plans, shard_count >= 2), OOM, BUDGET, CUDA.
 */
rimo_status rimo_build_holographic(rimo_plan_t plan, void* stream);

/*
 * Entries of the built holographic matrix of bin `bin`: out[q] = H_bin[c1][c2] for the
 * cell pairs pairs[4q .. 4q+3] = (u1, v1, u2, v2) (grid cells, taken modulo the grid);
 * zero where no footprint covers both cells.  pairs, out: host.  For tests and
 * inspection (one small copy per entry).  Synchronises `stream`.
 * Errors: INVALID_ARG, STATE (not built), CUDA.
 */
rimo_status rimo_plan_get_holographic(rimo_plan_t plan, int32_t bin, const int32_t* pairs, int64_t n,
                                      rimo_cfloat* out, void* stream);

/*
 * out = sum over the w-bins p with bin_mask[p] != 0 of Phi_p^dagger Phi_p x (the terms of
 * Eq. 7), for sharding the bins over devices or processes whose partial images are then
 * summed.  bin_mask: host, P bytes (rimo_plan_info.P); NULL selects every bin.  No
 * selected bin (or only empty ones) gives out = 0.  Layout, streams and errors as
 * rimo_apply_phi_adj_phi.
 */
rimo_status rimo_apply_phi_adj_phi_bins(rimo_plan_t plan, const rimo_cfloat* x_dev, rimo_cfloat* out_dev,
                                        int32_t real_part_only, const uint8_t* bin_mask, void* stream);

/* PSF: out = Phi^dagger Phi delta, delta at pixel (ny/2, nx/2); unnormalised. */
rimo_status rimo_psf(rimo_plan_t plan, rimo_cfloat* out_dev, void* stream);

/*
 * Stage timers (tracing).  When enabled, every kernel group the plan enqueues is
 * bracketed by CUDA events recorded on the same stream.  Stages:
 *   0 forward rows pass (Z_p and 2-D DFT along l)   1 forward cols pass
 *   2 grid clear                                   3 de-grid / grid / fused G^dagger G
 *   4 inverse cols pass                            5 inverse rows pass (Z_p^dagger, sum over p)
 *   6 G build                                      7 H build
 *   8 H apply                                      9 surrogate MLP (train / fused generation)
 *   10..15 reserved
 * rimo_profile_enable(plan, on) starts (on != 0) or stops recording; it does not reset.
 * rimo_profile_read synchronises the pending events, adds their durations to the
 * running totals and copies, for the first n stages, the total milliseconds (ms[n])
 * and the number of kernel launches (launches[n]); reset != 0 clears the totals after
 * copying.  Either output pointer may be NULL.  Errors: INVALID_ARG, CUDA.
 */
#define RIMO_N_STAGES 16
rimo_status rimo_profile_enable(rimo_plan_t plan, int32_t on);
rimo_status rimo_profile_read(rimo_plan_t plan, double* ms, int64_t* launches, int32_t n,
                              int32_t reset);

/*
 * Phi^dagger Phi without allocating device memory.  The paper has no counterpart: this
 * entry point exists for callers that may not allocate device memory when they apply
 * the operator - for example a program whose device memory is wholly owned by another
 * allocator (a framework's caching pool that has reserved the free memory, so that
 * cudaMalloc would fail or would have to evict its cache), or a processing loop that must
 * not call cudaMalloc / cudaFree after its set-up phase because those calls may
 * synchronise the device and take unbounded time.
 *
 * It computes exactly what rimo_apply_phi_adj_phi computes with the same arguments (see
 * there), but takes every scratch buffer of the apply (half-transformed rows, the
 * forward / gridded grid, the tile patches, the tile schedulers) from one array of
 * RIMO_NOALLOC_SCRATCH_BYTES (32 MiB) that the library allocates statically on every
 * device that loads it and keeps until the process exits.  The call itself performs no
 * cudaMalloc, cudaFree or other allocating call.  Of the plan's own device memory it
 * writes only the status word (read by rimo_plan_status) and the grid step's bound
 * words, as the regular apply does; for the duration of the call the plan's scratch
 * pointers are pointed at the array (and restored before it returns), so the plan must
 * not be applied from another thread meanwhile (plans are not re-entrant in any case).
 * Nothing of the array needs clearing between calls or between plans: the tile
 * schedulers are reset by every apply, and every grid cell an apply reads was written
 * earlier in the same apply (the forward column pass writes every cell of every uv-tile
 * that some tile patch of the bin reaches, which is every cell the grid step stages).
 *
 * Limit: the plan must fit the array: 8 (6 nx ny + max tiles per w-bin * (TS + H)^2) bytes
 * plus a little alignment, about nx = ny = 512 at most; larger plans are rejected with
 * RIMO_ERR_UNSUPPORTED and a message naming the bytes needed.
 * Set-up: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before any
 * stream capture.
 * Sharing: every call on a device uses the same array; each call clears what must start
 * at zero.  Calls whose work overlaps on the GPU (other streams, other threads, other
 * plans) race on the array and give wrong results: serialise them.
 * Errors: INVALID_ARG, UNSUPPORTED (scratch limit), CUDA.
 */
#define RIMO_NOALLOC_SCRATCH_BYTES (32u << 20)
rimo_status rimo_apply_phi_adj_phi_noalloc(rimo_plan_t plan, const rimo_cfloat* x_dev,
                                           rimo_cfloat* out_dev, int32_t real_part_only,
                                           void* stream);

/*
 * Device status of a plan: synchronises `stream`, then returns (and clears the flag)
 * RIMO_ERR_TIMEOUT if a kernel of this plan gave up a bounded wait, or RIMO_ERR_INVALID_ARG
 * if an input of Phi^dagger or Phi^dagger Phi held a non-finite value (the grid step
 * accumulates in fixed point from a bound on its inputs), since the last call - results
 * are then invalid - else RIMO_OK.  Kernels never spin without a bound.
 */
rimo_status rimo_plan_status(rimo_plan_t plan, void* stream);

/*
 * Failure-detection test of the device-side bounded waits (no counterpart in the paper;
 * the paper's workers fail on the host).  With stall = 1, the grid-step launches of this
 * plan's following applies run with their consumer warps never releasing a ring slot of
 * taps to the producer warp (a flag that nothing sets), and the producer's waits on the
 * other warps limited to `polls` (1 .. 32768) suspended polls of at most 100 us.  A block
 * whose producer has to reuse a slot then gives up: it records RIMO_ERR_TIMEOUT in the
 * plan's status, waits (with the normal bound) for its own bulk copies in flight, and
 * returns, and its consumer warps stop waiting for chunks that will not come.  Results of
 * applies made with stall = 1 are invalid; rimo_plan_status reports the timeout.
 * stall = 0 (polls ignored) restores normal operation.  Host-only call.
 * Errors: INVALID_ARG.
 */
rimo_status rimo_plan_set_wait_test(rimo_plan_t plan, int32_t stall, int32_t polls);

/*
 * Kernel surrogate (a learned replacement for the stored de-gridding taps; no
 * counterpart in the paper, which stores G or H or recomputes G on the fly, Section 3.4).
 * A multilayer perceptron maps the normalised inputs x = (2 phi_u - 1, 2 phi_v - 1,
 * w_r / w_scale) of a visibility - fractional grid offsets along u and v and residual w -
 * to its 15 x 15 complex tile: 3 -> 128 -> GELU -> 128 -> GELU -> 450 reals (the 225 real
 * parts row a along u major, then the 225 imaginary parts).  Weights and activations
 * enter the tensor cores (tcgen05) in bf16 with FP32 accumulation; Adam keeps FP32
 * masters.  Parameters as one FP32 vector of RIMO_SURROGATE_NPARAM values: W1 [128][3],
 * b1 [128], W2 [128][128], b2 [128], W3 [450][128], b3 [450].
 * Batches: B a positive multiple of 128; x_dev, t_dev, y_dev device FP32 row-major
 * (B x 3, B x 450, B x 450).  The surrogate owns its device memory.
 */
#define RIMO_SURROGATE_NPARAM 75074
typedef struct rimo_surrogate* rimo_surrogate_t;
/* New surrogate with weights drawn uniformly in +-1/sqrt(fan_in) from `seed`. */
rimo_status rimo_surrogate_create(uint64_t seed, rimo_surrogate_t* out);
rimo_status rimo_surrogate_destroy(rimo_surrogate_t s);
/* Copy the FP32 master parameters to / from the host (set also resets Adam). */
rimo_status rimo_surrogate_get_params(rimo_surrogate_t s, float* params);
rimo_status rimo_surrogate_set_params(rimo_surrogate_t s, const float* params);
/* y = MLP(x) for a batch, enqueued on `stream`. */
rimo_status rimo_surrogate_forward(rimo_surrogate_t s, const float* x_dev, int64_t B, float* y_dev,
                                   void* stream);
/*
 * Mean squared error over the batch and the 450 outputs, and its gradient with respect to
 * every parameter (grads: host, RIMO_SURROGATE_NPARAM values; loss: host; either may be
 * NULL).  Synchronises `stream`.  Errors: INVALID_ARG, TIMEOUT, CUDA.
 */
rimo_status rimo_surrogate_gradients(rimo_surrogate_t s, const float* x_dev, const float* t_dev,
                                     int64_t B, float* grads, float* loss, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at learning rate lr; loss (host, may be
 * NULL, then no synchronisation) receives the batch loss before the step. */
rimo_status rimo_surrogate_train_step(rimo_surrogate_t s, const float* x_dev, const float* t_dev,
                                      int64_t B, float lr, float* loss, void* stream);

/*
 * Batched wideband Phi^dagger Phi.  The wideband model applies the monochromatic operator
 * per frequency channel (Section 2; per-frequency worker pools, Section 3.5): a batch
 * groups independent plans, one per channel, each with its own uvw, w-stack and sizes of
 * w-bins, and all of the same image size.  The caller keeps owning the plans (destroy the
 * batch first); a plan may belong to one batch at a time and must not be applied on its
 * own while a batch call using it is in flight (plans have scratch).
 */
typedef struct rimo_batch* rimo_batch_t;
/* Errors: INVALID_ARG (no plans, NULL plan, a plan twice, image sizes differ, plans on
 * another device), OOM (staged scratch), CUDA.  Same as rimo_batch_create_form with
 * RIMO_BATCH_AUTO. */
rimo_status rimo_batch_create(const rimo_plan_t* plans, int32_t n_plans, rimo_batch_t* out);
/*
 * The form of a batch's recorded Phi^dagger Phi:
 *  RIMO_BATCH_STAGED   every (channel, w-bin) of the batch is a job with scratch of its own
 *                      (2 nx ny + 4 nx ny complex64 plus its tile patches, allocated once
 *                      here, freed by rimo_batch_destroy; rimo_batch_layout reports the
 *                      bytes), and each pass of Eq. 7-8 is ONE launch over all jobs: forward
 *                      rows and cols (F Z_p), the grid step G_p^H G_p as one persistent
 *                      launch whose blocks take the work units (uv-tiles or slices of heavy
 *                      ones) of every channel and bin from one heaviest-first queue, the
 *                      merge of split tiles, the fold, inverse cols, and inverse rows that
 *                      also sums each channel's bins.  Needs stored-G plans (no H) with
 *                      square images of one size (64 .. 4096) and one uv-tile size.
 *  RIMO_BATCH_BRANCHES each channel's own apply on a branch of a fork/join pattern.
 *  RIMO_BATCH_AUTO     staged when the plans allow it, else branches.
 * Results are the same in both forms, bit for bit (fixed-point grid step, same kernels).
 * Errors: as rimo_batch_create; UNSUPPORTED (STAGED asked for plans that do not allow it).
 */
#define RIMO_BATCH_AUTO 0
#define RIMO_BATCH_STAGED 1
#define RIMO_BATCH_BRANCHES 2
rimo_status rimo_batch_create_form(const rimo_plan_t* plans, int32_t n_plans, int32_t form, rimo_batch_t* out);
/* NULL is accepted. */
rimo_status rimo_batch_destroy(rimo_batch_t batch);
/*
 * out[c] = Phi_c^dagger Phi_c x[c] for every channel c of the batch, where x_dev and
 * out_dev hold n_plans images of ny x nx complex64 back to back (device, distinct,
 * non-overlapping).  The first call, and any call with other buffers or another
 * real_part_only, records the batch's form (see rimo_batch_create_form) into one CUDA
 * graph, after waiting for the device to finish earlier work (a staged batch rewrites
 * its job tables); each call then enqueues that graph with a single launch on `stream`.
 * Per-plan stage timers are not recorded inside the graph.  Device-side error flags are
 * per plan (rimo_plan_status).
 * Errors: INVALID_ARG, CUDA.
 */
rimo_status rimo_batch_apply_phi_adj_phi(rimo_batch_t batch, const rimo_cfloat* x_dev, rimo_cfloat* out_dev,
                                         int32_t real_part_only, void* stream);
/* Number of plans and how many times the graph was recorded (either may be NULL). */
rimo_status rimo_batch_info(rimo_batch_t batch, int32_t* n_plans, int64_t* captures);
/* The batch's form and work (any pointer may be NULL): staged (1) or branches (0); the
 * (channel, w-bin) jobs and the grid-step work units of the staged form; the bytes of its
 * job scratch. */
rimo_status rimo_batch_layout(rimo_batch_t batch, int32_t* staged, int64_t* jobs, int64_t* units,
                              int64_t* scratch_bytes);

/*
 * Tile-size autotuner (no counterpart in the paper: a scheduling choice of this design).
 * Times Phi^dagger Phi with uv-tile sizes 32 and 64 on plans built from a deterministic
 * subsample of uvw (every ceil(M / 2^20)-th row) with the other fields of `base`, and
 * writes the faster one to *tile_out.  cache_path (host string, may be NULL or ""): a JSON
 * object {"key": tile, ...} keyed by image size, FoV, log2 M, P, J and maximum tile side;
 * a hit returns without timing, a miss adds the result (the file is rewritten whole).
 * ms_out (host, 2 values, may be NULL): the measured ms per apply for 32 and 64, or -1
 * when not timed.  Allocates and frees two image buffers and two plans; synchronises
 * `stream`.  Errors: INVALID_ARG (also for an unwritable cache), OOM, BUDGET, CUDA.
 */
rimo_status rimo_autotune_tile(const double* uvw, int64_t M, const rimo_plan_params* base, const char* cache_path,
                               void* stream, int32_t* tile_out, double* ms_out);
/*
 * The same over both scheduling choices of the grid step: uv-tile size (32, 64) and the
 * order of visibilities within a tile (uv_order 0, 1, 2; see rimo_plan_params), six plans
 * timed on the subsample in the order (32, 0), (32, 1), (32, 2), (64, 0), (64, 1), (64, 2).
 * Writes the fastest to *tile_out and *order_out; ms_out (host, 6 values, may be NULL):
 * their ms per apply, or -1 when not timed.  Cache entries (key suffix "_tile_order")
 * hold tile * 10 + order.  Errors as rimo_autotune_tile.
 */
rimo_status rimo_autotune(const double* uvw, int64_t M, const rimo_plan_params* base, const char* cache_path,
                          void* stream, int32_t* tile_out, int32_t* order_out, double* ms_out);
/*
 * The same choice for a batch of workloads (the channels of a wideband batch, or a sample
 * of them): for every candidate, one plan per workload (every ceil(M[i] / 2^22)-th row) is
 * made and the plans are recorded as one batch (rimo_batch_create_form, RIMO_BATCH_AUTO),
 * whose Phi^dagger Phi is timed; the pick is the fastest batch.  (Timing the channels one
 * plan at a time does not rank the candidates as the batch does: there the per-bin launch
 * costs, which a batch amortises, hide the grid step's share.)  uvw[i] (host, M[i] x 3) and
 * base[i] describe workload i of n (base[i] with its own FoV and w-bins; one image size for
 * all).  ms_out (host, 6 values, may be NULL): the batch's ms per apply for each candidate,
 * or -1 when not timed.  Cache entries (key: the workloads' shape keys joined, suffix
 * "_batch_tile_order") hold tile * 10 + order.  Allocates and frees 2 n images, n plans and
 * one batch per candidate; synchronises `stream`.  Errors as rimo_autotune.
 */
rimo_status rimo_autotune_batch(const double* const* uvw, const int64_t* M, const rimo_plan_params* base, int32_t n,
                                const char* cache_path, void* stream, int32_t* tile_out, int32_t* order_out,
                                double* ms_out);

/*
 * Data weighting injected into the measurement operator (Section 2, Eq. 3: a weighting
 * such as Briggs' is applied to the data and injected into the model).  After this call
 * the plan's operator is W Phi with W = diag(w): Phi returns w_k y_k, Phi^dagger takes
 * W y, Phi^dagger Phi becomes Phi^dagger W^2 Phi and a holographic matrix built later is
 * G^dagger W^2 G.  The weights multiply the tiles of G (a stored-G plan rebuilds G on
 * `stream`; plans that generate tiles multiply them at generation), so an apply costs the
 * same as without weights.  rimo_plan_get_tiles then returns weighted tiles.
 * w: host, M values in caller order, finite and >= 0 (copied); NULL removes the weighting.
 * Errors: INVALID_ARG (null plan, negative or non-finite weight), STATE (the plan's
 * tiles were already folded into H), CUDA.  Synchronises `stream`.
 */
rimo_status rimo_plan_set_weights(rimo_plan_t plan, const float* w, void* stream);

/*
 * Briggs' robust weights of unit natural weights (the weighting Section 2 cites), on the
 * image's Fourier grid: nx x ny cells of 1/fov_x x 1/fov_y; visibility k falls in cell
 * (floor(u_k fov_x + 1/2) mod nx, floor(v_k fov_y + 1/2) mod ny); with D_c the number of
 * visibilities of cell c, f^2 = (5 10^-robust)^2 M / sum_c D_c^2 and
 * w_k = 1 / (1 + f^2 D_c(k)).  robust -> +inf gives natural weights (1), -inf uniform.
 * uvw: host, M x 3 (wavelengths); w_out: host, M floats.  Computed on the host (FP64).
 * Errors: INVALID_ARG (null pointer, M < 0, nx or ny < 1, non-positive field of view).
 */
rimo_status rimo_briggs_weights(const double* uvw, int64_t M, int32_t nx, int32_t ny, double fov_x,
                                double fov_y, double robust, float* w_out);

/*
 * One forward-backward update of Eq. 4 with the denoising step D = projection onto the
 * non-negative real images (the image model of Eq. 3): out = max(Re x + gamma (Re dirty -
 * Re g), 0) + 0i elementwise, where g = Phi^dagger Phi x (an apply's output) and dirty =
 * Phi^dagger y.  x, g, dirty, out: device, n complex values (out may alias x).
 * Enqueued on `stream`.  Errors: INVALID_ARG (null pointer, n < 0, gamma < 0 or not finite).
 */
rimo_status rimo_fb_step(const rimo_cfloat* x, const rimo_cfloat* g, const rimo_cfloat* dirty, float gamma,
                         rimo_cfloat* out, int64_t n, void* stream);

/*
 * *result = Re sum_i conj(a_i) b_i over n complex values (device buffers), accumulated in
 * FP64 in a fixed order (deterministic); for the data fidelity 1/2 ||Phi x - y||^2 =
 * 1/2 (<x, Phi^dagger Phi x> - 2 <x, Phi^dagger y> + ||y||^2) and power iterations.
 * result: host.  Synchronises `stream`; concurrent calls take turns.
 * Errors: INVALID_ARG (null pointer, n < 0), CUDA.
 */
rimo_status rimo_image_dot(const rimo_cfloat* a, const rimo_cfloat* b, int64_t n, double* result, void* stream);

/*
 * Kernel surrogate as the plan's tile generator.  A plan created with mode
 * RIMO_MODE_SURROGATE (kb_support + max_wsupport - 1 must be 15) places every visibility
 * with the largest support (15 x 15 tiles), keeps one Fourier block per w-bin and stores
 * no G: each apply generates one bin's tiles at a time with the attached network into a
 * scratch the size of the largest bin, then grids them as the stored-G path does.
 * rimo_plan_set_surrogate attaches s (not owned; it must outlive its use, and one
 * surrogate must not serve two applies at once) and allocates the generation buffers.
 * Applies and tile read-back of a surrogate plan without a surrogate fail with STATE;
 * rimo_build_holographic and the allocation-free apply return UNSUPPORTED.
 * The generator runs the whole network per 128 visibilities in one persistent kernel
 * (BF16 operands on the tensor cores, FP32 accumulation, layer 1 and GELU in FP32,
 * hidden activations rounded to BF16 as in rimo_surrogate_forward).
 * Errors: INVALID_ARG (plan not in surrogate mode, other device), OOM, CUDA.
 */
rimo_status rimo_plan_set_surrogate(rimo_plan_t plan, rimo_surrogate_t s);

/*
 * Train s on exact tiles: n_samples visibilities of `exact` (a stored-G plan with 15 x 15
 * tiles; smaller supports are embedded at the centre) drawn uniformly by a counter-based
 * SplitMix64 from `seed`, inputs (2 phi_u - 1, 2 phi_v - 1, w_r / w_scale) with w_scale =
 * the plan's largest |w_r|; `steps` Adam steps on batches of `batch` (a multiple of 128)
 * drawn from the samples, learning rate decaying from lr to lr / 100 (cosine).  losses
 * (host, `steps` values, may be NULL): each step's mean squared error before the update.
 * Sets the surrogate's w_scale.  Synchronises `stream`.  Errors: INVALID_ARG, OOM,
 * TIMEOUT, CUDA.
 */
rimo_status rimo_surrogate_fit(rimo_surrogate_t s, rimo_plan_t exact, int64_t n_samples, int32_t steps,
                               int32_t batch, float lr, uint64_t seed, float* losses, void* stream);
/* The w_r normalisation of the inputs (0 until fitted or set; then the plan's largest
 * |w_r| is used). */
rimo_status rimo_surrogate_get_w_scale(rimo_surrogate_t s, float* w_scale);
rimo_status rimo_surrogate_set_w_scale(rimo_surrogate_t s, float w_scale);

/* Thread-local description of the last failure on this thread ("" if none). */
const char* rimo_last_error(void);

/* Library version string. */
const char* rimo_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RIMO_H */
