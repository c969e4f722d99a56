// Plan creation (stages 1 - 3 of Fig. 3): planning, per-visibility placement on the
// oversampled grid, uv-tile sort, Fourier blocks (Section 3.2) and the device-side
// build of the de-gridding matrix G.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>

#include "internal.h"
#include "planner.h"

namespace rimo {

static thread_local std::string g_last_error;

void set_last_error(const std::string& msg) { g_last_error = msg; }

void fail(rimo_status s, const std::string& msg) { throw Error{s, msg}; }

void check_cuda(cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (e == cudaErrorMemoryAllocation)
            fail(RIMO_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
        fail(RIMO_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
}

void* dev_alloc(rimo_plan* p, size_t bytes) {
    void* ptr = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(RIMO_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                               cudaGetErrorString(e));
    }
    p->owned.push_back(ptr);
    return ptr;
}

template <class T>
static T* upload(rimo_plan* p, const std::vector<T>& v, cudaStream_t s) {
    T* d = (T*)dev_alloc(p, v.size() * sizeof(T));
    if (!v.empty()) RIMO_CUDA(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return d;
}

// ---------------------------------------------------------------------------
// Kaiser-Bessel helpers (FP64, host): I0 by its power series; the Fourier transform
// J sinh(sqrt(beta^2 - (pi J nu)^2)) / (I0(beta) sqrt(beta^2 - (pi J nu)^2)).
static double bessel_i0(double x) {
    double q = 0.25 * x * x, term = 1.0, sum = 1.0;
    for (int k = 1; k < 500; ++k) {
        term *= q / ((double)k * k);
        sum += term;
        if (term <= 1e-18 * sum) break;
    }
    return sum;
}

static double kb_hat(double nu, int J, double beta) {
    double a2 = beta * beta - (M_PI * J * nu) * (M_PI * J * nu);
    double r;
    if (a2 > 1e-12) r = std::sinh(std::sqrt(a2)) / std::sqrt(a2);
    else if (a2 < -1e-12) r = std::sin(std::sqrt(-a2)) / std::sqrt(-a2);
    else r = 1.0;
    return J * r / bessel_i0(beta);
}

static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

void validate_params(const rimo_plan_params& q) {
    auto bad = [](const std::string& m) { fail(RIMO_ERR_INVALID_ARG, m); };
    if (!is_pow2(q.nx) || !is_pow2(q.ny) || q.nx < 64 || q.ny < 64 || q.nx > 4096 || q.ny > 4096)
        bad("nx and ny must be powers of two in [64, 4096]");
    if (!(q.fov_x > 0) || !(q.fov_y > 0) || q.fov_x * q.fov_x + q.fov_y * q.fov_y >= 0.99)
        bad("fov_x and fov_y must be positive and keep (2 fov)^2 / 4 summed below 1");
    if (q.oversampling != 2) bad("oversampling must be 2");
    if (q.kb_support < 3 || q.kb_support > 11 || (q.kb_support & 1) == 0)
        bad("kb_support must be odd in [3, 11]");
    if (q.max_wsupport < 1 || q.max_wsupport > 9 || (q.max_wsupport & 1) == 0)
        bad("max_wsupport must be odd in [1, 9]");
    if (!(q.w_norm_frac > 0) || q.w_norm_frac > 1) bad("w_norm_frac must be in (0, 1]");
    if (q.n_wbins < 0 || q.n_wbins > 4096) bad("n_wbins must be in [0, 4096]");
    if (q.mode < 0 || q.mode > 4) bad("mode must be a rimo_mode");
    if (q.n_weight < 0 || q.n_weight > 1) bad("n_weight must be 0 or 1");
    if (q.plan_fraction <= 0 || q.plan_fraction > 1) bad("plan_fraction must be in (0, 1]");
    if (q.wkernel_L != 0 && (!is_pow2(q.wkernel_L) || q.wkernel_L < 16 || q.wkernel_L > 128))
        bad("wkernel_L must be 0 or a power of two in [16, 128]");
    if (q.tile_size != 0 && q.tile_size != 32 && q.tile_size != 64) bad("tile_size must be 0, 32 or 64");
    if (q.wkernel_table != 0 && (q.wkernel_table < 16 || q.wkernel_table > (1 << 22)))
        bad("wkernel_table must be 0 or in [16, 2^22]");
    if (q.uv_order < 0 || q.uv_order > 2) bad("uv_order must be 0, 1 or 2");
    if (q.shard_count < 0 || q.shard_count > 1024) bad("shard_count must be in [0, 1024]");
    if (q.shard_rank < 0 || q.shard_rank >= std::max(1, q.shard_count))
        bad("shard_rank must be in [0, shard_count)");
    if (q.kb_beta < 0) bad("kb_beta must be >= 0");
}

// Every coordinate finite and within the range where the placement (floor, integer
// conversion, wrap) and the k-means sums stay exact: |u| 2 fov_x, |v| 2 fov_y and |w|
// below 2^52.  Checked in parallel; the error is raised on the calling thread.
void validate_uvw(const double* uvw, int64_t M, const rimo_plan_params& q) {
    const double lim = 0x1.0p52;
    std::atomic<bool> bad{false};
    planner::parallel_for(M, [&](int64_t b, int64_t e) {
        bool ok = true;
        for (int64_t k = b; k < e; ++k) {
            const double u = std::fabs(uvw[3 * k] * (2.0 * q.fov_x)), v = std::fabs(uvw[3 * k + 1] * (2.0 * q.fov_y));
            const double w = std::fabs(uvw[3 * k + 2]);
            ok &= (u < lim) & (v < lim) & (w < lim);  // false for NaN as well
        }
        if (!ok) bad.store(true);
    }, 1 << 16);
    if (bad.load()) fail(RIMO_ERR_INVALID_ARG, "uvw holds a non-finite coordinate or one beyond 2^52 grid cells");
}

static planner::Params planner_params(const rimo_plan_params& q) {
    planner::Params pr;
    pr.nx = q.nx;
    pr.ny = q.ny;
    pr.J = q.kb_support;
    pr.kg.L = q.wkernel_L ? q.wkernel_L
                          : std::max(32, 1 << (int)std::ceil(std::log2(4.0 * q.max_wsupport)));
    pr.kg.max_wsupport = q.max_wsupport;
    pr.kg.fov_x = q.fov_x;
    pr.kg.fov_y = q.fov_y;
    pr.kg.eta = q.w_norm_frac;
    pr.kg.literal = q.taper_literal != 0;
    pr.seed = q.seed;
    pr.plan_fraction = q.plan_fraction;
    pr.n_wbins = q.n_wbins;
    pr.mode = q.mode;
    pr.budget = q.mem_budget_bytes;
    return pr;
}

static void fill_estimate(rimo_plan_info* info, const planner::Choice& ch, int64_t M, int L) {
    info->M = M;
    info->P = ch.P;
    info->mode = ch.mode;
    info->p_star = ch.p_star;
    info->subset = ch.subset;
    info->est_m_g = ch.est_m_g;
    info->est_cost = ch.est_cost;
    info->wsclean_p = ch.wsclean;
    info->wkernel_L = L;
    for (const auto& m : ch.models)
        if (m.P == ch.P) info->truncated = m.truncated ? 1 : 0;
}

// ---------------------------------------------------------------------------
// Device tables of one plan.
static void build_tables(rimo_plan* p, cudaStream_t s) {
    const int nx = p->nx, ny = p->ny, J = p->J, L = p->L;

    // Stockham stage tables: stage 2 combines NS = 16 points with radix R2, stage 3
    // NS = 256 with radix R3; entry [r NS + j] = W_{NS R}^{r j} = e^{-2 pi i r j / (NS R)}
    // stage twiddle tables of the L-point transforms (L = 2 n): stages 16 (NS 16),
    // 16 or L/256 (NS 256), L/4096 (NS 4096), laid out [r][j]
    auto stage_twiddles = [](int N) {
        const int R2 = N <= 256 ? N / 16 : 16;
        const int R3 = N <= 256 ? 0 : (N <= 4096 ? N / 256 : 16);
        const int R4 = N <= 4096 ? 0 : N / 4096;
        std::vector<float2> t((size_t)std::max(N, 256 + 256 * std::max(R3, 1) + 4096 * R4), make_float2(0.f, 0.f));
        auto fill = [&](size_t off, int NS, int R) {
            for (int r = 0; r < R; ++r)
                for (int j = 0; j < NS; ++j) {
                    double a = -2.0 * M_PI * (double)r * j / ((double)NS * R);
                    t[off + (size_t)r * NS + j] = make_float2((float)std::cos(a), (float)std::sin(a));
                }
        };
        fill(0, 16, R2);
        if (R3) fill(256, 256, R3);
        if (R4) fill(256 + 4096, 4096, R4);
        return t;
    };
    p->tab.tws_x = upload(p, stage_twiddles(2 * nx), s);
    p->tab.tws_y = upload(p, stage_twiddles(2 * ny), s);
    if (ny == 4096) {  // the 8192-point column passes run with 32 points per thread
        std::vector<float2> t(512 + 8192);
        for (int r = 0; r < 16; ++r) {
            for (int j = 0; j < 32; ++j) {
                const double a = -2.0 * M_PI * (double)r * j / 512.0;
                t[(size_t)r * 32 + j] = make_float2((float)std::cos(a), (float)std::sin(a));
            }
            for (int j = 0; j < 512; ++j) {
                const double a = -2.0 * M_PI * (double)r * j / 8192.0;
                t[512 + (size_t)r * 512 + j] = make_float2((float)std::cos(a), (float)std::sin(a));
            }
        }
        p->tab.tws32 = upload(p, t, s);
    }
    // Z_p on the quarter plane [|i_c|][|j_c|]: (n - 1) as a float pair for the w-phase and
    // |Z_p| = gc_x gc_y [/ n] (the grid correction is even in j_c and i_c), in FP64 then rounded
    const int qx = nx / 2 + 1, qy = ny / 2 + 1;
    std::vector<float4> zq((size_t)qx * qy);
    const double dl = p->prm.fov_x / nx, dm = p->prm.fov_y / ny;
    std::vector<double> gx_q(qx), gy_q(qy);
    for (int j = 0; j < qx; ++j) gx_q[j] = 1.0 / kb_hat((double)j / (2.0 * nx), J, p->beta);
    for (int i = 0; i < qy; ++i) gy_q[i] = 1.0 / kb_hat((double)i / (2.0 * ny), J, p->beta);
    const bool div_n = p->prm.n_weight == RIMO_NWEIGHT_DIV_N;
    for (int i = 0; i < qy; ++i)
        for (int j = 0; j < qx; ++j) {
            const double d = planner::dn(j * dl, i * dm);
            const float hi = (float)d;
            double g = gx_q[j] * gy_q[i];
            if (div_n) g /= 1.0 + d;
            zq[(size_t)i * qx + j] = make_float4(hi, (float)(d - (double)hi), (float)g, 0.f);
        }
    p->tab.zq = upload(p, zq, s);
    // KB(t) = sum_k e_k rho^k, rho = 1 - (2t/J)^2, e_k = (beta^2/4)^k / (k!)^2 / I0(beta)
    std::vector<float> coef;
    {
        double i0b = bessel_i0(p->beta), q0 = 0.25 * p->beta * p->beta, d = 1.0;
        for (int k = 0; k < 96; ++k) {
            if (k > 0) d *= q0 / ((double)k * k);
            coef.push_back((float)(d / i0b));
            if (k > 4 && d / i0b < 1e-13) break;
        }
    }
    p->tab.kb_nterm = (int)coef.size();
    p->tab.kb_coef = upload(p, coef, s);
    // residual w-kernel sampling grid over twice the field of view (Section 3.1, Fig. 1),
    // folded over the signs of (lam, mu): the chirp is even in both, the edge -L/2 is kept
    // once as a' = L/2 (same |lam|)
    const int Q = L / 2 + 1;
    std::vector<float> wdn((size_t)Q * Q), tx(Q), ty(Q);
    auto taper = [](double lam, double fov) {
        double a = std::fabs(lam), half = 0.5 * fov;
        return a <= half ? 1.0 : 0.54 + 0.46 * std::cos(M_PI * (a - half) / half);
    };
    for (int a = 0; a < Q; ++a) {
        double lam = a * (2.0 * p->prm.fov_x / L);
        double mu = a * (2.0 * p->prm.fov_y / L);
        tx[a] = (float)taper(lam, p->prm.fov_x);
        ty[a] = (float)taper(mu, p->prm.fov_y);
    }
    for (int a = 0; a < Q; ++a)
        for (int b = 0; b < Q; ++b) {
            double lam = a * (2.0 * p->prm.fov_x / L);
            double mu = b * (2.0 * p->prm.fov_y / L);
            wdn[(size_t)a * Q + b] = (float)planner::dn(lam, mu);
        }
    std::vector<float> wc((size_t)Q * 8, 0.f);  // rows of 8, offsets t in [0, 4]
    for (int a = 0; a < Q; ++a)
        for (int t = 0; t < 5; ++t) {
            const double m = (a == 0 || a == L / 2) ? 1.0 : 2.0;
            wc[(size_t)a * 8 + t] = (float)(m * std::cos(2.0 * M_PI * (double)a * (double)t / (double)L));
        }
    p->tab.wk_dn = upload(p, wdn, s);
    p->tab.wk_tau_x = upload(p, tx, s);
    p->tab.wk_tau_y = upload(p, ty, s);
    p->tab.wk_wc = upload(p, wc, s);
}

// ---------------------------------------------------------------------------
static void create_plan(const double* uvw, int64_t M, const rimo_plan_params& q, cudaStream_t s,
                        rimo_plan* p) {
    validate_params(q);
    p->prm = q;
    p->nx = q.nx;
    p->ny = q.ny;
    p->gx = 2 * q.nx;
    p->gy = 2 * q.ny;
    p->J = q.kb_support;
    p->beta = q.kb_beta > 0 ? q.kb_beta : 2.34 * q.kb_support;
    p->TS = q.tile_size ? q.tile_size : 32;
    p->info.tile_size = p->TS;
    p->M = M;
    planner::Params pr = planner_params(q);
    p->L = pr.kg.L;
    p->hmax = q.max_wsupport / 2;

    // ---- stage 1: planning on the subset (Section 3.4)
    planner::Choice ch = planner::choose(uvw, M, pr);
    fill_estimate(&p->info, ch, M, p->L);
    p->P = ch.P;
    p->mode = ch.mode;
    const bool surrogate = p->mode == RIMO_MODE_SURROGATE;
    // tiles generated per bin at apply time, by the network or exactly (no stored G)
    // (a holographic plan stores no G either: Phi and Phi^dagger, and Phi^dagger Phi until
    // rimo_build_holographic has run, generate exact tiles on the fly; Fig. 2 regimes b, c)
    const bool generated = surrogate || p->mode == RIMO_MODE_ONTHEFLY || p->mode == RIMO_MODE_HOLOGRAPHIC;
    const bool sharded = q.shard_count >= 2;
    if (sharded && p->mode != RIMO_MODE_STORED_G)
        fail(RIMO_ERR_UNSUPPORTED, "a shard plan (shard_count >= 2) stores G: its mode must be STORED_G");
    if (surrogate && (q.kb_support + q.max_wsupport - 1 != 15))
        fail(RIMO_ERR_UNSUPPORTED, "the kernel surrogate generates 15 x 15 tiles: kb_support + max_wsupport - 1 must be 15");

    // ---- w-bins on the subset, every visibility to its nearest bin (Section 3.1)
    std::vector<double> w_sub = planner::subset_w(uvw, M, q.seed, q.plan_fraction);
    p->w_stack = planner::kmeans1d(w_sub, p->P, 100);
    std::vector<int32_t> bin(M);
    planner::nearest_all(uvw + 2, M, 3, p->w_stack, bin.data());
    std::vector<double> wr(M);
    double wr_max = 0.0;
    for (int64_t k = 0; k < M; ++k) {
        wr[k] = uvw[3 * k + 2] - p->w_stack[bin[k]];
        wr_max = std::max(wr_max, std::fabs(wr[k]));
    }
    std::vector<int32_t> tab = planner::support_table(wr_max, pr.kg);
    p->info.wr_max = wr_max;
    p->info.truncated = planner::truncated_at(wr_max, pr.kg) ? 1 : 0;
    for (int i = 0; i < 64; ++i) p->info.support_table[i] = tab[i];

    // ---- placement on the oversampled grid: u~ = u * (2 fov_x), one FP64 multiply
    const int J = p->J, TS = p->TS, gx = p->gx, gy = p->gy;
    const int ntu = gx / TS, ntv = gy / TS;
    std::vector<int32_t> sw(M), g0(M), h0(M);
    std::vector<float> phiu(M), phiv(M);
    int max_sw = 1;
    planner::parallel_for(M, [&](int64_t b, int64_t e) {
        for (int64_t k = b; k < e; ++k) {
            // the surrogate generates every tile at the largest support
            int Sw = surrogate ? q.max_wsupport : tab[planner::support_bin(std::fabs(wr[k]), wr_max)];
            sw[k] = Sw;
            int h = (Sw - 1) / 2;
            double tu = uvw[3 * k + 0] * (2.0 * q.fov_x) - J / 2.0;
            double tv = uvw[3 * k + 1] * (2.0 * q.fov_y) - J / 2.0;
            double fu = std::floor(tu), fv = std::floor(tv);
            phiu[k] = (float)(tu - fu);
            phiv[k] = (float)(tv - fv);
            int64_t a = (int64_t)fu + 1 - h, c = (int64_t)fv + 1 - h;
            a %= gx; if (a < 0) a += gx;
            c %= gy; if (c < 0) c += gy;
            g0[k] = (int32_t)a;
            h0[k] = (int32_t)c;
        }
    }, 1 << 16);
    for (int64_t k = 0; k < M; ++k) max_sw = std::max(max_sw, sw[k]);
    p->max_S = max_sw + J - 1;
    p->H = p->max_S - 1;
    p->PW = TS + p->H;
    p->info.max_tile = p->max_S;

    // ---- sort by (bin, uv-tile): stable counting sort, bins first then tiles per bin
    const int P = p->P;
    std::vector<int64_t> bstart(P + 1, 0);
    for (int64_t k = 0; k < M; ++k) bstart[bin[k] + 1]++;
    for (int b = 0; b < P; ++b) bstart[b + 1] += bstart[b];
    std::vector<int32_t> by_bin(M);
    {
        std::vector<int64_t> cur(bstart.begin(), bstart.end() - 1);
        for (int64_t k = 0; k < M; ++k) by_bin[cur[bin[k]]++] = (int32_t)k;
    }
    std::vector<int32_t> order(M);
    const int64_t ntile = (int64_t)ntu * ntv;
    std::vector<std::vector<int64_t>> tstart(P);
    planner::parallel_for(P, [&](int64_t b0, int64_t b1) {
        for (int64_t b = b0; b < b1; ++b) {
            auto& st = tstart[b];
            st.assign(ntile + 1, 0);
            for (int64_t i = bstart[b]; i < bstart[b + 1]; ++i) {
                int k = by_bin[i];
                st[(int64_t)(g0[k] / TS) * ntv + h0[k] / TS + 1]++;
            }
            for (int64_t t = 0; t < ntile; ++t) st[t + 1] += st[t];
            std::vector<int64_t> cur(st.begin(), st.end() - 1);
            for (int64_t i = bstart[b]; i < bstart[b + 1]; ++i) {
                int k = by_bin[i];
                int64_t t = (int64_t)(g0[k] / TS) * ntv + h0[k] / TS;
                order[bstart[b] + cur[t]++] = k;
            }
        }
    }, 1);
    std::vector<int32_t>().swap(by_bin);

    // ---- active tiles, phases, Fourier blocks by radial sweep (Section 3.2)
    struct T {
        int32_t tu, tv;
        int64_t vb, ve;
        double r, bytes;
    };
    std::vector<std::vector<T>> tl(P);
    std::vector<int32_t> tmp;
    double total_bytes = 0.0;
    for (int b = 0; b < P; ++b) {
        for (int64_t t = 0; t < ntile; ++t) {
            int64_t vb = tstart[b][t], ve = tstart[b][t + 1];
            if (ve == vb) continue;
            T x;
            x.tu = (int32_t)(t / ntv);
            x.tv = (int32_t)(t % ntv);
            x.vb = bstart[b] + vb;
            x.ve = bstart[b] + ve;
            double cu = x.tu * TS + 0.5 * TS, cv = x.tv * TS + 0.5 * TS;
            if (cu >= gx / 2) cu -= gx;
            if (cv >= gy / 2) cv -= gy;
            x.r = std::sqrt(cu * cu + cv * cv);
            // Interleave the tile's visibilities (arrival order within a tile is time, so
            // neighbours are the same few baselines a fraction of a cell apart): viewed
            // as GTG_CHUNK rows of nc, the new order reads the list column by column, so
            // that the GTG_CHUNK consecutive visibilities of one ring chunk, de-gridded and
            // gridded at the same time by as many warps, come from far-apart instants and
            // rarely update the same grid cells.
            // (uv_order 0; 1 keeps the time order; 2 orders the tile's visibilities by a
            // SplitMix64 hash of their index)
            if (q.uv_order == 0) {
                const int64_t n = x.ve - x.vb, nc = (n + GTG_CHUNK - 1) / GTG_CHUNK;
                tmp.assign(order.begin() + x.vb, order.begin() + x.ve);
                int64_t o = x.vb;
                for (int64_t c = 0; c < nc; ++c)
                    for (int64_t r = 0; r < GTG_CHUNK; ++r)
                        if (r * nc + c < n) order[o++] = tmp[r * nc + c];
            } else if (q.uv_order == 2) {
                std::stable_sort(order.begin() + x.vb, order.begin() + x.ve, [](int32_t a, int32_t b) {
                    return planner::splitmix64((uint64_t)a) < planner::splitmix64((uint64_t)b);
                });
            }
            x.bytes = 0;
            for (int64_t i = x.vb; i < x.ve; ++i) {
                int64_t S = sw[order[i]] + J - 1;
                x.bytes += 8.0 * (double)(S * S + ((S * S) & 1));
            }
            total_bytes += x.bytes;
            tl[b].push_back(x);
        }
    }
    tstart.clear();
    if (sharded) {
        // level 2 (Section 3.5): this shard keeps the tiles of every bin whose place in the
        // bin's radial order (ties by row, then column) is shard_rank modulo shard_count
        total_bytes = 0.0;
        for (int b = 0; b < P; ++b) {
            std::vector<int> ix(tl[b].size());
            std::iota(ix.begin(), ix.end(), 0);
            std::sort(ix.begin(), ix.end(), [&](int x, int y) {
                const T& A = tl[b][x];
                const T& B = tl[b][y];
                if (A.r != B.r) return A.r < B.r;
                return A.tu != B.tu ? A.tu < B.tu : A.tv < B.tv;
            });
            std::vector<uint8_t> own(tl[b].size(), 0);
            for (size_t i = 0; i < ix.size(); ++i) own[ix[i]] = (int)(i % (size_t)q.shard_count) == q.shard_rank;
            std::vector<T> kept;
            for (size_t i = 0; i < tl[b].size(); ++i)
                if (own[i]) {
                    kept.push_back(tl[b][i]);
                    total_bytes += tl[b][i].bytes;
                }
            tl[b].swap(kept);
        }
    }
    double limit = q.block_bytes_max > 0 ? (double)q.block_bytes_max : 8.0 * 1073741824.0;
    if (q.n_blocks > 0) limit = std::ceil(total_bytes / q.n_blocks);
    limit = std::max(limit, std::ceil(total_bytes / 200.0));
    if (generated) limit = 1e300;  // one block per bin: its taps are generated into one scratch
    // visibilities of no tile of this plan (other shards') keep block SHARD_SKIP: no taps
    std::vector<VisMeta> meta(M, VisMeta{0, 0u, (uint32_t)SHARD_SKIP << 24});
    std::vector<float> wr_s(M), pu_s(M), pv_s(M);
    p->bins.assign(P, BinRange());
    p->block_bytes.clear();
    int64_t K = 0;
    for (int b = 0; b < P; ++b) {
        auto& v = tl[b];
        std::vector<int> rad(v.size());
        std::iota(rad.begin(), rad.end(), 0);
        std::stable_sort(rad.begin(), rad.end(), [&](int x, int y) { return v[x].r < v[y].r; });
        double cur = 0.0;
        int64_t off = 0;
        bool open = false;
        for (int id : rad) {
            if (!open || (cur + v[id].bytes > limit && cur > 0)) {
                p->block_bytes.push_back(0);
                cur = 0.0;
                off = 0;
                open = true;
            }
            int blk = (int)p->block_bytes.size() - 1;
            for (int64_t i = v[id].vb; i < v[id].ve; ++i) {
                int k = order[i];
                int S = sw[k] + J - 1;
                int du = g0[k] - v[id].tu * TS, dv = h0[k] - v[id].tv * TS;
                meta[i].off = off;
                meta[i].orig = (uint32_t)k;
                meta[i].pos = (uint32_t)du | ((uint32_t)dv << 8) | ((uint32_t)S << 16) |
                              ((uint32_t)blk << 24);
                int64_t n = (int64_t)S * S;
                off += n + (n & 1);
                K += n;
                wr_s[i] = (float)wr[k];
                pu_s[i] = phiu[k];
                pv_s[i] = phiv[k];
            }
            cur += v[id].bytes;
            p->block_bytes.back() = off * 8;
        }
        p->bins[b].vb = bstart[b];
        p->bins[b].ve = bstart[b + 1];
        p->bins[b].w = p->w_stack[b];
        p->bins[b].w_hi = (float)p->w_stack[b];
        p->bins[b].w_lo = (float)(p->w_stack[b] - (double)p->bins[b].w_hi);
    }
    if (p->block_bytes.size() > SHARD_SKIP) fail(RIMO_ERR_INVALID_ARG, "more than 255 Fourier blocks");
    // work units: active uv-tiles, split into units of at most `cap` visibilities so that
    // no unit outweighs a fraction of one SM's share of the bin; slots group the units of
    // a tile contiguously (merge groups), the schedule orders units heaviest first
    p->tiles_host.clear();
    p->sched_host.clear();
    p->merge_host.clear();
    int n_active = 0;
    std::vector<int32_t> slot((size_t)P * ntile, -1);
    int nsm_host = 0;
    {
        int dev = 0;
        RIMO_CUDA(cudaGetDevice(&dev));
        RIMO_CUDA(cudaDeviceGetAttribute(&nsm_host, cudaDevAttrMultiProcessorCount, dev));
    }
    for (int b = 0; b < P; ++b) {
        const int64_t bin_vis = bstart[b + 1] - bstart[b];
        const int64_t cap = std::min<int64_t>(
            FX_MAX_UNIT, std::max<int64_t>(256, (bin_vis + 2 * nsm_host - 1) / (2 * (int64_t)nsm_host)));
        p->bins[b].t0 = (int32_t)p->tiles_host.size();
        p->bins[b].m0 = (int32_t)p->merge_host.size();
        for (const auto& x : tl[b]) {
            const int32_t first = (int32_t)p->tiles_host.size() - p->bins[b].t0;
            const int64_t n = x.ve - x.vb;
            const int64_t k = (n + cap - 1) / cap;
            for (int64_t q = 0; q < k; ++q) {
                const int64_t a = x.vb + n * q / k, e = x.vb + n * (q + 1) / k;
                TileDesc u{x.tu, x.tv, a, e, 0, 0u, 0u};
                if (k > 1) {
                    u.box = box_pack(0, p->PW, 0, p->PW);  // the merge adds the slices' whole patches
                } else {
                    int a0 = p->PW, a1 = 0, b0 = p->PW, b1 = 0;
                    for (int64_t i = a; i < e; ++i) {
                        const uint32_t pos = meta[i].pos;
                        const int du = (int)(pos & 255u), dv = (int)((pos >> 8) & 255u), S = (int)((pos >> 16) & 255u);
                        a0 = std::min(a0, du);
                        a1 = std::max(a1, du + S);
                        b0 = std::min(b0, dv);
                        b1 = std::max(b1, dv + S);
                    }
                    u.box = box_pack(a0, a1, b0, b1);
                }
                p->tiles_host.push_back(u);
            }
            slot[(size_t)b * ntile + (size_t)x.tu * ntv + x.tv] = first;
            if (k > 1) p->merge_host.push_back(make_int2(first, (int)k));
        }
        p->bins[b].t1 = (int32_t)p->tiles_host.size();
        p->bins[b].m1 = (int32_t)p->merge_host.size();
        const int nu = p->bins[b].t1 - p->bins[b].t0;
        std::vector<int32_t> ord(nu);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int32_t i, int32_t j) {
            const auto& A = p->tiles_host[p->bins[b].t0 + i];
            const auto& B = p->tiles_host[p->bins[b].t0 + j];
            return (A.ve - A.vb) > (B.ve - B.vb);
        });
        p->sched_host.insert(p->sched_host.end(), ord.begin(), ord.end());
        n_active += (int)tl[b].size();
        p->max_tiles_bin = std::max(p->max_tiles_bin, nu);
    }

    // ---- caller-order host copies
    p->bins_user = bin;
    p->sw_user = sw;
    p->inv_perm.assign(M, 0);
    for (int64_t i = 0; i < M; ++i) p->inv_perm[order[i]] = (int32_t)i;

    // ---- device
    build_tables(p, s);
    if (q.wkernel_table > 0) {
        // folded kernels sampled over [-max|w_r|, max|w_r|] (one sample of margin each side)
        p->kw_n = q.wkernel_table;
        p->kw_dw = 2.0 * wr_max / p->kw_n;
        p->kw_w0 = -wr_max - p->kw_dw;
        p->d_kwtab = (float2*)dev_alloc(p, (size_t)(p->kw_n + 3) * 25 * sizeof(float2));
        launch_kwtab(p, s);
    }
    p->d_meta = upload(p, meta, s);
    // chunk descriptors: GTG_CHUNK consecutive visibilities of a unit share one tap range
    {
        std::vector<ChunkDesc> ch;
        for (auto& u : p->tiles_host) {
            u.cb = (int64_t)ch.size();
            for (int64_t v0 = u.vb; v0 < u.ve; v0 += GTG_CHUNK) {
                const int64_t v1 = std::min<int64_t>(u.ve, v0 + GTG_CHUNK);
                const VisMeta& m0 = meta[v0];
                const VisMeta& m1 = meta[v1 - 1];
                const int64_t S1 = (m1.pos >> 16) & 255;
                const int64_t end = m1.off + S1 * S1 + ((S1 * S1) & 1);
                ch.push_back(ChunkDesc{m0.off, (uint32_t)((end - m0.off) * 8), m0.pos >> 24});
            }
        }
        p->d_chunks = upload(p, ch, s);
    }
    p->d_tiles = upload(p, p->tiles_host, s);
    p->d_sched = upload(p, p->sched_host, s);
    p->d_merge = upload(p, p->merge_host, s);
    p->d_wr = upload(p, wr_s, s);
    p->d_phiu = upload(p, pu_s, s);
    p->d_phiv = upload(p, pv_s, s);
    int64_t gbytes = 0;
    std::vector<float2*> ptrs;
    if (generated) {
        // no stored G: every bin's (single) block points at one scratch that is refilled
        // for each bin of each apply
        int64_t mx = 16;
        for (int64_t bb : p->block_bytes) mx = std::max(mx, bb);
        p->d_sur_taps = (float2*)dev_alloc(p, (size_t)mx);
        p->sur_taps_bytes = mx;
        for (size_t i = 0; i < p->block_bytes.size(); ++i) ptrs.push_back(p->d_sur_taps);
    } else {
        for (int64_t bb : p->block_bytes) {
            p->d_gblocks.push_back((float2*)dev_alloc(p, (size_t)std::max<int64_t>(bb, 16)));
            gbytes += bb;
        }
        ptrs = p->d_gblocks;
    }
    p->d_gblock_ptrs = upload(p, ptrs, s);
    const size_t grid_elems = (size_t)gx * gy;
    p->d_X = (float2*)dev_alloc(p, grid_elems * sizeof(float2));
    // every cell finite from the start: the gridding step may stage cells that no footprint
    // of the current bin reaches
    RIMO_CUDA(cudaMemsetAsync(p->d_X, 0, grid_elems * sizeof(float2), s));
    {
        // the fold reads a tile's slot and the box of that slot's patch in one load
        std::vector<int2> sb(slot.size());
        for (int b = 0; b < P; ++b)
            for (int64_t t = 0; t < ntile; ++t) {
                const int32_t sl = slot[(size_t)b * ntile + t];
                sb[(size_t)b * ntile + t] =
                    make_int2(sl, sl < 0 ? 0 : (int)p->tiles_host[(size_t)p->bins[b].t0 + sl].box);
            }
        p->d_slot = upload(p, sb, s);
    }
    {
        // tiles of X read by the patch of some active tile: the tile itself and those of its
        // neighbours after it along u, v and both that the box of its patch reaches (a box
        // starts inside its own tile and ends at most H cells past it)
        std::vector<uint8_t> need((size_t)P * ntile, 0);
        for (int b = 0; b < P; ++b)
            for (int tu = 0; tu < ntu; ++tu)
                for (int tv = 0; tv < ntv; ++tv) {
                    const int32_t sl = slot[(size_t)b * ntile + (size_t)tu * ntv + tv];
                    if (sl < 0) continue;
                    const uint32_t box = p->tiles_host[(size_t)p->bins[b].t0 + sl].box;
                    const bool down = (int)((box >> 8) & 255u) > TS, right = (int)(box >> 24) > TS;
                    for (int du = 0; du < 2; ++du)
                        for (int dv = 0; dv < 2; ++dv)
                            if ((du == 0 || down) && (dv == 0 || right))
                                need[(size_t)b * ntile + (size_t)((tu + du) % ntu) * ntv + (tv + dv) % ntv] = 1;
                }
        p->d_need = upload(p, need, s);
        std::vector<int32_t> nl;
        for (int b = 0; b < P; ++b) {
            p->bins[b].n0 = (int32_t)nl.size();
            for (int64_t t = 0; t < ntile; ++t)
                if (need[(size_t)b * ntile + t]) nl.push_back((int32_t)t);
            p->bins[b].n1 = (int32_t)nl.size();
        }
        p->d_need_list = upload(p, nl, s);
        p->need_host = nl;
        p->info.n_needed = (int64_t)nl.size();
        // tile rows with a needed tile: the column passes transform only their grid rows
        p->trows.assign(P, {});
        for (int b = 0; b < P; ++b)
            for (int tu = 0; tu < ntu; ++tu)
                for (int tv = 0; tv < ntv; ++tv)
                    if (need[(size_t)b * ntile + (size_t)tu * ntv + tv]) {
                        p->trows[b].push_back((uint16_t)tu);
                        break;
                    }
        p->info.sel_rows = 0;
        for (int b = 0; b < P; ++b) p->info.sel_rows += (int64_t)p->trows[b].size() * TS;
    }
    p->d_patch = (float2*)dev_alloc(p, (size_t)std::max(1, p->max_tiles_bin) * p->PW * p->PW * sizeof(float2));
    p->d_counter = (int32_t*)dev_alloc(p, (size_t)P * sizeof(int32_t));
    p->d_status = (int32_t*)dev_alloc(p, sizeof(int32_t));
    RIMO_CUDA(cudaMemsetAsync(p->d_status, 0, sizeof(int32_t), s));
    p->d_fx = (uint32_t*)dev_alloc(p, FX_WORDS * sizeof(uint32_t));
    RIMO_CUDA(cudaMemsetAsync(p->d_fx, 0, FX_WORDS * sizeof(uint32_t), s));
    {
        int dev = 0;
        RIMO_CUDA(cudaGetDevice(&dev));
        RIMO_CUDA(cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, dev));
        p->device = dev;
        const int s2 = p->max_S * p->max_S;
        p->chunk_vis = GTG_CHUNK;
        p->chunk_bytes = p->chunk_vis * (s2 + (s2 & 1)) * (int)sizeof(float2);
    }
    p->d_AB = (float2*)dev_alloc(p, (size_t)2 * p->nx * p->ny * sizeof(float2));
    p->d_delta = (float2*)dev_alloc(p, (size_t)p->nx * p->ny * sizeof(float2));
    RIMO_CUDA(cudaMemsetAsync(p->d_delta, 0, (size_t)p->nx * p->ny * sizeof(float2), s));
    float2 one = make_float2(1.f, 0.f);
    RIMO_CUDA(cudaMemcpyAsync(p->d_delta + (size_t)(p->ny / 2) * p->nx + p->nx / 2, &one,
                              sizeof(float2), cudaMemcpyHostToDevice, s));
    p->info.K = K;
    p->info.g_bytes = gbytes + (int64_t)M * (int64_t)sizeof(VisMeta);
    p->info.scratch_bytes = (int64_t)(grid_elems + 3 * (size_t)p->nx * p->ny +
                                      (size_t)p->max_tiles_bin * p->PW * p->PW) * 8 + p->sur_taps_bytes;
    p->info.n_blocks = (int32_t)p->block_bytes.size();
    p->info.n_tiles = n_active;
    p->info.n_units = (int64_t)p->tiles_host.size();
    p->info.box_cells = 0;
    for (const TileDesc& u : p->tiles_host)
        p->info.box_cells += (int64_t)(((u.box >> 8) & 255u) - (u.box & 255u)) * (int64_t)((u.box >> 24) - ((u.box >> 16) & 255u));

    // ---- stage 3: precompute G on the device (the surrogate generates it at apply time)
    if (!generated) {
        prof_begin(p, ST_GBUILD, s);
        launch_gbuild(p, s);
        prof_end(p, 1, s);
    }
    RIMO_CUDA(cudaGetLastError());
    RIMO_CUDA(cudaStreamSynchronize(s));
}

}  // namespace rimo

using namespace rimo;

extern "C" {

void rimo_plan_params_default(rimo_plan_params* q, int32_t nx, int32_t ny, double fov_x,
                              double fov_y) {
    std::memset(q, 0, sizeof(*q));
    q->nx = nx;
    q->ny = ny;
    q->fov_x = fov_x;
    q->fov_y = fov_y;
    q->oversampling = 2;
    q->kb_support = 7;
    q->kb_beta = 0.0;
    q->max_wsupport = 9;
    q->w_norm_frac = 0.9999;
    q->plan_fraction = 0.01;
    q->seed = 12345;
    q->mode = RIMO_MODE_AUTO;
}

rimo_status rimo_plan_estimate(const double* uvw, int64_t M, const rimo_plan_params* q,
                               rimo_plan_info* info) {
    try {
        if (!uvw || M <= 0 || !q || !info) fail(RIMO_ERR_INVALID_ARG, "null pointer or M <= 0");
        validate_params(*q);
        validate_uvw(uvw, M, *q);
        planner::Params pr = planner_params(*q);
        planner::Choice ch = planner::choose(uvw, M, pr);
        std::memset(info, 0, sizeof(*info));
        fill_estimate(info, ch, M, pr.kg.L);
        return RIMO_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        return e.status;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return RIMO_ERR_OOM;
    }
}

rimo_status rimo_plan_create(const double* uvw, int64_t M, const rimo_plan_params* q,
                             void* stream, rimo_plan_t* out) {
    if (out) *out = nullptr;
    rimo_plan* p = nullptr;
    try {
        if (!uvw || M <= 0 || !q || !out) fail(RIMO_ERR_INVALID_ARG, "null pointer or M <= 0");
        if (M > 2000000000LL) fail(RIMO_ERR_INVALID_ARG, "M above 2e9 visibilities");
        validate_params(*q);
        validate_uvw(uvw, M, *q);
        p = new rimo_plan();
        create_plan(uvw, M, *q, (cudaStream_t)stream, p);
        *out = p;
        return RIMO_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        rimo_plan_destroy(p);
        return e.status;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        rimo_plan_destroy(p);
        return RIMO_ERR_OOM;
    }
}

rimo_status rimo_plan_destroy(rimo_plan_t p) {
    if (!p) return RIMO_OK;
    for (void* ptr : p->owned) cudaFree(ptr);
    for (auto& m : p->prof_pending) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    for (cudaEvent_t e : p->prof_pool) cudaEventDestroy(e);
    if (p->prof_open_event) cudaEventDestroy(p->prof_open_event);
    delete p;
    return RIMO_OK;
}

rimo_status rimo_plan_info_get(rimo_plan_t p, rimo_plan_info* info) {
    if (!p || !info) {
        set_last_error("null plan or info");
        return RIMO_ERR_INVALID_ARG;
    }
    *info = p->info;
    return RIMO_OK;
}

rimo_status rimo_plan_get_bins(rimo_plan_t p, double* w_stack, int32_t* bins, int32_t* s_w) {
    if (!p) {
        set_last_error("null plan");
        return RIMO_ERR_INVALID_ARG;
    }
    if (w_stack) std::memcpy(w_stack, p->w_stack.data(), p->w_stack.size() * sizeof(double));
    if (bins) std::memcpy(bins, p->bins_user.data(), p->bins_user.size() * sizeof(int32_t));
    if (s_w) std::memcpy(s_w, p->sw_user.data(), p->sw_user.size() * sizeof(int32_t));
    return RIMO_OK;
}

rimo_status rimo_plan_get_tiles(rimo_plan_t p, const int64_t* idx, int64_t n, int32_t* g0,
                                int32_t* h0, int32_t* S, rimo_cfloat* taps, void* stream) {
    try {
        if (!p || (n > 0 && (!idx || !g0 || !h0 || !S || !taps)) || n < 0)
            fail(RIMO_ERR_INVALID_ARG, "null pointer or n < 0");
        const bool generated = p->mode != RIMO_MODE_STORED_G;
        if (p->mode == RIMO_MODE_SURROGATE && !p->sur)
            fail(RIMO_ERR_STATE, "surrogate plan without a surrogate (rimo_plan_set_surrogate)");
        if (p->mode == RIMO_MODE_HOLOGRAPHIC && p->h_built)
            fail(RIMO_ERR_UNSUPPORTED, "holographic plan: its tiles were folded into H");
        cudaStream_t s = (cudaStream_t)stream;
        if (generated) reset_surrogate_bounds(p, s);
        int have_bin = -1;  // the bin whose tiles the tap scratch holds
        for (int64_t q = 0; q < n; ++q)
            if (idx[q] < 0 || idx[q] >= p->M) fail(RIMO_ERR_INVALID_ARG, "visibility index out of range");
        std::vector<int64_t> order(n);  // requests grouped by bin: one generation per bin
        for (int64_t q = 0; q < n; ++q) order[q] = q;
        if (generated)
            std::stable_sort(order.begin(), order.end(),
                             [&](int64_t a, int64_t b) { return p->bins_user[idx[a]] < p->bins_user[idx[b]]; });
        for (int64_t q : order) {
            int64_t i = p->inv_perm[idx[q]];
            VisMeta m;
            RIMO_CUDA(cudaMemcpyAsync(&m, p->d_meta + i, sizeof(m), cudaMemcpyDeviceToHost, s));
            RIMO_CUDA(cudaStreamSynchronize(s));
            int du = m.pos & 255, dv = (m.pos >> 8) & 255, Sq = (m.pos >> 16) & 255, blk = m.pos >> 24;
            if (blk == SHARD_SKIP) fail(RIMO_ERR_INVALID_ARG, "visibility held by another shard plan");
            // the tile containing sorted position i
            int b = p->bins_user[idx[q]];
            if (generated && b != have_bin) {  // tiles of generated plans: this bin, as an apply makes them
                RIMO_CUDA(cudaStreamSynchronize(s));  // earlier copies out of the scratch are done
                if (p->mode == RIMO_MODE_SURROGATE) surrogate_generate(p, b, s);
                else launch_gbuild_range(p, p->bins[b].vb, p->bins[b].ve - p->bins[b].vb, s);
                have_bin = b;
            }
            int tu = -1, tv = -1;
            for (int t = p->bins[b].t0; t < p->bins[b].t1; ++t)
                if (p->tiles_host[t].vb <= i && i < p->tiles_host[t].ve) {  // the unit holding i
                    tu = p->tiles_host[t].tu;
                    tv = p->tiles_host[t].tv;
                }
            g0[q] = tu * p->TS + du;
            h0[q] = tv * p->TS + dv;
            S[q] = Sq;
            // generated plans: every block is the one tap scratch
            const float2* src = generated ? p->d_sur_taps : p->d_gblocks.at((size_t)blk);
            RIMO_CUDA(cudaMemcpyAsync(taps + q * 361, src + m.off,
                                      (size_t)Sq * Sq * sizeof(float2), cudaMemcpyDeviceToHost, s));
        }
        RIMO_CUDA(cudaStreamSynchronize(s));
        return RIMO_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        return e.status;
    }
}

const char* rimo_last_error(void) { return g_last_error.c_str(); }

const char* rimo_version(void) { return "rimo 0.1 (sm_103a)"; }

}  // extern "C"
