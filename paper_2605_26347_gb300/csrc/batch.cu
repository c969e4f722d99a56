// Batched wideband Phi^dagger Phi and the tile-size autotuner.
//
// A batch groups independent plans (one per frequency channel, each with its own w-stack,
// Section 2 and Section 3.5: the wideband model applies the monochromatic one per
// channel).  Its Phi^dagger Phi is recorded once into a CUDA graph and replayed by one
// cudaGraphLaunch per call for as long as the buffers stay the same, in one of two forms:
//  * staged (plans with stored G and one image, uv-tile, patch and tap-ring shape): every
//    (channel, w-bin) is a job with its own scratch, and each pass runs as ONE launch over
//    all jobs - forward rows, forward cols, the grid step as one persistent launch that
//    takes the work units of every job heaviest first from one queue (channels and bins of
//    uneven visibility counts balance across the SMs), the merge of split tiles, the fold,
//    inverse cols, and inverse rows with the sum over each channel's bins;
//  * branches (any other batch): each channel's own apply on a branch of a fork/join
//    stream pattern, the branches running concurrently.
//
// The autotuner times the uv-tile size candidates of a plan (the tile shape drives the
// gridding schedule: patch halo overhead against work-unit count) on a deterministic
// subsample of the visibilities and keeps the winner in a JSON cache keyed by the
// workload's shape.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "internal.h"

using namespace rimo;

struct rimo_batch {
    std::vector<rimo_plan*> plans;
    int nx = 0, ny = 0, device = 0;
    cudaStream_t root = nullptr;        // recording stream (the caller's may be the legacy stream)
    std::vector<cudaStream_t> branches;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    cudaGraphExec_t exec = nullptr;
    // what the captured graph was recorded with
    const void* key_x = nullptr;
    void* key_out = nullptr;
    int key_real = -1;
    int64_t captures = 0;
    // staged form
    bool staged = false;
    std::vector<WideJob> jobs;          // (channel, w-bin) jobs, channel-major
    std::vector<bool> has_jobs;         // per channel: some bin holds visibilities
    void* scratch = nullptr;            // every job's scratch, one allocation
    int64_t scratch_bytes = 0;
    WideGtg* wgtg = nullptr;
    WideFft* wfft = nullptr;            // tables for the recorded (x, out)
};

namespace {

constexpr int BATCH_MAX_BRANCHES = 16;

void destroy_batch(rimo_batch* b) {
    if (!b) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(b->device);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->wfft) wide_fft_destroy(b->wfft);
    if (b->wgtg) wide_gtg_destroy(b->wgtg);
    if (b->scratch) cudaFree(b->scratch);
    for (auto e : b->joins) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    for (auto s : b->branches) cudaStreamDestroy(s);
    if (b->root) cudaStreamDestroy(b->root);
    cudaSetDevice(cur);
    delete b;
}

// Whether the plans can run as one staged pipeline: stored G (no H, no generated tiles),
// square images of one size and one uv-tile size (patch sides and tap chunks may differ).
bool stage_eligible(const std::vector<rimo_plan*>& plans) {
    const rimo_plan* a = plans[0];
    for (const rimo_plan* p : plans) {
        if (p->mode != RIMO_MODE_STORED_G || p->h_built) return false;
        if (p->nx != p->ny || p->nx != a->nx || p->TS != a->TS || p->nx > 4096 || p->nx < 64) return false;
    }
    return true;
}

// Jobs, their scratch (one allocation, 256-byte aligned parts) and the grid-step queue.
void stage(rimo_batch* b, cudaStream_t s) {
    auto al = [](int64_t x) { return (x + 255) & ~(int64_t)255; };
    int64_t total = 0;
    std::vector<std::array<int64_t, 3>> off;
    b->has_jobs.assign(b->plans.size(), false);
    for (size_t c = 0; c < b->plans.size(); ++c) {
        const rimo_plan* p = b->plans[c];
        for (int bin = 0; bin < p->P; ++bin) {
            if (p->bins[bin].ve == p->bins[bin].vb) continue;
            const int64_t ab = al((int64_t)2 * p->nx * p->ny * 8), gx = al((int64_t)p->gx * p->gy * 8);
            const int64_t pt = al((int64_t)std::max(1, p->bins[bin].t1 - p->bins[bin].t0) * p->PW * p->PW * 8);
            off.push_back({total, total + ab, total + ab + gx});
            total += ab + gx + pt;
            b->jobs.push_back(WideJob{p, bin, (int)c, nullptr, nullptr, nullptr});
            b->has_jobs[c] = true;
        }
    }
    if (b->jobs.empty()) return;
    if (cudaMalloc(&b->scratch, (size_t)total) != cudaSuccess) {
        cudaGetLastError();
        fail(RIMO_ERR_OOM, "batch scratch of " + std::to_string(total) + " bytes");
    }
    b->scratch_bytes = total;
    char* base = static_cast<char*>(b->scratch);
    for (size_t j = 0; j < b->jobs.size(); ++j) {
        b->jobs[j].AB = reinterpret_cast<float2*>(base + off[j][0]);
        b->jobs[j].X = reinterpret_cast<float2*>(base + off[j][1]);
        b->jobs[j].patch = reinterpret_cast<float2*>(base + off[j][2]);
    }
    b->wgtg = wide_gtg_create(b->jobs, s);
}

// Records the staged pipeline for (x, out): per channel the image bound (flags non-finite
// input in the plan's status), then one launch per pass over all jobs.
void record_staged(rimo_batch* b, const float2* x, float2* out, int real_only, cudaStream_t s) {
    const size_t img = (size_t)b->nx * b->ny;
    for (size_t c = 0; c < b->plans.size(); ++c) {
        if (b->has_jobs[c]) launch_image_bound(b->plans[c], x + c * img, s);
        else RIMO_CUDA(cudaMemsetAsync(out + c * img, 0, img * sizeof(float2), s));
    }
    if (b->jobs.empty()) return;
    wide_fwd(b->wfft, s);
    wide_gtg(b->wgtg, s);
    wide_inv(b->wfft, real_only, s);
}

// Records all channels' applies into a graph on the batch's own root stream (staged: one
// launch per pass; branches: fork, one branch stream per channel round robin over the
// branch pool, join back).  Nothing runs during recording; the graph is launched on the
// caller's stream afterwards.
void capture(rimo_batch* b, const float2* x, float2* out, int real_only) {
    cudaStream_t s = b->root;
    const size_t img = (size_t)b->nx * b->ny;
    std::vector<bool> prof(b->plans.size());
    for (size_t i = 0; i < b->plans.size(); ++i) {
        prof[i] = b->plans[i]->prof_on;
        b->plans[i]->prof_on = false;  // stage timers record events the graph cannot replay
    }
    if (b->staged && !b->jobs.empty()) {
        // the job tables point at (x, out); a graph of the previous tables may still run
        RIMO_CUDA(cudaDeviceSynchronize());
        if (b->wfft) wide_fft_destroy(b->wfft);
        b->wfft = nullptr;
        std::vector<const float2*> xs;
        std::vector<float2*> os;
        for (size_t c = 0; c < b->plans.size(); ++c) {
            xs.push_back(x + c * img);
            os.push_back(out + c * img);
        }
        b->wfft = wide_fft_create(b->jobs, xs, os, s);
    }
    RIMO_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaGraph_t graph = nullptr;
    try {
        if (b->staged) {
            record_staged(b, x, out, real_only, s);
        } else {
            RIMO_CUDA(cudaEventRecord(b->fork, s));
            for (size_t i = 0; i < b->plans.size(); ++i) {
                cudaStream_t br = b->branches[i % b->branches.size()];
                RIMO_CUDA(cudaStreamWaitEvent(br, b->fork, 0));
                apply_phi_adj_phi(b->plans[i], x + i * img, out + i * img, real_only, br);
                RIMO_CUDA(cudaEventRecord(b->joins[i], br));
                RIMO_CUDA(cudaStreamWaitEvent(s, b->joins[i], 0));
            }
        }
        RIMO_CUDA(cudaStreamEndCapture(s, &graph));
    } catch (...) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(s, &g);  // leave the caller's stream out of capture mode
        if (g) cudaGraphDestroy(g);
        for (size_t i = 0; i < b->plans.size(); ++i) b->plans[i]->prof_on = prof[i];
        throw;
    }
    for (size_t i = 0; i < b->plans.size(); ++i) b->plans[i]->prof_on = prof[i];
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    const cudaError_t e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    RIMO_CUDA(e);
    b->key_x = x;
    b->key_out = out;
    b->key_real = real_only;
    b->captures++;
}

// ---- autotuner cache: a flat JSON object {"key": tile, ...}
std::map<std::string, int> read_cache(const std::string& path) {
    std::map<std::string, int> m;
    std::ifstream f(path);
    if (!f) return m;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string t = ss.str();
    size_t i = 0;
    while ((i = t.find('"', i)) != std::string::npos) {
        const size_t j = t.find('"', i + 1);
        if (j == std::string::npos) break;
        const std::string key = t.substr(i + 1, j - i - 1);
        const size_t c = t.find(':', j);
        if (c == std::string::npos) break;
        m[key] = std::atoi(t.c_str() + c + 1);
        i = t.find_first_of(",}", c);
        if (i == std::string::npos) break;
    }
    return m;
}

void write_cache(const std::string& path, const std::map<std::string, int>& m) {
    const std::string tmp = path + ".tmp";
    {
        std::ofstream f(tmp);
        if (!f) fail(RIMO_ERR_INVALID_ARG, "cannot write autotuner cache " + path);
        f << "{";
        bool first = true;
        for (const auto& kv : m) {
            f << (first ? "\n" : ",\n") << "  \"" << kv.first << "\": " << kv.second;
            first = false;
        }
        f << "\n}\n";
    }
    if (std::rename(tmp.c_str(), path.c_str()) != 0) fail(RIMO_ERR_INVALID_ARG, "cannot replace " + path);
}

std::string tune_key(const rimo_plan_params& q, int64_t M, int P, int max_s) {
    char buf[256];
    const int mlog = M > 0 ? (int)std::lround(std::log2((double)M)) : 0;
    std::snprintf(buf, sizeof(buf), "n%dx%d_fov%.4fx%.4f_M2^%d_P%d_J%d_S%d", q.nx, q.ny, q.fov_x, q.fov_y, mlog, P,
                  q.kb_support, max_s);
    return buf;
}

}  // namespace

extern "C" {

rimo_status rimo_batch_create(const rimo_plan_t* plans, int32_t n_plans, rimo_batch_t* out) {
    return rimo_batch_create_form(plans, n_plans, RIMO_BATCH_AUTO, out);
}

rimo_status rimo_batch_create_form(const rimo_plan_t* plans, int32_t n_plans, int32_t form, rimo_batch_t* out) {
    if (out) *out = nullptr;
    rimo_batch* b = nullptr;
    RIMO_API_BEGIN
    if (!out || !plans || n_plans <= 0) fail(RIMO_ERR_INVALID_ARG, "need an output and at least one plan");
    if (form != RIMO_BATCH_AUTO && form != RIMO_BATCH_STAGED && form != RIMO_BATCH_BRANCHES)
        fail(RIMO_ERR_INVALID_ARG, "unknown batch form");
    b = new rimo_batch();
    RIMO_CUDA(cudaGetDevice(&b->device));
    for (int i = 0; i < n_plans; ++i) {
        rimo_plan* p = plans[i];
        if (!p) fail(RIMO_ERR_INVALID_ARG, "null plan in batch");
        if (i == 0) {
            b->nx = p->prm.nx;
            b->ny = p->prm.ny;
        } else if (p->prm.nx != b->nx || p->prm.ny != b->ny) {
            fail(RIMO_ERR_INVALID_ARG, "all plans of a batch need the same image size");
        }
        if (p->device != b->device) fail(RIMO_ERR_INVALID_ARG, "plans of a batch must live on the current device");
        for (int j = 0; j < i; ++j)
            if (plans[j] == p) fail(RIMO_ERR_INVALID_ARG, "a plan appears twice in the batch (it has scratch)");
        b->plans.push_back(p);
    }
    const bool eligible = stage_eligible(b->plans);
    if (form == RIMO_BATCH_STAGED && !eligible)
        fail(RIMO_ERR_UNSUPPORTED, "staged batches need stored-G plans of one image, tile, patch and ring shape");
    b->staged = form != RIMO_BATCH_BRANCHES && eligible;
    RIMO_CUDA(cudaStreamCreateWithFlags(&b->root, cudaStreamNonBlocking));
    if (b->staged) stage(b, b->root);
    const int nb = std::min(n_plans, BATCH_MAX_BRANCHES);
    for (int i = 0; i < nb; ++i) {
        cudaStream_t st = nullptr;
        RIMO_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        b->branches.push_back(st);
    }
    RIMO_CUDA(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    for (int i = 0; i < n_plans; ++i) {
        cudaEvent_t e = nullptr;
        RIMO_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        b->joins.push_back(e);
    }
    *out = b;
    b = nullptr;
    return RIMO_OK;
    }
    catch (const Error& e) {
        set_last_error(e.msg);
        destroy_batch(b);
        return e.status;
    }
    catch (const std::exception& e) {
        set_last_error(e.what());
        destroy_batch(b);
        return RIMO_ERR_OOM;
    }
}

rimo_status rimo_batch_destroy(rimo_batch_t b) {
    RIMO_API_BEGIN
    destroy_batch(b);
    RIMO_API_END
}

rimo_status rimo_batch_apply_phi_adj_phi(rimo_batch_t b, const rimo_cfloat* x_dev, rimo_cfloat* out_dev,
                                         int32_t real_part_only, void* stream) {
    RIMO_API_BEGIN
    if (!b) fail(RIMO_ERR_INVALID_ARG, "null batch");
    if (!x_dev || !out_dev) fail(RIMO_ERR_INVALID_ARG, "null buffer");
    const size_t bytes = b->plans.size() * (size_t)b->nx * b->ny * sizeof(float2);
    const char* xa = reinterpret_cast<const char*>(x_dev);
    const char* oa = reinterpret_cast<const char*>(out_dev);
    if (xa < oa + bytes && oa < xa + bytes) fail(RIMO_ERR_INVALID_ARG, "x and out overlap");
    int dev = 0;
    RIMO_CUDA(cudaGetDevice(&dev));
    if (dev != b->device) fail(RIMO_ERR_INVALID_ARG, "batch used on another device");
    cudaStream_t s = (cudaStream_t)stream;
    const int real = real_part_only ? 1 : 0;
    if (!b->exec || b->key_x != (const void*)x_dev || b->key_out != (void*)out_dev || b->key_real != real)
        capture(b, (const float2*)x_dev, (float2*)out_dev, real);
    RIMO_CUDA(cudaGraphLaunch(b->exec, s));
    RIMO_API_END
}

rimo_status rimo_batch_info(rimo_batch_t b, int32_t* n_plans, int64_t* captures) {
    RIMO_API_BEGIN
    if (!b) fail(RIMO_ERR_INVALID_ARG, "null batch");
    if (n_plans) *n_plans = (int32_t)b->plans.size();
    if (captures) *captures = b->captures;
    RIMO_API_END
}

rimo_status rimo_batch_layout(rimo_batch_t b, int32_t* staged, int64_t* jobs, int64_t* units,
                              int64_t* scratch_bytes) {
    RIMO_API_BEGIN
    if (!b) fail(RIMO_ERR_INVALID_ARG, "null batch");
    if (staged) *staged = b->staged ? 1 : 0;
    if (jobs) *jobs = (int64_t)b->jobs.size();
    if (units) *units = b->wgtg ? wide_gtg_units(b->wgtg) : 0;
    if (scratch_bytes) *scratch_bytes = b->scratch_bytes;
    RIMO_API_END
}

}  // extern "C"

namespace {

// Times Phi^dagger Phi for each candidate (uv-tile size, visibility order) on plans built
// from a deterministic subsample (every stride-th row, at most 2^20 rows) and returns the
// index of the fastest; ms[c] receives each candidate's ms per apply.
int tune(const double* uvw, int64_t M, const rimo_plan_params* base, const std::vector<std::pair<int, int>>& cands,
         void* stream, double* ms) {
    const int64_t cap = 1 << 20;
    const int64_t stride = (M + cap - 1) / cap;
    std::vector<double> sub;
    const double* src = uvw;
    int64_t Ms = M;
    if (stride > 1) {
        Ms = (M + stride - 1) / stride;
        sub.resize((size_t)Ms * 3);
        for (int64_t k = 0; k < Ms; ++k)
            for (int c = 0; c < 3; ++c) sub[(size_t)k * 3 + c] = uvw[(size_t)(k * stride) * 3 + c];
        src = sub.data();
    }
    rimo_plan_params q = *base;
    cudaStream_t s = (cudaStream_t)stream;
    float2 *x = nullptr, *o = nullptr;
    const size_t img = (size_t)q.nx * q.ny * sizeof(float2);
    RIMO_CUDA(cudaMalloc(&x, img));
    RIMO_CUDA(cudaMalloc(&o, img));
    double best = 1e300;
    int pick = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    try {
        // a point at the centre and one off-centre: every bin's grid is non-trivial
        RIMO_CUDA(cudaMemsetAsync(x, 0, img, s));
        const float2 one = make_float2(1.f, 0.f);
        RIMO_CUDA(cudaMemcpyAsync(x + (size_t)(q.ny / 2) * q.nx + q.nx / 2, &one, sizeof(one), cudaMemcpyHostToDevice, s));
        RIMO_CUDA(cudaMemcpyAsync(x + (size_t)(q.ny / 4) * q.nx + q.nx / 3, &one, sizeof(one), cudaMemcpyHostToDevice, s));
        RIMO_CUDA(cudaEventCreate(&e0));
        RIMO_CUDA(cudaEventCreate(&e1));
        for (size_t c = 0; c < cands.size(); ++c) {
            q.tile_size = cands[c].first;
            q.uv_order = cands[c].second;
            rimo_plan_t p = nullptr;
            if (rimo_plan_create(src, Ms, &q, stream, &p) != RIMO_OK) fail(RIMO_ERR_INVALID_ARG, rimo_last_error());
            float t = 0.f;
            try {
                apply_phi_adj_phi(p, x, o, 0, s);  // warm-up
                RIMO_CUDA(cudaEventRecord(e0, s));
                for (int r = 0; r < 3; ++r) apply_phi_adj_phi(p, x, o, 0, s);
                RIMO_CUDA(cudaEventRecord(e1, s));
                RIMO_CUDA(cudaEventSynchronize(e1));
                RIMO_CUDA(cudaEventElapsedTime(&t, e0, e1));
            } catch (...) {
                rimo_plan_destroy(p);
                throw;
            }
            rimo_plan_destroy(p);
            ms[c] = t / 3.0;
            if (ms[c] < best) {
                best = ms[c];
                pick = (int)c;
            }
        }
    } catch (...) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(x);
        cudaFree(o);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(x);
    cudaFree(o);
    return pick;
}

// The same for a batch: each candidate's plans (one per workload, every stride-th row of
// each, at most 2^22 rows) recorded as one batch (the staged form where eligible) and its
// Phi^dagger Phi timed; returns the index of the fastest, ms[c] the batch's ms per apply.
int tune_batch(const double* const* uvw, const int64_t* M, const rimo_plan_params* base, int n,
               const std::vector<std::pair<int, int>>& cands, void* stream, double* ms) {
    const int64_t cap = 1 << 22;
    std::vector<std::vector<double>> subs(n);
    std::vector<const double*> src(n);
    std::vector<int64_t> Ms(n);
    for (int i = 0; i < n; ++i) {
        if (base[i].nx != base[0].nx || base[i].ny != base[0].ny)
            fail(RIMO_ERR_INVALID_ARG, "the workloads of a batch share one image size");
        const int64_t stride = (M[i] + cap - 1) / cap;
        src[i] = uvw[i];
        Ms[i] = M[i];
        if (stride > 1) {
            Ms[i] = (M[i] + stride - 1) / stride;
            subs[i].resize((size_t)Ms[i] * 3);
            for (int64_t k = 0; k < Ms[i]; ++k)
                for (int c = 0; c < 3; ++c) subs[i][(size_t)k * 3 + c] = uvw[i][(size_t)(k * stride) * 3 + c];
            src[i] = subs[i].data();
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t img = (size_t)base[0].nx * base[0].ny;
    float2 *x = nullptr, *o = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<rimo_plan_t> plans;
    rimo_batch_t batch = nullptr;
    auto release = [&]() {
        rimo_batch_destroy(batch);
        batch = nullptr;
        for (rimo_plan_t p : plans) rimo_plan_destroy(p);
        plans.clear();
    };
    double best = 1e300;
    int pick = 0;
    try {
        RIMO_CUDA(cudaMalloc(&x, img * n * sizeof(float2)));
        RIMO_CUDA(cudaMalloc(&o, img * n * sizeof(float2)));
        RIMO_CUDA(cudaMemsetAsync(x, 0, img * n * sizeof(float2), s));
        const float2 one = make_float2(1.f, 0.f);
        for (int i = 0; i < n; ++i)  // a point at the centre of every image: every grid is non-trivial
            RIMO_CUDA(cudaMemcpyAsync(x + i * img + (size_t)(base[0].ny / 2) * base[0].nx + base[0].nx / 2, &one,
                                      sizeof(one), cudaMemcpyHostToDevice, s));
        RIMO_CUDA(cudaEventCreate(&e0));
        RIMO_CUDA(cudaEventCreate(&e1));
        for (size_t c = 0; c < cands.size(); ++c) {
            for (int i = 0; i < n; ++i) {
                rimo_plan_params q = base[i];
                q.tile_size = cands[c].first;
                q.uv_order = cands[c].second;
                rimo_plan_t p = nullptr;
                if (rimo_plan_create(src[i], Ms[i], &q, stream, &p) != RIMO_OK)
                    fail(RIMO_ERR_INVALID_ARG, rimo_last_error());
                plans.push_back(p);
            }
            if (rimo_batch_create_form(plans.data(), n, RIMO_BATCH_AUTO, &batch) != RIMO_OK)
                fail(RIMO_ERR_INVALID_ARG, rimo_last_error());
            auto apply = [&]() {
                if (rimo_batch_apply_phi_adj_phi(batch, (const rimo_cfloat*)x, (rimo_cfloat*)o, 0, stream) != RIMO_OK)
                    fail(RIMO_ERR_CUDA, rimo_last_error());
            };
            apply();  // records the graph
            RIMO_CUDA(cudaEventRecord(e0, s));
            for (int r = 0; r < 3; ++r) apply();
            RIMO_CUDA(cudaEventRecord(e1, s));
            RIMO_CUDA(cudaEventSynchronize(e1));
            float t = 0.f;
            RIMO_CUDA(cudaEventElapsedTime(&t, e0, e1));
            release();
            ms[c] = t / 3.0;
            if (ms[c] < best) {
                best = ms[c];
                pick = (int)c;
            }
        }
    } catch (...) {
        release();
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(x);
        cudaFree(o);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(x);
    cudaFree(o);
    return pick;
}

// cache key of a workload's shape (image, FoV, log2 M, P, J, largest tile side), from a
// host-only estimate on the same subsample the tuner times
std::string shape_key(const double* uvw, int64_t M, const rimo_plan_params* base, const char* suffix) {
    rimo_plan_params q = *base;
    q.tile_size = 0;
    rimo_plan_info est;
    if (rimo_plan_estimate(uvw, M, &q, &est) != RIMO_OK) fail(RIMO_ERR_INVALID_ARG, rimo_last_error());
    int max_s = 0;
    for (int i = 0; i < 64; ++i) max_s = std::max(max_s, (int)est.support_table[i]);
    return tune_key(q, M, est.P, max_s + q.kb_support - 1) + suffix;
}

}  // namespace

extern "C" {

rimo_status rimo_autotune_batch(const double* const* uvw, const int64_t* M, const rimo_plan_params* base, int32_t n,
                                const char* cache_path, void* stream, int32_t* tile_out, int32_t* order_out,
                                double* ms_out) {
    RIMO_API_BEGIN
    if (!uvw || !M || !base || n <= 0 || !tile_out || !order_out) fail(RIMO_ERR_INVALID_ARG, "null argument or n <= 0");
    for (int i = 0; i < n; ++i)
        if (!uvw[i] || M[i] <= 0) fail(RIMO_ERR_INVALID_ARG, "null or empty workload");
    if (ms_out)
        for (int i = 0; i < 6; ++i) ms_out[i] = -1.0;
    std::string key;
    for (int i = 0; i < n; ++i) key += (i ? "+" : "") + shape_key(uvw[i], M[i], &base[i], "");
    key += "_batch_tile_order";
    std::map<std::string, int> cache;
    if (cache_path && *cache_path) {
        cache = read_cache(cache_path);
        auto it = cache.find(key);
        if (it != cache.end() && (it->second / 10 == 32 || it->second / 10 == 64) && it->second % 10 <= 2) {
            *tile_out = it->second / 10;
            *order_out = it->second % 10;
            return RIMO_OK;
        }
    }
    std::vector<std::pair<int, int>> cands;
    for (int t : {32, 64})
        for (int o = 0; o < 3; ++o) cands.push_back({t, o});
    double ms[6];
    const int pick = tune_batch(uvw, M, base, n, cands, stream, ms);
    if (ms_out)
        for (int i = 0; i < 6; ++i) ms_out[i] = ms[i];
    *tile_out = cands[pick].first;
    *order_out = cands[pick].second;
    if (cache_path && *cache_path) {
        cache[key] = *tile_out * 10 + *order_out;
        write_cache(cache_path, cache);
    }
    RIMO_API_END
}

rimo_status rimo_autotune_tile(const double* uvw, int64_t M, const rimo_plan_params* base, const char* cache_path,
                               void* stream, int32_t* tile_out, double* ms_out) {
    RIMO_API_BEGIN
    if (!uvw || M <= 0 || !base || !tile_out) fail(RIMO_ERR_INVALID_ARG, "null argument or empty data");
    if (ms_out) ms_out[0] = ms_out[1] = -1.0;
    const std::string key = shape_key(uvw, M, base, "");
    std::map<std::string, int> cache;
    if (cache_path && *cache_path) {
        cache = read_cache(cache_path);
        auto it = cache.find(key);
        if (it != cache.end() && (it->second == 32 || it->second == 64)) {
            *tile_out = it->second;
            return RIMO_OK;
        }
    }
    const std::vector<std::pair<int, int>> cands = {{32, base->uv_order}, {64, base->uv_order}};
    double ms[2] = {-1.0, -1.0};
    const int pick = tune(uvw, M, base, cands, stream, ms);
    if (ms_out) ms_out[0] = ms[0], ms_out[1] = ms[1];
    *tile_out = cands[pick].first;
    if (cache_path && *cache_path) {
        cache[key] = *tile_out;
        write_cache(cache_path, cache);
    }
    RIMO_API_END
}

rimo_status rimo_autotune(const double* uvw, int64_t M, const rimo_plan_params* base, const char* cache_path,
                          void* stream, int32_t* tile_out, int32_t* order_out, double* ms_out) {
    RIMO_API_BEGIN
    if (!uvw || M <= 0 || !base || !tile_out || !order_out) fail(RIMO_ERR_INVALID_ARG, "null argument or empty data");
    if (ms_out)
        for (int i = 0; i < 6; ++i) ms_out[i] = -1.0;
    const std::string key = shape_key(uvw, M, base, "_tile_order");
    std::map<std::string, int> cache;
    if (cache_path && *cache_path) {
        cache = read_cache(cache_path);
        auto it = cache.find(key);
        if (it != cache.end() && (it->second / 10 == 32 || it->second / 10 == 64) && it->second % 10 <= 2) {
            *tile_out = it->second / 10;
            *order_out = it->second % 10;
            return RIMO_OK;
        }
    }
    std::vector<std::pair<int, int>> cands;
    for (int t : {32, 64})
        for (int o = 0; o < 3; ++o) cands.push_back({t, o});
    double ms[6];
    const int pick = tune(uvw, M, base, cands, stream, ms);
    if (ms_out)
        for (int i = 0; i < 6; ++i) ms_out[i] = ms[i];
    *tile_out = cands[pick].first;
    *order_out = cands[pick].second;
    if (cache_path && *cache_path) {
        cache[key] = *tile_out * 10 + *order_out;
        write_cache(cache_path, cache);
    }
    RIMO_API_END
}

}  // extern "C"
