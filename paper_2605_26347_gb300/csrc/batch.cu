// Batched wideband Phi^dagger Phi and the tile-size autotuner.
//
// A batch groups independent plans (one per frequency channel, each with its own w-stack,
// Section 2 and Section 3.5: the wideband model applies the monochromatic one per
// channel).  One call enqueues every channel's Phi^dagger Phi on its own branch of a
// fork/join stream pattern inside a single stream capture; the instantiated CUDA graph is
// then replayed by one cudaGraphLaunch per call for as long as the buffers stay the same.
// Channels share no state, so the branches run concurrently and the small per-channel
// kernels fill the GPU together.
//
// The autotuner times the uv-tile size candidates of a plan (the tile shape drives the
// gridding schedule: patch halo overhead against work-unit count) on a deterministic
// subsample of the visibilities and keeps the winner in a JSON cache keyed by the
// workload's shape.
#include <algorithm>
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
};

namespace {

constexpr int BATCH_MAX_BRANCHES = 16;

void destroy_batch(rimo_batch* b) {
    if (!b) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(b->device);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (auto e : b->joins) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    for (auto s : b->branches) cudaStreamDestroy(s);
    if (b->root) cudaStreamDestroy(b->root);
    cudaSetDevice(cur);
    delete b;
}

// Records all channels' applies into a graph on the batch's own root stream: fork, one
// branch stream per channel (round robin over the branch pool), join back.  Nothing runs
// during recording; the graph is launched on the caller's stream afterwards.
void capture(rimo_batch* b, const float2* x, float2* out, int real_only) {
    cudaStream_t s = b->root;
    const size_t img = (size_t)b->nx * b->ny;
    std::vector<bool> prof(b->plans.size());
    for (size_t i = 0; i < b->plans.size(); ++i) {
        prof[i] = b->plans[i]->prof_on;
        b->plans[i]->prof_on = false;  // stage timers record events the graph cannot replay
    }
    RIMO_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaGraph_t graph = nullptr;
    try {
        RIMO_CUDA(cudaEventRecord(b->fork, s));
        for (size_t i = 0; i < b->plans.size(); ++i) {
            cudaStream_t br = b->branches[i % b->branches.size()];
            RIMO_CUDA(cudaStreamWaitEvent(br, b->fork, 0));
            apply_phi_adj_phi(b->plans[i], x + i * img, out + i * img, real_only, br);
            RIMO_CUDA(cudaEventRecord(b->joins[i], br));
            RIMO_CUDA(cudaStreamWaitEvent(s, b->joins[i], 0));
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
    if (out) *out = nullptr;
    rimo_batch* b = nullptr;
    RIMO_API_BEGIN
    if (!out || !plans || n_plans <= 0) fail(RIMO_ERR_INVALID_ARG, "need an output and at least one plan");
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
    RIMO_CUDA(cudaStreamCreateWithFlags(&b->root, cudaStreamNonBlocking));
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

rimo_status rimo_autotune_tile(const double* uvw, int64_t M, const rimo_plan_params* base, const char* cache_path,
                               void* stream, int32_t* tile_out, double* ms_out) {
    RIMO_API_BEGIN
    if (!uvw || M <= 0 || !base || !tile_out) fail(RIMO_ERR_INVALID_ARG, "null argument or empty data");
    const int cands[2] = {32, 64};
    if (ms_out) ms_out[0] = ms_out[1] = -1.0;
    // deterministic subsample: every stride-th row, at most 1M rows
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
    q.tile_size = 0;
    rimo_plan_info est;
    if (rimo_plan_estimate(src, Ms, &q, &est) != RIMO_OK) fail(RIMO_ERR_INVALID_ARG, rimo_last_error());
    int max_s = 0;
    for (int i = 0; i < 64; ++i) max_s = std::max(max_s, (int)est.support_table[i]);
    const std::string key = tune_key(q, M, est.P, max_s + q.kb_support - 1);
    std::map<std::string, int> cache;
    if (cache_path && *cache_path) {
        cache = read_cache(cache_path);
        auto it = cache.find(key);
        if (it != cache.end() && (it->second == 32 || it->second == 64)) {
            *tile_out = it->second;
            return RIMO_OK;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    float2 *x = nullptr, *o = nullptr;
    const size_t img = (size_t)q.nx * q.ny * sizeof(float2);
    RIMO_CUDA(cudaMalloc(&x, img));
    RIMO_CUDA(cudaMalloc(&o, img));
    double best = 1e300;
    int pick = cands[0];
    try {
        // a point at the centre and one off-centre: every bin's grid is non-trivial
        RIMO_CUDA(cudaMemsetAsync(x, 0, img, s));
        const float2 one = make_float2(1.f, 0.f);
        RIMO_CUDA(cudaMemcpyAsync(x + (size_t)(q.ny / 2) * q.nx + q.nx / 2, &one, sizeof(one), cudaMemcpyHostToDevice, s));
        RIMO_CUDA(cudaMemcpyAsync(x + (size_t)(q.ny / 4) * q.nx + q.nx / 3, &one, sizeof(one), cudaMemcpyHostToDevice, s));
        cudaEvent_t e0, e1;
        RIMO_CUDA(cudaEventCreate(&e0));
        RIMO_CUDA(cudaEventCreate(&e1));
        for (int c = 0; c < 2; ++c) {
            q.tile_size = cands[c];
            rimo_plan_t p = nullptr;
            if (rimo_plan_create(src, Ms, &q, stream, &p) != RIMO_OK) fail(RIMO_ERR_INVALID_ARG, rimo_last_error());
            float ms = 0.f;
            try {
                apply_phi_adj_phi(p, x, o, 0, s);  // warm-up
                RIMO_CUDA(cudaEventRecord(e0, s));
                for (int r = 0; r < 3; ++r) apply_phi_adj_phi(p, x, o, 0, s);
                RIMO_CUDA(cudaEventRecord(e1, s));
                RIMO_CUDA(cudaEventSynchronize(e1));
                RIMO_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            } catch (...) {
                rimo_plan_destroy(p);
                throw;
            }
            rimo_plan_destroy(p);
            const double t = ms / 3.0;
            if (ms_out) ms_out[c] = t;
            if (t < best) {
                best = t;
                pick = cands[c];
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    } catch (...) {
        cudaFree(x);
        cudaFree(o);
        throw;
    }
    cudaFree(x);
    cudaFree(o);
    *tile_out = pick;
    if (cache_path && *cache_path) {
        cache[key] = pick;
        write_cache(cache_path, cache);
    }
    RIMO_API_END
}

}  // extern "C"
