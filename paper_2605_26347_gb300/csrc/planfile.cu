// Plan files: the inputs a plan is created from, so that the identical plan can be rebuilt
// in another process or later (Section 4: the planning stage may run on its own, and both
// stages read one parameter file and one observation file of (u, v, w) coordinates).  A
// plan is fully determined by its coordinates and parameters; the file holds those and,
// when given, the data weights injected into the operator (Section 2).
//
// Layout (the host's little-endian byte order):
//   offset  0  char[8]   "RIMOPLAN"
//           8  uint32    format version, 1
//          12  uint32    sizeof(rimo_plan_params)
//          16  int64     M
//          24  uint32    1 when M float32 data weights follow the coordinates, else 0
//          28  uint32    0
//          32  rimo_plan_params
//          ..  float64   uvw[M][3]
//          ..  float32   weights[M]                    (when present)
//          ..  uint64    checksum of every byte before it
// The checksum is FNV-1a (64-bit, Fowler-Noll-Vo) of each 1 MiB block, then FNV-1a of the
// block digests in order, each taken as 8 little-endian bytes; the blocks hash in parallel.
// Everything here runs on the host; only rimo_plan_create_from_file touches a GPU.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "internal.h"
#include "planner.h"

namespace rimo {
namespace {

constexpr char MAGIC[8] = {'R', 'I', 'M', 'O', 'P', 'L', 'A', 'N'};
constexpr uint32_t FORMAT = 1;
constexpr size_t HEAD = 32 + sizeof(rimo_plan_params);
constexpr size_t BLOCK = size_t(1) << 20;
constexpr uint64_t FNV_OFFSET = 14695981039346656037ull, FNV_PRIME = 1099511628211ull;

uint64_t fnv1a(const uint8_t* p, size_t n, uint64_t h) {
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= FNV_PRIME;
    }
    return h;
}

uint64_t checksum(const uint8_t* p, size_t n) {
    const int64_t nb = (int64_t)((n + BLOCK - 1) / BLOCK);
    std::vector<uint64_t> d((size_t)nb);
    planner::parallel_for(nb, [&](int64_t b, int64_t e) {
        for (int64_t i = b; i < e; ++i) {
            const size_t lo = (size_t)i * BLOCK;
            d[(size_t)i] = fnv1a(p + lo, std::min(BLOCK, n - lo), FNV_OFFSET);
        }
    }, 1);
    uint64_t h = FNV_OFFSET;
    for (uint64_t v : d) {
        uint8_t le[8];
        for (int k = 0; k < 8; ++k) le[k] = (uint8_t)(v >> (8 * k));
        h = fnv1a(le, 8, h);
    }
    return h;
}

size_t file_bytes(int64_t M, bool weights) {
    return HEAD + (size_t)M * 24 + (weights ? (size_t)M * 4 : 0) + 8;
}

void check_weights(const float* w, int64_t M) {
    for (int64_t k = 0; k < M; ++k)
        if (!(w[k] >= 0.f) || !std::isfinite(w[k])) fail(RIMO_ERR_INVALID_ARG, "weights must be finite and >= 0");
}

struct FileCloser {
    void operator()(FILE* f) const { std::fclose(f); }
};

// A plan file read whole and checked: header, size, checksum, parameters, coordinates and
// weights, each failure an INVALID_ARG naming what is wrong.
struct PlanFile {
    rimo_plan_params params{};
    int64_t M = 0;
    bool has_weights = false;
    std::vector<double> uvw;
    std::vector<float> weights;
};

PlanFile read_plan_file(const char* path) {
    if (!path) fail(RIMO_ERR_INVALID_ARG, "null path");
    std::unique_ptr<FILE, FileCloser> f(std::fopen(path, "rb"));
    if (!f) fail(RIMO_ERR_INVALID_ARG, std::string("cannot open plan file ") + path);
    if (std::fseek(f.get(), 0, SEEK_END) != 0) fail(RIMO_ERR_INVALID_ARG, "plan file: cannot seek");
    const long len = std::ftell(f.get());
    std::rewind(f.get());
    if (len < (long)(HEAD + 8)) fail(RIMO_ERR_INVALID_ARG, "plan file: shorter than its header");
    std::vector<uint8_t> head(HEAD);
    if (std::fread(head.data(), 1, HEAD, f.get()) != HEAD) fail(RIMO_ERR_INVALID_ARG, "plan file: short read");
    uint32_t version, pbytes, hw, zero;
    PlanFile pf;
    std::memcpy(&version, &head[8], 4);
    std::memcpy(&pbytes, &head[12], 4);
    std::memcpy(&pf.M, &head[16], 8);
    std::memcpy(&hw, &head[24], 4);
    std::memcpy(&zero, &head[28], 4);
    if (std::memcmp(head.data(), MAGIC, 8) != 0) fail(RIMO_ERR_INVALID_ARG, "plan file: not a plan file");
    if (version != FORMAT) fail(RIMO_ERR_INVALID_ARG, "plan file: unknown format version " + std::to_string(version));
    if (pbytes != sizeof(rimo_plan_params) || hw > 1 || zero != 0)
        fail(RIMO_ERR_INVALID_ARG, "plan file: header fields out of range");
    if (pf.M <= 0 || pf.M > 2000000000LL) fail(RIMO_ERR_INVALID_ARG, "plan file: M out of range");
    pf.has_weights = hw == 1;
    if ((size_t)len != file_bytes(pf.M, pf.has_weights))
        fail(RIMO_ERR_INVALID_ARG, "plan file: size does not match its header (truncated or extended)");
    std::vector<uint8_t> all((size_t)len);
    std::memcpy(all.data(), head.data(), HEAD);
    const size_t rest = (size_t)len - HEAD;
    if (std::fread(all.data() + HEAD, 1, rest, f.get()) != rest) fail(RIMO_ERR_INVALID_ARG, "plan file: short read");
    uint64_t stored;
    std::memcpy(&stored, all.data() + len - 8, 8);
    if (checksum(all.data(), (size_t)len - 8) != stored) fail(RIMO_ERR_INVALID_ARG, "plan file: checksum mismatch (corrupted)");
    std::memcpy(&pf.params, &head[32], sizeof(rimo_plan_params));
    pf.uvw.resize((size_t)pf.M * 3);
    std::memcpy(pf.uvw.data(), all.data() + HEAD, (size_t)pf.M * 24);
    if (pf.has_weights) {
        pf.weights.resize((size_t)pf.M);
        std::memcpy(pf.weights.data(), all.data() + HEAD + (size_t)pf.M * 24, (size_t)pf.M * 4);
    }
    validate_params(pf.params);
    validate_uvw(pf.uvw.data(), pf.M, pf.params);
    if (pf.has_weights) check_weights(pf.weights.data(), pf.M);
    return pf;
}

}  // namespace
}  // namespace rimo

using namespace rimo;

extern "C" {

rimo_status rimo_plan_file_write(const char* path, const double* uvw, int64_t M, const rimo_plan_params* q,
                                 const float* weights) {
    RIMO_API_BEGIN
    if (!path || !uvw || !q || M <= 0) fail(RIMO_ERR_INVALID_ARG, "null pointer or M <= 0");
    if (M > 2000000000LL) fail(RIMO_ERR_INVALID_ARG, "M above 2e9 visibilities");
    validate_params(*q);
    validate_uvw(uvw, M, *q);
    if (weights) check_weights(weights, M);
    const size_t len = file_bytes(M, weights != nullptr);
    std::vector<uint8_t> all(len, 0);
    std::memcpy(all.data(), MAGIC, 8);
    const uint32_t version = FORMAT, pbytes = sizeof(rimo_plan_params), hw = weights ? 1u : 0u;
    std::memcpy(&all[8], &version, 4);
    std::memcpy(&all[12], &pbytes, 4);
    std::memcpy(&all[16], &M, 8);
    std::memcpy(&all[24], &hw, 4);
    std::memcpy(&all[32], q, sizeof(rimo_plan_params));
    std::memcpy(&all[HEAD], uvw, (size_t)M * 24);
    if (weights) std::memcpy(&all[HEAD + (size_t)M * 24], weights, (size_t)M * 4);
    const uint64_t sum = checksum(all.data(), len - 8);
    std::memcpy(&all[len - 8], &sum, 8);
    std::unique_ptr<FILE, FileCloser> f(std::fopen(path, "wb"));
    if (!f) fail(RIMO_ERR_INVALID_ARG, std::string("cannot create plan file ") + path);
    if (std::fwrite(all.data(), 1, len, f.get()) != len || std::fflush(f.get()) != 0)
        fail(RIMO_ERR_INVALID_ARG, std::string("cannot write plan file ") + path);
    RIMO_API_END
}

rimo_status rimo_plan_file_info(const char* path, rimo_plan_params* params, int64_t* M, int32_t* has_weights) {
    RIMO_API_BEGIN
    PlanFile pf = read_plan_file(path);
    if (params) *params = pf.params;
    if (M) *M = pf.M;
    if (has_weights) *has_weights = pf.has_weights ? 1 : 0;
    RIMO_API_END
}

rimo_status rimo_plan_create_from_file(const char* path, void* stream, rimo_plan_t* out) {
    if (out) *out = nullptr;
    try {
        if (!out) fail(RIMO_ERR_INVALID_ARG, "null output");
        PlanFile pf = read_plan_file(path);
        rimo_plan_t p = nullptr;
        rimo_status st = rimo_plan_create(pf.uvw.data(), pf.M, &pf.params, stream, &p);
        if (st != RIMO_OK) return st;  // its message is already set
        if (pf.has_weights) {
            st = rimo_plan_set_weights(p, pf.weights.data(), stream);
            if (st != RIMO_OK) {
                const std::string msg = rimo_last_error();
                rimo_plan_destroy(p);
                set_last_error(msg);
                return st;
            }
        }
        *out = p;
        return RIMO_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        return e.status;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return RIMO_ERR_OOM;
    }
}

}  // extern "C"
