// Phi^dagger Phi without any device allocation: the scratch memory of the apply (half-
// transformed rows, the forward / folded grid, the tile patches and the tile schedulers)
// is carved from one statically allocated device array of this file instead of the
// plan's own scratch buffers.  The computation is the plan's regular apply, unchanged.
#include <mutex>

#include "internal.h"

namespace rimo {

constexpr size_t NOALLOC_BYTES = (size_t)RIMO_NOALLOC_SCRATCH_BYTES;

// One copy per device that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
static std::mutex g_noalloc_mutex;
static unsigned char* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device.  In host code the array's
// name is only a host-side stand-in, so the address comes from cudaGetSymbolAddress,
// once per device, with that device current.
static unsigned char* noalloc_scratch() {
    int dev = 0;
    RIMO_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) fail(RIMO_ERR_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            fail(RIMO_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch failed: ") +
                                    cudaGetErrorString(e));
        }
        g_noalloc_ptr[dev] = static_cast<unsigned char*>(ptr);
    }
    return g_noalloc_ptr[dev];
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }


}  // namespace rimo

using namespace rimo;

extern "C" rimo_status rimo_apply_phi_adj_phi_noalloc(rimo_plan_t p, const rimo_cfloat* x,
                                                       rimo_cfloat* out, int32_t real_part_only,
                                                       void* stream) {
    try {
        if (!p) fail(RIMO_ERR_INVALID_ARG, "null plan");
        if (!x || !out) fail(RIMO_ERR_INVALID_ARG, "null buffer");
        if ((const void*)x == (const void*)out) fail(RIMO_ERR_INVALID_ARG, "x and out must be distinct");
        if (p->mode != RIMO_MODE_STORED_G || p->h_built)
            fail(RIMO_ERR_UNSUPPORTED, "the allocation-free apply covers stored-G plans only");
        const size_t counters = align256((size_t)p->P * sizeof(int32_t));
        const size_t ab = align256((size_t)2 * p->nx * p->ny * sizeof(float2));
        const size_t grid = align256((size_t)p->gx * p->gy * sizeof(float2));
        const size_t patches = align256((size_t)std::max(1, p->max_tiles_bin) * p->PW * p->PW * sizeof(float2));
        const size_t need = counters + ab + grid + patches;
        if (need > NOALLOC_BYTES)
            fail(RIMO_ERR_UNSUPPORTED, "plan needs " + std::to_string(need) + " bytes of scratch, above the " +
                                           std::to_string(NOALLOC_BYTES) + "-byte static scratch");
        unsigned char* base = noalloc_scratch();
        cudaStream_t s = (cudaStream_t)stream;
        // run the regular apply with the plan's scratch pointers pointed into the array.
        // The array keeps the previous call's contents (possibly another plan's layout);
        // none of it is read before this apply writes it: the schedulers are cleared by
        // the apply itself, the forward column pass writes every cell of every needed
        // uv-tile (the tiles any active patch of the bin reaches, a superset of the cells
        // the grid step stages), the fold writes the needed tiles of the gridded grid, and
        // the inverse column pass reads needed tiles only.
        int32_t* own_counter = p->d_counter;
        float2* own_ab = p->d_AB;
        float2* own_x = p->d_X;
        float2* own_patch = p->d_patch;
        p->d_counter = reinterpret_cast<int32_t*>(base);
        p->d_AB = reinterpret_cast<float2*>(base + counters);
        p->d_X = reinterpret_cast<float2*>(base + counters + ab);
        p->d_patch = reinterpret_cast<float2*>(base + counters + ab + grid);
        try {
            apply_phi_adj_phi(p, (const float2*)x, (float2*)out, real_part_only, s);
            RIMO_CUDA(cudaGetLastError());
        } catch (...) {
            p->d_counter = own_counter;
            p->d_AB = own_ab;
            p->d_X = own_x;
            p->d_patch = own_patch;
            throw;
        }
        p->d_counter = own_counter;
        p->d_AB = own_ab;
        p->d_X = own_x;
        p->d_patch = own_patch;
        return RIMO_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        return e.status;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return RIMO_ERR_CUDA;
    }
}
