// gs_bin_sort_noalloc: the duplication + sort stage for callers that cannot
// allocate device memory, e.g. code running inside a framework whose
// allocator owns the device, plugins handed only their input and output
// buffers, or processes under a memory budget fixed up front.  The scratch
// gs_bin_sort takes from the caller lives here in one statically sized device
// array instead.  Every device that loads this library holds the array
// (kNoAllocScratchBytes) until the process exits.
#include <atomic>
#include <cstdio>

#include "internal.h"

namespace gs {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;  // 64 MiB

// Scratch of every gs_bin_sort_noalloc call on this device.  Calls share it,
// so calls that overlap on the GPU (different streams, or threads) race.
static __device__ __align__(256) unsigned char g_bin_sort_scratch[kNoAllocScratchBytes];

// Device address of g_bin_sort_scratch for the current device, looked up once
// per device (in host code the symbol only names a host-side stand-in).
void* scratch_address(gs_status* st) {
    static std::atomic<void*> addr[64] = {};  // per device; threads may look it up at once
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        *st = cuda_status(e, "gs_bin_sort_noalloc: current device");
        return nullptr;
    }
    if (dev < 0 || dev >= 64) {
        set_error("gs_bin_sort_noalloc: device ordinal %d out of range", dev);
        *st = GS_ERR_UNSUPPORTED;
        return nullptr;
    }
    void* a = addr[dev].load(std::memory_order_acquire);
    if (a == nullptr) {
        e = cudaGetSymbolAddress(&a, g_bin_sort_scratch);
        if (e != cudaSuccess) {
            *st = cuda_status(e, "gs_bin_sort_noalloc: scratch address");
            return nullptr;
        }
        addr[dev].store(a, std::memory_order_release);
    }
    *st = GS_OK;
    return a;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

size_t gs_bin_sort_noalloc_max_bytes(void) { return kNoAllocScratchBytes; }

gs_status gs_bin_sort_noalloc(int32_t n, const float* mean2d, const int32_t* radius, const float* depth,
                              int32_t width, int32_t height, int64_t capacity, uint64_t* keys_sorted,
                              uint32_t* ids_sorted, uint32_t* tile_ranges, int64_t* n_instances, gs_stream stream) {
    clear_error();
    SortViews sv{};
    sv.num_views = 1;
    sv.n_per_view = n;
    // the same view check as gs_bin_sort: each side 1..2^20 and fewer than 2^31 tiles
    if (n < 0 || capacity < 0 || capacity >= (int64_t(1) << 32) || !n_instances || !tile_ranges ||
        !fill_views(1, &width, &height, sv.views, &sv.total_tiles)) {
        set_error("gs_bin_sort_noalloc: bad arguments");
        return GS_ERR_INVALID_ARG;
    }
    if (n > 0 && (!mean2d || !radius || !depth)) {
        set_error("gs_bin_sort_noalloc: null pointer");
        return GS_ERR_INVALID_ARG;
    }
    if (capacity > 0 && !ids_sorted) {
        set_error("gs_bin_sort_noalloc: null output pointer");
        return GS_ERR_INVALID_ARG;
    }
    const size_t need = bin_sort_workspace_bytes(n, capacity, sv.total_tiles);
    if (need > kNoAllocScratchBytes) {
        set_error("gs_bin_sort_noalloc: n = %d and capacity = %lld need %zu bytes of scratch, more than the "
                  "built-in %zu; use gs_bin_sort with a caller workspace",
                  n, (long long)capacity, need, kNoAllocScratchBytes);
        return GS_ERR_WORKSPACE;
    }
    gs_status st = GS_OK;
    void* ws = scratch_address(&st);
    if (ws == nullptr) return st;
    return bin_sort_run(sv, mean2d, radius, depth, capacity, ws, kNoAllocScratchBytes, keys_sorted, ids_sorted,
                        tile_ranges, n_instances, nullptr, stream);
}

}  // extern "C"
