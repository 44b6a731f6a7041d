// Dispatch of the tensor-core blend over variants and pipeline shapes, and the
// per-device pool of tile-queue counters the persistent kernel consumes.
#include <atomic>

#include "blend_tc.cuh"

namespace gs {
namespace {

constexpr int kQueueSlots = 1024;
// Tile counters of the persistent blend.  Each launch takes the next slot
// (round robin) and zeroes it on its stream first, so launches in flight on
// different streams use different counters (up to kQueueSlots at once).
__device__ unsigned g_tile_queue[kQueueSlots];
std::atomic<unsigned> g_next_slot{0};

}  // namespace

unsigned* tile_queue_slot(cudaStream_t s, cudaError_t* err) {
    static std::atomic<unsigned*> base[64] = {};  // per device; threads may look it up at once
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess) return nullptr;
    if (dev < 0 || dev >= 64) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    unsigned* b = base[dev].load(std::memory_order_acquire);
    if (b == nullptr) {
        void* p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_tile_queue);
        if (*err != cudaSuccess) return nullptr;
        b = static_cast<unsigned*>(p);
        base[dev].store(b, std::memory_order_release);
    }
    unsigned* q = b + (g_next_slot.fetch_add(1, std::memory_order_relaxed) % kQueueSlots);
    *err = cudaMemsetAsync(q, 0, sizeof(unsigned), s);
    return *err == cudaSuccess ? q : nullptr;
}

bool tc_config_supported(int variant, int chunk, int stages) {
    if (variant < GS_BLEND_TC_FP16 || variant > GS_BLEND_PERSISTENT_FP32) return false;
    return (chunk == 32 && (stages == 2 || stages == 4)) || (chunk == 16 && stages == 4) ||
           (chunk == 16 && stages == 6);
}

cudaError_t launch_blend_tc(const BlendArgs& a0, int variant, int chunk, int stages, bool dump, int items,
                            cudaStream_t s) {
    BlendArgs a = a0;
    cudaError_t e = cudaSuccess;
    a.queue = tile_queue_slot(s, &e);
    if (a.queue == nullptr) return e;
    a.total_tiles = items;
    switch (variant) {
        case GS_BLEND_TC_FP16: return tc::launch_variant<GS_BLEND_TC_FP16>(a, chunk, stages, dump, items, s);
        case GS_BLEND_TC_BF16: return tc::launch_variant<GS_BLEND_TC_BF16>(a, chunk, stages, dump, items, s);
        case GS_BLEND_TC_FP16_SPLIT:
            return tc::launch_variant<GS_BLEND_TC_FP16_SPLIT>(a, chunk, stages, dump, items, s);
        case GS_BLEND_TC_BF16_SPLIT:
            return tc::launch_variant<GS_BLEND_TC_BF16_SPLIT>(a, chunk, stages, dump, items, s);
        case GS_BLEND_TC_FP8_SPLIT:
            return tc::launch_variant<GS_BLEND_TC_FP8_SPLIT>(a, chunk, stages, dump, items, s);
        case GS_BLEND_PERSISTENT_FP32:
            if (dump) return cudaErrorInvalidValue;
            return tc::launch_variant<GS_BLEND_PERSISTENT_FP32>(a, chunk, stages, dump, items, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gs
