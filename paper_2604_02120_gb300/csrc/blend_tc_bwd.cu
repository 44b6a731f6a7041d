// Dispatch of the tensor-core blend gradient over variants.
#include "blend_tc_bwd.cuh"

namespace gs {

cudaError_t launch_blend_tc_bwd(const BlendArgs& a0, const GradArgs& g, int variant, int stages, cudaStream_t s) {
    BlendArgs a = a0;
    cudaError_t e = cudaSuccess;
    a.queue = tile_queue_slot(s, &e);
    if (a.queue == nullptr) return e;
    a.total_tiles = shard_items(a0);  // queue length; item q is position q * shard_count + shard_index of the order
    switch (variant) {
        case GS_BLEND_TC_FP16: return tc::launch_bwd_variant<GS_BLEND_TC_FP16>(a, g, stages, s);
        case GS_BLEND_TC_BF16: return tc::launch_bwd_variant<GS_BLEND_TC_BF16>(a, g, stages, s);
        case GS_BLEND_TC_FP16_SPLIT: return tc::launch_bwd_variant<GS_BLEND_TC_FP16_SPLIT>(a, g, stages, s);
        case GS_BLEND_TC_BF16_SPLIT: return tc::launch_bwd_variant<GS_BLEND_TC_BF16_SPLIT>(a, g, stages, s);
        case GS_BLEND_TC_FP8_SPLIT: return tc::launch_bwd_variant<GS_BLEND_TC_FP8_SPLIT>(a, g, stages, s);
    }
    return cudaErrorInvalidValue;
}

bool tc_bwd_stages_supported(int stages) {
    return stages == 0 || stages == 2 || stages == 3 || stages == 4 || stages == 6;
}

}  // namespace gs
