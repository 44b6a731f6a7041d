// Dispatch of the tensor-core blend over variants and pipeline shapes.
#include "blend_tc.cuh"

namespace gs {

bool tc_config_supported(int variant, int chunk, int stages) {
    if (variant < GS_BLEND_TC_FP16 || variant > GS_BLEND_TC_BF16_SPLIT) return false;
    return (chunk == 32 && (stages == 2 || stages == 4)) || (chunk == 16 && stages == 4) ||
           (chunk == 64 && stages == 3);
}

cudaError_t launch_blend_tc(const BlendArgs& a, int variant, int chunk, int stages, bool dump, int grid,
                            cudaStream_t s) {
    switch (variant) {
        case GS_BLEND_TC_FP16: return tc::launch_variant<GS_BLEND_TC_FP16>(a, chunk, stages, dump, grid, s);
        case GS_BLEND_TC_BF16: return tc::launch_variant<GS_BLEND_TC_BF16>(a, chunk, stages, dump, grid, s);
        case GS_BLEND_TC_FP16_SPLIT:
            return tc::launch_variant<GS_BLEND_TC_FP16_SPLIT>(a, chunk, stages, dump, grid, s);
        case GS_BLEND_TC_BF16_SPLIT:
            return tc::launch_variant<GS_BLEND_TC_BF16_SPLIT>(a, chunk, stages, dump, grid, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gs
