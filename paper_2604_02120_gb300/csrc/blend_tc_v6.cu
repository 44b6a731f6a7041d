// Persistent-blend instantiations for gs_variant value 6 (GS_BLEND_PERSISTENT_FP32:
// the tensor-core kernel with the exponent contraction on CUDA cores; no tile-power dump).
#include "blend_tc.cuh"

namespace gs {
namespace tc {

template <>
cudaError_t launch_variant<6>(const BlendArgs& a, int chunk, int stages, bool dump, int grid, cudaStream_t s) {
    if (dump) return cudaErrorInvalidValue;
    if (chunk == 32 && stages == 4) return launch_inst<6, 32, 4, false>(a, grid, s);
    if (chunk == 32 && stages == 2) return launch_inst<6, 32, 2, false>(a, grid, s);
    if (chunk == 16 && stages == 4) return launch_inst<6, 16, 4, false>(a, grid, s);
    if (chunk == 16 && stages == 6) return launch_inst<6, 16, 6, false>(a, grid, s);
    return cudaErrorInvalidValue;
}

}  // namespace tc
}  // namespace gs
