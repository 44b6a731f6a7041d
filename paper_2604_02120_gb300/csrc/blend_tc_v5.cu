// Tensor-core blend instantiations for gs_variant value 5.
#include "blend_tc.cuh"

namespace gs {
namespace tc {

template <>
cudaError_t launch_variant<5>(const BlendArgs& a, int chunk, int stages, bool dump, int grid, cudaStream_t s) {
    if (dump) return launch_inst<5, 32, 2, true>(a, grid, s);
    if (chunk == 32 && stages == 4) return launch_inst<5, 32, 4, false>(a, grid, s);
    if (chunk == 32 && stages == 2) return launch_inst<5, 32, 2, false>(a, grid, s);
    if (chunk == 16 && stages == 4) return launch_inst<5, 16, 4, false>(a, grid, s);
    if (chunk == 16 && stages == 6) return launch_inst<5, 16, 6, false>(a, grid, s);
    return cudaErrorInvalidValue;
}

}  // namespace tc
}  // namespace gs
