// Tensor-core blend gradient for gs_variant value 3.
#include "blend_tc_bwd.cuh"

namespace gs {
namespace tc {

template <>
cudaError_t launch_bwd_variant<3>(const BlendArgs& a, const GradArgs& g, int stages, cudaStream_t s) {
    return launch_bwd_stages<3>(a, g, stages, s);
}

}  // namespace tc
}  // namespace gs
