// Preprocessing stage (Sec. 2.1 (a)): EWA projection of 3D Gaussians, one
// thread per Gaussian.  FP32 throughout; the 2D covariance and its inverse are
// recomputed in FP64 when the FP32 determinant is below 1e-6.
#include "project.cuh"

namespace gs {
namespace {

// blockIdx.y = view; outputs of view v, Gaussian g at index v * n + g.
template <int SH_DEGREE, bool VEC16>
__global__ void __launch_bounds__(256) k_project(int n, const float* __restrict__ means,
                                                 const float* __restrict__ scales, const float* __restrict__ quats,
                                                 const float* __restrict__ sh,
                                                 const __grid_constant__ CamViews views,
                                                 float2* __restrict__ mean2d_all, float* __restrict__ conic_all,
                                                 float* __restrict__ depth_all, int* __restrict__ radius_all,
                                                 float* __restrict__ rgb_all, uint32_t* __restrict__ touched_all) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    project_gaussian<SH_DEGREE, VEC16>(g, means, scales, quats, sh, views.cams[blockIdx.y], (size_t)blockIdx.y * n,
                                       mean2d_all, conic_all, depth_all, radius_all, rgb_all, touched_all);
}

}  // namespace

cudaError_t launch_project(int n, const float* means, const float* scales, const float* quats, const float* sh,
                           int sh_degree, const CamViews& cams, float* mean2d, float* conic, float* depth,
                           int* radius, float* rgb, uint32_t* tiles_touched, cudaStream_t s) {
    const int block = 256;
    const dim3 grid((n + block - 1) / block, cams.num_views);
    // 16-byte coefficient loads for degrees 1 and 3 (3K a multiple of 4) on an aligned array
    const bool vec = (reinterpret_cast<uintptr_t>(sh) & 15) == 0;
    switch (sh_degree) {
        case 0: k_project<0, false><<<grid, block, 0, s>>>(n, means, scales, quats, sh, cams, reinterpret_cast<float2*>(mean2d), conic, depth, radius, rgb,
                                       tiles_touched);
            break;
        case 1:
            if (vec) k_project<1, true><<<grid, block, 0, s>>>(n, means, scales, quats, sh, cams, reinterpret_cast<float2*>(mean2d), conic, depth, radius, rgb,
                                       tiles_touched);
            else k_project<1, false><<<grid, block, 0, s>>>(n, means, scales, quats, sh, cams, reinterpret_cast<float2*>(mean2d), conic, depth, radius, rgb,
                                       tiles_touched);
            break;
        case 2: k_project<2, false><<<grid, block, 0, s>>>(n, means, scales, quats, sh, cams, reinterpret_cast<float2*>(mean2d), conic, depth, radius, rgb,
                                       tiles_touched);
            break;
        default:
            if (vec) k_project<3, true><<<grid, block, 0, s>>>(n, means, scales, quats, sh, cams, reinterpret_cast<float2*>(mean2d), conic, depth, radius, rgb,
                                       tiles_touched);
            else k_project<3, false><<<grid, block, 0, s>>>(n, means, scales, quats, sh, cams, reinterpret_cast<float2*>(mean2d), conic, depth, radius, rgb,
                                       tiles_touched);
            break;
    }
    count_launches();
    return cudaGetLastError();
}

}  // namespace gs
