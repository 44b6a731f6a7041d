// Packed splat records and their TMA descriptor.
//
// The tensor-core blends stage the splats of each chunk into shared memory
// (Sec. 3.4 stages indices, then features, ahead of the contraction).  On
// this GPU the features come in by TMA: one 64-byte record per item holds
// everything a chunk's producer needs (mean, conic, log2 opacity and its cap
// at 0.99, 1/opacity, colour, the Gaussian index), so a chunk of 32 splats is
// eight tile::gather4 copies of four rows each instead of ten dependent loads
// per thread.
#include <mutex>

#include "internal.h"

namespace gs {
namespace {

constexpr float kLog2AlphaMax = -0.014499569695115089f;  // log2(0.99)

__global__ void k_pack_splats(int n_items, int n_per_view, const float2* __restrict__ mean2d,
                              const float* __restrict__ conic, const float* __restrict__ opac,
                              const float* __restrict__ rgb, float4* __restrict__ rec) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_items) return;
    const uint32_t g = (uint32_t)i - ((uint32_t)i / (uint32_t)n_per_view) * (uint32_t)n_per_view;
    const float2 m = mean2d[i];
    const float o = opac[g];
    // the same arithmetic as the load-based producers, so both give the same rows
    const float l2o = o > 0.f ? __log2f(o) : -INFINITY;
    float r = 0.f, gr = 0.f, b = 0.f;
    if (rgb) {
        r = rgb[3 * (size_t)i];
        gr = rgb[3 * (size_t)i + 1];
        b = rgb[3 * (size_t)i + 2];
    }
    float4* out = rec + 4 * (size_t)i;
    out[0] = make_float4(m.x, m.y, conic[3 * (size_t)i], conic[3 * (size_t)i + 1]);
    out[1] = make_float4(conic[3 * (size_t)i + 2], l2o, fminf(l2o, kLog2AlphaMax), o > 0.f ? 1.0f / o : 0.f);
    out[2] = make_float4(r, gr, b, __uint_as_float(g));
    out[3] = make_float4(0.f, 0.f, 0.f, 0.f);
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, looked up once per process.
EncodeTiled encoder(cudaError_t* err) {
    static std::mutex mu;
    static EncodeTiled fn = nullptr;
    std::lock_guard<std::mutex> lock(mu);
    *err = cudaSuccess;
    if (fn == nullptr) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        *err = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (*err == cudaSuccess && (q != cudaDriverEntryPointSuccess || p == nullptr)) *err = cudaErrorNotSupported;
        if (*err != cudaSuccess) return nullptr;
        fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

}  // namespace

cudaError_t launch_pack_splats(int n_items, int n_per_view, const float2* mean2d, const float* conic,
                               const float* opac, const float* rgb, float* rec, cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    k_pack_splats<<<(n_items + 255) / 256, 256, 0, s>>>(n_items, n_per_view, mean2d, conic, opac, rgb,
                                                        reinterpret_cast<float4*>(rec));
    count_launches();
    return cudaGetLastError();
}

// 2D table: kRecFloats float32 per row (64 bytes), n_items rows; one box is a
// whole row (16 x 1), the shape tile::gather4 takes (four such rows per copy).
// Rows outside the table read as zeros.
cudaError_t encode_rec_map(CUtensorMap* map, const void* rec, int n_items) {
    cudaError_t e = cudaSuccess;
    EncodeTiled enc = encoder(&e);
    if (enc == nullptr) return e;
    const cuuint64_t dims[2] = {(cuuint64_t)kRecFloats, (cuuint64_t)n_items};
    const cuuint64_t strides[1] = {(cuuint64_t)kRecBytes};
    const cuuint32_t box[2] = {(cuuint32_t)kRecFloats, 1u};
    const cuuint32_t elem[2] = {1u, 1u};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(rec), dims, strides, box, elem,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace gs
