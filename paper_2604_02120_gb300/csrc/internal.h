// Host-side declarations shared by the translation units of the library.
#pragma once

#include "common.cuh"

namespace gs {

constexpr int kMaxViews = 32;

// One rendered view (camera) of a blend call.  Its tiles are numbered
// [tile_begin, tile_begin + tiles_x * tiles_y) in the call's global tile
// space; its outputs start at pixel offset pix_off of the packed per-view
// arrays (image: 3 * pix_off floats in, CHW per view).
struct ViewDesc {
    int W, H, tiles_x, tile_begin;
    long long pix_off;
};

struct BlendArgs {
    int W, H, tiles_x, num_tiles;  // single-view shape (the FP32 kernels)
    int num_views, total_tiles;    // view table (the tensor-core kernel)
    ViewDesc views[kMaxViews];
    unsigned* queue;               // tile counter, zero at launch (tensor-core kernel)
    const uint32_t* ranges;
    const uint32_t* ids;
    const float2* mean2d;
    const float* conic;
    const float* opac;
    const float* rgb;
    float bg[3];
    float* image;
    float* T_final;
    int* n_contrib;
    unsigned* err;
    uint64_t timeout_ns;
    int ref_origin;
    // gs_tile_power only
    const int* tiles;
    int max_len;
    float* dump;
};

struct GradArgs {
    const float* T_final;
    const int* n_contrib;
    const float* dL_dimage;
    float2* dmean2d;
    float* dconic;
    float* dopac;
    float* drgb;
};

// Thread-local error text (gs_last_error).
void set_error(const char* fmt, ...);
// A CUDA error from the last launch or runtime call, mapped to a status.
gs_status cuda_status(cudaError_t e, const char* what);
// Device address of the current device's error word.
unsigned* error_word();
// Count `k` kernel launches (gs_launch_count).
void count_launches(int k = 1);

cudaError_t launch_project(int n, const float* means, const float* scales, const float* quats, const float* sh,
                           int sh_degree, const CamDev& cam, float* mean2d, float* conic, float* depth,
                           int* radius, float* rgb, uint32_t* tiles_touched, cudaStream_t s);

size_t bin_sort_workspace_bytes(int n, int64_t capacity, int num_tiles);
gs_status bin_sort_run(int n, const float* mean2d, const int* radius, const float* depth, int W, int H,
                       int64_t capacity, void* ws, size_t ws_bytes, uint64_t* keys_sorted, uint32_t* ids_sorted,
                       uint32_t* tile_ranges, int64_t* n_instances, cudaStream_t s);

cudaError_t launch_blend_fp32_fwd(const BlendArgs& a, cudaStream_t s);
cudaError_t launch_blend_fp32_bwd(const BlendArgs& a, const GradArgs& g, cudaStream_t s);
// variant: 1..4 (gs_variant TC values); dump = gs_tile_power mode
cudaError_t launch_blend_tc(const BlendArgs& a, int variant, int chunk, int stages, bool dump, int grid,
                            cudaStream_t s);
bool tc_config_supported(int variant, int chunk, int stages);

}  // namespace gs
