// Host-side declarations shared by the translation units of the library.
#pragma once

#include <cuda.h>

#include <mutex>

#include "common.cuh"

namespace gs {

// Launch shape of a persistent kernel: blocks resident per SM and SM count.
// `make` computes it once per process, under the lock, because host threads
// may launch at the same time; a failed computation is retried by the next
// call.  `make` sets per_sm >= 1.
struct LaunchShape {
    int per_sm = 0, sms = 0;
};
template <typename F>
cudaError_t cached_shape(std::mutex& mu, LaunchShape& cache, LaunchShape& out, F make) {
    std::lock_guard<std::mutex> lock(mu);
    if (cache.per_sm == 0) {
        LaunchShape s;
        const cudaError_t e = make(s);
        if (e != cudaSuccess) return e;
        cache = s;
    }
    out = cache;
    return cudaSuccess;
}

constexpr int kMaxViews = 32;

// One rendered view (camera) of a blend call.  Its tiles are numbered
// [tile_begin, tile_begin + tiles_x * tiles_y) in the call's global tile
// space; its outputs start at pixel offset pix_off of the packed per-view
// arrays (image: 3 * pix_off floats in, CHW per view).
struct ViewDesc {
    int W, H, tiles_x, tile_begin;
    long long pix_off;
};

// View of a global tile id (views are ordered by tile_begin).
template <class A>
__host__ __device__ inline int view_of(const A& a, int tile) {
    int v = 0;
    while (v + 1 < a.num_views && a.views[v + 1].tile_begin <= tile) ++v;
    return v;
}

struct BlendArgs {
    int W, H, tiles_x, num_tiles;  // shape of view 0
    int num_views, total_tiles;    // all views: tiles [0, total_tiles)
    ViewDesc views[kMaxViews];
    int n_per_view;                // ids are v * n_per_view + g; opacity is indexed by g
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
    int shard_count, shard_index;  // queue item q takes position p = q * count + index of the tile order
    const uint32_t* order;         // the tile at position p: order[p] (nullptr: tile p)
    int order_tiles;               // the call's tile count; order entries are clamped below it
    unsigned long long* issued;    // if set, the TC forward adds 256 x the splats of every chunk it issues
    // gs_tile_power only
    const int* tiles;
    int max_len;
    float* dump;
    // Packed splat records (kRecFloats floats per item, gs_pack_splats) and
    // the TMA descriptor of that table (2D: kRecFloats x items, box 16 x 1):
    // when use_rec is set the tensor-core kernels stage each chunk's records
    // into shared memory with tile::gather4 copies instead of loading the
    // splat arrays thread by thread.
    int use_rec;
    alignas(64) CUtensorMap rec_map;
};

// Packed per-item splat record of gs_pack_splats, in floats:
// [0] mean x, [1] mean y, [2..4] conic A, B, C, [5] log2 opacity (-inf if 0),
// [6] min(log2 opacity, log2 0.99), [7] 1 / opacity (0 if 0), [8..10] rgb,
// [11] the Gaussian index g of item v * n_per_view + g (as bits), [12..15] 0.
constexpr int kRecFloats = 16;
constexpr int kRecBytes = 4 * kRecFloats;
cudaError_t launch_pack_splats(int n_items, int n_per_view, const float2* mean2d, const float* conic,
                               const float* opac, const float* rgb, float* rec, cudaStream_t s);
// Encode the TMA descriptor of a record table of n_items rows (16-byte aligned).
cudaError_t encode_rec_map(CUtensorMap* map, const void* rec, int n_items);

// The tile at position p of the call's tile order.
// A bad order entry is clamped, so a corrupt order gives a wrong image, never
// an access outside the tile ranges.
__host__ __device__ inline int tile_at(const BlendArgs& a, int p) {
    if (!a.order) return p;
    const uint32_t t = a.order[p];
    return t < (uint32_t)a.order_tiles ? (int)t : a.order_tiles - 1;
}

// Number of the call's tiles in its shard.
inline int shard_items(const BlendArgs& a) {
    return a.total_tiles > a.shard_index ? (a.total_tiles - a.shard_index + a.shard_count - 1) / a.shard_count : 0;
}

struct GradArgs {
    const float* T_final;
    const int* n_contrib;
    const float* dL_dimage;
    float2* dmean2d;
    float* dconic;
    float* dopac;
    float* drgb;
};

// Thread-local error text (gs_last_error); clear_error empties it at the
// start of a call.
void set_error(const char* fmt, ...);
void clear_error();
// View table of n_views images (HOST width/height arrays) and their total
// tile count; false if a size is out of range (each side 1..2^20) or the
// views hold 2^31 tiles or more.
bool fill_views(int32_t n_views, const int32_t* widths, const int32_t* heights, ViewDesc* views, int* total_tiles);
// A CUDA error from the last launch or runtime call, mapped to a status.
gs_status cuda_status(cudaError_t e, const char* what);
// Device address of the current device's error word.
unsigned* error_word();
// Count `k` kernel launches (gs_launch_count).
void count_launches(int k = 1);
// gs_set_kernel_events: store the pair, and record the start (end = false) or end
// event of `kernel` on `s` as an external record when set.
void set_kernel_events(int kernel, void* start, void* end);
cudaError_t record_kernel_event(int kernel, bool end, cudaStream_t s);

struct CamViews {
    int num_views;
    CamDev cams[kMaxViews];
};

// outputs are view-major: view v, Gaussian g at index v * n + g
cudaError_t launch_project(int n, const float* means, const float* scales, const float* quats, const float* sh,
                           int sh_degree, const CamViews& cams, float* mean2d, float* conic, float* depth,
                           int* radius, float* rgb, uint32_t* tiles_touched, cudaStream_t s);
// tiles by decreasing list length (a permutation of 0..ntiles-1)
cudaError_t launch_tile_order(int ntiles, const uint32_t* ranges, uint32_t* order, cudaStream_t s);
// projection + per-tile lists in one cooperative launch (one view, small scenes)
cudaError_t launch_project_bin_small(int n, const float* means, const float* scales, const float* quats,
                                     const float* sh, int sh_degree, const CamViews& cams, const float* power_min,
                                     int max_per_tile, float* mean2d, float* conic, float* depth, int* radius,
                                     float* rgb, uint32_t* touched, uint32_t* ids, uint32_t* ranges, cudaStream_t s);
// the same, then each tile blended (fp16-split tensor-core exponents) by the block that ordered its list
cudaError_t launch_render_small(int n, const float* means, const float* scales, const float* quats, const float* sh,
                                int sh_degree, const CamViews& cams, const float* power_min, int max_per_tile,
                                float* mean2d, float* conic, float* depth, int* radius, float* rgb, uint32_t* touched,
                                uint32_t* ids, uint32_t* ranges, const float* opacity, const float bg[3],
                                float* image, float* T_final, int* n_contrib, cudaStream_t s);
// gradient of launch_project summed over the views (inputs view-major, outputs per Gaussian)
cudaError_t launch_project_bwd(int n, const float* means, const float* scales, const float* quats, const float* sh,
                               int sh_degree, const CamViews& cams, const int* radius, const float* dmean2d,
                               const float* dconic, const float* drgb, float* dmeans, float* dscales, float* dquats,
                               float* dsh, cudaStream_t s);

// Bin/sort geometry: items are (view, Gaussian) pairs, item = v * n_per_view + g.
struct SortViews {
    int num_views, total_tiles, n_per_view;
    ViewDesc views[kMaxViews];
    // opacity-aware tile lists when both are set: conic per item, power_min per Gaussian
    const float* conic;
    const float* power_min;
    // supertiles (4 x 4 tiles) of each view, numbered [st_begin[v], st_begin[v] +
    // st_x[v] * ceil(tiles_y / 4)) in one space of total_st (filled by bin_sort_run)
    int st_begin[kMaxViews], st_x[kMaxViews];
    int total_st;
};

size_t bin_sort_workspace_bytes(int n_items, int64_t capacity, int num_tiles);
cudaError_t launch_alpha_power_min(int n, const float* opacity, float* out, cudaStream_t s);
// n_instances_host != nullptr: synchronise once, read the count, exact grids.
// otherwise (graph mode): no synchronisation; grids sized by capacity; the count
// goes to n_instances_dev and overflow sets kErrCapacity in the error word.
gs_status bin_sort_run(const SortViews& sv, const float* mean2d, const int* radius, const float* depth,
                       int64_t capacity, void* ws, size_t ws_bytes, uint64_t* keys_sorted, uint32_t* ids_sorted,
                       uint32_t* tile_ranges, int64_t* n_instances_host, int64_t* n_instances_dev, cudaStream_t s);

cudaError_t launch_blend_fp32_fwd(const BlendArgs& a, cudaStream_t s);
cudaError_t launch_blend_fp32_bwd(const BlendArgs& a, const GradArgs& g, cudaStream_t s);
// variant: 1..4 (gs_variant TC values); dump = gs_tile_power mode
cudaError_t launch_blend_tc(const BlendArgs& a, int variant, int chunk, int stages, bool dump, int grid,
                            cudaStream_t s);
bool tc_config_supported(int variant, int chunk, int stages);
// Gradient of the tensor-core blend of `variant` (exponents recomputed with the
// forward pass's tensor-core arithmetic).
cudaError_t launch_blend_tc_bwd(const BlendArgs& a, const GradArgs& g, int variant, int stages, cudaStream_t s);
bool tc_bwd_stages_supported(int stages);
// A zeroed tile-queue counter for one persistent launch on stream s.
unsigned* tile_queue_slot(cudaStream_t s, cudaError_t* err);

}  // namespace gs
