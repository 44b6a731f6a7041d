// C ABI entry points: argument checks, status reporting, the per-device error
// word, and dispatch to the kernels of the other translation units.
#include <atomic>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace gs {

namespace {
thread_local char g_last_error[512] = "";
std::atomic<int64_t> g_launches{0};
__device__ unsigned g_error_word;

// bounded-wait self test: wait on an mbarrier nobody arrives on
__global__ void k_selftest_wait(uint64_t limit_ns, unsigned* err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!mbar_wait_bounded(smem_u32(&bar), 0, limit_ns, nullptr)) atomicOr(err, kErrTimeout);
    }
}
}  // namespace

void clear_error() { g_last_error[0] = 0; }

static bool size_ok(int32_t W, int32_t H) { return W > 0 && H > 0 && W <= (1 << 20) && H <= (1 << 20); }

bool fill_views(int32_t n_views, const int32_t* widths, const int32_t* heights, ViewDesc* views, int* total_tiles) {
    long long tiles = 0, pix = 0;
    for (int v = 0; v < n_views; ++v) {
        if (!size_ok(widths[v], heights[v])) return false;
        views[v] = ViewDesc{widths[v], heights[v], tiles_x(widths[v]), (int)tiles, pix};
        tiles += (long long)tiles_x(widths[v]) * tiles_y(heights[v]);
        pix += (long long)widths[v] * heights[v];
        if (tiles >= (1ll << 31)) return false;
    }
    *total_tiles = (int)tiles;
    return true;
}

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

gs_status cuda_status(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return GS_OK;
    set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    if (e == cudaErrorNoKernelImageForDevice || e == cudaErrorInvalidDeviceFunction) return GS_ERR_UNSUPPORTED;
    return GS_ERR_CUDA;
}

void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// gs_set_kernel_events: one (start, end) pair per timed kernel
std::atomic<void*> g_kernel_events[2][2] = {};
void set_kernel_events(int kernel, void* start, void* end) {
    g_kernel_events[kernel][0].store(start, std::memory_order_relaxed);
    g_kernel_events[kernel][1].store(end, std::memory_order_relaxed);
}
cudaError_t record_kernel_event(int kernel, bool end, cudaStream_t s) {
    void* ev = g_kernel_events[kernel][end ? 1 : 0].load(std::memory_order_relaxed);
    if (ev == nullptr) return cudaSuccess;
    // inside a stream capture the record becomes an external event node of the
    // graph (recorded at every replay); outside one it is a plain record
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    return cs == cudaStreamCaptureStatusActive
               ? cudaEventRecordWithFlags(static_cast<cudaEvent_t>(ev), s, cudaEventRecordExternal)
               : cudaEventRecord(static_cast<cudaEvent_t>(ev), s);
}

unsigned* error_word() {
    static std::atomic<unsigned*> addr[64] = {};  // per device; threads may look it up at once
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    unsigned* a = addr[dev].load(std::memory_order_acquire);
    if (a == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_error_word) != cudaSuccess) return nullptr;
        a = static_cast<unsigned*>(p);
        addr[dev].store(a, std::memory_order_release);
    }
    return a;
}

}  // namespace gs

using namespace gs;

// The options struct is part of the ABI (the Python binding mirrors it).
static_assert(sizeof(gs_blend_opts) == 80, "gs_blend_opts layout");
static_assert(offsetof(gs_blend_opts, splat_records) == 64, "gs_blend_opts layout");

namespace {

gs_status check_views(const char* who, int32_t n_views, const int32_t* widths, const int32_t* heights) {
    if (n_views < 1 || n_views > kMaxViews || !widths || !heights) {
        set_error("%s: n_views must be 1..%d with width/height arrays", who, kMaxViews);
        return GS_ERR_INVALID_ARG;
    }
    return GS_OK;
}


gs_status check_blend_common(const uint32_t* ranges, const uint32_t* ids, const float* mean2d, const float* conic,
                             const float* opacity) {
    if (!ranges || !ids || !mean2d || !conic || !opacity) {
        set_error("null input pointer");
        return GS_ERR_INVALID_ARG;
    }
    return GS_OK;
}

// Blend arguments for n_views views of n_per_view Gaussians each (false: bad sizes).
bool make_args(BlendArgs& a, int32_t n_views, const int32_t* widths, const int32_t* heights, int32_t n_per_view,
               const uint32_t* ranges, const uint32_t* ids, const float* mean2d, const float* conic,
               const float* opacity, const float* rgb, const gs_blend_opts* o) {
    a = BlendArgs{};
    if (!fill_views(n_views, widths, heights, a.views, &a.total_tiles)) return false;
    a.num_views = n_views;
    a.n_per_view = n_per_view;
    a.W = widths[0];
    a.H = heights[0];
    a.tiles_x = tiles_x(a.W);
    a.num_tiles = tiles_x(a.W) * tiles_y(a.H);
    a.ranges = ranges;
    a.ids = ids;
    a.mean2d = reinterpret_cast<const float2*>(mean2d);
    a.conic = conic;
    a.opac = opacity;
    a.rgb = rgb;
    for (int c = 0; c < 3; ++c) a.bg[c] = o ? o->bg[c] : 0.0f;
    a.timeout_ns = (o && o->timeout_ns > 0) ? (uint64_t)o->timeout_ns : 1000000000ull;
    a.ref_origin = o ? o->ref_origin : 0;
    a.shard_count = (o && o->shard_count > 1) ? o->shard_count : 1;
    a.shard_index = o ? o->shard_index : 0;
    if (a.shard_index < 0 || a.shard_index >= a.shard_count) return false;
    a.order = o ? o->tile_order : nullptr;
    a.order_tiles = a.total_tiles;
    a.issued = o ? reinterpret_cast<unsigned long long*>(o->issued_pairs) : nullptr;  // same width, 64 bits
    a.err = error_word();
    a.use_rec = 0;
    if (o && o->splat_records) {
        if (o->splat_record_count < 1 || o->splat_record_count >= (int64_t(1) << 31) ||
            (reinterpret_cast<uintptr_t>(o->splat_records) & 15u) != 0)
            return false;
        if (encode_rec_map(&a.rec_map, o->splat_records, (int)o->splat_record_count) != cudaSuccess) return false;
        a.use_rec = 1;
    }
    return true;
}

bool is_tc(int v) { return v >= GS_BLEND_TC_FP16 && v <= GS_BLEND_TC_FP8_SPLIT; }
// the persistent kernel: the TC variants, and the same kernel with the exponent on CUDA cores
bool is_persistent(int v) { return is_tc(v) || v == GS_BLEND_PERSISTENT_FP32; }

}  // namespace

extern "C" {

int32_t gs_version(void) { return 100; }

int64_t gs_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

gs_status gs_set_kernel_events(int32_t kernel, void* start, void* end) {
    g_last_error[0] = 0;
    if (kernel != GS_KERNEL_DUPLICATE || (start == nullptr) != (end == nullptr)) {
        set_error("gs_set_kernel_events: kernel must be GS_KERNEL_DUPLICATE and the events both set or both NULL");
        return GS_ERR_INVALID_ARG;
    }
    gs::set_kernel_events(kernel, start, end);
    return GS_OK;
}

const char* gs_status_string(gs_status s) {
    switch (s) {
        case GS_OK: return "ok";
        case GS_ERR_INVALID_ARG: return "invalid argument";
        case GS_ERR_CUDA: return "CUDA error";
        case GS_ERR_CAPACITY: return "instance capacity exceeded";
        case GS_ERR_TIMEOUT: return "device wait timed out";
        case GS_ERR_UNSUPPORTED: return "unsupported device or option";
        case GS_ERR_WORKSPACE: return "workspace too small";
    }
    return "unknown status";
}

const char* gs_last_error(void) { return g_last_error; }

// Host cameras -> the kernels' camera table (n_views <= kMaxViews).
static gs_status make_cam_views(const char* who, const gs_camera* cams, int32_t n_views, CamViews& cv) {
    cv = CamViews{};
    cv.num_views = n_views;
    for (int v = 0; v < n_views; ++v) {
        const gs_camera* cam = cams + v;
        if (!size_ok(cam->width, cam->height)) {
            set_error("%s: image size %d x %d out of range", who, cam->width, cam->height);
            return GS_ERR_INVALID_ARG;
        }
        CamDev& c = cv.cams[v];
        c.W = cam->width;
        c.H = cam->height;
        c.fx = cam->fx;
        c.fy = cam->fy;
        c.cx = cam->cx;
        c.cy = cam->cy;
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) c.R[3 * i + j] = cam->world_to_cam[4 * i + j];
            c.t[i] = cam->world_to_cam[4 * i + 3];
        }
        c.znear = cam->znear;
        c.lowpass = cam->lowpass;
    }
    return GS_OK;
}

static gs_status check_project_args(const char* who, int32_t n, int32_t sh_degree, const gs_camera* cams,
                                    int32_t n_views) {
    if (n < 0 || sh_degree < 0 || sh_degree > 3 || !cams || n_views < 1 || n_views > kMaxViews) {
        set_error("%s: bad n (%d), sh_degree (%d), cameras or n_views (%d)", who, n, sh_degree, n_views);
        return GS_ERR_INVALID_ARG;
    }
    if ((long long)n * n_views >= (1ll << 32)) {
        set_error("%s: n * n_views must be below 2^32", who);
        return GS_ERR_INVALID_ARG;
    }
    return GS_OK;
}

gs_status gs_project_views(int32_t n, const float* means, const float* scales, const float* quats, const float* sh,
                           int32_t sh_degree, const gs_camera* cams, int32_t n_views, float* mean2d, float* conic,
                           float* depth, int32_t* radius, float* rgb, uint32_t* tiles_touched, gs_stream stream) {
    g_last_error[0] = 0;
    gs_status st = check_project_args("gs_project", n, sh_degree, cams, n_views);
    if (st != GS_OK) return st;
    CamViews cv;
    if ((st = make_cam_views("gs_project", cams, n_views, cv)) != GS_OK) return st;
    if (n == 0) return GS_OK;
    if (!means || !scales || !quats || !sh || !mean2d || !conic || !depth || !radius || !rgb || !tiles_touched) {
        set_error("gs_project: null pointer");
        return GS_ERR_INVALID_ARG;
    }
    return cuda_status(launch_project(n, means, scales, quats, sh, sh_degree, cv, mean2d, conic, depth, radius, rgb,
                                      tiles_touched, static_cast<cudaStream_t>(stream)),
                       "gs_project");
}

gs_status gs_project_backward(int32_t n, const float* means, const float* scales, const float* quats,
                              const float* sh, int32_t sh_degree, const gs_camera* cams, int32_t n_views,
                              const int32_t* radius, const float* dmean2d, const float* dconic, const float* drgb,
                              float* dmeans, float* dscales, float* dquats, float* dsh, gs_stream stream) {
    g_last_error[0] = 0;
    gs_status st = check_project_args("gs_project_backward", n, sh_degree, cams, n_views);
    if (st != GS_OK) return st;
    CamViews cv;
    if ((st = make_cam_views("gs_project_backward", cams, n_views, cv)) != GS_OK) return st;
    if (n == 0) return GS_OK;
    if (!means || !scales || !quats || !sh || !radius || !dmean2d || !dconic || !drgb || !dmeans || !dscales ||
        !dquats || !dsh) {
        set_error("gs_project_backward: null pointer");
        return GS_ERR_INVALID_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(dmean2d) & 7) != 0) {
        set_error("gs_project_backward: dmean2d must be 8-byte aligned");
        return GS_ERR_INVALID_ARG;
    }
    return cuda_status(launch_project_bwd(n, means, scales, quats, sh, sh_degree, cv, radius, dmean2d, dconic, drgb,
                                          dmeans, dscales, dquats, dsh, static_cast<cudaStream_t>(stream)),
                       "gs_project_backward");
}

gs_status gs_project_bin_small(int32_t n, const float* means, const float* scales, const float* quats,
                               const float* sh, int32_t sh_degree, const gs_camera* cam, const float* power_min,
                               int32_t max_per_tile, float* mean2d, float* conic, float* depth, int32_t* radius,
                               float* rgb, uint32_t* tiles_touched, uint32_t* ids, uint32_t* tile_ranges,
                               gs_stream stream) {
    g_last_error[0] = 0;
    gs_status st = check_project_args("gs_project_bin_small", n, sh_degree, cam, 1);
    if (st != GS_OK) return st;
    CamViews cv;
    if ((st = make_cam_views("gs_project_bin_small", cam, 1, cv)) != GS_OK) return st;
    const long long ntiles = (long long)tiles_x(cam->width) * tiles_y(cam->height);
    if (max_per_tile < 1 || max_per_tile > GS_SMALL_MAX_PER_TILE || ntiles * max_per_tile >= (1ll << 32) || n < 1) {
        set_error("gs_project_bin_small: need n >= 1, 1 <= max_per_tile <= %d and tiles * max_per_tile < 2^32",
                  GS_SMALL_MAX_PER_TILE);
        return GS_ERR_INVALID_ARG;
    }
    if (!means || !scales || !quats || !sh || !mean2d || !conic || !depth || !radius || !rgb || !tiles_touched ||
        !ids || !tile_ranges) {
        set_error("gs_project_bin_small: null pointer");
        return GS_ERR_INVALID_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(mean2d) & 7) != 0) {
        set_error("gs_project_bin_small: mean2d must be 8-byte aligned");
        return GS_ERR_INVALID_ARG;
    }
    return cuda_status(launch_project_bin_small(n, means, scales, quats, sh, sh_degree, cv, power_min, max_per_tile,
                                                mean2d, conic, depth, radius, rgb, tiles_touched, ids, tile_ranges,
                                                static_cast<cudaStream_t>(stream)),
                       "gs_project_bin_small");
}

gs_status gs_render_small(int32_t n, const float* means, const float* scales, const float* quats, const float* sh,
                          int32_t sh_degree, const gs_camera* cam, const float* power_min, int32_t max_per_tile,
                          const float* opacity, const float* bg, float* mean2d, float* conic, float* depth,
                          int32_t* radius, float* rgb, uint32_t* tiles_touched, uint32_t* ids, uint32_t* tile_ranges,
                          float* image, float* T_final, int32_t* n_contrib, gs_stream stream) {
    g_last_error[0] = 0;
    gs_status st = check_project_args("gs_render_small", n, sh_degree, cam, 1);
    if (st != GS_OK) return st;
    CamViews cv;
    if ((st = make_cam_views("gs_render_small", cam, 1, cv)) != GS_OK) return st;
    const long long ntiles = (long long)tiles_x(cam->width) * tiles_y(cam->height);
    if (max_per_tile < 1 || max_per_tile > GS_SMALL_MAX_PER_TILE || ntiles * max_per_tile >= (1ll << 32) || n < 1) {
        set_error("gs_render_small: need n >= 1, 1 <= max_per_tile <= %d and tiles * max_per_tile < 2^32",
                  GS_SMALL_MAX_PER_TILE);
        return GS_ERR_INVALID_ARG;
    }
    if (!means || !scales || !quats || !sh || !opacity || !bg || !mean2d || !conic || !depth || !radius || !rgb ||
        !tiles_touched || !ids || !tile_ranges || !image || !T_final || !n_contrib) {
        set_error("gs_render_small: null pointer");
        return GS_ERR_INVALID_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(mean2d) & 7) != 0) {
        set_error("gs_render_small: mean2d must be 8-byte aligned");
        return GS_ERR_INVALID_ARG;
    }
    const float bgv[3] = {bg[0], bg[1], bg[2]};
    return cuda_status(launch_render_small(n, means, scales, quats, sh, sh_degree, cv, power_min, max_per_tile, mean2d,
                                           conic, depth, radius, rgb, tiles_touched, ids, tile_ranges, opacity, bgv,
                                           image, T_final, n_contrib, static_cast<cudaStream_t>(stream)),
                       "gs_render_small");
}

gs_status gs_project(int32_t n, const float* means, const float* scales, const float* quats, const float* sh,
                     int32_t sh_degree, const gs_camera* cam, float* mean2d, float* conic, float* depth,
                     int32_t* radius, float* rgb, uint32_t* tiles_touched, gs_stream stream) {
    return gs_project_views(n, means, scales, quats, sh, sh_degree, cam, 1, mean2d, conic, depth, radius, rgb,
                            tiles_touched, stream);
}

gs_status gs_bin_sort_workspace_size(int32_t n, int64_t capacity, int32_t width, int32_t height, size_t* bytes) {
    g_last_error[0] = 0;
    ViewDesc view;
    int total_tiles = 0;
    if (n < 0 || capacity < 0 || capacity >= (int64_t(1) << 32) || !bytes ||
        !fill_views(1, &width, &height, &view, &total_tiles)) {
        set_error("gs_bin_sort_workspace_size: bad arguments");
        return GS_ERR_INVALID_ARG;
    }
    *bytes = bin_sort_workspace_bytes(n, capacity, total_tiles);
    return GS_OK;
}

gs_status gs_tile_order(int32_t n_views, const int32_t* widths, const int32_t* heights, const uint32_t* tile_ranges,
                        uint32_t* tile_order, gs_stream stream) {
    g_last_error[0] = 0;
    gs_status st = check_views("gs_tile_order", n_views, widths, heights);
    if (st != GS_OK) return st;
    ViewDesc views[kMaxViews];
    int total = 0;
    if (!fill_views(n_views, widths, heights, views, &total)) {
        set_error("gs_tile_order: bad views");
        return GS_ERR_INVALID_ARG;
    }
    if (!tile_ranges || !tile_order) {
        set_error("gs_tile_order: null pointer");
        return GS_ERR_INVALID_ARG;
    }
    return cuda_status(launch_tile_order(total, tile_ranges, tile_order, static_cast<cudaStream_t>(stream)),
                       "gs_tile_order");
}

gs_status gs_pack_splats(int32_t n_items, int32_t n_per_view, const float* mean2d, const float* conic,
                         const float* opacity, const float* rgb, float* records, gs_stream stream) {
    g_last_error[0] = 0;
    if (n_items < 0 || n_per_view < 0 || (n_items > 0 && (n_per_view == 0 || n_items % n_per_view != 0)) ||
        (n_items > 0 && (!mean2d || !conic || !opacity || !records)) ||
        (reinterpret_cast<uintptr_t>(records) & 15u) != 0 || (reinterpret_cast<uintptr_t>(mean2d) & 7u) != 0) {
        set_error("gs_pack_splats: bad arguments (n_items a multiple of n_per_view > 0, 16-byte aligned records, "
                  "8-byte aligned mean2d)");
        return GS_ERR_INVALID_ARG;
    }
    return cuda_status(launch_pack_splats(n_items, n_per_view, reinterpret_cast<const float2*>(mean2d), conic, opacity,
                                          rgb, records, static_cast<cudaStream_t>(stream)),
                       "gs_pack_splats");
}

gs_status gs_alpha_power_min(int32_t n, const float* opacity, float* power_min, gs_stream stream) {
    g_last_error[0] = 0;
    if (n < 0 || (n > 0 && (!opacity || !power_min))) {
        set_error("gs_alpha_power_min: bad arguments");
        return GS_ERR_INVALID_ARG;
    }
    return cuda_status(launch_alpha_power_min(n, opacity, power_min, static_cast<cudaStream_t>(stream)),
                       "gs_alpha_power_min");
}

gs_status gs_bin_sort_views(int32_t n_views, int32_t n_per_view, const float* mean2d, const int32_t* radius,
                            const float* depth, const float* conic, const float* power_min, const int32_t* widths,
                            const int32_t* heights, int64_t capacity,
                            void* workspace, size_t workspace_bytes, uint64_t* keys_sorted, uint32_t* ids_sorted,
                            uint32_t* tile_ranges, int64_t* n_instances, int64_t* n_instances_dev, gs_stream stream) {
    g_last_error[0] = 0;
    gs_status st = check_views("gs_bin_sort", n_views, widths, heights);
    if (st != GS_OK) return st;
    if (n_per_view < 0 || capacity < 0 || capacity >= (int64_t(1) << 32) || !tile_ranges ||
        (!n_instances && !n_instances_dev) || (long long)n_per_view * n_views >= (1ll << 31)) {
        set_error("gs_bin_sort: bad arguments");
        return GS_ERR_INVALID_ARG;
    }
    SortViews sv{};
    sv.num_views = n_views;
    sv.n_per_view = n_per_view;
    if ((conic == nullptr) != (power_min == nullptr)) {
        set_error("gs_bin_sort: conic and power_min go together");
        return GS_ERR_INVALID_ARG;
    }
    sv.conic = conic;
    sv.power_min = power_min;
    if (!fill_views(n_views, widths, heights, sv.views, &sv.total_tiles)) {
        set_error("gs_bin_sort: image size out of range");
        return GS_ERR_INVALID_ARG;
    }
    const int items = n_views * n_per_view;
    if (items > 0 && (!mean2d || !radius || !depth || !workspace)) {
        set_error("gs_bin_sort: null pointer");
        return GS_ERR_INVALID_ARG;
    }
    if (capacity > 0 && !ids_sorted) {
        set_error("gs_bin_sort: null output pointer");
        return GS_ERR_INVALID_ARG;
    }
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) {
        set_error("gs_bin_sort: workspace must be 256-byte aligned");
        return GS_ERR_INVALID_ARG;
    }
    const size_t need = bin_sort_workspace_bytes(items, capacity, sv.total_tiles);
    if (workspace_bytes < need) {
        set_error("gs_bin_sort: workspace %zu bytes < %zu needed", workspace_bytes, need);
        return GS_ERR_WORKSPACE;
    }
    return bin_sort_run(sv, mean2d, radius, depth, capacity, workspace, workspace_bytes, keys_sorted, ids_sorted,
                        tile_ranges, n_instances, n_instances ? nullptr : n_instances_dev, stream);
}

gs_status gs_bin_sort(int32_t n, const float* mean2d, const int32_t* radius, const float* depth, int32_t width,
                      int32_t height, int64_t capacity, void* workspace, size_t workspace_bytes,
                      uint64_t* keys_sorted, uint32_t* ids_sorted, uint32_t* tile_ranges, int64_t* n_instances,
                      gs_stream stream) {
    if (!n_instances) {
        set_error("gs_bin_sort: n_instances must be a host pointer");
        return GS_ERR_INVALID_ARG;
    }
    return gs_bin_sort_views(1, n, mean2d, radius, depth, nullptr, nullptr, &width, &height, capacity, workspace,
                             workspace_bytes,
                             keys_sorted, ids_sorted, tile_ranges, n_instances, nullptr, stream);
}

gs_status gs_blend_forward_views(int32_t n_views, const int32_t* widths, const int32_t* heights,
                                 int32_t n_per_view, const uint32_t* tile_ranges, const uint32_t* ids_sorted,
                                 const float* mean2d, const float* conic, const float* opacity, const float* rgb,
                                 const gs_blend_opts* opts, float* image, float* T_final, int32_t* n_contrib,
                                 gs_stream stream) {
    g_last_error[0] = 0;
    gs_status st = check_views("gs_blend_forward", n_views, widths, heights);
    if (st != GS_OK) return st;
    st = check_blend_common(tile_ranges, ids_sorted, mean2d, conic, opacity);
    if (st != GS_OK) return st;
    if (!rgb || !image || !T_final || !n_contrib || n_per_view < 0) {
        set_error("gs_blend_forward: null pointer or negative n_per_view");
        return GS_ERR_INVALID_ARG;
    }
    gs_blend_opts def{};
    const gs_blend_opts* o = opts ? opts : &def;
    BlendArgs a;
    if (!make_args(a, n_views, widths, heights, n_per_view, tile_ranges, ids_sorted, mean2d, conic, opacity, rgb, o)) {
        set_error("gs_blend_forward: image size, shard or splat records out of range");
        return GS_ERR_INVALID_ARG;
    }
    a.image = image;
    a.T_final = T_final;
    a.n_contrib = n_contrib;
    if (!a.err) return cuda_status(cudaGetLastError(), "gs_blend_forward: error word");
    if (o->variant == GS_BLEND_FP32) return cuda_status(launch_blend_fp32_fwd(a, stream), "gs_blend_forward fp32");
    if (!is_persistent(o->variant)) {
        set_error("gs_blend_forward: unknown variant %d", o->variant);
        return GS_ERR_INVALID_ARG;
    }
    int chunk = o->chunk ? o->chunk : 32, stages = o->stages ? o->stages : 2;
    if (!tc_config_supported(o->variant, chunk, stages)) {
        set_error("gs_blend_forward: chunk %d / stages %d not built", chunk, stages);
        return GS_ERR_UNSUPPORTED;
    }
    return cuda_status(launch_blend_tc(a, o->variant, chunk, stages, false, shard_items(a), stream),
                       "gs_blend_forward tc");
}

gs_status gs_blend_forward(int32_t width, int32_t height, const uint32_t* tile_ranges, const uint32_t* ids_sorted,
                           const float* mean2d, const float* conic, const float* opacity, const float* rgb,
                           const gs_blend_opts* opts, float* image, float* T_final, int32_t* n_contrib,
                           gs_stream stream) {
    return gs_blend_forward_views(1, &width, &height, 0, tile_ranges, ids_sorted, mean2d, conic, opacity, rgb, opts,
                                  image, T_final, n_contrib, stream);
}

gs_status gs_blend_backward_views(int32_t n_views, const int32_t* widths, const int32_t* heights,
                                  int32_t n_per_view, const uint32_t* tile_ranges, const uint32_t* ids_sorted,
                                  const float* mean2d, const float* conic, const float* opacity, const float* rgb,
                                  const gs_blend_opts* opts, const float* T_final, const int32_t* n_contrib,
                                  const float* dL_dimage, float* dmean2d, float* dconic, float* dopacity,
                                  float* drgb, gs_stream stream) {
    g_last_error[0] = 0;
    gs_status st = check_views("gs_blend_backward", n_views, widths, heights);
    if (st != GS_OK) return st;
    st = check_blend_common(tile_ranges, ids_sorted, mean2d, conic, opacity);
    if (st != GS_OK) return st;
    if (!rgb || !T_final || !n_contrib || !dL_dimage || !dmean2d || !dconic || !dopacity || !drgb ||
        n_per_view < 0) {
        set_error("gs_blend_backward: null pointer or negative n_per_view");
        return GS_ERR_INVALID_ARG;
    }
    gs_blend_opts def{};
    const gs_blend_opts* o = opts ? opts : &def;
    if (o->variant == GS_BLEND_PERSISTENT_FP32) {
        set_error("gs_blend_backward: variant %d is forward only", o->variant);
        return GS_ERR_UNSUPPORTED;
    }
    if (o->variant != GS_BLEND_FP32 && !is_tc(o->variant)) {
        set_error("gs_blend_backward: unknown variant %d", o->variant);
        return GS_ERR_INVALID_ARG;
    }
    BlendArgs a;
    if (!make_args(a, n_views, widths, heights, n_per_view, tile_ranges, ids_sorted, mean2d, conic, opacity, rgb, o)) {
        set_error("gs_blend_backward: image size, shard or splat records out of range");
        return GS_ERR_INVALID_ARG;
    }
    GradArgs g{T_final, n_contrib, dL_dimage, reinterpret_cast<float2*>(dmean2d), dconic, dopacity, drgb};
    if (is_tc(o->variant)) {
        if (!tc_bwd_stages_supported(o->bwd_stages)) {
            set_error("gs_blend_backward: bwd_stages %d not built (0, 2, 3, 4, 6)", o->bwd_stages);
            return GS_ERR_UNSUPPORTED;
        }
        return cuda_status(launch_blend_tc_bwd(a, g, o->variant, o->bwd_stages, stream), "gs_blend_backward");
    }
    return cuda_status(launch_blend_fp32_bwd(a, g, stream), "gs_blend_backward");
}

gs_status gs_blend_backward(int32_t width, int32_t height, const uint32_t* tile_ranges, const uint32_t* ids_sorted,
                            const float* mean2d, const float* conic, const float* opacity, const float* rgb,
                            const gs_blend_opts* opts, const float* T_final, const int32_t* n_contrib,
                            const float* dL_dimage, float* dmean2d, float* dconic, float* dopacity, float* drgb,
                            gs_stream stream) {
    return gs_blend_backward_views(1, &width, &height, 0, tile_ranges, ids_sorted, mean2d, conic, opacity, rgb, opts,
                                   T_final, n_contrib, dL_dimage, dmean2d, dconic, dopacity, drgb, stream);
}

gs_status gs_blend_autotune(int32_t n_views, const int32_t* widths, const int32_t* heights, int32_t n_per_view,
                            const uint32_t* tile_ranges, const uint32_t* ids_sorted, const float* mean2d,
                            const float* conic, const float* opacity, const float* rgb, gs_blend_opts* opts,
                            float* image, float* T_final, int32_t* n_contrib, int32_t reps, float* best_ms,
                            gs_stream stream) {
    g_last_error[0] = 0;
    if (!opts || !is_persistent(opts->variant) || reps < 1) {
        set_error("gs_blend_autotune: needs a TC (or the persistent FP32) variant and reps >= 1");
        return GS_ERR_INVALID_ARG;
    }
    static const int kShapes[][2] = {{32, 2}, {32, 4}, {16, 4}, {16, 6}};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gs_status st = cuda_status(cudaEventCreate(&e0), "gs_blend_autotune: event");
    if (st == GS_OK) st = cuda_status(cudaEventCreate(&e1), "gs_blend_autotune: event");
    float best = 1e30f;
    int best_i = -1;
    for (int i = 0; st == GS_OK && i < (int)(sizeof(kShapes) / sizeof(kShapes[0])); ++i) {
        gs_blend_opts o = *opts;
        o.chunk = kShapes[i][0];
        o.stages = kShapes[i][1];
        if (!tc_config_supported(o.variant, o.chunk, o.stages)) continue;
        st = gs_blend_forward_views(n_views, widths, heights, n_per_view, tile_ranges, ids_sorted, mean2d, conic,
                                    opacity, rgb, &o, image, T_final, n_contrib, stream);
        if (st != GS_OK) break;
        if ((st = cuda_status(cudaEventRecord(e0, stream), "gs_blend_autotune: record")) != GS_OK) break;
        for (int r = 0; st == GS_OK && r < reps; ++r)
            st = gs_blend_forward_views(n_views, widths, heights, n_per_view, tile_ranges, ids_sorted, mean2d, conic,
                                        opacity, rgb, &o, image, T_final, n_contrib, stream);
        if (st != GS_OK) break;
        if ((st = cuda_status(cudaEventRecord(e1, stream), "gs_blend_autotune: record")) != GS_OK) break;
        if ((st = cuda_status(cudaEventSynchronize(e1), "gs_blend_autotune: synchronize")) != GS_OK) break;
        float ms = 0.f;
        if ((st = cuda_status(cudaEventElapsedTime(&ms, e0, e1), "gs_blend_autotune: elapsed")) != GS_OK) break;
        ms /= (float)reps;
        if (ms < best) {
            best = ms;
            best_i = i;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st != GS_OK) return st;
    if (best_i < 0) {
        set_error("gs_blend_autotune: no pipeline shape built for variant %d", opts->variant);
        return GS_ERR_UNSUPPORTED;
    }
    opts->chunk = kShapes[best_i][0];
    opts->stages = kShapes[best_i][1];
    if (best_ms) *best_ms = best;
    return gs_sync_status(stream);
}

gs_status gs_blend_autotune_backward(int32_t n_views, const int32_t* widths, const int32_t* heights,
                                     int32_t n_per_view, const uint32_t* tile_ranges, const uint32_t* ids_sorted,
                                     const float* mean2d, const float* conic, const float* opacity, const float* rgb,
                                     gs_blend_opts* opts, const float* T_final, const int32_t* n_contrib,
                                     const float* dL_dimage, float* dmean2d, float* dconic, float* dopacity,
                                     float* drgb, int32_t reps, float* best_ms, gs_stream stream) {
    g_last_error[0] = 0;
    if (!opts || !is_tc(opts->variant) || reps < 1) {
        set_error("gs_blend_autotune_backward: needs a TC variant and reps >= 1");
        return GS_ERR_INVALID_ARG;
    }
    static const int kStages[] = {2, 3, 4, 6};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gs_status st = cuda_status(cudaEventCreate(&e0), "gs_blend_autotune_backward: event");
    if (st == GS_OK) st = cuda_status(cudaEventCreate(&e1), "gs_blend_autotune_backward: event");
    float best = 1e30f;
    int best_i = -1;
    for (int i = 0; st == GS_OK && i < 3; ++i) {
        gs_blend_opts o = *opts;
        o.bwd_stages = kStages[i];
        auto run = [&]() {
            return gs_blend_backward_views(n_views, widths, heights, n_per_view, tile_ranges, ids_sorted, mean2d,
                                           conic, opacity, rgb, &o, T_final, n_contrib, dL_dimage, dmean2d, dconic,
                                           dopacity, drgb, stream);
        };
        if ((st = run()) != GS_OK) break;
        if ((st = cuda_status(cudaEventRecord(e0, stream), "gs_blend_autotune_backward: record")) != GS_OK) break;
        for (int r = 0; st == GS_OK && r < reps; ++r) st = run();
        if (st != GS_OK) break;
        if ((st = cuda_status(cudaEventRecord(e1, stream), "gs_blend_autotune_backward: record")) != GS_OK) break;
        if ((st = cuda_status(cudaEventSynchronize(e1), "gs_blend_autotune_backward: synchronize")) != GS_OK) break;
        float ms = 0.f;
        if ((st = cuda_status(cudaEventElapsedTime(&ms, e0, e1), "gs_blend_autotune_backward: elapsed")) != GS_OK)
            break;
        ms /= (float)reps;
        if (ms < best) {
            best = ms;
            best_i = i;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st != GS_OK) return st;
    opts->bwd_stages = kStages[best_i];
    if (best_ms) *best_ms = best;
    return gs_sync_status(stream);
}

gs_status gs_tile_power(int32_t width, int32_t height, const uint32_t* tile_ranges, const uint32_t* ids_sorted,
                        const float* mean2d, const float* conic, const float* opacity, const gs_blend_opts* opts,
                        const int32_t* tiles, int32_t n_tiles, int32_t max_len, float* out, gs_stream stream) {
    g_last_error[0] = 0;
    gs_status st = check_blend_common(tile_ranges, ids_sorted, mean2d, conic, opacity);
    if (st != GS_OK) return st;
    if (!opts || !is_tc(opts->variant) || n_tiles < 0 || max_len < 0 || (n_tiles > 0 && (!tiles || !out))) {
        set_error("gs_tile_power: bad arguments");
        return GS_ERR_INVALID_ARG;
    }
    if (n_tiles == 0 || max_len == 0) return GS_OK;
    int chunk = opts->chunk ? opts->chunk : 32, stages = opts->stages ? opts->stages : 2;
    if (!tc_config_supported(opts->variant, chunk, stages)) {
        set_error("gs_tile_power: chunk %d / stages %d not built", chunk, stages);
        return GS_ERR_UNSUPPORTED;
    }
    BlendArgs a;
    if (!make_args(a, 1, &width, &height, 0, tile_ranges, ids_sorted, mean2d, conic, opacity, nullptr, opts)) {
        set_error("gs_tile_power: image size out of range");
        return GS_ERR_INVALID_ARG;
    }
    a.tiles = tiles;
    a.max_len = max_len;
    a.dump = out;
    return cuda_status(launch_blend_tc(a, opts->variant, chunk, stages, true, n_tiles, stream), "gs_tile_power");
}

gs_status gs_sync_status(gs_stream stream) {
    g_last_error[0] = 0;
    gs_status st = cuda_status(cudaStreamSynchronize(stream), "gs_sync_status: synchronize");
    if (st != GS_OK) return st;
    unsigned* w = error_word();
    if (!w) return cuda_status(cudaGetLastError(), "gs_sync_status: error word");
    unsigned v = 0;
    st = cuda_status(cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost), "gs_sync_status: read");
    if (st != GS_OK) return st;
    if (v == 0) return GS_OK;
    unsigned zero = 0;
    st = cuda_status(cudaMemcpy(w, &zero, sizeof(zero), cudaMemcpyHostToDevice), "gs_sync_status: clear");
    if (st != GS_OK) return st;
    if (v & kErrTimeout) {
        set_error("a device-side wait exceeded its time limit");
        return GS_ERR_TIMEOUT;
    }
    if (v & kErrCapacity) {
        set_error("a bin/sort without synchronisation had more instances than its capacity");
        return GS_ERR_CAPACITY;
    }
    set_error("device error word 0x%x", v);
    return GS_ERR_CUDA;
}

gs_status gs_selftest_bounded_wait(int64_t timeout_ns, gs_stream stream) {
    g_last_error[0] = 0;
    if (timeout_ns < 0) {
        set_error("gs_selftest_bounded_wait: negative timeout");
        return GS_ERR_INVALID_ARG;
    }
    uint64_t lim = timeout_ns > 1000000000ll ? 1000000000ull : (uint64_t)timeout_ns;
    unsigned* w = error_word();
    if (!w) return cuda_status(cudaGetLastError(), "gs_selftest_bounded_wait: error word");
    k_selftest_wait<<<1, 32, 0, stream>>>(lim, w);
    count_launches();
    return cuda_status(cudaGetLastError(), "gs_selftest_bounded_wait launch");
}

}  // extern "C"
