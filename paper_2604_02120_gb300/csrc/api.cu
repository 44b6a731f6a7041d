// C ABI entry points: argument checks, status reporting, the per-device error
// word, and dispatch to the kernels of the other translation units.
#include <atomic>
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

unsigned* error_word() {
    static unsigned* addr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (addr[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_error_word) != cudaSuccess) return nullptr;
        addr[dev] = static_cast<unsigned*>(p);
    }
    return addr[dev];
}

}  // namespace gs

using namespace gs;

namespace {

gs_status check_blend_common(int32_t W, int32_t H, const uint32_t* ranges, const uint32_t* ids, const float* mean2d,
                             const float* conic, const float* opacity) {
    if (W <= 0 || H <= 0 || W > (1 << 20) || H > (1 << 20)) {
        set_error("image size %d x %d out of range", W, H);
        return GS_ERR_INVALID_ARG;
    }
    if (!ranges || !ids || !mean2d || !conic || !opacity) {
        set_error("null input pointer");
        return GS_ERR_INVALID_ARG;
    }
    return GS_OK;
}

BlendArgs make_args(int32_t W, int32_t H, const uint32_t* ranges, const uint32_t* ids, const float* mean2d,
                    const float* conic, const float* opacity, const float* rgb, const gs_blend_opts* o) {
    BlendArgs a{};
    a.W = W;
    a.H = H;
    a.tiles_x = tiles_x(W);
    a.num_tiles = tiles_x(W) * tiles_y(H);
    a.ranges = ranges;
    a.ids = ids;
    a.mean2d = reinterpret_cast<const float2*>(mean2d);
    a.conic = conic;
    a.opac = opacity;
    a.rgb = rgb;
    for (int c = 0; c < 3; ++c) a.bg[c] = o ? o->bg[c] : 0.0f;
    a.timeout_ns = (o && o->timeout_ns > 0) ? (uint64_t)o->timeout_ns : 1000000000ull;
    a.ref_origin = o ? o->ref_origin : 0;
    a.err = error_word();
    a.num_views = 1;
    a.total_tiles = a.num_tiles;
    a.views[0] = ViewDesc{W, H, a.tiles_x, 0, 0};
    return a;
}

bool is_tc(int v) { return v >= GS_BLEND_TC_FP16 && v <= GS_BLEND_TC_BF16_SPLIT; }

}  // namespace

extern "C" {

int32_t gs_version(void) { return 100; }

int64_t gs_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

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

gs_status gs_project(int32_t n, const float* means, const float* scales, const float* quats, const float* sh,
                     int32_t sh_degree, const gs_camera* cam, float* mean2d, float* conic, float* depth,
                     int32_t* radius, float* rgb, uint32_t* tiles_touched, gs_stream stream) {
    g_last_error[0] = 0;
    if (n < 0 || sh_degree < 0 || sh_degree > 3 || !cam) {
        set_error("gs_project: bad n (%d), sh_degree (%d) or camera", n, sh_degree);
        return GS_ERR_INVALID_ARG;
    }
    if (cam->width <= 0 || cam->height <= 0 || cam->width > (1 << 20) || cam->height > (1 << 20)) {
        set_error("gs_project: image size %d x %d out of range", cam->width, cam->height);
        return GS_ERR_INVALID_ARG;
    }
    if (n == 0) return GS_OK;
    if (!means || !scales || !quats || !sh || !mean2d || !conic || !depth || !radius || !rgb || !tiles_touched) {
        set_error("gs_project: null pointer");
        return GS_ERR_INVALID_ARG;
    }
    CamDev c{};
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
    return cuda_status(launch_project(n, means, scales, quats, sh, sh_degree, c, mean2d, conic, depth, radius, rgb,
                                      tiles_touched, stream),
                       "gs_project launch");
}

gs_status gs_bin_sort_workspace_size(int32_t n, int64_t capacity, int32_t width, int32_t height, size_t* bytes) {
    g_last_error[0] = 0;
    if (n < 0 || capacity < 0 || capacity >= (int64_t(1) << 32) || width <= 0 || height <= 0 || !bytes ||
        width > (1 << 20) || height > (1 << 20)) {
        set_error("gs_bin_sort_workspace_size: bad arguments");
        return GS_ERR_INVALID_ARG;
    }
    *bytes = bin_sort_workspace_bytes(n, capacity, tiles_x(width) * tiles_y(height));
    return GS_OK;
}

gs_status gs_bin_sort(int32_t n, const float* mean2d, const int32_t* radius, const float* depth, int32_t width,
                      int32_t height, int64_t capacity, void* workspace, size_t workspace_bytes,
                      uint64_t* keys_sorted, uint32_t* ids_sorted, uint32_t* tile_ranges, int64_t* n_instances,
                      gs_stream stream) {
    g_last_error[0] = 0;
    if (n < 0 || capacity < 0 || capacity >= (int64_t(1) << 32) || width <= 0 || height <= 0 ||
        width > (1 << 20) || height > (1 << 20) || !n_instances || !tile_ranges) {
        set_error("gs_bin_sort: bad arguments");
        return GS_ERR_INVALID_ARG;
    }
    if (n > 0 && (!mean2d || !radius || !depth || !workspace)) {
        set_error("gs_bin_sort: null pointer");
        return GS_ERR_INVALID_ARG;
    }
    if (capacity > 0 && (!keys_sorted || !ids_sorted)) {
        set_error("gs_bin_sort: null output pointer");
        return GS_ERR_INVALID_ARG;
    }
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) {
        set_error("gs_bin_sort: workspace must be 256-byte aligned");
        return GS_ERR_INVALID_ARG;
    }
    size_t need = bin_sort_workspace_bytes(n, capacity, tiles_x(width) * tiles_y(height));
    if (workspace_bytes < need) {
        set_error("gs_bin_sort: workspace %zu bytes < %zu needed", workspace_bytes, need);
        return GS_ERR_WORKSPACE;
    }
    return bin_sort_run(n, mean2d, radius, depth, width, height, capacity, workspace, workspace_bytes, keys_sorted,
                        ids_sorted, tile_ranges, n_instances, stream);
}

gs_status gs_blend_forward(int32_t width, int32_t height, const uint32_t* tile_ranges, const uint32_t* ids_sorted,
                           const float* mean2d, const float* conic, const float* opacity, const float* rgb,
                           const gs_blend_opts* opts, float* image, float* T_final, int32_t* n_contrib,
                           gs_stream stream) {
    g_last_error[0] = 0;
    gs_status st = check_blend_common(width, height, tile_ranges, ids_sorted, mean2d, conic, opacity);
    if (st != GS_OK) return st;
    if (!rgb || !image || !T_final || !n_contrib) {
        set_error("gs_blend_forward: null pointer");
        return GS_ERR_INVALID_ARG;
    }
    gs_blend_opts def{};
    const gs_blend_opts* o = opts ? opts : &def;
    BlendArgs a = make_args(width, height, tile_ranges, ids_sorted, mean2d, conic, opacity, rgb, o);
    a.image = image;
    a.T_final = T_final;
    a.n_contrib = n_contrib;
    if (!a.err) return cuda_status(cudaGetLastError(), "gs_blend_forward: error word");
    if (o->variant == GS_BLEND_FP32) return cuda_status(launch_blend_fp32_fwd(a, stream), "gs_blend_forward fp32");
    if (!is_tc(o->variant)) {
        set_error("gs_blend_forward: unknown variant %d", o->variant);
        return GS_ERR_INVALID_ARG;
    }
    int chunk = o->chunk ? o->chunk : 32, stages = o->stages ? o->stages : 2;
    if (!tc_config_supported(o->variant, chunk, stages)) {
        set_error("gs_blend_forward: chunk %d / stages %d not built", chunk, stages);
        return GS_ERR_UNSUPPORTED;
    }
    return cuda_status(launch_blend_tc(a, o->variant, chunk, stages, false, a.num_tiles, stream),
                       "gs_blend_forward tc");
}

gs_status gs_blend_backward(int32_t width, int32_t height, const uint32_t* tile_ranges, const uint32_t* ids_sorted,
                            const float* mean2d, const float* conic, const float* opacity, const float* rgb,
                            const gs_blend_opts* opts, const float* T_final, const int32_t* n_contrib,
                            const float* dL_dimage, float* dmean2d, float* dconic, float* dopacity, float* drgb,
                            gs_stream stream) {
    g_last_error[0] = 0;
    gs_status st = check_blend_common(width, height, tile_ranges, ids_sorted, mean2d, conic, opacity);
    if (st != GS_OK) return st;
    if (!rgb || !T_final || !n_contrib || !dL_dimage || !dmean2d || !dconic || !dopacity || !drgb) {
        set_error("gs_blend_backward: null pointer");
        return GS_ERR_INVALID_ARG;
    }
    gs_blend_opts def{};
    const gs_blend_opts* o = opts ? opts : &def;
    if (o->variant != GS_BLEND_FP32 && !is_tc(o->variant)) {
        set_error("gs_blend_backward: unknown variant %d", o->variant);
        return GS_ERR_INVALID_ARG;
    }
    BlendArgs a = make_args(width, height, tile_ranges, ids_sorted, mean2d, conic, opacity, rgb, o);
    GradArgs g{T_final, n_contrib, dL_dimage, reinterpret_cast<float2*>(dmean2d), dconic, dopacity, drgb};
    return cuda_status(launch_blend_fp32_bwd(a, g, stream), "gs_blend_backward");
}

gs_status gs_tile_power(int32_t width, int32_t height, const uint32_t* tile_ranges, const uint32_t* ids_sorted,
                        const float* mean2d, const float* conic, const float* opacity, const gs_blend_opts* opts,
                        const int32_t* tiles, int32_t n_tiles, int32_t max_len, float* out, gs_stream stream) {
    g_last_error[0] = 0;
    gs_status st = check_blend_common(width, height, tile_ranges, ids_sorted, mean2d, conic, opacity);
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
    BlendArgs a = make_args(width, height, tile_ranges, ids_sorted, mean2d, conic, opacity, nullptr, opts);
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
