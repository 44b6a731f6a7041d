// CUDA-core blending (Alg. 1) and its gradient.  One 256-thread block per
// 16 x 16 tile, one thread per pixel; the tile's list is staged through shared
// memory in batches of 256 splats (Sec. 2.1 (d)).  The exponent is evaluated
// per pixel as the quadratic of Eq. 3 in FP32.
#include "internal.h"

namespace gs {
namespace {

constexpr int kBatch = 256;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

struct SplatSm {
    float4 geo;  // mx, my, A, B
    float4 oc;   // C, o, r, g
    float b;
};

// alpha of a splat at a pixel; `e` receives exp(min(power, 0)) and `pw` power.
// Shared by the forward and backward kernels so both take identical decisions.
__device__ __forceinline__ float splat_alpha(const float4& geo, const float4& oc, float xp, float yp, float& e,
                                             float& pw, float& dx, float& dy) {
    dx = geo.x - xp;
    dy = geo.y - yp;
    const float q = __fmaf_rn(geo.z * dx, dx, __fmul_rn(oc.x * dy, dy));
    pw = __fmaf_rn(-geo.w * dx, dy, -0.5f * q);
    e = __expf(fminf(pw, 0.0f));
    return fminf(kAlphaMax, oc.y * e);
}

// item g of view v: projected data at g, opacity at g - v * n_per_view
__device__ __forceinline__ void load_splat(const BlendArgs& a, uint32_t g, uint32_t opac_off, SplatSm& s) {
    const float2 m = a.mean2d[g];
    s.geo = make_float4(m.x, m.y, a.conic[3 * g], a.conic[3 * g + 1]);
    s.oc = make_float4(a.conic[3 * g + 2], a.opac[g - opac_off], a.rgb[3 * g], a.rgb[3 * g + 1]);
    s.b = a.rgb[3 * g + 2];
}

// Geometry of the block's tile (blockIdx.x is a global tile id).
struct TileGeo {
    int W, H, px, py;
    long long pix_off;
    uint32_t opac_off;
};

__device__ __forceinline__ TileGeo tile_geo(const BlendArgs& a, int tile) {
    const int v = view_of(a, tile);
    const ViewDesc& vd = a.views[v];
    const int lt = tile - vd.tile_begin;
    TileGeo t;
    t.W = vd.W;
    t.H = vd.H;
    t.px = (lt % vd.tiles_x) * kTile + (threadIdx.x & 15);
    t.py = (lt / vd.tiles_x) * kTile + (threadIdx.x >> 4);
    t.pix_off = vd.pix_off;
    t.opac_off = (uint32_t)(v * a.n_per_view);
    return t;
}

__global__ void __launch_bounds__(kBatch) k_blend_fp32_fwd(const __grid_constant__ BlendArgs a) {
    __shared__ float4 s_geo[kBatch];
    __shared__ float4 s_oc[kBatch];
    __shared__ float s_b[kBatch];
    const int tile = tile_at(a, blockIdx.x * a.shard_count + a.shard_index);
    const TileGeo tg = tile_geo(a, tile);
    const int px = tg.px, py = tg.py;
    const bool inside = px < tg.W && py < tg.H;
    const float xp = px + 0.5f, yp = py + 0.5f;
    const uint32_t start = a.ranges[2 * tile], end = a.ranges[2 * tile + 1];
    const int len = end > start ? (int)(end - start) : 0;

    float T = 1.0f, cr = 0.f, cg = 0.f, cb = 0.f;
    int last = 0;
    bool done = !inside;
    for (int base = 0; base < len; base += kBatch) {
        if (__syncthreads_count(done) == kBatch) break;
        const int i = base + threadIdx.x;
        if (i < len) {
            SplatSm s;
            load_splat(a, a.ids[start + i], tg.opac_off, s);
            s_geo[threadIdx.x] = s.geo;
            s_oc[threadIdx.x] = s.oc;
            s_b[threadIdx.x] = s.b;
        }
        __syncthreads();
        const int nb = min(kBatch, len - base);
        for (int j = 0; !done && j < nb; ++j) {
            const float4 geo = s_geo[j], oc = s_oc[j];
            float e, pw, dx, dy;
            const float alpha = splat_alpha(geo, oc, xp, yp, e, pw, dx, dy);
            if (alpha < kAlphaMin) continue;
            const float tT = T * (1.0f - alpha);
            if (tT < kTMin) {
                done = true;
                break;
            }
            const float w = alpha * T;
            cr = __fmaf_rn(oc.z, w, cr);
            cg = __fmaf_rn(oc.w, w, cg);
            cb = __fmaf_rn(s_b[j], w, cb);
            T = tT;
            last = base + j + 1;
        }
    }
    if (inside) {
        const size_t pix = (size_t)py * tg.W + px, plane = (size_t)tg.W * tg.H;
        float* img = a.image + 3 * tg.pix_off;
        img[pix] = cr + T * a.bg[0];
        img[plane + pix] = cg + T * a.bg[1];
        img[2 * plane + pix] = cb + T * a.bg[2];
        a.T_final[tg.pix_off + pix] = T;
        a.n_contrib[tg.pix_off + pix] = last;
    }
}

// Sums of nine per-lane values over the warp.  v[0..7] are reduced by
// recursive halving (each level halves the values a lane carries while
// exchanging the other half with its partner), leaving the total of v[k] in
// the lanes with (lane >> 2) == k; v[8] by a plain butterfly (all lanes).
__device__ __forceinline__ void warp_reduce9(const float (&v)[9], int lane, float& vk, float& v8) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float k4[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = b4 ? v[i] : v[i + 4];
        const float keep = b4 ? v[i + 4] : v[i];
        k4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float k2[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = b3 ? k4[i] : k4[i + 2];
        const float keep = b3 ? k4[i + 2] : k4[i];
        k2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float k1 = (b2 ? k2[1] : k2[0]) + __shfl_xor_sync(0xffffffffu, b2 ? k2[0] : k2[1], 4);
    k1 += __shfl_xor_sync(0xffffffffu, k1, 2);
    k1 += __shfl_xor_sync(0xffffffffu, k1, 1);
    vk = k1;
    float s8 = v[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s8 += __shfl_xor_sync(0xffffffffu, s8, o);
    v8 = s8;
}

// Address of gradient component k (0..8) of Gaussian g:
// dmean2d.x, dmean2d.y, dA, dB, dC, dopacity, dr, dg, db.
__device__ __forceinline__ float* grad_slot(const GradArgs& gr, uint32_t g, uint32_t opac_off, int k) {
    if (k < 2) return reinterpret_cast<float*>(gr.dmean2d) + 2 * (size_t)g + k;
    if (k < 5) return gr.dconic + 3 * (size_t)g + (k - 2);
    if (k == 5) return gr.dopac + (g - opac_off);
    return gr.drgb + 3 * (size_t)g + (k - 6);
}

// Back-to-front walk per pixel.  Per (splat, warp) the nine gradient values
// are either added directly by the few lanes that have them, or summed over
// the warp (warp_reduce9) and added by nine lanes.
__global__ void __launch_bounds__(kBatch) k_blend_fp32_bwd(const __grid_constant__ BlendArgs a, GradArgs gr) {
    __shared__ float4 s_geo[kBatch];
    __shared__ float4 s_oc[kBatch];
    __shared__ float s_b[kBatch];
    __shared__ uint32_t s_id[kBatch];
    __shared__ int s_max;
    const int tile = tile_at(a, blockIdx.x * a.shard_count + a.shard_index);
    const TileGeo tg = tile_geo(a, tile);
    const int px = tg.px, py = tg.py;
    const bool inside = px < tg.W && py < tg.H;
    const float xp = px + 0.5f, yp = py + 0.5f;
    const uint32_t start = a.ranges[2 * tile];
    const int lane = threadIdx.x & 31;

    const size_t pix = (size_t)tg.pix_off + (size_t)py * tg.W + px, plane = (size_t)tg.W * tg.H;
    const size_t gpix = 3 * (size_t)tg.pix_off + (size_t)py * tg.W + px;
    int nc = 0;
    float T = 1.0f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
    if (inside) {
        nc = gr.n_contrib[pix];
        T = gr.T_final[pix];
        g0 = gr.dL_dimage[gpix];
        g1 = gr.dL_dimage[plane + gpix];
        g2 = gr.dL_dimage[2 * plane + gpix];
    }
    float S0 = a.bg[0], S1 = a.bg[1], S2 = a.bg[2];  // colour behind the current splat
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    int wmax = nc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    if (lane == 0) atomicMax(&s_max, wmax);
    __syncthreads();
    const int maxn = s_max;

    for (int hi = maxn; hi > 0; hi -= kBatch) {
        const int lo = max(0, hi - kBatch);
        __syncthreads();
        const int i = lo + threadIdx.x;
        if (i < hi) {
            const uint32_t g = a.ids[start + i];
            SplatSm s;
            load_splat(a, g, tg.opac_off, s);
            s_geo[threadIdx.x] = s.geo;
            s_oc[threadIdx.x] = s.oc;
            s_b[threadIdx.x] = s.b;
            s_id[threadIdx.x] = g;
        }
        __syncthreads();
        // this warp only needs list positions below its largest n_contrib
        for (int j = min(hi, wmax) - 1; j >= lo; --j) {
            const int k = j - lo;
            const float4 geo = s_geo[k], oc = s_oc[k];
            const float cb = s_b[k];
            float v[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) v[q] = 0.f;
            bool contrib = false;
            if (j < nc) {
                float e, pw, dx, dy;
                const float alpha = splat_alpha(geo, oc, xp, yp, e, pw, dx, dy);
                if (alpha >= kAlphaMin) {
                    contrib = true;
                    const float Ti = __fdividef(T, 1.0f - alpha);
                    const float wgt = alpha * Ti;
                    v[6] = wgt * g0;
                    v[7] = wgt * g1;
                    v[8] = wgt * g2;
                    const float dL_dalpha = Ti * ((oc.z - S0) * g0 + (oc.w - S1) * g1 + (cb - S2) * g2);
                    S0 = fmaf(alpha, oc.z - S0, S0);
                    S1 = fmaf(alpha, oc.w - S1, S1);
                    S2 = fmaf(alpha, cb - S2, S2);
                    T = Ti;
                    if (oc.y * e <= kAlphaMax) {  // not clamped
                        v[5] = dL_dalpha * e;
                        if (pw <= 0.0f) {
                            const float dp = dL_dalpha * alpha;
                            v[0] = -dp * (geo.z * dx + geo.w * dy);
                            v[1] = -dp * (geo.w * dx + oc.x * dy);
                            v[2] = -0.5f * dp * dx * dx;
                            v[3] = -dp * dx * dy;
                            v[4] = -0.5f * dp * dy * dy;
                        }
                    }
                }
            }
            const unsigned who = __ballot_sync(0xffffffffu, contrib);
            if (who == 0u) continue;
            const uint32_t g = s_id[k];
            if (__popc(who) <= 3) {
                if (contrib) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) atomicAdd(grad_slot(gr, g, tg.opac_off, q), v[q]);
                }
            } else {
                float vk, v8;
                warp_reduce9(v, lane, vk, v8);
                if ((lane & 3) == 0) atomicAdd(grad_slot(gr, g, tg.opac_off, lane >> 2), vk);
                if (lane == 0) atomicAdd(grad_slot(gr, g, tg.opac_off, 8), v8);
            }
        }
    }
}

}  // namespace

cudaError_t launch_blend_fp32_fwd(const BlendArgs& a, cudaStream_t s) {
    const int items = shard_items(a);
    if (items == 0) return cudaSuccess;
    k_blend_fp32_fwd<<<items, kBatch, 0, s>>>(a);
    count_launches();
    return cudaGetLastError();
}

cudaError_t launch_blend_fp32_bwd(const BlendArgs& a, const GradArgs& g, cudaStream_t s) {
    const int items = shard_items(a);
    if (items == 0) return cudaSuccess;
    k_blend_fp32_bwd<<<items, kBatch, 0, s>>>(a, g);
    count_launches();
    return cudaGetLastError();
}

}  // namespace gs
