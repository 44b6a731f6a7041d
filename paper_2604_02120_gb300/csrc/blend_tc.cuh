// Tensor-core blending (Alg. 2, Eqs. 4-8) for sm_100-family GPUs.
//
// One CTA per 16 x 16 tile, 10 warps:
//   warps 0-7  epilogue: one thread per pixel.  Warp w reads TMEM lanes
//              32 (w % 4) .. +31 of the accumulator half w / 4 (pixels
//              128 (w / 4) + 32 (w % 4) + lane), walks the chunk's columns in
//              depth order and does exp2 / skip / clamp / composite / stop.
//   warp 8     producer: gathers each splat of the next chunk (mean, conic,
//              opacity, colour), forms its coefficient row v_g of Eq. 6 (scaled
//              by log2 e, with log2 o folded into the constant term) split into
//              operand-type terms, writes it in the UMMA shared-memory layout.
//   warp 9     lane 0 issues two tcgen05.mma (M = 128 pixels each, N = chunk
//              splats, K = 16 or 32) per chunk into a TMEM stage; the warp owns
//              the TMEM allocation.
// Stages form a ring of S shared-memory + TMEM buffers guarded by three
// mbarriers each (full: producer -> MMA, tfull: MMA -> epilogue, empty:
// epilogue -> producer).  Every wait is bounded by opts.timeout_ns; on expiry
// the CTA records GS_ERR_TIMEOUT in the device error word, all roles leave,
// the MMA thread waits (bounded, 1 s) for its last commit and TMEM is freed.
//
// The pixel matrix M_p (A operand, 256 x K) holds [xb^2, yb^2, xb yb, xb, yb, 1]
// once per split term; with the reference pixel at the tile centre every
// entry is a multiple of 1/4 of magnitude <= 56.25 (exact in fp16 and bf16).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"

namespace gs {
namespace tc {

constexpr int kEpiWarps = 8;
constexpr int kThreads = 320;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLog2AlphaMin = -7.9943534368588578f;  // log2(1/255)
constexpr float kDeadPower = -200.0f;

template <int V>
struct Traits {
    static constexpr int K = (V == GS_BLEND_TC_BF16_SPLIT) ? 32 : 16;
    static constexpr int TERMS = (V == GS_BLEND_TC_FP16_SPLIT) ? 2 : (V == GS_BLEND_TC_BF16_SPLIT ? 3 : 1);
    static constexpr uint32_t FMT = (V == GS_BLEND_TC_BF16 || V == GS_BLEND_TC_BF16_SPLIT) ? 1u : 0u;
    static constexpr bool HALF = (FMT == 0);
    static constexpr int KSTEPS = K / 16;
    static constexpr int ROW_BYTES = K * 2;
    static constexpr int SBO = (K / 8) * 128;  // bytes between 8-row core-matrix groups
};

template <bool HALF>
__device__ __forceinline__ uint16_t to_op(float x) {
    if constexpr (HALF) return __half_as_ushort(__float2half_rn(x));
    else return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
template <bool HALF>
__device__ __forceinline__ float from_op(uint16_t b) {
    if constexpr (HALF) return __half2float(__ushort_as_half(b));
    else return __bfloat162float(__ushort_as_bfloat16(b));
}

template <int S, int CH, int V>
struct Layout {
    static constexpr int A_BYTES = 256 * Traits<V>::ROW_BYTES;
    static constexpr int B_BYTES = CH * Traits<V>::ROW_BYTES;
    static constexpr int OFF_B = A_BYTES;
    static constexpr int OFF_REC = OFF_B + S * B_BYTES;
    static constexpr int OFF_BAR = OFF_REC + S * CH * 16;
    static constexpr int OFF_N = OFF_BAR + 3 * S * 8;
    static constexpr int OFF_MISC = OFF_N + S * 4;
    static constexpr int BYTES = OFF_MISC + 16;
    static constexpr uint32_t TCOLS_RAW = 2u * S * CH;
    static constexpr uint32_t TCOLS = TCOLS_RAW <= 32 ? 32 : TCOLS_RAW <= 64 ? 64 : TCOLS_RAW <= 128 ? 128
                                      : TCOLS_RAW <= 256 ? 256 : 512;
    static_assert(TCOLS_RAW <= 512, "TMEM stages exceed 512 columns");
};

// Store 8 consecutive K elements (one 16-byte core-matrix row) of row r.
template <int V>
__device__ __forceinline__ void store_row_chunk(uint8_t* mat, int r, int kc, const uint16_t (&e)[8]) {
    uint4 u;
    u.x = (uint32_t)e[0] | ((uint32_t)e[1] << 16);
    u.y = (uint32_t)e[2] | ((uint32_t)e[3] << 16);
    u.z = (uint32_t)e[4] | ((uint32_t)e[5] << 16);
    u.w = (uint32_t)e[6] | ((uint32_t)e[7] << 16);
    *reinterpret_cast<uint4*>(mat + (r >> 3) * Traits<V>::SBO + kc * 128 + (r & 7) * 16) = u;
}

// Maximum of q(d) = -1/2 d^T [[A, B], [B, C]] d over the box [bx0, bx1] x [by0, by1].
__device__ __forceinline__ float box_max_quadratic(float A, float B, float C, float bx0, float bx1, float by0,
                                                   float by1) {
    if (!(A > 0.f) || !(C > 0.f)) return 0.f;  // not positive definite: never skipped
    if (bx0 <= 0.f && bx1 >= 0.f && by0 <= 0.f && by1 >= 0.f) return 0.f;
    float best = -INFINITY;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float ex = e ? bx1 : bx0;
        const float dy = fminf(fmaxf(-B * ex / C, by0), by1);
        best = fmaxf(best, -0.5f * (A * ex * ex + 2.f * B * ex * dy + C * dy * dy));
        const float ey = e ? by1 : by0;
        const float dx = fminf(fmaxf(-B * ey / A, bx0), bx1);
        best = fmaxf(best, -0.5f * (A * dx * dx + 2.f * B * dx * ey + C * ey * ey));
    }
    return best;
}

template <int V, int CH, int S, bool DUMP>
__global__ void __launch_bounds__(kThreads, 1) k_blend_tc(BlendArgs a) {
    using TR = Traits<V>;
    using LY = Layout<S, CH, V>;
    constexpr int K = TR::K;
    constexpr int SBO = TR::SBO;
    constexpr uint32_t IDESC = idesc_f16(TR::FMT, 128, CH);
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sA = smem;
    uint8_t* sB = smem + LY::OFF_B;
    float4* sRec = reinterpret_cast<float4*>(smem + LY::OFF_REC);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + LY::OFF_BAR);
    int* sN = reinterpret_cast<int*>(smem + LY::OFF_N);
    uint32_t* sTmem = reinterpret_cast<uint32_t*>(smem + LY::OFF_MISC);
    volatile int* sDone = reinterpret_cast<volatile int*>(smem + LY::OFF_MISC + 4);
    volatile int* sAbort = reinterpret_cast<volatile int*>(smem + LY::OFF_MISC + 8);
    auto bar_full = [&](int s) { return smem_u32(bars + s); };
    auto bar_tfull = [&](int s) { return smem_u32(bars + S + s); };
    auto bar_empty = [&](int s) { return smem_u32(bars + 2 * S + s); };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = DUMP ? a.tiles[blockIdx.x] : (int)blockIdx.x;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int x0 = tx * kTile, y0 = ty * kTile;
    const uint32_t start = a.ranges[2 * tile], end = a.ranges[2 * tile + 1];
    int len = end > start ? (int)(end - start) : 0;
    if (DUMP && len > a.max_len) len = a.max_len;

    // epilogue pixel of this thread
    const int half = (warp >> 2) & 1, quad = warp & 3;
    const int pix = half * 128 + quad * 32 + lane;
    const int px = x0 + (pix & 15), py = y0 + (pix >> 4);
    const bool inside = warp < kEpiWarps && px < a.W && py < a.H;

    if (len == 0) {  // uniform over the CTA: nothing to blend
        if (!DUMP && inside) {
            const size_t p = (size_t)py * a.W + px, plane = (size_t)a.W * a.H;
            a.image[p] = a.bg[0];
            a.image[plane + p] = a.bg[1];
            a.image[2 * plane + p] = a.bg[2];
            a.T_final[p] = 1.0f;
            a.n_contrib[p] = 0;
        }
        return;
    }
    const int nchunks = (len + CH - 1) / CH;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(bar_full(s), 1);
            mbar_init(bar_tfull(s), 1);
            mbar_init(bar_empty(s), kEpiWarps);
        }
        *sDone = 0;
        *sAbort = 0;
        mbar_fence_init();
    }
    // pixel matrix M_p (A operand)
    const bool origin = a.ref_origin != 0;
    for (int idx = threadIdx.x; idx < 256 * (K / 8); idx += kThreads) {
        const int r = idx / (K / 8), kc = idx % (K / 8);
        const float xb = origin ? -(float)(r & 15) : 7.5f - (float)(r & 15);
        const float yb = origin ? -(float)(r >> 4) : 7.5f - (float)(r >> 4);
        const float vp[6] = {xb * xb, yb * yb, xb * yb, xb, yb, 1.0f};
        uint16_t e[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = kc * 8 + i;
            e[i] = (k < 6 * TR::TERMS) ? to_op<TR::HALF>(vp[k % 6]) : (uint16_t)0;
        }
        store_row_chunk<V>(sA, r, kc, e);
    }
    fence_proxy_async_smem();
    if (warp == 9) {
        tmem_alloc(smem_u32(sTmem), LY::TCOLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *sTmem;
    const uint64_t tmo = a.timeout_ns;

    if (warp < kEpiWarps) {
        // ------------------------------------------------------- epilogue --
        float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
        int last = 0;
        bool done = DUMP ? false : !inside;
        bool wdone = DUMP ? false : __all_sync(0xffffffffu, done);
        if (!DUMP && wdone && lane == 0) atomicAdd((int*)sDone, 1);
        for (int k = 0;; ++k) {
            const int s = k % S;
            const uint32_t ph = (uint32_t)(k / S) & 1u;
            if (!mbar_wait_bounded(bar_tfull(s), ph, tmo, sAbort) || !mbar_wait_bounded(bar_full(s), ph, tmo, sAbort)) {
                *sAbort = 1;
                atomicOr(a.err, kErrTimeout);
                break;
            }
            const int n = sN[s];
            if (n == 0) break;
            tc_fence_after();
            if (!wdone) {
                const uint32_t tb = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(s * 2 * CH + half * CH);
                const float4* rec = sRec + s * CH;
#pragma unroll 1
                for (int c0 = 0; c0 < CH && c0 < n; c0 += 32) {
                    uint32_t v[32];
                    tmem_ld_32x32b_x32(tb + (uint32_t)c0, v);
                    tmem_ld_wait();
                    if constexpr (DUMP) {
#pragma unroll
                        for (int c = 0; c < 32; ++c) {
                            const int j = c0 + c;
                            if (j < n)
                                a.dump[((size_t)blockIdx.x * a.max_len + (size_t)k * CH + j) * 256 + pix] =
                                    __uint_as_float(v[c]);
                        }
                    } else {
                        const int gbase = k * CH + c0;
#pragma unroll
                        for (int c = 0; c < 32; ++c) {
                            if (c0 + c < n) {
                                const float4 rc = rec[c0 + c];
                                float al = ex2_approx(fminf(__uint_as_float(v[c]), rc.w));
                                al = fminf(al, kAlphaMax);
                                if (!done && al >= kAlphaMin) {
                                    const float tT = T * (1.0f - al);
                                    if (tT < kTMin) {
                                        done = true;
                                    } else {
                                        const float w = al * T;
                                        C0 = fmaf(rc.x, w, C0);
                                        C1 = fmaf(rc.y, w, C1);
                                        C2 = fmaf(rc.z, w, C2);
                                        T = tT;
                                        last = gbase + c + 1;
                                    }
                                }
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (!DUMP && !wdone) {
                wdone = __all_sync(0xffffffffu, done);
                if (wdone && lane == 0) atomicAdd((int*)sDone, 1);
            }
            if (lane == 0) mbar_arrive(bar_empty(s));
        }
        if (!DUMP && inside) {
            const size_t p = (size_t)py * a.W + px, plane = (size_t)a.W * a.H;
            a.image[p] = C0 + T * a.bg[0];
            a.image[plane + p] = C1 + T * a.bg[1];
            a.image[2 * plane + p] = C2 + T * a.bg[2];
            a.T_final[p] = T;
            a.n_contrib[p] = last;
        }
    } else if (warp == kEpiWarps) {
        // ------------------------------------------------------- producer --
        const float xc = (float)x0 + (origin ? 0.5f : 8.0f), yc = (float)y0 + (origin ? 0.5f : 8.0f);
        const float bmin = origin ? -15.0f : -7.5f, bmax = origin ? 0.0f : 7.5f;
        for (int k = 0;; ++k) {
            const int s = k % S;
            const uint32_t ph = (uint32_t)(k / S) & 1u;
            if (!mbar_wait_bounded(bar_empty(s), ph ^ 1u, tmo, sAbort)) {
                *sAbort = 1;
                atomicOr(a.err, kErrTimeout);
                break;
            }
            const bool stop = k >= nchunks || (!DUMP && *sDone >= kEpiWarps) || *sAbort;
            if (stop) {
                if (lane == 0) {
                    sN[s] = 0;
                    mbar_arrive(bar_full(s));
                }
                break;
            }
            const int base = k * CH;
            const int n = min(CH, len - base);
            uint8_t* mB = sB + s * LY::B_BYTES;
            for (int j = lane; j < CH; j += 32) {
                float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                float4 rc = make_float4(0.f, 0.f, 0.f, 0.f);
                if (j < n) {
                    const uint32_t g = a.ids[start + base + j];
                    const float2 m = a.mean2d[g];
                    const float A = a.conic[3 * g], B = a.conic[3 * g + 1], C = a.conic[3 * g + 2];
                    const float o = a.opac[g];
                    const float xh = m.x - xc, yh = m.y - yc;
                    const float ux = fmaf(A, xh, B * yh), uy = fmaf(B, xh, C * yh);
                    const float P0 = -0.5f * fmaf(xh, ux, yh * uy);
                    const float l2o = o > 0.f ? __log2f(o) : -INFINITY;
                    const float qmax = box_max_quadratic(A, B, C, xh + bmin, xh + bmax, yh + bmin, yh + bmax);
                    const bool live = fmaf(qmax, kLog2e, l2o) >= kLog2AlphaMin - 0.25f;
                    if (live) {
                        v[0] = -0.5f * A * kLog2e;
                        v[1] = -0.5f * C * kLog2e;
                        v[2] = -B * kLog2e;
                        v[3] = -ux * kLog2e;
                        v[4] = -uy * kLog2e;
                        v[5] = fmaf(P0, kLog2e, l2o);
                        if constexpr (TR::HALF) {
#pragma unroll
                            for (int i = 0; i < 6; ++i) v[i] = fminf(fmaxf(v[i], -30000.f), 30000.f);
                        }
                    } else {
                        v[5] = kDeadPower;
                    }
                    if (a.rgb) rc = make_float4(a.rgb[3 * g], a.rgb[3 * g + 1], a.rgb[3 * g + 2], live ? l2o : 0.f);
                }
                // split v into TERMS operand-type terms: v ~ t0 + t1 (+ t2)
                uint16_t terms[3][6];
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    float r = v[i];
#pragma unroll
                    for (int t = 0; t < TR::TERMS; ++t) {
                        terms[t][i] = to_op<TR::HALF>(r);
                        r -= from_op<TR::HALF>(terms[t][i]);
                    }
                }
#pragma unroll
                for (int kc = 0; kc < K / 8; ++kc) {
                    uint16_t e[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int kk = kc * 8 + i;
                        e[i] = (kk < 6 * TR::TERMS) ? terms[kk / 6][kk % 6] : (uint16_t)0;
                    }
                    store_row_chunk<V>(mB, j, kc, e);
                }
                sRec[s * CH + j] = rc;
            }
            if (lane == 0) sN[s] = n;
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_full(s));
        }
    } else if (lane == 0) {
        // ------------------------------------------------------ MMA issue --
        int last_s = -1;
        uint32_t last_ph = 0;
        const uint32_t aA = smem_u32(sA);
        for (int k = 0;; ++k) {
            const int s = k % S;
            const uint32_t ph = (uint32_t)(k / S) & 1u;
            if (!mbar_wait_bounded(bar_full(s), ph, tmo, sAbort)) {
                *sAbort = 1;
                atomicOr(a.err, kErrTimeout);
                break;
            }
            if (sN[s] == 0) {
                mbar_arrive(bar_tfull(s));
                break;
            }
            tc_fence_after();
            const uint32_t aB = smem_u32(sB + s * LY::B_BYTES);
#pragma unroll
            for (int ks = 0; ks < TR::KSTEPS; ++ks) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint64_t ad = smem_desc(aA + (uint32_t)(h * 16 * SBO + ks * 256), 128, SBO);
                    const uint64_t bd = smem_desc(aB + (uint32_t)(ks * 256), 128, SBO);
                    tc_mma_f16(tmem + (uint32_t)(s * 2 * CH + h * CH), ad, bd, IDESC, ks > 0 ? 1u : 0u);
                }
            }
            tc_commit(bar_tfull(s));
            last_s = s;
            last_ph = ph;
        }
        if (last_s >= 0) mbar_wait_bounded(bar_tfull(last_s), last_ph, 1000000000ull, nullptr);
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 9) tmem_dealloc(tmem, LY::TCOLS);
}

template <int V, int CH, int S, bool DUMP>
cudaError_t launch_inst(const BlendArgs& a, int grid, cudaStream_t s) {
    constexpr int bytes = Layout<S, CH, V>::BYTES;
    auto kern = k_blend_tc<V, CH, S, DUMP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    kern<<<grid, kThreads, bytes, s>>>(a);
    count_launches();
    return cudaGetLastError();
}

// Instantiated per variant in blend_tc_v<V>.cu
template <int V>
cudaError_t launch_variant(const BlendArgs& a, int chunk, int stages, bool dump, int grid, cudaStream_t s);
template <>
cudaError_t launch_variant<1>(const BlendArgs&, int, int, bool, int, cudaStream_t);
template <>
cudaError_t launch_variant<2>(const BlendArgs&, int, int, bool, int, cudaStream_t);
template <>
cudaError_t launch_variant<3>(const BlendArgs&, int, int, bool, int, cudaStream_t);
template <>
cudaError_t launch_variant<4>(const BlendArgs&, int, int, bool, int, cudaStream_t);

}  // namespace tc
}  // namespace gs
