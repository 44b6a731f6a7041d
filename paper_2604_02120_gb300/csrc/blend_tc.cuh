// Tensor-core blending (Alg. 2, Eqs. 4-8) for sm_100-family GPUs.
//
// One CTA per 16 x 16 tile.  The tile is split into an upper and a lower
// 16 x 8 half; M_p (A operand, 128 x K) holds the monomials
// [xb^2, yb^2, xb yb, xb, yb, 1] of the 128 pixels of a half relative to the
// half's reference pixel.  For every chunk of CH splats the producer writes
// 2 CH coefficient rows v_g (Eq. 6): rows [0, CH) referred to the upper half's
// reference, rows [CH, 2 CH) to the lower half's (8 pixels further down).
// One tcgen05.mma (M = 128, N = 2 CH, K = 16 or 32) then leaves in TMEM lane
// r, column j the exponent of splat j at upper pixel r and, at column CH + j,
// at lower pixel r: each epilogue thread owns two pixels of one lane and
// composites both with packed f32x2 arithmetic.
//
// Warps: 0-3 epilogue (warp w reads TMEM lanes 32 w .. 32 w + 31), 4 producer,
// 5 MMA issue (lane 0) and TMEM owner.  The producer fills a ring of SS
// shared-memory stages (v_g rows + per-splat colour), the MMA writes a ring of
// 2 TMEM stages; a stage of either ring is reused once the epilogue (and, for
// shared memory, the MMA) is done with it.  All waits are bounded by
// opts.timeout_ns; on expiry the CTA records GS_ERR_TIMEOUT in the device
// error word, every role leaves its loop, the MMA thread waits (bounded, 1 s)
// for its last commit and TMEM is freed.
//
// Compositing without branches (per pixel, alpha already clamped):
//   cull = sat((1/255 - alpha) 2^36)        1 iff alpha < 1/255 (exact: one rounding)
//   a    = alpha - alpha cull
//   T'   = T - a T;  stop = sat((1e-4 - T') 2^40)   1 iff T' < 1e-4
//   T_stop += T stop;  a2 = a - a stop;  w = a2 T;  T = T' - T' stop
//   C += c w;  used = sat(a2 2^36);  last += used (index + 1 - last)
// A pixel that stops keeps T = 0 from then on (so it never contributes
// again, and T' = 0 keeps `stop` at 1 while T_stop stays put); T_final =
// T + T_stop.  Pixels outside the image start with T = 0.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"

namespace gs {
namespace tc {

constexpr int kEpiWarps = 4;
constexpr int kThreads = 192;
constexpr int kTStages = 2;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLog2AlphaMin = -7.9943534368588578f;    // log2(1/255)
constexpr float kLog2AlphaMax = -0.014499569695115089f;  // log2(0.99)
constexpr float kDeadPower = -200.0f;
constexpr float kCullScale = 68719476736.0f;    // 2^36
constexpr float kStopScale = 1099511627776.0f;  // 2^40

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

// Per-splat record the epilogue reads: colour duplicated for both pixels of a
// lane and the exponent ceiling min(log2 0.99, log2 o).
struct alignas(16) Rec {
    float4 rg;  // r, r, g, g
    float4 bc;  // b, b, cap, cap
};

template <int SS, int CH, int V>
struct Layout {
    static constexpr int A_BYTES = 128 * Traits<V>::ROW_BYTES;
    static constexpr int B_BYTES = 2 * CH * Traits<V>::ROW_BYTES;
    static constexpr int OFF_B = A_BYTES;
    static constexpr int OFF_REC = OFF_B + SS * B_BYTES;
    static constexpr int OFF_BAR = OFF_REC + SS * CH * (int)sizeof(Rec);
    static constexpr int NBAR = 2 * SS + 2 * kTStages;
    static constexpr int OFF_N = OFF_BAR + NBAR * 8;
    static constexpr int OFF_MISC = OFF_N + SS * 4;
    static constexpr int BYTES = OFF_MISC + 16;
    static constexpr uint32_t TCOLS_RAW = 2u * kTStages * CH;
    static constexpr uint32_t TCOLS = TCOLS_RAW <= 32 ? 32 : TCOLS_RAW <= 64 ? 64 : TCOLS_RAW <= 128 ? 128
                                      : TCOLS_RAW <= 256 ? 256 : 512;
    static_assert(TCOLS_RAW <= 512, "TMEM stages exceed 512 columns");
    static_assert(CH % 16 == 0 && 2 * CH <= 256, "chunk must be a multiple of 16 and at most 128");
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

// Coefficient row of Eq. 6 for one splat and one reference pixel, in base-2
// units with log2(o) folded into the constant term: v . v_p = log2(e) power + log2 o.
// (xh, yh) = splat centre minus reference pixel; (bx0..by1) = the range of the
// pixel offsets of the half-tile.  A splat that cannot reach alpha >= 1/255 at
// any point of the half gets a dead row (exponent -200 everywhere).
template <bool HALF>
__device__ __forceinline__ void coeff_row(float A, float B, float C, float l2o, float xh, float yh, float bx0,
                                          float bx1, float by0, float by1, float (&v)[6]) {
    const float ux = fmaf(A, xh, B * yh), uy = fmaf(B, xh, C * yh);
    const float P0 = -0.5f * fmaf(xh, ux, yh * uy);
    const float qmax = box_max_quadratic(A, B, C, xh + bx0, xh + bx1, yh + by0, yh + by1);
    const bool live = fmaf(qmax, kLog2e, l2o) >= kLog2AlphaMin - 0.25f;
    if (live) {
        v[0] = -0.5f * A * kLog2e;
        v[1] = -0.5f * C * kLog2e;
        v[2] = -B * kLog2e;
        v[3] = -ux * kLog2e;
        v[4] = -uy * kLog2e;
        v[5] = fmaf(P0, kLog2e, l2o);
        if constexpr (HALF) {
#pragma unroll
            for (int i = 0; i < 6; ++i) v[i] = fminf(fmaxf(v[i], -30000.f), 30000.f);
        }
    } else {
#pragma unroll
        for (int i = 0; i < 5; ++i) v[i] = 0.f;
        v[5] = kDeadPower;
    }
}

// Write row r of a B stage: v split into TERMS operand-type terms, each in its
// own 6-wide K slot, zero padding up to K.
template <int V>
__device__ __forceinline__ void store_coeff_row(uint8_t* mB, int r, const float (&v)[6]) {
    using TR = Traits<V>;
    uint16_t terms[3][6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        float rem = v[i];
#pragma unroll
        for (int t = 0; t < TR::TERMS; ++t) {
            terms[t][i] = to_op<TR::HALF>(rem);
            rem -= from_op<TR::HALF>(terms[t][i]);
        }
    }
#pragma unroll
    for (int kc = 0; kc < TR::K / 8; ++kc) {
        uint16_t e[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int kk = kc * 8 + i;
            e[i] = (kk < 6 * TR::TERMS) ? terms[kk / 6][kk % 6] : (uint16_t)0;
        }
        store_row_chunk<V>(mB, r, kc, e);
    }
}

__device__ __forceinline__ void tmem_ld_32x32b_x16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

__device__ __forceinline__ float sat(float x) { return __saturatef(x); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

template <int V, int CH, int SS, bool DUMP>
__global__ void __launch_bounds__(kThreads, 4) k_blend_tc(BlendArgs a) {
    using TR = Traits<V>;
    using LY = Layout<SS, CH, V>;
    constexpr int K = TR::K;
    constexpr int SBO = TR::SBO;
    constexpr uint32_t IDESC = idesc_f16(TR::FMT, 128, 2 * CH);
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sA = smem;
    uint8_t* sB = smem + LY::OFF_B;
    Rec* sRec = reinterpret_cast<Rec*>(smem + LY::OFF_REC);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + LY::OFF_BAR);
    int* sN = reinterpret_cast<int*>(smem + LY::OFF_N);
    uint32_t* sTmem = reinterpret_cast<uint32_t*>(smem + LY::OFF_MISC);
    volatile int* sDone = reinterpret_cast<volatile int*>(smem + LY::OFF_MISC + 4);
    volatile int* sAbort = reinterpret_cast<volatile int*>(smem + LY::OFF_MISC + 8);
    auto bar_full = [&](int s) { return smem_u32(bars + s); };
    auto bar_empty = [&](int s) { return smem_u32(bars + SS + s); };
    auto bar_tfull = [&](int t) { return smem_u32(bars + 2 * SS + t); };
    auto bar_tempty = [&](int t) { return smem_u32(bars + 2 * SS + kTStages + t); };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = DUMP ? a.tiles[blockIdx.x] : (int)blockIdx.x;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int x0 = tx * kTile, y0 = ty * kTile;
    const uint32_t start = a.ranges[2 * tile], end = a.ranges[2 * tile + 1];
    int len = end > start ? (int)(end - start) : 0;
    if (DUMP && len > a.max_len) len = a.max_len;

    // the two pixels of this epilogue thread: lane r of the accumulator
    const int r = warp * 32 + lane;  // 0..127 for warps 0-3
    const int px = x0 + (r & 15), py_up = y0 + (r >> 4), py_lo = py_up + 8;
    const bool epi = warp < kEpiWarps;
    const bool in_up = epi && px < a.W && py_up < a.H;
    const bool in_lo = epi && px < a.W && py_lo < a.H;

    if (len == 0) {  // uniform over the CTA: nothing to blend
        if (!DUMP) {
            const size_t plane = (size_t)a.W * a.H;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h ? in_lo : in_up) {
                    const size_t p = (size_t)(h ? py_lo : py_up) * a.W + px;
                    a.image[p] = a.bg[0];
                    a.image[plane + p] = a.bg[1];
                    a.image[2 * plane + p] = a.bg[2];
                    a.T_final[p] = 1.0f;
                    a.n_contrib[p] = 0;
                }
            }
        }
        return;
    }
    const int nchunks = (len + CH - 1) / CH;

    if (threadIdx.x == 0) {
        for (int s = 0; s < SS; ++s) {
            mbar_init(bar_full(s), 1);
            mbar_init(bar_empty(s), 1 + kEpiWarps);
        }
        for (int t = 0; t < kTStages; ++t) {
            mbar_init(bar_tfull(t), 1);
            mbar_init(bar_tempty(t), kEpiWarps);
        }
        *sDone = 0;
        *sAbort = 0;
        mbar_fence_init();
    }
    // pixel matrix M_p of a 16 x 8 half-tile (A operand)
    const bool origin = a.ref_origin != 0;
    for (int idx = threadIdx.x; idx < 128 * (K / 8); idx += kThreads) {
        const int row = idx / (K / 8), kc = idx % (K / 8);
        const float xb = origin ? -(float)(row & 15) : 7.5f - (float)(row & 15);
        const float yb = origin ? -(float)(row >> 4) : 3.5f - (float)(row >> 4);
        const float vp[6] = {xb * xb, yb * yb, xb * yb, xb, yb, 1.0f};
        uint16_t e[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = kc * 8 + i;
            e[i] = (k < 6 * TR::TERMS) ? to_op<TR::HALF>(vp[k % 6]) : (uint16_t)0;
        }
        store_row_chunk<V>(sA, row, kc, e);
    }
    fence_proxy_async_smem();
    if (warp == 5) {
        tmem_alloc(smem_u32(sTmem), LY::TCOLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *sTmem;
    const uint64_t tmo = a.timeout_ns;

    if (epi) {
        // ------------------------------------------------------- epilogue --
        float2 T = make_float2(in_up || DUMP ? 1.f : 0.f, in_lo || DUMP ? 1.f : 0.f);
        float2 Tstop = make_float2(0.f, 0.f), last = make_float2(0.f, 0.f);
        float2 Cr = make_float2(0.f, 0.f), Cg = Cr, Cb = Cr;
        bool wdone = DUMP ? false : __all_sync(0xffffffffu, T.x == 0.f && T.y == 0.f);
        if (!DUMP && wdone && lane == 0) atomicAdd((int*)sDone, 1);
        for (int k = 0;; ++k) {
            const int s = k % SS, t = k % kTStages;
            const uint32_t ps = (uint32_t)(k / SS) & 1u, pt = (uint32_t)(k / kTStages) & 1u;
            if (!mbar_wait_bounded(bar_tfull(t), pt, tmo, sAbort) || !mbar_wait_bounded(bar_full(s), ps, tmo, sAbort)) {
                *sAbort = 1;
                atomicOr(a.err, kErrTimeout);
                break;
            }
            const int n = sN[s];
            if (n == 0) break;
            tc_fence_after();
            if (!wdone) {
                const uint32_t tb = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * 2 * CH);
                const Rec* rec = sRec + s * CH;
#pragma unroll 1
                for (int c0 = 0; c0 < n; c0 += 16) {
                    uint32_t vu[16], vl[16];
                    tmem_ld_32x32b_x16(tb + (uint32_t)c0, vu);
                    tmem_ld_32x32b_x16(tb + (uint32_t)(CH + c0), vl);
                    tmem_ld_wait();
                    if constexpr (DUMP) {
#pragma unroll
                        for (int c = 0; c < 16; ++c) {
                            const int j = c0 + c;
                            if (j < n) {
                                float* o = a.dump + ((size_t)blockIdx.x * a.max_len + (size_t)k * CH + j) * 256;
                                o[r] = __uint_as_float(vu[c]);
                                o[r + 128] = __uint_as_float(vl[c]);
                            }
                        }
                    } else {
                        const float base1 = (float)(k * CH + c0 + 1);
#pragma unroll
                        for (int c = 0; c < 16; ++c) {
                            const Rec rc = rec[c0 + c];
                            float2 al;
                            al.x = ex2_approx(fminf(__uint_as_float(vu[c]), rc.bc.z));
                            al.y = ex2_approx(fminf(__uint_as_float(vl[c]), rc.bc.w));
                            float2 cull;
                            cull.x = sat(fmaf(al.x, -kCullScale, kAlphaMin * kCullScale));
                            cull.y = sat(fmaf(al.y, -kCullScale, kAlphaMin * kCullScale));
                            al = __ffma2_rn(neg2(al), cull, al);
                            const float2 tT = __ffma2_rn(neg2(al), T, T);
                            float2 stop;
                            stop.x = sat(fmaf(tT.x, -kStopScale, kTMin * kStopScale));
                            stop.y = sat(fmaf(tT.y, -kStopScale, kTMin * kStopScale));
                            Tstop = __ffma2_rn(T, stop, Tstop);
                            const float2 a2 = __ffma2_rn(neg2(al), stop, al);
                            const float2 w = __fmul2_rn(a2, T);
                            T = __ffma2_rn(neg2(tT), stop, tT);
                            Cr = __ffma2_rn(make_float2(rc.rg.x, rc.rg.y), w, Cr);
                            Cg = __ffma2_rn(make_float2(rc.rg.z, rc.rg.w), w, Cg);
                            Cb = __ffma2_rn(make_float2(rc.bc.x, rc.bc.y), w, Cb);
                            float2 used;
                            used.x = sat(a2.x * kCullScale);
                            used.y = sat(a2.y * kCullScale);
                            const float idx1 = base1 + (float)c;
                            last = __ffma2_rn(used, __fadd2_rn(make_float2(idx1, idx1), neg2(last)), last);
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (!DUMP && !wdone) {
                wdone = __all_sync(0xffffffffu, T.x == 0.f && T.y == 0.f);
                if (wdone && lane == 0) atomicAdd((int*)sDone, 1);
            }
            if (lane == 0) {
                mbar_arrive(bar_tempty(t));
                mbar_arrive(bar_empty(s));
            }
        }
        if (!DUMP) {
            const size_t plane = (size_t)a.W * a.H;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h ? in_lo : in_up) {
                    const size_t p = (size_t)(h ? py_lo : py_up) * a.W + px;
                    const float Tf = h ? T.y + Tstop.y : T.x + Tstop.x;
                    a.image[p] = (h ? Cr.y : Cr.x) + Tf * a.bg[0];
                    a.image[plane + p] = (h ? Cg.y : Cg.x) + Tf * a.bg[1];
                    a.image[2 * plane + p] = (h ? Cb.y : Cb.x) + Tf * a.bg[2];
                    a.T_final[p] = Tf;
                    a.n_contrib[p] = (int)(h ? last.y : last.x);
                }
            }
        }
    } else if (warp == kEpiWarps) {
        // ------------------------------------------------------- producer --
        // reference pixels of the two halves and the pixel-offset box of a half
        const float xc = (float)x0 + (origin ? 0.5f : 8.0f);
        const float yc_up = (float)y0 + (origin ? 0.5f : 4.0f), yc_lo = yc_up + 8.0f;
        const float bx0 = origin ? -15.0f : -7.5f, bx1 = origin ? 0.0f : 7.5f;
        const float by0 = origin ? -7.0f : -3.5f, by1 = origin ? 0.0f : 3.5f;
        for (int k = 0;; ++k) {
            const int s = k % SS;
            const uint32_t ps = (uint32_t)(k / SS) & 1u;
            if (!mbar_wait_bounded(bar_empty(s), ps ^ 1u, tmo, sAbort)) {
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
                float vu[6], vl[6];
                Rec rc;
                if (j < n) {
                    const uint32_t g = a.ids[start + base + j];
                    const float2 m = a.mean2d[g];
                    const float A = a.conic[3 * g], B = a.conic[3 * g + 1], C = a.conic[3 * g + 2];
                    const float o = a.opac[g];
                    const float l2o = o > 0.f ? __log2f(o) : -INFINITY;
                    const float xh = m.x - xc;
                    coeff_row<TR::HALF>(A, B, C, l2o, xh, m.y - yc_up, bx0, bx1, by0, by1, vu);
                    coeff_row<TR::HALF>(A, B, C, l2o, xh, m.y - yc_lo, bx0, bx1, by0, by1, vl);
                    const float cap = fminf(l2o, kLog2AlphaMax);
                    float cr = 0.f, cg = 0.f, cb = 0.f;
                    if (a.rgb) {
                        cr = a.rgb[3 * g];
                        cg = a.rgb[3 * g + 1];
                        cb = a.rgb[3 * g + 2];
                    }
                    rc.rg = make_float4(cr, cr, cg, cg);
                    rc.bc = make_float4(cb, cb, cap, cap);
                } else {  // padding column: dead rows, no colour
#pragma unroll
                    for (int i = 0; i < 5; ++i) vu[i] = vl[i] = 0.f;
                    vu[5] = vl[5] = kDeadPower;
                    rc.rg = make_float4(0.f, 0.f, 0.f, 0.f);
                    rc.bc = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                store_coeff_row<V>(mB, j, vu);
                store_coeff_row<V>(mB, CH + j, vl);
                sRec[s * CH + j] = rc;
            }
            if (lane == 0) sN[s] = n;
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_full(s));
        }
    } else if (lane == 0) {
        // ------------------------------------------------------ MMA issue --
        int last_t = -1;
        uint32_t last_pt = 0;
        const uint32_t aA = smem_u32(sA);
        for (int k = 0;; ++k) {
            const int s = k % SS, t = k % kTStages;
            const uint32_t ps = (uint32_t)(k / SS) & 1u, pt = (uint32_t)(k / kTStages) & 1u;
            if (!mbar_wait_bounded(bar_full(s), ps, tmo, sAbort)) {
                *sAbort = 1;
                atomicOr(a.err, kErrTimeout);
                break;
            }
            if (sN[s] == 0) {
                mbar_arrive(bar_tfull(t));
                break;
            }
            if (!mbar_wait_bounded(bar_tempty(t), pt ^ 1u, tmo, sAbort)) {
                *sAbort = 1;
                atomicOr(a.err, kErrTimeout);
                break;
            }
            tc_fence_after();
            const uint32_t aB = smem_u32(sB + s * LY::B_BYTES);
#pragma unroll
            for (int ks = 0; ks < TR::KSTEPS; ++ks) {
                const uint64_t ad = smem_desc(aA + (uint32_t)(ks * 256), 128, SBO);
                const uint64_t bd = smem_desc(aB + (uint32_t)(ks * 256), 128, SBO);
                tc_mma_f16(tmem + (uint32_t)(t * 2 * CH), ad, bd, IDESC, ks > 0 ? 1u : 0u);
            }
            tc_commit(bar_tfull(t));
            tc_commit(bar_empty(s));
            last_t = t;
            last_pt = pt;
        }
        if (last_t >= 0) mbar_wait_bounded(bar_tfull(last_t), last_pt, 1000000000ull, nullptr);
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 5) tmem_dealloc(tmem, LY::TCOLS);
}

template <int V, int CH, int SS, bool DUMP>
cudaError_t launch_inst(const BlendArgs& a, int grid, cudaStream_t s) {
    constexpr int bytes = Layout<SS, CH, V>::BYTES;
    auto kern = k_blend_tc<V, CH, SS, DUMP>;
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
