// Tensor-core blending (Alg. 2, Eqs. 4-8) for sm_100-family GPUs.
//
// Persistent kernel: each CTA pulls tiles from a global queue (an atomic
// counter) until the queue is empty; the tiles of all views of the call form
// one queue.  Every 16 x 16 tile is split into an upper and a lower 16 x 8
// half; M_p (A operand, 128 x K) holds the monomials
// [xb^2, yb^2, xb yb, xb, yb, 1] of the 128 pixels of a half relative to the
// half's reference pixel and is built once per CTA.  For every chunk of CH
// splats of a tile the producer writes 2 CH coefficient rows v_g (Eq. 6):
// rows [0, CH) referred to the upper half's reference, rows [CH, 2 CH) to the
// lower half's (8 pixels further down).  One tcgen05.mma (M = 128, N = 2 CH,
// K = 16 or 32) then leaves in TMEM lane r, column j the exponent of splat j
// at upper pixel r and, at column CH + j, at lower pixel r: each epilogue
// thread owns two pixels of one lane and composites both with packed f32x2
// arithmetic.
//
// Warps: 0-3 epilogue (warp w reads TMEM lanes 32 w .. 32 w + 31), 4 producer,
// 5 MMA issue (lane 0) and TMEM owner.  The producer streams (tile, chunk)
// items through a ring of SS shared-memory stages (header, v_g rows,
// per-splat colour) across tile boundaries, so the next tile's gathers
// overlap the current tile's compositing; the MMA writes a ring of 2 TMEM
// stages.  An empty tile travels as one stage with n = 0, the end of the
// queue as n = -1.  When all four epilogue warps of a tile are
// done (every pixel stopped) the producer skips that tile's remaining chunks.
// All waits are bounded by opts.timeout_ns; on expiry the CTA records
// GS_ERR_TIMEOUT in the device error word, every role leaves its loop, the
// MMA thread commits to a drain barrier of its own and waits (bounded, 1 s)
// until every MMA it issued has completed; then TMEM is freed.
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
#include <cuda_fp8.h>

#include "internal.h"

namespace gs {
namespace tc {

constexpr int kEpiWarps = 4;
constexpr int kThreads = 192;
constexpr int kTStages = 2;
constexpr int kDoneRing = 16;  // tiles in flight between producer and epilogue < kDoneRing
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLog2AlphaMin = -7.9943534368588578f;    // log2(1/255)
constexpr float kLog2AlphaMax = -0.014499569695115089f;  // log2(0.99)
constexpr float kDeadPower = -200.0f;
constexpr float kCullScale = 68719476736.0f;    // 2^36
constexpr float kStopScale = 1099511627776.0f;  // 2^40

// Operand encoding of a variant.  K elements of a row: TERMS operand-type terms
// of v_g times PTERMS terms of the monomials, 6 each (every product of a v_g
// term with a monomial term gets its own K slot), zero-padded.  FP8: e4m3
// operands (tcgen05 kind::f8f6f4), each v_g row scaled by a power of two so
// that its largest coefficient lies in [128, 256), the monomials split into 2
// exact terms.
template <int V>
struct Traits {
    // CC: the exponent v_g . v_p by FP32 FMAs on the CUDA cores; the B stage
    // then holds each splat's two FP32 rows (12 floats) and no MMA runs
    static constexpr bool CC = (V == GS_BLEND_PERSISTENT_FP32);
    static constexpr bool FP8 = (V == GS_BLEND_TC_FP8_SPLIT);
    static constexpr int TERMS = FP8 ? 5 : (V == GS_BLEND_TC_FP16_SPLIT) ? 2 : (V == GS_BLEND_TC_BF16_SPLIT ? 3 : 1);
    static constexpr int PTERMS = FP8 ? 2 : 1;
    static constexpr int K = FP8 ? 64 : (V == GS_BLEND_TC_BF16_SPLIT) ? 32 : 16;
    static constexpr uint32_t FMT = (V == GS_BLEND_TC_BF16 || V == GS_BLEND_TC_BF16_SPLIT) ? 1u : 0u;  // e4m3: 0
    static constexpr bool HALF = (FMT == 0);
    static constexpr int ROW_BYTES = FP8 ? K : 2 * K;
    static constexpr int KSTEPS = ROW_BYTES / 32;               // one MMA consumes 32 bytes of every row
    static constexpr int SBO = (ROW_BYTES / 16) * 128;          // bytes between 8-row core-matrix groups
    static_assert(6 * TERMS * PTERMS <= K, "operand terms exceed K");
};

// FP8 term t of v_g is stored multiplied by 2^kFp8Shift[t] and the monomial
// slots it meets by 2^-kFp8Shift[t] (products unchanged): the small terms move
// up into e4m3's normal range, the monomials (>= 1/4) stay normal.
__device__ __forceinline__ float fp8_term_shift(int t) { return t >= 2 ? 16.0f : 1.0f; }

// e4m3 encoding (round to nearest, saturating) and its value
__device__ __forceinline__ uint8_t to_e4m3(float x) {
    return (uint8_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}
__device__ __forceinline__ float from_e4m3(uint8_t b) {
    const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)b, __NV_E4M3);
    return __half2float(__half(h));
}

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

// tcgen05.mma of the variant's operand kind (f16/bf16 or e4m3)
template <int V>
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    if constexpr (Traits<V>::FP8)
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    else
        tc_mma_f16(d_tmem, adesc, bdesc, idesc, accumulate);
}

// A work item of the TMA producer: one chunk of a tile (n > 0), an empty
// tile (n == 0) or the end of the queue (n < 0).
struct ProdItem {
    int tile, seq, base, n, q, vview;
    uint32_t start;
    float xc, yc;
    int pad[3];
};

constexpr int kRecStages = 4;  // TMA record stages: copies run this many chunks minus one ahead

template <int SS, int CH, int V>
struct Layout {
    static constexpr int A_BYTES = 128 * Traits<V>::ROW_BYTES;
    static constexpr int B_BYTES = 2 * CH * Traits<V>::ROW_BYTES;
    static constexpr int OFF_B = A_BYTES;
    static constexpr int OFF_REC = OFF_B + SS * B_BYTES;
    static constexpr int OFF_SCL = OFF_REC + SS * CH * (int)sizeof(Rec);  // FP8: row scales (float2 per splat)
    static constexpr int RS = kRecStages;
    static constexpr int OFF_RECT = (OFF_SCL + SS * CH * 8 + 255) / 256 * 256;  // TMA record ring (256-aligned)
    static constexpr int OFF_BAR = OFF_RECT + RS * CH * kRecBytes;
    static constexpr int NBAR = 2 * SS + 2 * kTStages + 1 + RS;  // + one drain barrier + the record stages
    static constexpr int OFF_HDR = OFF_BAR + NBAR * 8;
    static constexpr int OFF_ITEM = OFF_HDR + SS * 32;
    static constexpr int OFF_MISC = OFF_ITEM + RS * (int)sizeof(ProdItem);
    static constexpr int BYTES = OFF_MISC + 16 + 4 * kDoneRing;
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
// (xh, yh) = splat centre minus reference pixel.  fp16 operands cannot hold
// coefficients beyond 65504: if any would exceed 30000, the splat is tested
// against the half-tile's pixel-offset box (bx0..by1) and, if it cannot reach
// alpha >= 1/255 there, gets a dead row (exponent -200 everywhere); otherwise
// the coefficients are clamped (only splats far from the tile relative to
// their size reach this, and the error is stated in the design notes).
template <bool HALF>
__device__ __forceinline__ void coeff_row(float A, float B, float C, float l2o, float xh, float yh, float bx0,
                                          float bx1, float by0, float by1, float (&v)[6]) {
    const float ux = fmaf(A, xh, B * yh), uy = fmaf(B, xh, C * yh);
    const float P0 = -0.5f * fmaf(xh, ux, yh * uy);
    v[0] = -0.5f * A * kLog2e;
    v[1] = -0.5f * C * kLog2e;
    v[2] = -B * kLog2e;
    v[3] = -ux * kLog2e;
    v[4] = -uy * kLog2e;
    v[5] = fmaf(P0, kLog2e, l2o);
    if constexpr (HALF) {
        float big = 0.f;
#pragma unroll
        for (int i = 0; i < 6; ++i) big = fmaxf(big, fabsf(v[i]));
        if (big > 30000.f) {
            const float qmax = box_max_quadratic(A, B, C, xh + bx0, xh + bx1, yh + by0, yh + by1);
            if (fmaf(qmax, kLog2e, l2o) >= kLog2AlphaMin - 0.25f) {
#pragma unroll
                for (int i = 0; i < 6; ++i) v[i] = fminf(fmaxf(v[i], -30000.f), 30000.f);
            } else {
#pragma unroll
                for (int i = 0; i < 5; ++i) v[i] = 0.f;
                v[5] = kDeadPower;
            }
        }
    }
}

// Write row r of a B stage: v split into TERMS operand-type terms, each in its
// own K slots (once per monomial term), zero padding up to K.  Returns the
// factor that maps the MMA result back to v . v_p (1 unless FP8, whose rows
// are scaled by a power of two first).
template <int V>
__device__ __forceinline__ float store_coeff_row(uint8_t* mB, int r, const float (&v)[6]) {
    using TR = Traits<V>;
    if constexpr (TR::FP8) {
        float big = 0.f;
#pragma unroll
        for (int i = 0; i < 6; ++i) big = fmaxf(big, fabsf(v[i]));
        // 2^E <= big < 2^(E+1); scale 2^(7-E) puts the largest coefficient in [128, 256)
        const int E = big > 0.f ? ((__float_as_int(big) >> 23) & 0xff) - 127 : 0;
        const int sh = max(-100, min(100, 7 - E));
        const float scale = __int_as_float((127 + sh) << 23), inv = __int_as_float((127 - sh) << 23);
        uint8_t terms[TR::TERMS][6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            float rem = v[i] * scale;
#pragma unroll
            for (int t = 0; t < TR::TERMS; ++t) {
                const float sh = fp8_term_shift(t);
                terms[t][i] = to_e4m3(rem * sh);
                rem -= from_e4m3(terms[t][i]) / sh;
            }
        }
        // slot k = (t * PTERMS + s) * 6 + i holds term t of v_i (for every monomial term s)
#pragma unroll
        for (int kc = 0; kc < TR::ROW_BYTES / 16; ++kc) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t word = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int k = kc * 16 + q * 4 + b;
                    const uint32_t e = (k < 6 * TR::TERMS * TR::PTERMS)
                                           ? terms[k / (6 * TR::PTERMS)][k % 6] : 0u;
                    word |= e << (8 * b);
                }
                w[q] = word;
            }
            *reinterpret_cast<uint4*>(mB + (r >> 3) * TR::SBO + kc * 128 + (r & 7) * 16) =
                make_uint4(w[0], w[1], w[2], w[3]);
        }
        return inv;
    } else {
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
        return 1.0f;
    }
}

// The CUDA-core variant's B stage: splat j's two FP32 rows, 12 floats at 48 j
// (upper row 0..5, lower row 6..11).
__device__ __forceinline__ void store_cc_rows(uint8_t* mB, int j, const float (&vu)[6], const float (&vl)[6]) {
    float4* d = reinterpret_cast<float4*>(mB + 48 * j);
    d[0] = make_float4(vu[0], vu[1], vu[2], vu[3]);
    d[1] = make_float4(vu[4], vu[5], vl[0], vl[1]);
    d[2] = make_float4(vl[2], vl[3], vl[4], vl[5]);
}

// Row `row` of M_p, the pixel-monomial operand: the 6 monomials of the pixel
// (offsets xb, yb from its half's reference), in the slot order of
// store_coeff_row (for FP8 each monomial as 2 exact e4m3 terms).
template <int V>
__device__ __forceinline__ void store_mp_row(uint8_t* sA, int row, float xb, float yb) {
    using TR = Traits<V>;
    const float vp[6] = {xb * xb, yb * yb, xb * yb, xb, yb, 1.0f};
    if constexpr (TR::FP8) {
        float pv[2][6];  // the 2 exact e4m3 terms of each monomial
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            pv[0][i] = from_e4m3(to_e4m3(vp[i]));
            pv[1][i] = vp[i] - pv[0][i];
        }
#pragma unroll
        for (int kc = 0; kc < TR::ROW_BYTES / 16; ++kc) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t word = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int k = kc * 16 + q * 4 + b;
                    const uint32_t e = (k < 6 * TR::TERMS * TR::PTERMS)
                                           ? to_e4m3(pv[(k / 6) % TR::PTERMS][k % 6] / fp8_term_shift(k / (6 * TR::PTERMS)))
                                           : 0u;
                    word |= e << (8 * b);
                }
                w[q] = word;
            }
            *reinterpret_cast<uint4*>(sA + (row >> 3) * TR::SBO + kc * 128 + (row & 7) * 16) =
                make_uint4(w[0], w[1], w[2], w[3]);
        }
    } else {
#pragma unroll
        for (int kc = 0; kc < TR::K / 8; ++kc) {
            uint16_t e[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int k = kc * 8 + i;
                e[i] = (k < 6 * TR::TERMS) ? to_op<TR::HALF>(vp[k % 6]) : (uint16_t)0;
            }
            store_row_chunk<V>(sA, row, kc, e);
        }
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

// Work item of one pipeline stage.  n > 0: chunk [base, base + n) of the
// tile's list; n == 0: the tile is empty; n < 0: end of the queue.
struct StageHdr {
    int tile;  // global tile id
    int seq;   // this CTA's running tile number
    int base;  // list position of the chunk's first splat
    int n;
    int slot;  // queue position of the tile (gs_tile_power output row)
    int pad[3];
};


__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

template <int V, int CH, int SS, bool DUMP>
__global__ void __launch_bounds__(kThreads, 4) k_blend_tc(const __grid_constant__ BlendArgs a) {
    using TR = Traits<V>;
    using LY = Layout<SS, CH, V>;
    constexpr int K = TR::K;
    constexpr int SBO = TR::SBO;
    constexpr uint32_t IDESC = idesc_f16(TR::FMT, 128, 2 * CH);
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sA = smem;
    uint8_t* sB = smem + LY::OFF_B;
    Rec* sRec = reinterpret_cast<Rec*>(smem + LY::OFF_REC);
    float2* sScl = reinterpret_cast<float2*>(smem + LY::OFF_SCL);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + LY::OFF_BAR);
    StageHdr* sHdr = reinterpret_cast<StageHdr*>(smem + LY::OFF_HDR);
    uint32_t* sTmem = reinterpret_cast<uint32_t*>(smem + LY::OFF_MISC);
    volatile int* sAbort = reinterpret_cast<volatile int*>(smem + LY::OFF_MISC + 4);
    volatile int* sDoneRing = reinterpret_cast<volatile int*>(smem + LY::OFF_MISC + 16);
    auto bar_full = [&](int s) { return smem_u32(bars + s); };
    auto bar_empty = [&](int s) { return smem_u32(bars + SS + s); };
    auto bar_tfull = [&](int t) { return smem_u32(bars + 2 * SS + t); };
    auto bar_tempty = [&](int t) { return smem_u32(bars + 2 * SS + kTStages + t); };
    const uint32_t bar_drain = smem_u32(bars + 2 * SS + 2 * kTStages);
    auto bar_rec = [&](int r) { return smem_u32(bars + 2 * SS + 2 * kTStages + 1 + r); };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_items = a.total_tiles;  // gs_tile_power: the number of listed tiles
    const bool origin = a.ref_origin != 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < SS; ++s) {
            mbar_init(bar_full(s), 1);
            mbar_init(bar_empty(s), 1 + kEpiWarps);
        }
        for (int t = 0; t < kTStages; ++t) {
            mbar_init(bar_tfull(t), 1);
            mbar_init(bar_tempty(t), kEpiWarps);
        }
        mbar_init(bar_drain, 1);
        for (int r = 0; r < LY::RS; ++r) mbar_init(bar_rec(r), 1);
        *sAbort = 0;
        mbar_fence_init();
    }
    // pixel matrix M_p of a 16 x 8 half-tile (A operand)
    for (int row = threadIdx.x; row < 128; row += kThreads) {
        const float xb = origin ? -(float)(row & 15) : 7.5f - (float)(row & 15);
        const float yb = origin ? -(float)(row >> 4) : 3.5f - (float)(row >> 4);
        store_mp_row<V>(sA, row, xb, yb);
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

    if (warp < kEpiWarps) {
        // ------------------------------------------------------- epilogue --
        const int r = warp * 32 + lane;  // accumulator lane: pixel r of each half
        // this lane's pixel monomials (the same in both halves), as M_p holds them
        float mp[5];
        {
            const float xb = origin ? -(float)(r & 15) : 7.5f - (float)(r & 15);
            const float yb = origin ? -(float)(r >> 4) : 3.5f - (float)(r >> 4);
            mp[0] = xb * xb;
            mp[1] = yb * yb;
            mp[2] = xb * yb;
            mp[3] = xb;
            mp[4] = yb;
        }
        int cur_seq = -1, slot = 0;
        int px = 0, py_up = 0, W = 0, H = 0;
        bool in_up = false, in_lo = false, wdone = true;
        long long pix_off = 0;
        float2 T = make_float2(0.f, 0.f), Tstop = T, last = T, Cr = T, Cg = T, Cb = T;
        for (int k = 0;; ++k) {
            const int s = k % SS, t = k % kTStages;
            const uint32_t ps = (uint32_t)(k / SS) & 1u, pt = (uint32_t)(k / kTStages) & 1u;
            if (!mbar_wait_bounded(bar_tfull(t), pt, tmo, sAbort) || !mbar_wait_bounded(bar_full(s), ps, tmo, sAbort)) {
                *sAbort = 1;
                atomicOr(a.err, kErrTimeout);
                break;
            }
            const StageHdr hd = sHdr[s];
            if (hd.seq != cur_seq) {
                if (!DUMP && cur_seq >= 0) {  // write the finished tile's pixels
                    const size_t plane = (size_t)W * H;
                    float* img = a.image + 3 * pix_off;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (h ? in_lo : in_up) {
                            const size_t p = (size_t)(py_up + 8 * h) * W + px;
                            const float Tf = h ? T.y + Tstop.y : T.x + Tstop.x;
                            img[p] = (h ? Cr.y : Cr.x) + Tf * a.bg[0];
                            img[plane + p] = (h ? Cg.y : Cg.x) + Tf * a.bg[1];
                            img[2 * plane + p] = (h ? Cb.y : Cb.x) + Tf * a.bg[2];
                            a.T_final[pix_off + p] = Tf;
                            a.n_contrib[pix_off + p] = (int)(h ? last.y : last.x);
                        }
                    }
                }
                if (hd.n < 0) break;
                cur_seq = hd.seq;
                const int v = view_of(a, hd.tile);
                const ViewDesc vd = a.views[v];
                const int lt = hd.tile - vd.tile_begin;
                W = vd.W;
                H = vd.H;
                pix_off = vd.pix_off;
                px = (lt % vd.tiles_x) * kTile + (r & 15);
                py_up = (lt / vd.tiles_x) * kTile + (r >> 4);
                in_up = px < W && py_up < H;
                in_lo = px < W && py_up + 8 < H;
                slot = hd.slot;
                T = make_float2(in_up || DUMP ? 1.f : 0.f, in_lo || DUMP ? 1.f : 0.f);
                Tstop = last = Cr = Cg = Cb = make_float2(0.f, 0.f);
                wdone = DUMP ? false : __all_sync(0xffffffffu, T.x == 0.f && T.y == 0.f);
                if (!DUMP && wdone && lane == 0) atomicAdd((int*)&sDoneRing[cur_seq % kDoneRing], 1);
            }
            tc_fence_after();
            const int n = hd.n;
            const int base = hd.base;
            if (n > 0 && !wdone) {
                const uint32_t tb = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * 2 * CH);
                const Rec* rec = sRec + s * CH;
#pragma unroll 1
                for (int c0 = 0; c0 < n; c0 += 16) {
                    // every pixel of this warp has stopped: the chunk's later splats change nothing
                    if (!DUMP && c0 > 0 && __all_sync(0xffffffffu, T.x == 0.f && T.y == 0.f)) break;
                    uint32_t vu[16], vl[16];
                    // CC: Eq. 6 on the CUDA cores, column by column below (both pixels of
                    // the lane share their monomials)
                    const float* rows = reinterpret_cast<const float*>(sB + s * LY::B_BYTES) + (size_t)c0 * 12;
                    auto cc_power = [&](int c) {
                        const float4 a0 = *reinterpret_cast<const float4*>(rows + 12 * c);
                        const float4 a1 = *reinterpret_cast<const float4*>(rows + 12 * c + 4);
                        const float4 a2 = *reinterpret_cast<const float4*>(rows + 12 * c + 8);
                        float2 p = __fmul2_rn(make_float2(a0.x, a1.z), make_float2(mp[0], mp[0]));
                        p = __ffma2_rn(make_float2(a0.y, a1.w), make_float2(mp[1], mp[1]), p);
                        p = __ffma2_rn(make_float2(a0.z, a2.x), make_float2(mp[2], mp[2]), p);
                        p = __ffma2_rn(make_float2(a0.w, a2.y), make_float2(mp[3], mp[3]), p);
                        p = __ffma2_rn(make_float2(a1.x, a2.z), make_float2(mp[4], mp[4]), p);
                        return __fadd2_rn(make_float2(a1.y, a2.w), p);
                    };
                    if constexpr (!TR::CC) {
                        tmem_ld_32x32b_x16(tb + (uint32_t)c0, vu);
                        tmem_ld_32x32b_x16(tb + (uint32_t)(CH + c0), vl);
                        tmem_ld_wait();
                    }
                    if constexpr (TR::FP8) {  // undo the per-row scaling of the e4m3 operands
                        const float2* scl = sScl + s * CH;
#pragma unroll
                        for (int c = 0; c < 16; ++c) {
                            const float2 z = __fmul2_rn(make_float2(__uint_as_float(vu[c]), __uint_as_float(vl[c])),
                                                        scl[c0 + c]);
                            vu[c] = __float_as_uint(z.x);
                            vl[c] = __float_as_uint(z.y);
                        }
                    }
                    if constexpr (DUMP) {
#pragma unroll
                        for (int c = 0; c < 16; ++c) {
                            const int j = c0 + c;
                            if (j < n) {
                                float* o = a.dump + ((size_t)slot * a.max_len + (size_t)base + j) * 256;
                                o[r] = __uint_as_float(vu[c]);
                                o[r + 128] = __uint_as_float(vl[c]);
                            }
                        }
                    } else {
                        const float base1 = (float)(base + c0 + 1);
#pragma unroll
                        for (int c = 0; c < 16; ++c) {
                            const Rec rc = rec[c0 + c];
                            float2 pw;
                            if constexpr (TR::CC) pw = cc_power(c);
                            else pw = make_float2(__uint_as_float(vu[c]), __uint_as_float(vl[c]));
                            float2 al;
                            al.x = ex2_approx(fminf(pw.x, rc.bc.z));
                            al.y = ex2_approx(fminf(pw.y, rc.bc.w));
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
            if (lane == 0) mbar_arrive(bar_tempty(t));
            if (!DUMP && !wdone) {
                wdone = __all_sync(0xffffffffu, T.x == 0.f && T.y == 0.f);
                if (wdone && lane == 0) atomicAdd((int*)&sDoneRing[cur_seq % kDoneRing], 1);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_empty(s));
        }
    } else if (warp == kEpiWarps && !DUMP && a.use_rec) {
        // ------------------------------------------------ producer (TMA) --
        // Three stages per chunk, as in Sec. 3.4, each a step ahead of the
        // next: (1) the work item (tile ticket, its range, the chunk's ids),
        // (2) the chunk's splat records gathered into a shared-memory ring by
        // TMA (tile::gather4: four 64-byte rows per copy) RS - 1 items before
        // (3) its v_g rows are built from that ring into the B stage.  The
        // copies of the next chunks, across tile boundaries, are in flight
        // while this chunk's rows are built.
        constexpr int RS = LY::RS;
        ProdItem* sIt = reinterpret_cast<ProdItem*>(smem + LY::OFF_ITEM);
        const float* sRecT = reinterpret_cast<const float*>(smem + LY::OFF_RECT);
        const float bx0 = origin ? -15.0f : -7.5f, bx1 = origin ? 0.0f : 7.5f;
        const float by0 = origin ? -7.0f : -3.5f, by1 = origin ? 0.0f : 3.5f;
        // generator state (warp-uniform)
        int g_seq = -1, g_tile = 0, g_q = 0, g_view = 0, g_len = 0, g_nch = 0, g_c = 0;
        uint32_t g_start = 0;
        float g_xc = 0.f, g_yc = 0.f;
        bool g_end = false;
        auto gen_next = [&]() -> ProdItem {
            for (;;) {
                if (g_end) return ProdItem{0, -2, 0, -1, g_q, 0, 0u, 0.f, 0.f, {0, 0, 0}};
                // the next chunk of this tile, unless every pixel of the tile has stopped
                if (g_c < g_nch && !(g_c > 0 && sDoneRing[g_seq % kDoneRing] >= kEpiWarps)) break;
                int q = 0;
                if (lane == 0) q = (int)atomicAdd(a.queue, 1u);
                q = __shfl_sync(0xffffffffu, q, 0);
                g_q = q;
                if (q >= n_items) {
                    g_end = true;
                    continue;
                }
                ++g_seq;
                g_tile = tile_at(a, q * a.shard_count + a.shard_index);
                g_start = a.ranges[2 * g_tile];
                const uint32_t stop = a.ranges[2 * g_tile + 1];
                g_len = stop > g_start ? (int)(stop - g_start) : 0;
                g_view = view_of(a, g_tile);
                const ViewDesc vd = a.views[g_view];
                const int lt = g_tile - vd.tile_begin;
                g_xc = (float)((lt % vd.tiles_x) * kTile) + (origin ? 0.5f : 8.0f);
                g_yc = (float)((lt / vd.tiles_x) * kTile) + (origin ? 0.5f : 4.0f);
                g_nch = max(1, (g_len + CH - 1) / CH);
                g_c = 0;
                if (lane == 0) sDoneRing[g_seq % kDoneRing] = 0;
            }
            const int base = g_c * CH;
            ++g_c;
            return ProdItem{g_tile, g_seq, base, g_len > 0 ? min(CH, g_len - base) : 0, g_q, g_view, g_start,
                            g_xc, g_yc, {0, 0, 0}};
        };
        // stage (2) for an item in record stage rs: the ids, then ceil(n / 4)
        // gather copies (rows past n repeat id 0, a row of the table); an item
        // without splats just completes the stage's phase
        auto issue = [&](const ProdItem& it, int rs) {
            if (it.n <= 0) {
                if (lane == 0) mbar_arrive(bar_rec(rs));
                return;
            }
            const uint32_t g = lane < it.n ? a.ids[it.start + it.base + lane] : 0u;
            const int src = 4 * (lane & 7);
            const uint32_t g0 = __shfl_sync(0xffffffffu, g, src), g1 = __shfl_sync(0xffffffffu, g, src + 1);
            const uint32_t g2 = __shfl_sync(0xffffffffu, g, src + 2), g3 = __shfl_sync(0xffffffffu, g, src + 3);
            const int ng = (it.n + 3) >> 2;
            if (lane == 0) mbar_arrive_expect_tx(bar_rec(rs), (uint32_t)(ng * 4 * kRecBytes));
            __syncwarp();
            if (lane < ng)
                tma_gather4(smem_u32(sRecT + ((size_t)rs * CH + 4 * lane) * kRecFloats), &a.rec_map, 0, g0, g1, g2,
                            g3, bar_rec(rs));
        };
        int k = 0, ri = 0, wi = 0;
        bool gen_done = false, quit = false;
        unsigned long long issued = 0;
        for (; ri < RS - 1 && !gen_done; ++ri) {
            const ProdItem it = gen_next();
            __syncwarp();
            if (lane == 0) sIt[ri % RS] = it;
            issue(it, ri % RS);
            gen_done = it.n < 0;
        }
        while (!quit) {
            if (!gen_done) {  // keep RS - 1 items in flight
                const ProdItem it = gen_next();
                __syncwarp();
                if (lane == 0) sIt[ri % RS] = it;
                issue(it, ri % RS);
                gen_done = it.n < 0;
                ++ri;
            }
            __syncwarp();
            const ProdItem it = sIt[wi % RS];
            const int rs = wi % RS;
            if (!mbar_wait_bounded(bar_rec(rs), (uint32_t)(wi / RS) & 1u, tmo, sAbort)) {
                *sAbort = 1;
                atomicOr(a.err, kErrTimeout);
                break;
            }
            ++wi;
            // a later chunk of a tile whose pixels have all stopped is dropped
            if (it.n > 0 && it.base > 0 && sDoneRing[it.seq % kDoneRing] >= kEpiWarps) continue;
            const int s = k % SS;
            const uint32_t ps = (uint32_t)(k / SS) & 1u;
            if (!mbar_wait_bounded(bar_empty(s), ps ^ 1u, tmo, sAbort)) {
                *sAbort = 1;
                atomicOr(a.err, kErrTimeout);
                break;
            }
            if (*sAbort) break;
            const int n = it.n;
            if (n > 0) {
                issued += (unsigned long long)n;
                uint8_t* mB = sB + s * LY::B_BYTES;
                const float yc_lo = it.yc + 8.0f;
                for (int j = lane; j < CH; j += 32) {
                    float vu[6], vl[6];
                    Rec rc;
                    if (j < n) {
                        const float4* rp = reinterpret_cast<const float4*>(sRecT + ((size_t)rs * CH + j) * kRecFloats);
                        const float4 r0 = rp[0], r1 = rp[1], r2 = rp[2];
                        const float xh = r0.x - it.xc;
                        coeff_row<TR::HALF && !TR::CC>(r0.z, r0.w, r1.x, r1.y, xh, r0.y - it.yc, bx0, bx1, by0, by1, vu);
                        coeff_row<TR::HALF && !TR::CC>(r0.z, r0.w, r1.x, r1.y, xh, r0.y - yc_lo, bx0, bx1, by0, by1, vl);
                        rc.rg = make_float4(r2.x, r2.x, r2.y, r2.y);
                        rc.bc = make_float4(r2.z, r2.z, r1.z, r1.z);
                    } else {  // padding column: dead rows, no colour
#pragma unroll
                        for (int i = 0; i < 5; ++i) vu[i] = vl[i] = 0.f;
                        vu[5] = vl[5] = kDeadPower;
                        rc.rg = make_float4(0.f, 0.f, 0.f, 0.f);
                        rc.bc = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                    if constexpr (TR::CC) {
                        store_cc_rows(mB, j, vu, vl);
                    } else {
                        const float su = store_coeff_row<V>(mB, j, vu);
                        const float sl = store_coeff_row<V>(mB, CH + j, vl);
                        if constexpr (TR::FP8) sScl[s * CH + j] = make_float2(su, sl);
                    }
                    sRec[s * CH + j] = rc;
                }
            }
            if (lane == 0) sHdr[s] = StageHdr{it.tile, n < 0 ? -2 : it.seq, it.base, n, it.q, {0, 0, 0}};
            // orders this warp's shared-memory reads and writes before the MMA's
            // reads and before the next TMA copies into the record ring
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_full(s));
            ++k;
            if (n < 0) quit = true;
        }
        // copies still in flight (after a timeout) land before the block leaves
        for (; wi < ri; ++wi) mbar_wait_bounded(bar_rec(wi % RS), (uint32_t)(wi / RS) & 1u, 1000000000ull, nullptr);
        if (lane == 0 && a.issued != nullptr && issued) atomicAdd(a.issued, issued * 256ull);
    } else if (warp == kEpiWarps) {
        // ------------------------------------------------------- producer --
        int k = 0;
        bool quit = false;
        unsigned long long issued = 0;  // splats of the chunks this block issued
        // The next tile's queue item is taken when a tile starts and its range
        // read once the tile's first chunk is out, so those dependent loads
        // overlap the chunk work instead of preceding the next tile.
        auto fetch = [&](int qq, int& tl, uint32_t& st, int& ln) {
            tl = DUMP ? a.tiles[qq] : tile_at(a, qq * a.shard_count + a.shard_index);
            st = a.ranges[2 * tl];
            const uint32_t sp = a.ranges[2 * tl + 1];
            ln = sp > st ? (int)(sp - st) : 0;
        };
        int q_next = 0, nt_tile = 0, nt_len = 0;
        uint32_t nt_start = 0;
        if (lane == 0) q_next = (int)atomicAdd(a.queue, 1u);
        q_next = __shfl_sync(0xffffffffu, q_next, 0);
        if (q_next < n_items) fetch(q_next, nt_tile, nt_start, nt_len);
        for (int seq = 0; !quit; ++seq) {
            const int q = q_next;
            const bool end = q >= n_items;
            int tile = 0, len = 0, vview = 0;
            uint32_t start = 0;
            float xc = 0.f, yc_up = 0.f;
            if (!end && lane == 0) q_next = (int)atomicAdd(a.queue, 1u);  // used after this tile's first chunk
            if (!end) {
                tile = nt_tile;
                start = nt_start;
                len = nt_len;
                if (DUMP && len > a.max_len) len = a.max_len;
                vview = view_of(a, tile);
                const ViewDesc vd = a.views[vview];
                const int lt = tile - vd.tile_begin;
                xc = (float)((lt % vd.tiles_x) * kTile) + (origin ? 0.5f : 8.0f);
                yc_up = (float)((lt / vd.tiles_x) * kTile) + (origin ? 0.5f : 4.0f);
                if (lane == 0) sDoneRing[seq % kDoneRing] = 0;
            }
            const float yc_lo = yc_up + 8.0f;
            const float bx0 = origin ? -15.0f : -7.5f, bx1 = origin ? 0.0f : 7.5f;
            const float by0 = origin ? -7.0f : -3.5f, by1 = origin ? 0.0f : 3.5f;
            const int nch = end ? 1 : max(1, (len + CH - 1) / CH);
            for (int c = 0; c < nch; ++c) {
                const int s = k % SS;
                const uint32_t ps = (uint32_t)(k / SS) & 1u;
                if (!mbar_wait_bounded(bar_empty(s), ps ^ 1u, tmo, sAbort)) {
                    *sAbort = 1;
                    atomicOr(a.err, kErrTimeout);
                    quit = true;
                    break;
                }
                if (*sAbort) {
                    quit = true;
                    break;
                }
                // every pixel of this tile has stopped: skip its remaining chunks
                if (!DUMP && c > 0 && sDoneRing[seq % kDoneRing] >= kEpiWarps) break;
                const int base = c * CH;
                const int n = end ? -1 : min(CH, len - base);
                if (n > 0) {
                    issued += (unsigned long long)n;
                    uint8_t* mB = sB + s * LY::B_BYTES;
                    for (int j = lane; j < CH; j += 32) {
                        float vu[6], vl[6];
                        Rec rc;
                        if (j < n) {
                            const uint32_t g = a.ids[start + base + j];
                            const float2 m = a.mean2d[g];
                            const float A = a.conic[3 * g], B = a.conic[3 * g + 1], C = a.conic[3 * g + 2];
                            const float o = a.opac[g - (uint32_t)(vview * a.n_per_view)];
                            const float l2o = o > 0.f ? __log2f(o) : -INFINITY;
                            const float xh = m.x - xc;
                            coeff_row<TR::HALF && !TR::CC>(A, B, C, l2o, xh, m.y - yc_up, bx0, bx1, by0, by1, vu);
                            coeff_row<TR::HALF && !TR::CC>(A, B, C, l2o, xh, m.y - yc_lo, bx0, bx1, by0, by1, vl);
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
                        if constexpr (TR::CC) {
                            store_cc_rows(mB, j, vu, vl);
                        } else {
                            const float su = store_coeff_row<V>(mB, j, vu);
                            const float sl = store_coeff_row<V>(mB, CH + j, vl);
                            if constexpr (TR::FP8) sScl[s * CH + j] = make_float2(su, sl);
                        }
                        sRec[s * CH + j] = rc;
                    }
                }
                if (lane == 0) sHdr[s] = StageHdr{tile, end ? -2 : seq, base, n, q, {0, 0, 0}};
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_full(s));
                ++k;
                if (c == 0 && !end) {  // the next tile's range, while this tile's chunks are consumed
                    q_next = __shfl_sync(0xffffffffu, q_next, 0);
                    if (q_next < n_items) fetch(q_next, nt_tile, nt_start, nt_len);
                }
            }
            if (end) quit = true;
        }
        // issued pairs: every chunk is evaluated at all 256 pixels of its tile
        if (!DUMP && lane == 0 && a.issued != nullptr && issued) atomicAdd(a.issued, issued * 256ull);
    } else if (lane == 0) {
        // ------------------------------------------------------ MMA issue --
        const uint32_t aA = smem_u32(sA);
        for (int k = 0;; ++k) {
            const int s = k % SS, t = k % kTStages;
            const uint32_t ps = (uint32_t)(k / SS) & 1u, pt = (uint32_t)(k / kTStages) & 1u;
            if (!mbar_wait_bounded(bar_full(s), ps, tmo, sAbort)) {
                *sAbort = 1;
                atomicOr(a.err, kErrTimeout);
                break;
            }
            // the TMEM stage must be free even for a stage without an MMA, so
            // that tfull[t] never runs two phases ahead of a waiting epilogue warp
            if (!mbar_wait_bounded(bar_tempty(t), pt ^ 1u, tmo, sAbort)) {
                *sAbort = 1;
                atomicOr(a.err, kErrTimeout);
                break;
            }
            const int n = sHdr[s].n;
            if (n <= 0) {
                mbar_arrive(bar_tfull(t));
                if (n < 0) break;
                mbar_arrive(bar_empty(s));
                continue;
            }
            if constexpr (TR::CC) {  // the epilogue contracts the rows itself
                mbar_arrive(bar_tfull(t));
                mbar_arrive(bar_empty(s));
                continue;
            }
            tc_fence_after();
            const uint32_t aB = smem_u32(sB + s * LY::B_BYTES);
#pragma unroll
            for (int ks = 0; ks < TR::KSTEPS; ++ks) {
                const uint64_t ad = smem_desc(aA + (uint32_t)(ks * 256), 128, SBO);
                const uint64_t bd = smem_desc(aB + (uint32_t)(ks * 256), 128, SBO);
                tc_mma<V>(tmem + (uint32_t)(t * 2 * CH), ad, bd, IDESC, ks > 0 ? 1u : 0u);
            }
            tc_commit(bar_tfull(t));
            tc_commit(bar_empty(s));
        }
        // every MMA this thread issued has finished before TMEM is freed (a
        // fresh barrier: no phase of another stage can be mistaken for it)
        tc_commit(bar_drain);
        mbar_wait_bounded(bar_drain, 0, 1000000000ull, nullptr);
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 5) tmem_dealloc(tmem, LY::TCOLS);
}

// Persistent grid: as many CTAs as fit on the GPU at once, from the kernel's
// registers, shared memory and threads and the SM's 512 TMEM columns.
template <int V, int CH, int SS, bool DUMP>
cudaError_t launch_inst(const BlendArgs& a, int items, cudaStream_t s) {
    using LY = Layout<SS, CH, V>;
    constexpr int bytes = LY::BYTES;
    auto kern = k_blend_tc<V, CH, SS, DUMP>;
    static std::mutex mu;
    static LaunchShape cache;
    LaunchShape sh;
    const cudaError_t es = cached_shape(mu, cache, sh, [&](LaunchShape& r) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
        int dev = 0, smem_sm = 0;
        cudaFuncAttributes fa{};
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&r.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
            return e;
        if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
        // registers are granted per warp in units of 256
        const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
        const int by_regs = 65536 / (regs_warp * (kThreads / 32));
        const int by_smem = smem_sm / (bytes + (int)fa.sharedSizeBytes + 1024);
        const int by_threads = 2048 / kThreads;
        const int by_tmem = (int)(512 / LY::TCOLS);
        r.per_sm = by_regs;
        if (by_smem < r.per_sm) r.per_sm = by_smem;
        if (by_threads < r.per_sm) r.per_sm = by_threads;
        if (by_tmem < r.per_sm) r.per_sm = by_tmem;
        if (r.per_sm < 1) r.per_sm = 1;
        return cudaSuccess;
    });
    if (es != cudaSuccess) return es;
    const int grid = items < sh.per_sm * sh.sms ? (items > 0 ? items : 1) : sh.per_sm * sh.sms;
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
template <>
cudaError_t launch_variant<5>(const BlendArgs&, int, int, bool, int, cudaStream_t);
template <>
cudaError_t launch_variant<6>(const BlendArgs&, int, int, bool, int, cudaStream_t);

}  // namespace tc
}  // namespace gs
