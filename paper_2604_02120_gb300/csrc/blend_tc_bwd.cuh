// Gradient of the tensor-core blend (the backward pass of Alg. 2).
//
// Same persistent structure as the forward kernel: warps 0-3 work on pixels
// (warp w owns TMEM lanes 32 w .. 32 w + 31; thread r holds pixel r of the
// tile's upper 16 x 8 half and pixel r of the lower half), warp 4 produces
// chunks of CH = 16 splats from the global tile queue, warp 5 issues the MMAs.
// Two MMAs per chunk:
//  1. exponents, exactly as in the forward pass (Eq. 6): D1 (128 pixels x 32)
//     = M_p (128 x K) . [v_g of the 16 splats for the upper and the lower
//     reference pixel], so the backward pass recomputes the forward's alpha;
//  2. the sums over pixels that make up each splat's gradient: every pixel
//     thread writes two per-(splat, pixel) values, the exponent gradient
//     dL/dpower (fp16 hi + lo) and the blending weight w = alpha T (fp16),
//     into A2 (96 rows = dpow {upper, lower half} x {hi, lo} x 16 splats and
//     w {upper, lower} x 16 splats, K = the 128 pixels of a half, stored
//     MN-major so that a thread writes 8 splats of its pixel with one 16-byte
//     store), and D2 (128 x 32) = A2 . B2 where B2 holds per pixel the
//     monomials [xb^2, yb^2, xb yb, xb, yb, 1] of Eq. 6 (exact in fp16) and
//     the pixel's dL/dimage (hi + lo, separately for each half).  Row
//     (dpow, h, s, j) of D2 then holds sum_p dpow m_p for splat j over half
//     h, from which the conic, mean and opacity gradients follow by the chain
//     rule; row (w, h, j) holds sum_p w dL/dC_p, the colour gradient.  The MMA
//     runs with M = 128: rows 96..127 of D2 read past the 96 rows (the next
//     8-pixel group, or the buffer's padding) and are ignored.
//
// Per pixel the splats are visited back to front (chunks in reverse order,
// splats inside a chunk from last to first), starting from T_final and the
// background: for each splat j < n_contrib that passes the 1/255 test,
//   T_j = T_{j+1} / (1 - a_j),  w_j = a_j T_j,
//   dL/da_j = T_j (c_j . g - S_j . g),  S_{j-1} . g = S_j . g + a_j (c_j . g - S_j . g)
// (S = the colour behind splat j, starting at the background), and
// dL/dpower = a dL/da (0 where alpha is clamped at 0.99), dL/do = sum dpow / o.
// Scaling keeps the fp16 operands in range: dL/dimage is multiplied by
// 2^(-E) with 2^E the largest |dL/dimage| of the tile, T by 2^12; the sums
// are scaled back in the finishing step.
//
// A2 and D2 are double buffered: chunk c writes A2[c % 2] while the MMA of
// chunk c - 1 runs, and the finishing step of chunk c - 1 (reading D2, chain
// rule, atomics) follows chunk c's stores, so the MMA's latency is hidden
// behind a whole chunk.  At a new tile the pending chunk is finished first
// (B2 changes).  Each epilogue warp finishes its own rows, so the four warps
// never wait for one another.  All waits are bounded by
// opts.timeout_ns as in the forward kernel.
#pragma once

#include "blend_tc.cuh"

namespace gs {
namespace tc {

constexpr int kBwdChunk = 16;
// Built depths of the shared-memory ring: 6 (fp16 operands: the deepest that
// keeps 3 blocks per SM, 75.9 KB each), 3 (bf16 and FP8 rows are twice as
// wide: 76.4 KB, the deepest that keeps 3 blocks per SM for them), 4 and 2.
constexpr int kBwdStagesBuilt[4] = {2, 3, 4, 6};
template <int V>
constexpr int bwd_default_stages() {
    return (V == GS_BLEND_TC_BF16_SPLIT || V == GS_BLEND_TC_FP8_SPLIT) ? 3 : 6;
}
constexpr float kTScale = 4096.0f;  // 2^12

__device__ __forceinline__ void tmem_ld_32x32b_x8(uint32_t taddr, uint32_t (&v)[8]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
        : "r"(taddr));
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Per-splat data of the finishing step.
struct alignas(16) Fin {
    uint32_t g;     // item index (0xffffffff: padding)
    uint32_t og;    // opacity index
    float xh, yh;   // splat centre minus the upper half's reference pixel
    float A, B, C;  // conic
    float inv_o;    // 1 / opacity
};

// Stage header of the backward pipeline.
struct BwdHdr {
    int tile, seq, base, n;  // n > 0 chunk, 0 nothing to do for the tile, < 0 end
    float gscale;            // 2^(-E-12): dL/dimage scale for the pixel arithmetic
    float bscale;            // 2^(-E): dL/dimage scale in B2
    float undp, uncol;       // 2^E, 2^(E-12): scale of the D2 sums back
};

template <int SS, int V>
struct BwdLayout {
    static constexpr int CH = kBwdChunk;
    static constexpr int A2_ROWS = 96;
    static constexpr int A2_LBO = A2_ROWS / 8 * 128;            // bytes per 8-pixel group: 1536
    static constexpr int A2_BYTES = 16 * A2_LBO + 512;           // + what the M = 128 MMA reads past row 96
    static constexpr int B2_BYTES = 32 * 128 * 2;   // 32 columns x 128 pixels, fp16
    static constexpr int A1_BYTES = 128 * Traits<V>::ROW_BYTES;
    static constexpr int B1_BYTES = 2 * CH * Traits<V>::ROW_BYTES;
    static constexpr int OFF_A2 = 0;
    static constexpr int OFF_B2 = OFF_A2 + 2 * A2_BYTES;
    static constexpr int OFF_A1 = OFF_B2 + B2_BYTES;
    static constexpr int OFF_B1 = OFF_A1 + A1_BYTES;
    static constexpr int OFF_REC = OFF_B1 + SS * B1_BYTES;
    static constexpr int OFF_SCL = OFF_REC + SS * CH * (int)sizeof(Rec);  // FP8 only: row scales
    static constexpr int OFF_FIN = OFF_SCL + (Traits<V>::FP8 ? SS * CH * 8 : 0);
    static constexpr int OFF_BAR = OFF_FIN + SS * CH * (int)sizeof(Fin);
    // full[SS], empty[SS], tfull[2], tempty[2], a2full[2], m2done[2], drain
    static constexpr int NBAR = 2 * SS + 2 * kTStages + 5;
    static constexpr int OFF_HDR = OFF_BAR + NBAR * 8;
    static constexpr int OFF_MISC = OFF_HDR + SS * (int)sizeof(BwdHdr);
    static constexpr int BYTES = OFF_MISC + 16;
    static constexpr uint32_t D2_COL = 2 * kTStages * CH;  // 64: after the two exponent stages; 2 x 32
    static constexpr uint32_t TCOLS = 128;
    static_assert(D2_COL + 64 <= TCOLS, "TMEM columns");
};

// 16-byte store into A2 (MN-major: core matrix = 8 pixels x 8 rows; rows
// contiguous, SBO = 128 B between 8-row groups, LBO = 1536 B between 8-pixel groups).
__device__ __forceinline__ void a2_store(uint8_t* A2, int pix, int mblk, const uint4& v) {
    *reinterpret_cast<uint4*>(A2 + (pix >> 3) * 1536 + mblk * 128 + (pix & 7) * 16) = v;
}
// One fp16 element of B2 (K-major: core matrix = 8 columns x 8 pixels).
__device__ __forceinline__ void b2_store(uint8_t* B2, int col, int pix, __half v) {
    *reinterpret_cast<__half*>(B2 + (col >> 3) * 2048 + (pix >> 3) * 128 + (col & 7) * 16 + (pix & 7) * 2) = v;
}

// x0, x1 -> fp16 hi (x0 in the low half) and the fp16 of the remainder.
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
    const __half2 h = __floats2half2_rn(x0, x1);
    const float2 hf = __half22float2(h);
    const float2 r = __fadd2_rn(make_float2(x0, x1), neg2(hf));
    const __half2 l = __floats2half2_rn(r.x, r.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

template <int V, int SS>
__global__ void __launch_bounds__(kThreads, 3) k_blend_tc_bwd(const __grid_constant__ BlendArgs a, const GradArgs gr) {
    using TR = Traits<V>;
    using LY = BwdLayout<SS, V>;
    constexpr int CH = LY::CH;
    constexpr uint32_t IDESC1 = idesc_f16(TR::FMT, 128, 2 * CH);
    constexpr uint32_t IDESC2 = idesc_f16(0u, 128, 32) | (1u << 15);  // fp16, A MN-major
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sA2 = smem + LY::OFF_A2;
    uint8_t* sB2 = smem + LY::OFF_B2;
    uint8_t* sA1 = smem + LY::OFF_A1;
    uint8_t* sB1 = smem + LY::OFF_B1;
    Rec* sRec = reinterpret_cast<Rec*>(smem + LY::OFF_REC);
    Fin* sFin = reinterpret_cast<Fin*>(smem + LY::OFF_FIN);
    float2* sScl = reinterpret_cast<float2*>(smem + LY::OFF_SCL);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + LY::OFF_BAR);
    BwdHdr* sHdr = reinterpret_cast<BwdHdr*>(smem + LY::OFF_HDR);
    uint32_t* sTmem = reinterpret_cast<uint32_t*>(smem + LY::OFF_MISC);
    volatile int* sAbort = reinterpret_cast<volatile int*>(smem + LY::OFF_MISC + 4);
    auto bar_full = [&](int s) { return smem_u32(bars + s); };
    auto bar_empty = [&](int s) { return smem_u32(bars + SS + s); };
    auto bar_tfull = [&](int t) { return smem_u32(bars + 2 * SS + t); };
    auto bar_tempty = [&](int t) { return smem_u32(bars + 2 * SS + kTStages + t); };
    auto bar_a2full = [&](int b) { return smem_u32(bars + 2 * SS + 2 * kTStages + b); };
    auto bar_m2done = [&](int b) { return smem_u32(bars + 2 * SS + 2 * kTStages + 2 + b); };
    const uint32_t bar_drain = smem_u32(bars + 2 * SS + 2 * kTStages + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
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
        for (int b = 0; b < 2; ++b) {
            mbar_init(bar_a2full(b), kEpiWarps);
            mbar_init(bar_m2done(b), 1);
        }
        mbar_init(bar_drain, 1);
        *sAbort = 0;
        mbar_fence_init();
    }
    // M_p of a 16 x 8 half (A operand of the exponent MMA), as in the forward kernel
    for (int row = threadIdx.x; row < 128; row += kThreads) {
        const float xb = origin ? -(float)(row & 15) : 7.5f - (float)(row & 15);
        const float yb = origin ? -(float)(row >> 4) : 3.5f - (float)(row >> 4);
        store_mp_row<V>(sA1, row, xb, yb);
    }
    // B2: zero, then the monomial columns 0..5 (the dL/dimage columns are per tile)
    for (int i = threadIdx.x; i < LY::B2_BYTES / 16; i += kThreads)
        reinterpret_cast<uint4*>(sB2)[i] = make_uint4(0, 0, 0, 0);
    for (int i = threadIdx.x; i < 2 * LY::A2_BYTES / 16; i += kThreads)
        reinterpret_cast<uint4*>(sA2)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    if (threadIdx.x < 128) {
        const int pix = threadIdx.x;
        const float xb = origin ? -(float)(pix & 15) : 7.5f - (float)(pix & 15);
        const float yb = origin ? -(float)(pix >> 4) : 3.5f - (float)(pix >> 4);
        const float vp[6] = {xb * xb, yb * yb, xb * yb, xb, yb, 1.0f};
#pragma unroll
        for (int i = 0; i < 6; ++i) b2_store(sB2, i, pix, __float2half_rn(vp[i]));
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
    auto fail = [&]() {
        *sAbort = 1;
        atomicOr(a.err, kErrTimeout);
    };

    if (warp < kEpiWarps) {
        // ------------------------------------------------------- epilogue --
        const int r = warp * 32 + lane;
        int cur_seq = -1;
        float2 T = make_float2(0.f, 0.f), Sg = T, ncf = T, g0 = T, g1 = T, g2 = T;
        // pending chunk (finishing step not done yet)
        int p_stage = -1, p_n = 0;
        uint32_t p_c2 = 0;
        float p_undp = 0.f, p_uncol = 0.f;
        uint32_t c2 = 0;  // chunks with an A2/MMA2 so far

        auto finish = [&]() -> bool {
            const int pb = (int)(p_c2 & 1u);
            if (!mbar_wait_bounded(bar_m2done(pb), (p_c2 >> 1) & 1u, tmo, sAbort)) {
                fail();
                return false;
            }
            tc_fence_after();
            if (warp < 3) {
                uint32_t v[16];
                const uint32_t d2 = tmem + ((uint32_t)(warp * 32) << 16) + LY::D2_COL + (uint32_t)(32 * pb);
                if (warp < 2) {
                    uint32_t v8[8];
                    tmem_ld_32x32b_x8(d2, v8);
                    tmem_ld_wait();
#pragma unroll
                    for (int k = 0; k < 8; ++k) v[k] = v8[k];
                } else {
                    tmem_ld_32x32b_x16(d2 + 8u, v);  // columns 8..23: dL/dimage of both halves
                    tmem_ld_wait();
                }
                float S[6];
                if (warp < 2) {
                    // rows (h = warp, s = lane >> 4, j = lane & 15): monomial moments, hi + lo
#pragma unroll
                    for (int k = 0; k < 6; ++k) S[k] = __uint_as_float(v[k]);
                } else {
                    // rows (h = lane >> 4, j = lane & 15): w . dL/dimage (hi + lo columns)
                    const bool lower = (lane >> 4) != 0;
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch)
                        S[ch] = lower ? __uint_as_float(v[8 + ch]) + __uint_as_float(v[11 + ch])
                                      : __uint_as_float(v[ch]) + __uint_as_float(v[3 + ch]);
                    S[3] = S[4] = S[5] = 0.f;
                }
#pragma unroll
                for (int k = 0; k < 6; ++k) S[k] += __shfl_xor_sync(0xffffffffu, S[k], 16);
                const int j = lane & 15;
                const Fin f = sFin[p_stage * CH + j];
                if (lane < 16 && j < p_n && f.g != 0xffffffffu) {
                    if (warp < 2) {
                        const float xh = f.xh, yh = warp ? f.yh - 8.0f : f.yh;
#pragma unroll
                        for (int k = 0; k < 6; ++k) S[k] *= p_undp;
                        const float Sx = fmaf(xh, S[5], S[3]), Sy = fmaf(yh, S[5], S[4]);
                        const float Sxx = fmaf(xh, fmaf(xh, S[5], 2.0f * S[3]), S[0]);
                        const float Syy = fmaf(yh, fmaf(yh, S[5], 2.0f * S[4]), S[1]);
                        const float Sxy = fmaf(xh, fmaf(yh, S[5], S[4]), fmaf(yh, S[3], S[2]));
                        float* dm = reinterpret_cast<float*>(gr.dmean2d) + 2 * (size_t)f.g;
                        atomicAdd(dm, -fmaf(f.A, Sx, f.B * Sy));
                        atomicAdd(dm + 1, -fmaf(f.B, Sx, f.C * Sy));
                        float* dc = gr.dconic + 3 * (size_t)f.g;
                        atomicAdd(dc, -0.5f * Sxx);
                        atomicAdd(dc + 1, -Sxy);
                        atomicAdd(dc + 2, -0.5f * Syy);
                        atomicAdd(gr.dopac + f.og, S[5] * f.inv_o);
                    } else {
                        float* dr = gr.drgb + 3 * (size_t)f.g;
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) atomicAdd(dr + ch, S[ch] * p_uncol);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_empty(p_stage));
            p_stage = -1;
            return true;
        };

        for (int k = 0;; ++k) {
            const int s = k % SS, t = k % kTStages;
            const uint32_t ps = (uint32_t)(k / SS) & 1u, pt = (uint32_t)(k / kTStages) & 1u;
            if (!mbar_wait_bounded(bar_tfull(t), pt, tmo, sAbort) || !mbar_wait_bounded(bar_full(s), ps, tmo, sAbort)) {
                fail();
                break;
            }
            const BwdHdr hd = sHdr[s];
            const int n = hd.n;
            if (n <= 0 || hd.seq != cur_seq) {
                // the pending chunk belongs to an earlier tile (or the queue ended):
                // finish it before B2 changes
                if (p_stage >= 0 && !finish()) break;
            }
            if (n < 0) break;
            if (n > 0 && hd.seq != cur_seq) {
                cur_seq = hd.seq;
                const int v = view_of(a, hd.tile);
                const ViewDesc vd = a.views[v];
                const int lt = hd.tile - vd.tile_begin;
                const int px = (lt % vd.tiles_x) * kTile + (r & 15);
                const int py = (lt / vd.tiles_x) * kTile + (r >> 4);
                const size_t plane = (size_t)vd.W * vd.H;
                float gv[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
                float Tf[2] = {0.f, 0.f}, nc[2] = {0.f, 0.f};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int y = py + 8 * h;
                    if (px < vd.W && y < vd.H) {
                        const size_t p = (size_t)y * vd.W + px;
                        nc[h] = (float)gr.n_contrib[vd.pix_off + p];
                        Tf[h] = gr.T_final[vd.pix_off + p];
                        const float* dl = gr.dL_dimage + 3 * vd.pix_off + p;
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) gv[h][ch] = dl[ch * plane];
                    }
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) {
                        const float bg = gv[h][ch] * hd.bscale;
                        const __half hi = __float2half_rn(bg);
                        const __half lo = __float2half_rn(bg - __half2float(hi));
                        b2_store(sB2, 8 + 8 * h + ch, r, hi);
                        b2_store(sB2, 8 + 8 * h + 3 + ch, r, lo);
                    }
                }
                T = make_float2(Tf[0] * kTScale, Tf[1] * kTScale);
                ncf = make_float2(nc[0], nc[1]);
                g0 = make_float2(gv[0][0] * hd.gscale, gv[1][0] * hd.gscale);
                g1 = make_float2(gv[0][1] * hd.gscale, gv[1][1] * hd.gscale);
                g2 = make_float2(gv[0][2] * hd.gscale, gv[1][2] * hd.gscale);
                Sg = __ffma2_rn(make_float2(a.bg[0], a.bg[0]), g0,
                                __ffma2_rn(make_float2(a.bg[1], a.bg[1]), g1, __fmul2_rn(make_float2(a.bg[2], a.bg[2]), g2)));
            }
            tc_fence_after();
            if (n == 0) {
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(bar_tempty(t));
                    mbar_arrive(bar_empty(s));
                }
                continue;
            }
            // exponents of the chunk's 16 splats at both pixels
            uint32_t pu[16], pl[16];
            const uint32_t tb = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * 2 * CH);
            tmem_ld_32x32b_x16(tb, pu);
            tmem_ld_32x32b_x16(tb + (uint32_t)CH, pl);
            tmem_ld_wait();
            if constexpr (TR::FP8) {  // undo the per-row scaling of the e4m3 operands
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float2 z = __fmul2_rn(make_float2(__uint_as_float(pu[j]), __uint_as_float(pl[j])),
                                                sScl[s * CH + j]);
                    pu[j] = __float_as_uint(z.x);
                    pl[j] = __float_as_uint(z.y);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_tempty(t));
            const Rec* rec = sRec + s * CH;
            const float base = (float)hd.base;

            // back to front over the chunk in two groups of 8 splats (group 1 =
            // splats 8..15 first), each group stored to A2[b] as it is done
            // (the MMA that last read A2[b] finished with chunk c2 - 2)
            const int b = (int)(c2 & 1u);
            uint8_t* A2 = sA2 + b * LY::A2_BYTES;
            auto splat = [&](int j, float2& dp, float2& wt) {
                const Rec rc = rec[j];
                const float zx = __uint_as_float(pu[j]), zy = __uint_as_float(pl[j]);
                float2 al;
                al.x = ex2_approx(fminf(zx, rc.bc.z));
                al.y = ex2_approx(fminf(zy, rc.bc.w));
                float2 cull;
                cull.x = sat(fmaf(al.x, -kCullScale, kAlphaMin * kCullScale));
                cull.y = sat(fmaf(al.y, -kCullScale, kAlphaMin * kCullScale));
                al = __ffma2_rn(neg2(al), cull, al);
                const float idx = base + (float)j;
                float2 in;
                in.x = sat(ncf.x - idx);
                in.y = sat(ncf.y - idx);
                const float2 aa = __fmul2_rn(al, in);
                const float2 om = __fadd2_rn(make_float2(1.f, 1.f), neg2(aa));
                const float2 inv = make_float2(rcp_approx(om.x), rcp_approx(om.y));
                const float2 Tj = __fmul2_rn(T, inv);
                wt = __fmul2_rn(aa, Tj);
                float2 cg = __fmul2_rn(make_float2(rc.rg.x, rc.rg.y), g0);
                cg = __ffma2_rn(make_float2(rc.rg.z, rc.rg.w), g1, cg);
                cg = __ffma2_rn(make_float2(rc.bc.x, rc.bc.y), g2, cg);
                const float2 diff = __fadd2_rn(cg, neg2(Sg));
                const float2 dLda = __fmul2_rn(Tj, diff);
                Sg = __ffma2_rn(aa, diff, Sg);
                T = Tj;
                float2 un;  // 0 where alpha is clamped at 0.99
                un.x = sat(fmaf(zx, -kStopScale, kLog2AlphaMax * kStopScale));
                un.y = sat(fmaf(zy, -kStopScale, kLog2AlphaMax * kStopScale));
                dp = __fmul2_rn(dLda, __fmul2_rn(aa, un));
            };
#pragma unroll
            for (int grp = 1; grp >= 0; --grp) {
                uint32_t wv[3][2][4];  // [dpow hi, dpow lo, w][h][word]
#pragma unroll
                for (int pr = 3; pr >= 0; --pr) {
                    float2 dpA, wA, dpB, wB;
                    splat(8 * grp + 2 * pr + 1, dpA, wA);
                    splat(8 * grp + 2 * pr, dpB, wB);
                    split2(dpB.x, dpA.x, wv[0][0][pr], wv[1][0][pr]);
                    split2(dpB.y, dpA.y, wv[0][1][pr], wv[1][1][pr]);
                    const __half2 hu = __floats2half2_rn(wB.x, wA.x), hl = __floats2half2_rn(wB.y, wA.y);
                    wv[2][0][pr] = *reinterpret_cast<const uint32_t*>(&hu);
                    wv[2][1][pr] = *reinterpret_cast<const uint32_t*>(&hl);
                }
                // rows: dpow (h, s, j) = 32 h + 16 s + j; w (h, j) = 64 + 16 h + j
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    a2_store(A2, r, 4 * h + grp, make_uint4(wv[0][h][0], wv[0][h][1], wv[0][h][2], wv[0][h][3]));
                    a2_store(A2, r, 4 * h + 2 + grp, make_uint4(wv[1][h][0], wv[1][h][1], wv[1][h][2], wv[1][h][3]));
                    a2_store(A2, r, 8 + 2 * h + grp, make_uint4(wv[2][h][0], wv[2][h][1], wv[2][h][2], wv[2][h][3]));
                }
            }
            fence_proxy_async_smem();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_a2full(b));
            // the previous chunk's sums (its MMA has had this whole chunk to finish)
            if (p_stage >= 0 && !finish()) break;
            p_stage = s;
            p_n = n;
            p_c2 = c2++;
            p_undp = hd.undp;
            p_uncol = hd.uncol;
        }
    } else if (warp == kEpiWarps) {
        // ------------------------------------------------------- producer --
        // A tile's header (queue item, range, the largest n_contrib and
        // |dL/dimage| of its pixels, the scales) is worked out for the next
        // tile once the current tile's first stage is out, so those loads
        // overlap the current tile's chunks and leave the tile's pixel data in
        // the cache for the epilogue.
        struct TileHead {
            int q, tile, len, vview, nch;
            uint32_t start;
            float xc, yc_up;
            BwdHdr hd;
        };
        auto head = [&](int qi) {
            TileHead th{};
            th.q = qi;
            if (qi >= a.total_tiles) return th;
            th.tile = tile_at(a, qi * a.shard_count + a.shard_index);
            th.start = a.ranges[2 * th.tile];
            const uint32_t stop = a.ranges[2 * th.tile + 1];
            th.len = stop > th.start ? (int)(stop - th.start) : 0;
            th.vview = view_of(a, th.tile);
            const ViewDesc vd = a.views[th.vview];
            const int lt = th.tile - vd.tile_begin;
            const int x0 = (lt % vd.tiles_x) * kTile, y0 = (lt / vd.tiles_x) * kTile;
            th.xc = (float)x0 + (origin ? 0.5f : 8.0f);
            th.yc_up = (float)y0 + (origin ? 0.5f : 4.0f);
            // largest n_contrib and |dL/dimage| over the tile's pixels
            int maxnc = 0;
            float gmax = 0.f;
            const size_t plane = (size_t)vd.W * vd.H;
            for (int p = lane; p < kTilePixels; p += 32) {
                const int px = x0 + (p & 15), py = y0 + (p >> 4);
                if (px < vd.W && py < vd.H) {
                    const size_t pp = (size_t)py * vd.W + px;
                    // T_final is read by the epilogue when the tile starts (n_contrib and
                    // dL/dimage pass through the cache here already)
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(gr.T_final + vd.pix_off + pp));
                    maxnc = max(maxnc, gr.n_contrib[vd.pix_off + pp]);
                    const float* dl = gr.dL_dimage + 3 * vd.pix_off + pp;
                    gmax = fmaxf(gmax, fmaxf(fabsf(dl[0]), fmaxf(fabsf(dl[plane]), fabsf(dl[2 * plane]))));
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                maxnc = max(maxnc, __shfl_xor_sync(0xffffffffu, maxnc, o));
                gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
            }
            maxnc = min(maxnc, th.len);
            th.nch = (maxnc + CH - 1) / CH;
            // 2^E <= gmax < 2^(E + 1), E clamped so that every scale is a normal float
            int E = 0;
            if (gmax > 0.f) E = ((__float_as_int(gmax) >> 23) & 0xff) - 127;
            E = max(-100, min(100, E));
            th.hd.gscale = __int_as_float((127 - E - 12) << 23);
            th.hd.bscale = __int_as_float((127 - E) << 23);
            th.hd.undp = __int_as_float((127 + E) << 23);
            th.hd.uncol = __int_as_float((127 + E - 12) << 23);
            return th;
        };
        // The splat data of the next chunk to build, loaded while the current
        // one is published and its stage's release is awaited (ids, then
        // position, conic, opacity and colour; lane j and j + 16 the same splat).
        struct Pre {
            int seq, c;  // the chunk it belongs to (seq -1: none)
            uint32_t g, og;
            float2 m;
            float A, B, C, o, cr, cg, cb;
        };
        Pre pf{};
        pf.seq = -1;
        auto prefetch = [&](int pseq, int c, uint32_t start, int len, int vview) {
            pf.seq = pseq;
            pf.c = c;
            const int j = lane & 15, n = min(CH, len - c * CH);
            if (j < n) {
                pf.g = a.ids[start + (uint32_t)(c * CH + j)];
                pf.m = a.mean2d[pf.g];
                pf.A = a.conic[3 * pf.g];
                pf.B = a.conic[3 * pf.g + 1];
                pf.C = a.conic[3 * pf.g + 2];
                pf.og = pf.g - (uint32_t)(vview * a.n_per_view);
                pf.o = a.opac[pf.og];
                if (lane < 16) {
                    pf.cr = a.rgb[3 * pf.g];
                    pf.cg = a.rgb[3 * pf.g + 1];
                    pf.cb = a.rgb[3 * pf.g + 2];
                }
            }
        };
        int k = 0;
        bool quit = false;
        int q_next = 0;
        if (lane == 0) q_next = (int)atomicAdd(a.queue, 1u);
        TileHead nxt = head(__shfl_sync(0xffffffffu, q_next, 0));
        for (int seq = 0; !quit; ++seq) {
            const TileHead cur = nxt;
            const bool end = cur.q >= a.total_tiles;
            if (!end && lane == 0) q_next = (int)atomicAdd(a.queue, 1u);  // read after this tile's first stage
            const int tile = cur.tile, len = cur.len, vview = cur.vview, nch = cur.nch;
            const uint32_t start = cur.start;
            const float xc = cur.xc, yc_up = cur.yc_up;
            BwdHdr hd = cur.hd;
            const int nst = end ? 1 : max(1, nch);
            const float bx0 = origin ? -15.0f : -7.5f, bx1 = origin ? 0.0f : 7.5f;
            const float by0 = origin ? -7.0f : -3.5f, by1 = origin ? 0.0f : 3.5f;
            for (int cc = 0; cc < nst; ++cc) {
                const int c = nch - 1 - cc;  // chunks back to front
                const int base = c * CH;
                const int n = end ? -1 : (nch == 0 ? 0 : min(CH, len - base));
                if (n > 0 && !(pf.seq == seq && pf.c == c)) prefetch(seq, c, start, len, vview);
                const int s = k % SS;
                const uint32_t ps = (uint32_t)(k / SS) & 1u;
                if (!mbar_wait_bounded(bar_empty(s), ps ^ 1u, tmo, sAbort)) {
                    fail();
                    quit = true;
                    break;
                }
                if (*sAbort) {
                    quit = true;
                    break;
                }
                if (n > 0) {
                    // lanes 0..15: upper reference rows, 16..31: lower, for splat j = lane & 15
                    const int j = lane & 15;
                    const bool upper = lane < 16;
                    uint8_t* mB = sB1 + s * LY::B1_BYTES;
                    float vrow[6];
                    if (j < n) {
                        const uint32_t g = pf.g, og = pf.og;
                        const float A = pf.A, B = pf.B, C = pf.C, o = pf.o;
                        const float l2o = o > 0.f ? __log2f(o) : -INFINITY;
                        const float xh = pf.m.x - xc, yh = pf.m.y - yc_up;
                        coeff_row<TR::HALF>(A, B, C, l2o, xh, upper ? yh : yh - 8.0f, bx0, bx1, by0, by1, vrow);
                        if (upper) {
                            const float cap = fminf(l2o, kLog2AlphaMax);
                            Rec rc;
                            rc.rg = make_float4(pf.cr, pf.cr, pf.cg, pf.cg);
                            rc.bc = make_float4(pf.cb, pf.cb, cap, cap);
                            sRec[s * CH + j] = rc;
                            sFin[s * CH + j] = Fin{g, og, xh, yh, A, B, C, o > 0.f ? 1.0f / o : 0.f};
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 5; ++i) vrow[i] = 0.f;
                        vrow[5] = kDeadPower;
                        if (upper) {
                            Rec rc;
                            rc.rg = make_float4(0.f, 0.f, 0.f, 0.f);
                            rc.bc = make_float4(0.f, 0.f, kDeadPower, kDeadPower);
                            sRec[s * CH + j] = rc;
                            sFin[s * CH + j] = Fin{0xffffffffu, 0u, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                        }
                    }
                    const float rs = store_coeff_row<V>(mB, upper ? j : CH + j, vrow);
                    if constexpr (TR::FP8) reinterpret_cast<float*>(sScl + s * CH + j)[upper ? 0 : 1] = rs;
                }
                if (lane == 0) {
                    hd.tile = tile;
                    hd.seq = end ? -2 : seq;
                    hd.base = base;
                    hd.n = n;
                    sHdr[s] = hd;
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_full(s));
                ++k;
                if (cc == 0 && !end) nxt = head(__shfl_sync(0xffffffffu, q_next, 0));  // the next tile's header
                // the next chunk's splats: this tile's next chunk, or the next tile's first
                if (!end) {
                    if (cc + 1 < nst) {
                        if (c - 1 >= 0) prefetch(seq, c - 1, start, len, vview);
                    } else if (nxt.q < a.total_tiles && nxt.nch > 0) {
                        prefetch(seq + 1, nxt.nch - 1, nxt.start, nxt.len, nxt.vview);
                    }
                }
            }
            if (end) quit = true;
        }
    } else if (lane == 0) {
        // ------------------------------------------------------ MMA issue --
        const uint32_t aA1 = smem_u32(sA1), aB2 = smem_u32(sB2);
        bool have_prev = false;
        uint32_t prev_c2 = 0, c2 = 0;
        for (int k = 0;; ++k) {
            const int s = k % SS, t = k % kTStages;
            const uint32_t ps = (uint32_t)(k / SS) & 1u, pt = (uint32_t)(k / kTStages) & 1u;
            if (!mbar_wait_bounded(bar_full(s), ps, tmo, sAbort) ||
                !mbar_wait_bounded(bar_tempty(t), pt ^ 1u, tmo, sAbort)) {
                fail();
                break;
            }
            const int n = sHdr[s].n;
            if (n > 0) {
                tc_fence_after();
                const uint32_t aB1 = smem_u32(sB1 + s * LY::B1_BYTES);
#pragma unroll
                for (int ks = 0; ks < TR::KSTEPS; ++ks) {
                    const uint64_t ad = smem_desc(aA1 + (uint32_t)(ks * 256), 128, TR::SBO);
                    const uint64_t bd = smem_desc(aB1 + (uint32_t)(ks * 256), 128, TR::SBO);
                    tc_mma<V>(tmem + (uint32_t)(t * 2 * CH), ad, bd, IDESC1, ks > 0 ? 1u : 0u);
                }
                tc_commit(bar_tfull(t));
                tc_commit(bar_empty(s));
            } else {
                mbar_arrive(bar_tfull(t));
                if (n == 0) mbar_arrive(bar_empty(s));
            }
            // the previous chunk's sums, once its A2 is written
            if (have_prev) {
                const int pb = (int)(prev_c2 & 1u);
                if (!mbar_wait_bounded(bar_a2full(pb), (prev_c2 >> 1) & 1u, tmo, sAbort)) {
                    fail();
                    break;
                }
                tc_fence_after();
                const uint32_t aA2 = smem_u32(sA2 + pb * LY::A2_BYTES);
#pragma unroll
                for (int ks = 0; ks < 8; ++ks) {
                    const uint64_t ad = smem_desc(aA2 + (uint32_t)(ks * 2 * LY::A2_LBO), LY::A2_LBO, 128);
                    const uint64_t bd = smem_desc(aB2 + (uint32_t)(ks * 256), 128, 2048);
                    tc_mma_f16(tmem + LY::D2_COL + (uint32_t)(32 * pb), ad, bd, IDESC2, ks > 0 ? 1u : 0u);
                }
                tc_commit(bar_m2done(pb));
                have_prev = false;
            }
            if (n > 0) {
                have_prev = true;
                prev_c2 = c2++;
            }
            if (n < 0) break;
        }
        tc_commit(bar_drain);
        mbar_wait_bounded(bar_drain, 0, 1000000000ull, nullptr);
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 5) tmem_dealloc(tmem, LY::TCOLS);
}

template <int V, int SS>
cudaError_t launch_bwd_inst(const BlendArgs& a, const GradArgs& g, cudaStream_t s) {
    using LY = BwdLayout<SS, V>;
    constexpr int bytes = LY::BYTES;
    auto kern = k_blend_tc_bwd<V, SS>;
    static std::mutex mu;
    static LaunchShape cache;
    LaunchShape sh;
    const cudaError_t es = cached_shape(mu, cache, sh, [&](LaunchShape& r) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
        // all of the SM's unified L1/shared storage as shared memory, so that
        // the residency computed below is what the hardware grants
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess)
            return e;
        int dev = 0, smem_sm = 0;
        cudaFuncAttributes fa{};
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&r.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
            return e;
        if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
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
    const int items = a.total_tiles;
    const int grid = items < sh.per_sm * sh.sms ? (items > 0 ? items : 1) : sh.per_sm * sh.sms;
    kern<<<grid, kThreads, bytes, s>>>(a, g);
    count_launches();
    return cudaGetLastError();
}

// stages 0: the variant's default; otherwise one of kBwdStagesBuilt
template <int V>
cudaError_t launch_bwd_stages(const BlendArgs& a, const GradArgs& g, int stages, cudaStream_t s) {
    if (stages == 0) stages = bwd_default_stages<V>();
    if (stages == 2) return launch_bwd_inst<V, 2>(a, g, s);
    if (stages == 3) return launch_bwd_inst<V, 3>(a, g, s);
    if (stages == 4) return launch_bwd_inst<V, 4>(a, g, s);
    if (stages == 6) return launch_bwd_inst<V, 6>(a, g, s);
    return cudaErrorInvalidValue;
}

// Instantiated per variant in blend_tc_bwd_v<V>.cu
template <int V>
cudaError_t launch_bwd_variant(const BlendArgs& a, const GradArgs& g, int stages, cudaStream_t s);
template <>
cudaError_t launch_bwd_variant<1>(const BlendArgs&, const GradArgs&, int, cudaStream_t);
template <>
cudaError_t launch_bwd_variant<2>(const BlendArgs&, const GradArgs&, int, cudaStream_t);
template <>
cudaError_t launch_bwd_variant<3>(const BlendArgs&, const GradArgs&, int, cudaStream_t);
template <>
cudaError_t launch_bwd_variant<4>(const BlendArgs&, const GradArgs&, int, cudaStream_t);
template <>
cudaError_t launch_bwd_variant<5>(const BlendArgs&, const GradArgs&, int, cudaStream_t);

}  // namespace tc
}  // namespace gs
