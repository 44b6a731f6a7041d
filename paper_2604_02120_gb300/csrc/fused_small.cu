// Fused projection + binning (+ blend) for small scenes (not in the paper;
// the steps it replaces are Sec. 2.1 (a)-(c), and with the blend also (d)).
// For a scene of a few thousand to tens of thousands of Gaussians the usual
// bin/sort stage is a chain of nine launches that each do microseconds of
// work, so launch and look-back latency is most of its time.  Here one
// cooperative launch does it all:
//   1. every block projects Gaussians (grid-stride), exactly as gs_project,
//      and clears the per-tile counters;
//   2. a grid barrier (bounded wait: on expiry the timeout bit is set and the
//      blocks leave);
//   3. every splat appends its index to each tile of its rectangle (with
//      power_min, of its opacity-aware runs) in the tile's fixed slot range
//      of `ids`, by an atomic counter per tile;
//   4. a second grid barrier;
//   5. each block orders its tiles' lists by (depth bits, Gaussian index) --
//      the order of the global stable sort -- with a bitonic sort in shared
//      memory and writes them back;
//   6. (BLEND) the same block then blends the tile from the ordered list it
//      holds in shared memory: per chunk of 32 splats, warp 0 builds the
//      Eq. 6 coefficient rows of both 16 x 8 halves (fp16 hi + lo, as
//      GS_BLEND_TC_FP16_SPLIT), one tcgen05.mma (M = 128 pixels, N = 64 rows,
//      K = 16) leaves the exponents in TMEM, and warps w and w + 4 composite
//      the upper and lower pixel of TMEM lane quarter w with the persistent
//      blend's branch-free arithmetic (Eq. 1, Alg. 1's skip and stop rules),
//      until every pixel of the tile has stopped.
// The lists equal gs_bin_sort's lists tile by tile, so the blend kernels take
// them unchanged, and the blended tiles equal gs_blend_forward's
// (GS_BLEND_TC_FP16_SPLIT) on those lists.  One tile's list is sorted by one
// block in shared memory, which is what limits this path to small scenes.
#include <algorithm>

#include "blend_tc.cuh"
#include "project.cuh"
#include "tight.cuh"

namespace gs {
namespace {

constexpr int kFusedThreads = 256;
constexpr int kScatterBatch = 8;  // a splat's tile counters incremented together
constexpr uint64_t kFusedBarrierNs = 1000000000ull;  // 1 s

// One-shot grid barrier of a cooperative launch; *count is 0 at launch (one
// counter per barrier).
// Returns false (with the timeout bit set) if not every block arrived in time.
__device__ bool grid_barrier(unsigned* count, unsigned blocks, unsigned* err) {
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(count, 1u);
        const uint64_t t0 = globaltimer_ns();
        unsigned seen;
        do {
            asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(seen) : "l"(count) : "memory");
            if (seen >= blocks) break;
            if (globaltimer_ns() - t0 > kFusedBarrierNs) {
                atomicOr(err, kErrTimeout);
                ok = 0;
                break;
            }
            __nanosleep(64);
        } while (true);
    }
    return __syncthreads_and(ok) != 0;
}

// Pointers and scalars of one launch (the blend's only with BLEND).
struct SmallArgs {
    int n, max_per_tile;
    const float *means, *scales, *quats, *sh, *power_min;
    float2* mean2d;
    float *conic, *depth, *rgb;
    int* radius;
    uint32_t *touched, *ids, *ranges;
    unsigned *barrier, *err;
    const float* opacity;
    float bg[3];
    float *image, *T_final;
    int* n_contrib;
};

// The blend's shared memory after the sort keys: M_p, two stages of a chunk's
// coefficient rows and records, three mbarriers (MMA done per stage, drain)
// and the TMEM address.
constexpr int kBlendV = GS_BLEND_TC_FP16_SPLIT;
using BTR = tc::Traits<kBlendV>;
constexpr int kBlendCh = 32;                       // splats per MMA
constexpr int kSmA = 128 * BTR::ROW_BYTES;         // 4 KB
constexpr int kSmB = 2 * kBlendCh * BTR::ROW_BYTES;  // 2 KB per stage
constexpr int kSmRec = kBlendCh * (int)sizeof(tc::Rec);
constexpr int kSmBlend = kSmA + 2 * kSmB + 2 * kSmRec + 32;
constexpr uint32_t kBlendCols = 4 * kBlendCh;      // 2 stages x 64 TMEM columns (upper splats, lower splats)
__host__ __device__ inline size_t blend_smem_offset(int pow2) { return ((size_t)8 * pow2 + 1023) / 1024 * 1024; }

template <int SH_DEGREE, bool VEC16, bool BLEND>
__global__ void __launch_bounds__(kFusedThreads) k_project_bin_small(const __grid_constant__ SmallArgs a,
                                                                     const __grid_constant__ CamViews views,
                                                                     int pow2) {
    extern __shared__ __align__(1024) unsigned long long s_key[];  // (depth bits << 32) | index, pow2 of them
    const CamDev& cam = views.cams[0];
    const int n = a.n, max_per_tile = a.max_per_tile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t* sm = reinterpret_cast<uint8_t*>(s_key) + blend_smem_offset(pow2);
    uint8_t* sA = sm;
    uint8_t* sB = sm + kSmA;                                               // stage b at sB + b kSmB
    tc::Rec* sRec = reinterpret_cast<tc::Rec*>(sm + kSmA + 2 * kSmB);     // stage b at sRec + b kBlendCh
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kSmA + 2 * kSmB + 2 * kSmRec);  // [2]: drain
    uint32_t* sTmem = reinterpret_cast<uint32_t*>(bars + 3);
    uint32_t tmem = 0, mma_phase[2] = {0u, 0u};
    bool blend_ok = true;  // false once an MMA wait gave up: no further MMA is issued
    if constexpr (BLEND) {
        if (threadIdx.x == 0) {
            for (int b = 0; b < 3; ++b) mbar_init(smem_u32(bars + b), 1);
            mbar_fence_init();
        }
        for (int row = threadIdx.x; row < 128; row += kFusedThreads)  // M_p of a 16 x 8 half, centre reference
            tc::store_mp_row<kBlendV>(sA, row, 7.5f - (float)(row & 15), 3.5f - (float)(row >> 4));
        fence_proxy_async_smem();
        if (warp == 0) {
            tmem_alloc(smem_u32(sTmem), kBlendCols);
            tmem_relinquish();
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        tmem = *sTmem;
    }

    // 1. projection
    for (int g = blockIdx.x * kFusedThreads + threadIdx.x; g < n; g += gridDim.x * kFusedThreads)
        project_gaussian<SH_DEGREE, VEC16>(g, a.means, a.scales, a.quats, a.sh, cam, 0, a.mean2d, a.conic, a.depth,
                                           a.radius, a.rgb, a.touched);
    const int tx_n = tiles_x(cam.W), ntiles = tx_n * tiles_y(cam.H);
    for (int t = blockIdx.x * kFusedThreads + threadIdx.x; t < ntiles; t += gridDim.x * kFusedThreads)
        a.ranges[2 * t + 1] = 0;  // the tiles' instance counters of step 3
    // 2. every projection written, every counter cleared
    bool ok = grid_barrier(a.barrier, gridDim.x, a.err);

    // 3. every splat appends its index to the tiles it covers (the other
    // blocks' outputs are read through L2: this SM's L1 may hold lines from
    // before the barrier)
    for (int g = blockIdx.x * kFusedThreads + threadIdx.x; ok && g < n; g += gridDim.x * kFusedThreads) {
        const int r = __ldcg(a.radius + g);
        if (r <= 0) continue;
        const float2 m = __ldcg(a.mean2d + g);
        int x0, x1, y0, y1;
        if (!tile_rect(m.x, m.y, r, cam.W, cam.H, x0, x1, y0, y1)) continue;
        TightRows tr{};
        if (a.power_min != nullptr)
            tr = tight_rows(m.x, m.y, __ldcg(a.conic + 3 * g), __ldcg(a.conic + 3 * g + 1),
                            __ldcg(a.conic + 3 * g + 2), a.power_min[g]);
        for (int y = y0; y <= y1; ++y) {
            int f = x0, l = x1;
            if (a.power_min != nullptr) tight_row(tr, y, x0, x1, f, l);
            for (int xb = f; xb <= l; xb += kScatterBatch) {  // the batch's atomics in flight together
                unsigned pos[kScatterBatch];
#pragma unroll
                for (int u = 0; u < kScatterBatch; ++u)
                    if (xb + u <= l) pos[u] = atomicAdd(&a.ranges[2 * (y * tx_n + xb + u) + 1], 1u);
#pragma unroll
                for (int u = 0; u < kScatterBatch; ++u)
                    if (xb + u <= l && pos[u] < (unsigned)max_per_tile)
                        a.ids[(size_t)(y * tx_n + xb + u) * max_per_tile + pos[u]] = (uint32_t)g;
            }
        }
    }
    if (ok) ok = grid_barrier(a.barrier + 1, gridDim.x, a.err);

    // 4. per tile: (depth bits, index) keys, bitonic sort padded to a power of
    // two with keys above any real one, the list written back in order
    for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
        const unsigned total = __ldcg(&a.ranges[2 * t + 1]);
        const int cnt = (int)min(total, (unsigned)max_per_tile);
        uint32_t* list = a.ids + (size_t)t * max_per_tile;
        int P = 2;
        while (P < cnt) P <<= 1;
        for (int i = threadIdx.x; i < P; i += kFusedThreads) {
            unsigned long long k = ~0ull;
            if (i < cnt) {
                const uint32_t g = __ldcg(list + i);
                k = ((unsigned long long)__float_as_uint(__ldcg(a.depth + g)) << 32) | g;
            }
            s_key[i] = k;
        }
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < P; i += kFusedThreads) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const unsigned long long x = s_key[i], y = s_key[ixj];
                        if ((x > y) == ((i & k) == 0)) {
                            s_key[i] = y;
                            s_key[ixj] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int i = threadIdx.x; i < cnt; i += kFusedThreads) list[i] = (uint32_t)s_key[i];
        if (threadIdx.x == 0) {
            if (total > (unsigned)max_per_tile) atomicOr(a.err, kErrCapacity);
            a.ranges[2 * t] = (uint32_t)t * (uint32_t)max_per_tile;
            a.ranges[2 * t + 1] = (uint32_t)t * (uint32_t)max_per_tile + (uint32_t)cnt;
        }
        if constexpr (BLEND) {
            // 5. the tile's blend from the ordered list in s_key
            const int lx = (t % tx_n) * kTile, ly = (t / tx_n) * kTile;
            const int r = (warp & 3) * 32 + lane, h = warp >> 2;  // TMEM lane r, half h
            const int px = lx + (r & 15), py = ly + (r >> 4) + 8 * h;
            const bool in = px < cam.W && py < cam.H;
            float T = in ? 1.f : 0.f, Tstop = 0.f, last = 0.f, Cr = 0.f, Cg = 0.f, Cb = 0.f;
            const float xc = (float)lx + 8.0f, yc_up = (float)ly + 4.0f, yc_lo = (float)ly + 12.0f;
            // chunk c in stage c & 1: warp 0 builds chunk c + 1's rows (and loads
            // chunk c + 2's splats) while the MMA of chunk c runs and its
            // exponents are composited
            // warp 0's registers: the parameters of splat c0 + lane of the next chunk to build,
            // loaded a chunk ahead so that their latency overlaps the compositing
            bool pv = false;
            float2 pm = make_float2(0.f, 0.f);
            float pA = 0.f, pB = 0.f, pC = 0.f, po = 0.f, pr = 0.f, pg = 0.f, pb = 0.f;
            auto fetch = [&](int c0) {
                pv = c0 + lane < cnt;
                if (pv) {
                    const uint32_t g = (uint32_t)s_key[c0 + lane];
                    pm = __ldcg(a.mean2d + g);
                    pA = __ldcg(a.conic + 3 * g);
                    pB = __ldcg(a.conic + 3 * g + 1);
                    pC = __ldcg(a.conic + 3 * g + 2);
                    po = a.opacity[g];
                    pr = __ldcg(a.rgb + 3 * g);
                    pg = __ldcg(a.rgb + 3 * g + 1);
                    pb = __ldcg(a.rgb + 3 * g + 2);
                }
            };
            auto build = [&](int st) {  // warp 0: the fetched splat's rows of both halves and record
                uint8_t* mB = sB + st * kSmB;
                float vu[6], vl[6];
                tc::Rec rc;
                if (pv) {
                    const float l2o = po > 0.f ? __log2f(po) : -INFINITY;
                    const float xh = pm.x - xc;
                    tc::coeff_row<true>(pA, pB, pC, l2o, xh, pm.y - yc_up, -7.5f, 7.5f, -3.5f, 3.5f, vu);
                    tc::coeff_row<true>(pA, pB, pC, l2o, xh, pm.y - yc_lo, -7.5f, 7.5f, -3.5f, 3.5f, vl);
                    const float cap = fminf(l2o, tc::kLog2AlphaMax);
                    rc.rg = make_float4(pr, pr, pg, pg);
                    rc.bc = make_float4(pb, pb, cap, cap);
                } else {  // padding: dead rows, no colour
#pragma unroll
                    for (int i = 0; i < 5; ++i) vu[i] = vl[i] = 0.f;
                    vu[5] = vl[5] = tc::kDeadPower;
                    rc.rg = rc.bc = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                tc::store_coeff_row<kBlendV>(mB, lane, vu);
                tc::store_coeff_row<kBlendV>(mB, kBlendCh + lane, vl);
                sRec[st * kBlendCh + lane] = rc;
                fence_proxy_async_smem();
            };
            auto issue = [&](int st) {  // thread 0: the MMA of stage st, committed to its barrier
                tc_fence_after();
                constexpr uint32_t IDESC = idesc_f16(BTR::FMT, 128, 2 * kBlendCh);
                tc::tc_mma<kBlendV>(tmem + (uint32_t)(st * 2 * kBlendCh), smem_desc(smem_u32(sA), 128, BTR::SBO),
                                    smem_desc(smem_u32(sB + st * kSmB), 128, BTR::SBO), IDESC, 0u);
                tc_commit(smem_u32(bars + st));
            };
            const int nchunk = blend_ok ? (cnt + kBlendCh - 1) / kBlendCh : 0;
            if (nchunk > 0) {
                if (warp == 0) {
                    fetch(0);
                    build(0);
                    if (nchunk > 1) fetch(kBlendCh);
                }
                __syncthreads();
                if (threadIdx.x == 0) issue(0);
            }
            int c = 0;
            bool pending = false;  // an MMA issued and not yet waited for (chunk c + 1's)
            for (; c < nchunk; ++c) {
                const int st = c & 1;
                const bool more = c + 1 < nchunk;
                if (more && warp == 0) {
                    build(st ^ 1);
                    if (c + 2 < nchunk) fetch((c + 2) * kBlendCh);
                }
                const bool got = mbar_wait_bounded(smem_u32(bars + st), mma_phase[st], kFusedBarrierNs, nullptr);
                mma_phase[st] ^= 1u;
                if (!__syncthreads_and(got)) {  // (also: chunk c + 1's rows are in place)
                    if (threadIdx.x == 0) atomicOr(a.err, kErrTimeout);
                    blend_ok = false;
                    pending = false;  // whatever is in flight, the final drain waits for it
                    break;
                }
                if (more && threadIdx.x == 0) issue(st ^ 1);
                pending = more;
                tc_fence_after();
                const int c0 = c * kBlendCh;
                const tc::Rec* rec = sRec + st * kBlendCh;
                const uint32_t tcol = tmem + ((uint32_t)((warp & 3) * 32) << 16) +
                                      (uint32_t)(st * 2 * kBlendCh + h * kBlendCh);
#pragma unroll 1
                for (int q0 = 0; q0 < kBlendCh; q0 += 16) {  // 16 columns at a time
                    uint32_t v[16];
                    tc::tmem_ld_32x32b_x16(tcol + (uint32_t)q0, v);
                    tmem_ld_wait();
#pragma unroll
                    for (int q = 0; q < 16; ++q) {  // the persistent blend's compositing, one pixel
                        const tc::Rec rc = rec[q0 + q];
                        float al = ex2_approx(fminf(__uint_as_float(v[q]), rc.bc.z));
                        const float cull = tc::sat(fmaf(al, -tc::kCullScale, tc::kAlphaMin * tc::kCullScale));
                        al = fmaf(-al, cull, al);
                        const float tT = fmaf(-al, T, T);
                        const float stop = tc::sat(fmaf(tT, -tc::kStopScale, tc::kTMin * tc::kStopScale));
                        Tstop = fmaf(T, stop, Tstop);
                        const float a2 = fmaf(-al, stop, al);
                        const float w = __fmul_rn(a2, T);
                        T = fmaf(-tT, stop, tT);
                        Cr = fmaf(rc.rg.x, w, Cr);
                        Cg = fmaf(rc.rg.z, w, Cg);
                        Cb = fmaf(rc.bc.x, w, Cb);
                        const float used = tc::sat(__fmul_rn(a2, tc::kCullScale));
                        const float idx1 = (float)(c0 + q0 + q + 1);
                        last = fmaf(used, __fadd_rn(idx1, -last), last);
                    }
                }
                tc_fence_before();
                if (__syncthreads_and(T == 0.f)) {  // every pixel of the tile has stopped
                    ++c;
                    break;
                }
            }
            if (pending) {  // the MMA issued for a chunk that is not composited: let it finish
                const int st = c & 1;
                const bool got = mbar_wait_bounded(smem_u32(bars + st), mma_phase[st], kFusedBarrierNs, nullptr);
                mma_phase[st] ^= 1u;
                if (!__syncthreads_and(got)) {
                    if (threadIdx.x == 0) atomicOr(a.err, kErrTimeout);
                    blend_ok = false;
                }
            }
            if (in) {
                const size_t plane = (size_t)cam.W * cam.H, p = (size_t)py * cam.W + px;
                const float Tf = T + Tstop;
                a.image[p] = Cr + Tf * a.bg[0];
                a.image[plane + p] = Cg + Tf * a.bg[1];
                a.image[2 * plane + p] = Cb + Tf * a.bg[2];
                a.T_final[p] = Tf;
                a.n_contrib[p] = (int)last;
            }
        }
        __syncthreads();
    }
    if constexpr (BLEND) {
        // every MMA this block issued has completed before TMEM is freed
        if (threadIdx.x == 0) {
            tc_commit(smem_u32(bars + 2));
            mbar_wait_bounded(smem_u32(bars + 2), 0, kFusedBarrierNs, nullptr);
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (warp == 0) tmem_dealloc(tmem, kBlendCols);
    }
}

template <int D, bool V, bool BLEND>
cudaError_t launch_fused(const SmallArgs& args, const CamViews& cams, cudaStream_t s) {
    auto kern = k_project_bin_small<D, V, BLEND>;
    int pow2 = 2;  // the sort pads a tile's keys to a power of two
    while (pow2 < args.max_per_tile) pow2 <<= 1;
    const size_t smem = BLEND ? blend_smem_offset(pow2) + kSmBlend : sizeof(unsigned long long) * (size_t)pow2;
    // residency for the last shared-memory size, as for the other kernels once per process
    // (under a lock: host threads may call at the same time)
    static std::mutex mu;
    static size_t cached_smem = 0;
    static int cached_per_sm = 0, cached_sms = 0;
    int per_sm = 0, sms = 0;
    cudaError_t e;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (smem != cached_smem) {
            if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
                cudaSuccess)
                return e;
            // all of the SM's unified L1 as shared memory: the blend's stages would otherwise
            // leave room for one block per SM under the default split
            if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          (int)cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
                return e;
            int dev = 0, s_sms = 0, s_per_sm = 0;
            if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
            if ((e = cudaDeviceGetAttribute(&s_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s_per_sm, kern, kFusedThreads, smem)) !=
                cudaSuccess)
                return e;
            // BLEND: every resident block holds kBlendCols of the SM's 512 TMEM columns
            if (BLEND) s_per_sm = std::min(s_per_sm, (int)(512 / kBlendCols));
            cached_sms = s_sms;
            cached_per_sm = s_per_sm;
            cached_smem = smem;
        }
        per_sm = cached_per_sm;
        sms = cached_sms;
    }
    const int ntiles = tiles_x(cams.cams[0].W) * tiles_y(cams.cams[0].H);
    // every block must be resident (cooperative launch); no more blocks than the larger phase needs
    const int need = std::max(ntiles, (args.n + kFusedThreads - 1) / kFusedThreads);
    const int grid = std::max(1, std::min(need, std::max(per_sm, 1) * sms));
    if ((e = cudaMemsetAsync(args.barrier, 0, 2 * sizeof(unsigned), s)) != cudaSuccess) return e;
    void* kargs[] = {(void*)&args, (void*)&cams, (void*)&pow2};
    e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(kFusedThreads), kargs, smem, s);
    count_launches();
    return e;
}

template <bool BLEND>
cudaError_t launch_fused_sh(int sh_degree, const SmallArgs& args, const CamViews& cams, cudaStream_t s) {
    const bool vec = (reinterpret_cast<uintptr_t>(args.sh) & 15) == 0;
    switch (sh_degree) {
        case 0: return launch_fused<0, false, BLEND>(args, cams, s);
        case 1: return vec ? launch_fused<1, true, BLEND>(args, cams, s) : launch_fused<1, false, BLEND>(args, cams, s);
        case 2: return launch_fused<2, false, BLEND>(args, cams, s);
        default:
            return vec ? launch_fused<3, true, BLEND>(args, cams, s) : launch_fused<3, false, BLEND>(args, cams, s);
    }
}

// Scratch of the grid barrier (the library allocates no device memory).
static __device__ unsigned g_fused_barrier[2];

cudaError_t fill_small_args(SmallArgs& x, int n, const float* means, const float* scales, const float* quats,
                            const float* sh, const float* power_min, int max_per_tile, float* mean2d, float* conic,
                            float* depth, int* radius, float* rgb, uint32_t* touched, uint32_t* ids,
                            uint32_t* ranges) {
    x = SmallArgs{};
    x.err = error_word();
    if (x.err == nullptr) return cudaErrorUnknown;
    void* bar = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&bar, g_fused_barrier);
    if (e != cudaSuccess) return e;
    x.barrier = static_cast<unsigned*>(bar);
    x.n = n;
    x.max_per_tile = max_per_tile;
    x.means = means;
    x.scales = scales;
    x.quats = quats;
    x.sh = sh;
    x.power_min = power_min;
    x.mean2d = reinterpret_cast<float2*>(mean2d);
    x.conic = conic;
    x.depth = depth;
    x.rgb = rgb;
    x.radius = radius;
    x.touched = touched;
    x.ids = ids;
    x.ranges = ranges;
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_project_bin_small(int n, const float* means, const float* scales, const float* quats,
                                     const float* sh, int sh_degree, const CamViews& cams, const float* power_min,
                                     int max_per_tile, float* mean2d, float* conic, float* depth, int* radius,
                                     float* rgb, uint32_t* touched, uint32_t* ids, uint32_t* ranges,
                                     cudaStream_t s) {
    SmallArgs x;
    const cudaError_t e = fill_small_args(x, n, means, scales, quats, sh, power_min, max_per_tile, mean2d, conic,
                                          depth, radius, rgb, touched, ids, ranges);
    if (e != cudaSuccess) return e;
    return launch_fused_sh<false>(sh_degree, x, cams, s);
}

cudaError_t launch_render_small(int n, const float* means, const float* scales, const float* quats, const float* sh,
                                int sh_degree, const CamViews& cams, const float* power_min, int max_per_tile,
                                float* mean2d, float* conic, float* depth, int* radius, float* rgb, uint32_t* touched,
                                uint32_t* ids, uint32_t* ranges, const float* opacity, const float bg[3],
                                float* image, float* T_final, int* n_contrib, cudaStream_t s) {
    SmallArgs x;
    const cudaError_t e = fill_small_args(x, n, means, scales, quats, sh, power_min, max_per_tile, mean2d, conic,
                                          depth, radius, rgb, touched, ids, ranges);
    if (e != cudaSuccess) return e;
    x.opacity = opacity;
    for (int c = 0; c < 3; ++c) x.bg[c] = bg[c];
    x.image = image;
    x.T_final = T_final;
    x.n_contrib = n_contrib;
    return launch_fused_sh<true>(sh_degree, x, cams, s);
}

}  // namespace gs
