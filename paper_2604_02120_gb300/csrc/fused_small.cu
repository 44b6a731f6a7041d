// Fused projection + binning for small scenes (not in the paper; the step it
// replaces is Sec. 2.1 (a)-(c)).  For a scene of a few thousand to tens of
// thousands of Gaussians the usual bin/sort stage is a chain of nine launches
// that each do microseconds of work, so launch and look-back latency is most
// of its time.  Here one cooperative launch does it all:
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
//      memory and writes them back.
// The lists equal gs_bin_sort's lists tile by tile, so the blend kernels take
// them unchanged.  One tile's list is sorted by one block in shared memory,
// which is what limits this path to small scenes.
#include <algorithm>

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

template <int SH_DEGREE, bool VEC16>
__global__ void __launch_bounds__(kFusedThreads) k_project_bin_small(
    int n, const float* __restrict__ means, const float* __restrict__ scales, const float* __restrict__ quats,
    const float* __restrict__ sh, const __grid_constant__ CamViews views, const float* __restrict__ power_min,
    int max_per_tile, float2* mean2d, float* conic, float* depth, int* radius, float* rgb, uint32_t* touched,
    uint32_t* __restrict__ ids, uint32_t* __restrict__ ranges, unsigned* barrier, unsigned* err) {
    extern __shared__ unsigned long long s_key[];  // (depth bits << 32) | Gaussian index; a power of two >= max_per_tile
    const CamDev& cam = views.cams[0];

    // 1. projection
    for (int g = blockIdx.x * kFusedThreads + threadIdx.x; g < n; g += gridDim.x * kFusedThreads)
        project_gaussian<SH_DEGREE, VEC16>(g, means, scales, quats, sh, cam, 0, mean2d, conic, depth, radius, rgb,
                                           touched);
    const int tx_n = tiles_x(cam.W), ntiles = tx_n * tiles_y(cam.H);
    for (int t = blockIdx.x * kFusedThreads + threadIdx.x; t < ntiles; t += gridDim.x * kFusedThreads)
        ranges[2 * t + 1] = 0;  // the tiles' instance counters of step 3
    // 2. every projection written, every counter cleared
    if (!grid_barrier(barrier, gridDim.x, err)) return;

    // 3. every splat appends its index to the tiles it covers (the other
    // blocks' outputs are read through L2: this SM's L1 may hold lines from
    // before the barrier)
    for (int g = blockIdx.x * kFusedThreads + threadIdx.x; g < n; g += gridDim.x * kFusedThreads) {
        const int r = __ldcg(radius + g);
        if (r <= 0) continue;
        const float2 m = __ldcg(mean2d + g);
        int x0, x1, y0, y1;
        if (!tile_rect(m.x, m.y, r, cam.W, cam.H, x0, x1, y0, y1)) continue;
        TightRows tr{};
        if (power_min != nullptr)
            tr = tight_rows(m.x, m.y, __ldcg(conic + 3 * g), __ldcg(conic + 3 * g + 1), __ldcg(conic + 3 * g + 2),
                            power_min[g]);
        for (int y = y0; y <= y1; ++y) {
            int f = x0, l = x1;
            if (power_min != nullptr) tight_row(tr, y, x0, x1, f, l);
            for (int xb = f; xb <= l; xb += kScatterBatch) {  // the batch's atomics in flight together
                unsigned pos[kScatterBatch];
#pragma unroll
                for (int u = 0; u < kScatterBatch; ++u)
                    if (xb + u <= l) pos[u] = atomicAdd(&ranges[2 * (y * tx_n + xb + u) + 1], 1u);
#pragma unroll
                for (int u = 0; u < kScatterBatch; ++u)
                    if (xb + u <= l && pos[u] < (unsigned)max_per_tile)
                        ids[(size_t)(y * tx_n + xb + u) * max_per_tile + pos[u]] = (uint32_t)g;
            }
        }
    }
    if (!grid_barrier(barrier + 1, gridDim.x, err)) return;

    // 4. per tile: (depth bits, index) keys, bitonic sort padded to a power of
    // two with keys above any real one, the list written back in order
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const unsigned total = __ldcg(&ranges[2 * t + 1]);
        const int cnt = (int)min(total, (unsigned)max_per_tile);
        uint32_t* list = ids + (size_t)t * max_per_tile;
        int P = 2;
        while (P < cnt) P <<= 1;
        for (int i = threadIdx.x; i < P; i += kFusedThreads) {
            unsigned long long k = ~0ull;
            if (i < cnt) {
                const uint32_t g = __ldcg(list + i);
                k = ((unsigned long long)__float_as_uint(__ldcg(depth + g)) << 32) | g;
            }
            s_key[i] = k;
        }
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < P; i += kFusedThreads) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const unsigned long long a = s_key[i], b = s_key[ixj];
                        if ((a > b) == ((i & k) == 0)) {
                            s_key[i] = b;
                            s_key[ixj] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int i = threadIdx.x; i < cnt; i += kFusedThreads) list[i] = (uint32_t)s_key[i];
        if (threadIdx.x == 0) {
            if (total > (unsigned)max_per_tile) atomicOr(err, kErrCapacity);
            ranges[2 * t] = (uint32_t)t * (uint32_t)max_per_tile;
            ranges[2 * t + 1] = (uint32_t)t * (uint32_t)max_per_tile + (uint32_t)cnt;
        }
        __syncthreads();
    }
}

template <int D, bool V>
cudaError_t launch_fused(int n, const float* means, const float* scales, const float* quats, const float* sh,
                         const CamViews& cams, const float* power_min, int max_per_tile, float* mean2d, float* conic,
                         float* depth, int* radius, float* rgb, uint32_t* touched, uint32_t* ids, uint32_t* ranges,
                         unsigned* barrier, unsigned* err, cudaStream_t s) {
    auto kern = k_project_bin_small<D, V>;
    int pow2 = 2;  // the sort pads a tile's keys to a power of two
    while (pow2 < max_per_tile) pow2 <<= 1;
    const size_t smem = sizeof(unsigned long long) * (size_t)pow2;
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
            int dev = 0, s_sms = 0, s_per_sm = 0;
            if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
            if ((e = cudaDeviceGetAttribute(&s_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s_per_sm, kern, kFusedThreads, smem)) !=
                cudaSuccess)
                return e;
            cached_sms = s_sms;
            cached_per_sm = s_per_sm;
            cached_smem = smem;
        }
        per_sm = cached_per_sm;
        sms = cached_sms;
    }
    const int ntiles = tiles_x(cams.cams[0].W) * tiles_y(cams.cams[0].H);
    // every block must be resident (cooperative launch); no more blocks than the larger phase needs
    const int need = std::max(ntiles, (n + kFusedThreads - 1) / kFusedThreads);
    const int grid = std::max(1, std::min(need, std::max(per_sm, 1) * sms));
    if ((e = cudaMemsetAsync(barrier, 0, 2 * sizeof(unsigned), s)) != cudaSuccess) return e;
    float2* m2 = reinterpret_cast<float2*>(mean2d);
    void* args[] = {&n,      (void*)&means, (void*)&scales, (void*)&quats, (void*)&sh,   (void*)&cams,
                    (void*)&power_min, &max_per_tile, &m2,   &conic,  &depth, &radius, &rgb, &touched,
                    &ids,    &ranges,  &barrier, &err};
    e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(kFusedThreads), args, smem, s);
    count_launches();
    return e;
}

// Scratch of the grid barrier (the library allocates no device memory).
static __device__ unsigned g_fused_barrier[2];

}  // namespace

cudaError_t launch_project_bin_small(int n, const float* means, const float* scales, const float* quats,
                                     const float* sh, int sh_degree, const CamViews& cams, const float* power_min,
                                     int max_per_tile, float* mean2d, float* conic, float* depth, int* radius,
                                     float* rgb, uint32_t* touched, uint32_t* ids, uint32_t* ranges,
                                     cudaStream_t s) {
    unsigned* err = error_word();
    if (err == nullptr) return cudaErrorUnknown;
    void* bar = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&bar, g_fused_barrier);
    if (e != cudaSuccess) return e;
    unsigned* b = static_cast<unsigned*>(bar);
    const bool vec = (reinterpret_cast<uintptr_t>(sh) & 15) == 0;
    switch (sh_degree) {
        case 0: return launch_fused<0, false>(n, means, scales, quats, sh, cams, power_min, max_per_tile, mean2d,
                                              conic, depth, radius, rgb, touched, ids, ranges, b, err, s);
        case 1:
            return vec ? launch_fused<1, true>(n, means, scales, quats, sh, cams, power_min, max_per_tile, mean2d,
                                               conic, depth, radius, rgb, touched, ids, ranges, b, err, s)
                       : launch_fused<1, false>(n, means, scales, quats, sh, cams, power_min, max_per_tile, mean2d,
                                                conic, depth, radius, rgb, touched, ids, ranges, b, err, s);
        case 2: return launch_fused<2, false>(n, means, scales, quats, sh, cams, power_min, max_per_tile, mean2d,
                                              conic, depth, radius, rgb, touched, ids, ranges, b, err, s);
        default:
            return vec ? launch_fused<3, true>(n, means, scales, quats, sh, cams, power_min, max_per_tile, mean2d,
                                               conic, depth, radius, rgb, touched, ids, ranges, b, err, s)
                       : launch_fused<3, false>(n, means, scales, quats, sh, cams, power_min, max_per_tile, mean2d,
                                                conic, depth, radius, rgb, touched, ids, ranges, b, err, s);
    }
}

}  // namespace gs
