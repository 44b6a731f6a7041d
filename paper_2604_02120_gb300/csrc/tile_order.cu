// Longest-list-first tile order for the persistent blend kernels (not in the
// paper).  A persistent kernel's time is its busiest block's; blocks pull
// tiles from a queue, and a long list taken last leaves the other SMs idle
// while it finishes.  Taking tiles by decreasing list length (the greedy
// longest-processing-time rule) keeps that tail short.  One block of 1024
// threads counts the tiles per length bucket (quarter octaves: the leading
// bit and the two after it), places the buckets longest first and scatters
// the tile ids; within a bucket the order is the order of the atomic
// increments, since any order gives the same image.
#include "internal.h"

namespace gs {
namespace {

constexpr int kOrderThreads = 1024;
constexpr int kBuckets = 4 * 32;
constexpr int kOrderBatch = 8;

__device__ __forceinline__ int length_bucket(uint32_t len) {
    if (len < 4) return (int)len;
    const int lg = 31 - __clz(len);  // >= 2
    return 4 * lg + (int)((len >> (lg - 2)) & 3u) - 4;
}

__global__ void __launch_bounds__(kOrderThreads) k_tile_order(int ntiles, const uint32_t* __restrict__ ranges,
                                                              uint32_t* __restrict__ order) {
    __shared__ unsigned s_count[kBuckets], s_next[kBuckets];
    for (int b = threadIdx.x; b < kBuckets; b += kOrderThreads) s_count[b] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    // kOrderBatch tiles per thread and round, all loads issued before any use;
    // one shared atomic per distinct bucket in a warp (most tiles share a few)
    for (int pass = 0; pass < 2; ++pass) {
        for (int t0 = 0; t0 < ntiles; t0 += kOrderThreads * kOrderBatch) {
            uint2 rg[kOrderBatch];
#pragma unroll
            for (int u = 0; u < kOrderBatch; ++u) {
                const int t = t0 + u * kOrderThreads + (int)threadIdx.x;
                rg[u] = t < ntiles ? make_uint2(ranges[2 * t], ranges[2 * t + 1]) : make_uint2(0u, 0u);
            }
#pragma unroll
            for (int u = 0; u < kOrderBatch; ++u) {
                const int t = t0 + u * kOrderThreads + (int)threadIdx.x;
                const bool ok = t < ntiles;
                const int bk = ok ? length_bucket(rg[u].y > rg[u].x ? rg[u].y - rg[u].x : 0u) : -1;
                const unsigned peers = __match_any_sync(0xffffffffu, bk);
                const int leader = __ffs(peers) - 1;
                if (pass == 0) {
                    if (ok && lane == leader) atomicAdd(&s_count[bk], (unsigned)__popc(peers));
                } else {
                    unsigned base = 0;
                    if (ok && lane == leader) base = atomicAdd(&s_next[bk], (unsigned)__popc(peers));
                    base = __shfl_sync(0xffffffffu, base, leader);
                    if (ok) order[base + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)t;
                }
            }
        }
        __syncthreads();
        if (pass == 0 && threadIdx.x < 32) {  // longest bucket first: lane l takes buckets from the top down
            unsigned c[kBuckets / 32], sum = 0;
#pragma unroll
            for (int i = 0; i < kBuckets / 32; ++i) sum += (c[i] = s_count[kBuckets - 1 - (kBuckets / 32) * lane - i]);
            unsigned incl = sum;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned v = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += v;
            }
            unsigned acc = incl - sum;
#pragma unroll
            for (int i = 0; i < kBuckets / 32; ++i) {
                s_next[kBuckets - 1 - (kBuckets / 32) * lane - i] = acc;
                acc += c[i];
            }
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_tile_order(int ntiles, const uint32_t* ranges, uint32_t* order, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    k_tile_order<<<1, kOrderThreads, 0, s>>>(ntiles, ranges, order);
    count_launches();
    return cudaGetLastError();
}

}  // namespace gs
