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
    for (int t = threadIdx.x; t < ntiles; t += kOrderThreads) {
        const uint32_t a = ranges[2 * t], b = ranges[2 * t + 1];
        atomicAdd(&s_count[length_bucket(b > a ? b - a : 0u)], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // longest bucket first
        unsigned acc = 0;
        for (int b = kBuckets - 1; b >= 0; --b) {
            s_next[b] = acc;
            acc += s_count[b];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ntiles; t += kOrderThreads) {
        const uint32_t a = ranges[2 * t], b = ranges[2 * t + 1];
        order[atomicAdd(&s_next[length_bucket(b > a ? b - a : 0u)], 1u)] = (uint32_t)t;
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
