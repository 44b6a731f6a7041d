// gs_measure_peaks: microbenchmarks of the arithmetic units the blend kernels
// are bound by — MUFU ex2 and reciprocal (one of each per pair in the backward
// pass, one ex2 per pair in the forward pass) and FP32 FMA — and of the SM
// clock while they run.  Every thread runs 8 independent dependent chains so
// that the unit, not the latency, is the limit; the grid fills every SM.
#include <algorithm>
#include <vector>

#include "internal.h"

namespace gs {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;
constexpr int kMaxBlocks = 4096;  // 8 blocks of 256 threads per SM, up to 512 SMs

// Scratch of the microbenchmarks (the library allocates no device memory).
static __device__ float g_peak_sink[kMaxBlocks];
static __device__ long long g_peak_clocks[4 * kMaxBlocks];

enum PeakOp { kOpEx2 = 0, kOpRcp = 1, kOpFma = 2 };

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_op(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// clocks[blockIdx.x] = {clock64 at start, at end, globaltimer at start, at end}
template <int OP>
__global__ void __launch_bounds__(kPeakThreads) k_peak(int iters, float* __restrict__ sink,
                                                       long long* __restrict__ clocks) {
    const long long c0 = clock64();
    const long long t0 = (long long)globaltimer_ns();
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = 0.5f + 1e-3f * (float)((threadIdx.x + c) & 63);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if constexpr (OP == kOpEx2) v[c] = ex2_op(-v[c]);          // stays in [0.5, 1]
            else if constexpr (OP == kOpRcp) v[c] = rcp_approx(v[c] + 1.0f);  // stays in [0.5, 1]
            else v[c] = fmaf(v[c], 0.999f, 0.0005f);                 // stays near 0.5
        }
    }
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc += v[c];
    if (acc == 12345.678f) sink[blockIdx.x] = acc;  // keeps the chains alive
    __syncthreads();
    if (threadIdx.x == 0) {
        clocks[4 * blockIdx.x + 0] = c0;
        clocks[4 * blockIdx.x + 1] = clock64();
        clocks[4 * blockIdx.x + 2] = t0;
        clocks[4 * blockIdx.x + 3] = (long long)globaltimer_ns();
    }
}

// Best of `reps` timed launches: operations per second and the mean SM clock.
template <int OP>
cudaError_t time_op(int blocks, int iters, int reps, float* sink, long long* clocks_dev, cudaStream_t s,
                    double* ops_per_s, double* mhz) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    k_peak<OP><<<blocks, kPeakThreads, 0, s>>>(iters / 8, sink, clocks_dev);  // warm-up
    count_launches();
    double best = 0.0, best_mhz = 0.0;
    std::vector<long long> host((size_t)4 * blocks);
    for (int r = 0; e == cudaSuccess && r < reps; ++r) {
        if ((e = cudaEventRecord(e0, s)) != cudaSuccess) break;
        k_peak<OP><<<blocks, kPeakThreads, 0, s>>>(iters, sink, clocks_dev);
        count_launches();
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = cudaEventRecord(e1, s)) != cudaSuccess) break;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
        if ((e = cudaMemcpy(host.data(), clocks_dev, host.size() * sizeof(long long), cudaMemcpyDeviceToHost)) !=
            cudaSuccess)
            break;
        double cyc = 0.0, ns = 0.0;
        for (int b = 0; b < blocks; ++b) {
            cyc += (double)(host[4 * b + 1] - host[4 * b + 0]);
            ns += (double)(host[4 * b + 3] - host[4 * b + 2]);
        }
        const double ops = (double)blocks * kPeakThreads * kChains * (double)iters;
        const double rate = ops / (ms * 1e-3);
        if (rate > best) {
            best = rate;
            best_mhz = ns > 0.0 ? cyc / ns * 1e3 : 0.0;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    *ops_per_s = best;
    *mhz = best_mhz;
    return e;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_measure_peaks(gs_peaks* out, gs_stream stream) {
    if (out == nullptr) {
        set_error("gs_measure_peaks: null output");
        return GS_ERR_INVALID_ARG;
    }
    *out = gs_peaks{};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_status(e, "gs_measure_peaks: device");
    const int blocks = std::min(kMaxBlocks, sms * (2048 / kPeakThreads));  // every thread slot of every SM
    void* sink = nullptr;
    void* clocks = nullptr;
    if ((e = cudaGetSymbolAddress(&sink, g_peak_sink)) != cudaSuccess ||
        (e = cudaGetSymbolAddress(&clocks, g_peak_clocks)) != cudaSuccess)
        return cuda_status(e, "gs_measure_peaks: scratch");
    float* sk = static_cast<float*>(sink);
    long long* ck = static_cast<long long*>(clocks);
    double mhz[3] = {0, 0, 0};
    e = time_op<kOpEx2>(blocks, 4096, 3, sk, ck, s, &out->ex2_per_s, &mhz[0]);
    if (e == cudaSuccess) e = time_op<kOpRcp>(blocks, 4096, 3, sk, ck, s, &out->rcp_per_s, &mhz[1]);
    if (e == cudaSuccess) e = time_op<kOpFma>(blocks, 16384, 3, sk, ck, s, &out->fma_per_s, &mhz[2]);
    if (e != cudaSuccess) return cuda_status(e, "gs_measure_peaks");
    out->sm_mhz = (mhz[0] + mhz[1] + mhz[2]) / 3.0;
    out->sms = sms;
    return GS_OK;
}
