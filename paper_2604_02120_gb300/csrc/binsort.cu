// Duplication and sorting stages (Sec. 2.1 (b), (c)).
//
// The result equals a stable sort of (tile << 32 | depth_bits) keys emitted in
// Gaussian order, i.e. every tile's list ordered by (depth bits, Gaussian
// index).  It is produced in two sorts instead of one wide one:
//   1. stable LSD radix sort of the N Gaussians by depth bits (32-bit keys);
//   2. duplication in that depth order (one instance per touched tile);
//   3. stable LSD radix sort of the I instances by tile id alone
//      (ceil(log2 tiles / 8) passes instead of ceil((32 + log2 tiles) / 8)).
// Stability of step 3 keeps the depth order (and the index order of equal
// depths from step 1) inside each tile.
#include "internal.h"

namespace gs {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTileItems = kThreads * kItems;  // 4096 items per block

inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// ------------------------------------------------------------ scan (excl) --

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// exclusive scan of one value per thread across a block of NT threads;
// returns the thread's exclusive prefix, `total` receives the block's sum.
template <typename T, int NT>
__device__ __forceinline__ T block_excl_scan(T v, T& total, T* s_warp /*[NT/32 + 1]*/) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < NT / 32 ? s_warp[lane] : T(0);
        T wi = warp_incl_scan(w);
        if (lane < NT / 32) s_warp[lane] = wi - w;
        if (lane == NT / 32 - 1) s_warp[NT / 32] = wi;
    }
    __syncthreads();
    T res = inc - v + s_warp[warp];
    total = s_warp[NT / 32];
    __syncthreads();
    return res;
}

// Scans run on 1024-thread blocks; a block covers kScanItems<T>() * 1024 elements
// staged through 64 KB of dynamic shared memory.
constexpr int kScanThreads = 1024;
template <typename T>
constexpr int scan_items() { return sizeof(T) == 8 ? 8 : 16; }
template <typename T>
constexpr int scan_tile() { return kScanThreads * scan_items<T>(); }

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const T* __restrict__ in, int64_t n, T* __restrict__ sums) {
    __shared__ T s_warp[kScanThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * scan_tile<T>();
    T acc = 0;
#pragma unroll
    for (int r = 0; r < scan_items<T>(); ++r) {
        int64_t i = base + r * kScanThreads + threadIdx.x;
        if (i < n) acc += in[i];
    }
    T total;
    block_excl_scan<T, kScanThreads>(acc, total, s_warp);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// out[i] = sum_{k<i} in[k]; the block's offset is the sum of sums[0 .. block)
// (each block adds up the block sums before it, at most kScanThreads of them);
// if write_total, out[n] = sum of all.
template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const T* in, int64_t n, const T* __restrict__ sums,
                                                             int sums_scanned, T* out, int write_total) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    T* s_items = reinterpret_cast<T*>(s_raw);
    __shared__ T s_warp[kScanThreads / 32 + 1];
    constexpr int IT = scan_items<T>();
    const int64_t base = (int64_t)blockIdx.x * scan_tile<T>();
    T off = 0;
    if (sums != nullptr && sums_scanned) {
        off = sums[blockIdx.x];
    } else if (sums != nullptr) {
        T mine = (int)threadIdx.x < (int)blockIdx.x ? sums[threadIdx.x] : T(0);
        T tot;
        block_excl_scan<T, kScanThreads>(mine, tot, s_warp);
        off = tot;
    }
#pragma unroll
    for (int r = 0; r < IT; ++r) {
        int64_t i = base + r * kScanThreads + threadIdx.x;
        s_items[r * kScanThreads + threadIdx.x] = i < n ? in[i] : T(0);
    }
    __syncthreads();
    T loc[IT];
    T acc = 0;
#pragma unroll
    for (int k = 0; k < IT; ++k) {
        loc[k] = s_items[threadIdx.x * IT + k];
        acc += loc[k];
    }
    T total;
    T pre = block_excl_scan<T, kScanThreads>(acc, total, s_warp) + off;
#pragma unroll
    for (int k = 0; k < IT; ++k) {
        s_items[threadIdx.x * IT + k] = pre;
        pre += loc[k];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < IT; ++r) {
        int64_t i = base + r * kScanThreads + threadIdx.x;
        if (i < n) out[i] = s_items[r * kScanThreads + threadIdx.x];
    }
    if (write_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = off + total;
}

// number of scratch elements the scan of n items needs
size_t scan_scratch_elems(int64_t n) {
    size_t total = 0;
    int64_t m = n;
    const int64_t tile = scan_tile<uint64_t>();  // the smaller tile of the two element types
    while (m > tile) {
        m = cdiv(m, tile);
        total += (size_t)m + 64;
    }
    return total + 64;
}

// exclusive scan in -> out (may alias), out[n] = total if write_total.
// One launch up to one block's tile, two up to kScanThreads blocks, else the
// block sums are scanned recursively first.
template <typename T>
cudaError_t scan_exclusive(const T* in, T* out, int64_t n, T* scratch, bool write_total, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    constexpr int smem = scan_tile<T>() * (int)sizeof(T);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_scan_apply<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int nb = cdiv(n, scan_tile<T>());
    if (nb == 1) {
        k_scan_apply<T><<<1, kScanThreads, smem, s>>>(in, n, nullptr, 0, out, write_total ? 1 : 0);
        count_launches();
        return cudaGetLastError();
    }
    T* sums = scratch;
    k_scan_reduce<T><<<nb, kScanThreads, 0, s>>>(in, n, sums);
    count_launches();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int scanned = 0;
    if (nb > kScanThreads) {
        // too many blocks for a block to add up its predecessors: turn the sums
        // into exclusive offsets first
        if ((e = scan_exclusive<T>(sums, sums, nb, scratch + nb + 64, false, s)) != cudaSuccess) return e;
        scanned = 1;
    }
    k_scan_apply<T><<<nb, kScanThreads, smem, s>>>(in, n, sums, scanned, out, write_total ? 1 : 0);
    count_launches();
    return cudaGetLastError();
}

// ------------------------------------------------------------- radix sort --

// Item count of a pass: the host value, or min(*n_dev, host value) in graph mode.
__device__ __forceinline__ uint32_t pass_count(uint32_t n_host, const uint64_t* n_dev) {
    if (n_dev == nullptr) return n_host;
    const uint64_t v = *n_dev;
    return v < n_host ? (uint32_t)v : n_host;
}

__global__ void __launch_bounds__(kThreads) k_radix_hist(const uint32_t* __restrict__ keys, uint32_t n_host,
                                                         const uint64_t* __restrict__ n_dev, int shift,
                                                         uint32_t* __restrict__ hist, int nblk) {
    __shared__ uint32_t s_cnt[256];
    const uint32_t n = pass_count(n_host, n_dev);
    s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTileItems;
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        int64_t i = base + r * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&s_cnt[(keys[i] >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nblk + blockIdx.x] = s_cnt[threadIdx.x];
}

// Stable scatter: warp w owns the contiguous items [w*512, w*512 + 512) of the
// block's tile, walked in rounds of 32 so lane order = input order.
__global__ void __launch_bounds__(kThreads) k_radix_scatter(const uint32_t* __restrict__ kin,
                                                            const uint32_t* __restrict__ vin, uint32_t n_host,
                                                            const uint64_t* __restrict__ n_dev, int shift,
                                                            const uint32_t* __restrict__ offs, int nblk,
                                                            uint32_t* __restrict__ kout, uint32_t* __restrict__ vout) {
    __shared__ uint32_t s_w[kThreads / 32][256];
    const uint32_t n = pass_count(n_host, n_dev);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < (kThreads / 32) * 256; i += kThreads) (&s_w[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTileItems + warp * (kItems * 32);
    uint32_t k[kItems], v[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        int64_t i = base + r * 32 + lane;
        k[r] = i < n ? kin[i] : 0u;
        v[r] = i < n ? vin[i] : 0u;
    }
    const unsigned lt = (1u << lane) - 1u;
    // per-warp digit counts
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const bool valid = base + r * 32 + lane < n;
        const uint32_t d = valid ? ((k[r] >> shift) & 0xFFu) : (0x100u + lane);
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid && (peers & lt) == 0) s_w[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // exclusive bases per (warp, digit)
    {
        const int d = threadIdx.x;
        uint32_t run = offs[(size_t)d * nblk + blockIdx.x];
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) {
            uint32_t c = s_w[w][d];
            s_w[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const bool valid = base + r * 32 + lane < n;
        const uint32_t d = valid ? ((k[r] >> shift) & 0xFFu) : (0x100u + lane);
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t pos = 0;
        if (valid) pos = s_w[warp][d] + __popc(peers & lt);
        __syncwarp();
        if (valid) {
            kout[pos] = k[r];
            vout[pos] = v[r];
            if ((peers & lt) == 0) s_w[warp][d] += __popc(peers);
        }
        __syncwarp();
    }
}

struct RadixScratch {
    uint32_t* hist;
    uint32_t* scan;
};

// One stable pass on bits [shift, shift + 8) over n items (at most n, the
// actual count in *n_dev, in graph mode).
cudaError_t radix_pass(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout, uint32_t n,
                       const uint64_t* n_dev, int shift, RadixScratch rs, cudaStream_t s) {
    const int nblk = cdiv(n, kTileItems);
    k_radix_hist<<<nblk, kThreads, 0, s>>>(kin, n, n_dev, shift, rs.hist, nblk);
    count_launches();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan_exclusive<uint32_t>(rs.hist, rs.hist, (int64_t)256 * nblk, rs.scan, false, s);
    if (e != cudaSuccess) return e;
    k_radix_scatter<<<nblk, kThreads, 0, s>>>(kin, vin, n, n_dev, shift, rs.hist, nblk, kout, vout);
    count_launches();
    return cudaGetLastError();
}

// Sorts (k[0], v[0]) on bits [0, bits); the result ends in buffer *which.
cudaError_t radix_sort(uint32_t* k[2], uint32_t* v[2], uint32_t n, const uint64_t* n_dev, int bits, RadixScratch rs,
                       int* which, cudaStream_t s) {
    int cur = 0;
    for (int shift = 0; shift < bits; shift += 8) {
        cudaError_t e = radix_pass(k[cur], v[cur], k[cur ^ 1], v[cur ^ 1], n, n_dev, shift, rs, s);
        if (e != cudaSuccess) return e;
        cur ^= 1;
    }
    *which = cur;
    return cudaSuccess;
}

// ------------------------------------------------------ duplicate/finalize --

__global__ void k_count(int n_items, const __grid_constant__ SortViews sv, const float2* __restrict__ mean2d,
                        const int* __restrict__ radius, const float* __restrict__ depth, uint32_t* __restrict__ cnt,
                        uint32_t* __restrict__ dkey, uint32_t* __restrict__ dval) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_items) return;
    const ViewDesc& vd = sv.views[i / sv.n_per_view];
    int x0, x1, y0, y1;
    const float2 m = mean2d[i];
    uint32_t c = 0;
    if (tile_rect(m.x, m.y, radius[i], vd.W, vd.H, x0, x1, y0, y1)) c = (uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1));
    cnt[i] = c;
    dkey[i] = __float_as_uint(depth[i]);
    dval[i] = (uint32_t)i;
}

__global__ void k_gather_counts(int n, const uint32_t* __restrict__ perm, const uint32_t* __restrict__ cnt,
                                uint64_t* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = cnt[perm[k]];
}

// One thread per instance: find its item by binary search over the
// depth-ordered exclusive offsets, then its tile inside the rectangle.  In
// graph mode the count comes from offs[n_items] and is clamped to capacity
// (overflow sets kErrCapacity); block 0 also stores the count for the caller.
__global__ void k_duplicate(uint32_t I_host, int64_t capacity, int n_items, const uint64_t* __restrict__ offs,
                            const uint32_t* __restrict__ perm, const __grid_constant__ SortViews sv,
                            const float2* __restrict__ mean2d, const int* __restrict__ radius,
                            uint32_t* __restrict__ tkey, uint32_t* __restrict__ tval, int64_t* __restrict__ count_out,
                            unsigned* __restrict__ err) {
    uint32_t I = I_host;
    if (count_out != nullptr) {  // graph mode
        const uint64_t total = offs[n_items];
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            *count_out = (int64_t)total;
            if (total > (uint64_t)capacity) atomicOr(err, kErrCapacity);
        }
        I = total < (uint64_t)capacity ? (uint32_t)total : (uint32_t)capacity;
    }
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= I) return;
    // largest k with offs[k] <= i
    int lo = 0, hi = n_items - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (offs[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    const uint32_t item = perm[lo];
    const uint32_t j = i - (uint32_t)offs[lo];
    const ViewDesc& vd = sv.views[item / (uint32_t)sv.n_per_view];
    int x0, x1, y0, y1;
    const float2 m = mean2d[item];
    tile_rect(m.x, m.y, radius[item], vd.W, vd.H, x0, x1, y0, y1);
    const uint32_t w = (uint32_t)(x1 - x0 + 1);
    const uint32_t ty = (uint32_t)y0 + j / w, tx = (uint32_t)x0 + j % w;
    tkey[i] = (uint32_t)vd.tile_begin + ty * (uint32_t)vd.tiles_x + tx;
    tval[i] = item;
}

__global__ void k_finalize(uint32_t I_host, const uint64_t* __restrict__ I_dev, const uint32_t* __restrict__ tkey,
                           const uint32_t* __restrict__ tval, const float* __restrict__ depth,
                           uint64_t* __restrict__ keys_sorted, uint32_t* __restrict__ ids_sorted,
                           uint32_t* __restrict__ ranges) {
    const uint32_t I = pass_count(I_host, I_dev);
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= I) return;
    const uint32_t t = tkey[i], g = tval[i];
    keys_sorted[i] = ((uint64_t)t << 32) | __float_as_uint(depth[g]);
    ids_sorted[i] = g;
    if (i == 0 || tkey[i - 1] != t) ranges[2 * t] = i;
    if (i == I - 1 || tkey[i + 1] != t) ranges[2 * t + 1] = i + 1;
}

struct Layout {
    size_t cnt, dk0, dk1, dv0, dv1, c64, offs, sscan, hist, hscan, tk0, tk1, tv0, tv1, total;
};

Layout make_layout(int n, int64_t capacity) {
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align256(o + bytes);
        return at;
    };
    const size_t N = (size_t)(n > 0 ? n : 1), C = (size_t)(capacity > 0 ? capacity : 1);
    L.cnt = take(4 * N);
    L.dk0 = take(4 * N);
    L.dk1 = take(4 * N);
    L.dv0 = take(4 * N);
    L.dv1 = take(4 * N);
    L.c64 = take(8 * N);
    L.offs = take(8 * (N + 1));
    L.sscan = take(8 * scan_scratch_elems((int64_t)N));
    const int64_t most = (int64_t)(N > C ? N : C);
    const int64_t hist_elems = (int64_t)256 * cdiv(most, kTileItems);
    L.hist = take(4 * (size_t)hist_elems);
    L.hscan = take(4 * scan_scratch_elems(hist_elems));
    L.tk0 = take(4 * C);
    L.tk1 = take(4 * C);
    L.tv0 = take(4 * C);
    L.tv1 = take(4 * C);
    L.total = o;
    return L;
}

}  // namespace

size_t bin_sort_workspace_bytes(int n_items, int64_t capacity, int /*num_tiles*/) {
    return make_layout(n_items, capacity).total;
}

gs_status bin_sort_run(const SortViews& sv, const float* mean2d_f, const int* radius, const float* depth,
                       int64_t capacity, void* ws, size_t /*ws_bytes*/, uint64_t* keys_sorted, uint32_t* ids_sorted,
                       uint32_t* tile_ranges, int64_t* n_instances_host, int64_t* n_instances_dev, cudaStream_t s) {
    const int ntiles = sv.total_tiles;
    const int n = sv.num_views * sv.n_per_view;  // items
    const bool graph = n_instances_host == nullptr;
    cudaError_t e = cudaMemsetAsync(tile_ranges, 0, sizeof(uint32_t) * 2 * (size_t)ntiles, s);
    if (e != cudaSuccess) return cuda_status(e, "gs_bin_sort: clear ranges");
    if (!graph) *n_instances_host = 0;
    if (n == 0) {
        if (graph && (e = cudaMemsetAsync(n_instances_dev, 0, sizeof(int64_t), s)) != cudaSuccess)
            return cuda_status(e, "gs_bin_sort: count");
        return GS_OK;
    }
    unsigned* err = error_word();
    if (err == nullptr) return cuda_status(cudaGetLastError(), "gs_bin_sort: error word");
    const Layout L = make_layout(n, capacity);
    char* base = static_cast<char*>(ws);
    auto U32 = [&](size_t off) { return reinterpret_cast<uint32_t*>(base + off); };
    const float2* mean2d = reinterpret_cast<const float2*>(mean2d_f);
    RadixScratch rs{U32(L.hist), U32(L.hscan)};

    // 1. counts and depth keys; depth sort of all items
    k_count<<<cdiv(n, 256), 256, 0, s>>>(n, sv, mean2d, radius, depth, U32(L.cnt), U32(L.dk0), U32(L.dv0));
    count_launches();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e, "gs_bin_sort: count");
    uint32_t* dk[2] = {U32(L.dk0), U32(L.dk1)};
    uint32_t* dv[2] = {U32(L.dv0), U32(L.dv1)};
    int which = 0;
    if ((e = radix_sort(dk, dv, (uint32_t)n, nullptr, 32, rs, &which, s)) != cudaSuccess)
        return cuda_status(e, "gs_bin_sort: depth sort");
    const uint32_t* perm = dv[which];

    // 2. offsets of each item's instances in depth order
    uint64_t* c64 = reinterpret_cast<uint64_t*>(base + L.c64);
    uint64_t* offs = reinterpret_cast<uint64_t*>(base + L.offs);
    k_gather_counts<<<cdiv(n, 256), 256, 0, s>>>(n, perm, U32(L.cnt), c64);
    count_launches();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e, "gs_bin_sort: gather");
    if ((e = scan_exclusive<uint64_t>(c64, offs, n, reinterpret_cast<uint64_t*>(base + L.sscan), true, s)) !=
        cudaSuccess)
        return cuda_status(e, "gs_bin_sort: scan");
    uint64_t I = 0;
    const uint64_t* I_dev = nullptr;
    uint32_t I_grid = 0;  // items the remaining kernels are launched for
    if (!graph) {
        if ((e = cudaMemcpyAsync(&I, offs + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return cuda_status(e, "gs_bin_sort: read count");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_status(e, "gs_bin_sort: synchronize");
        *n_instances_host = (int64_t)I;
        if ((int64_t)I > capacity) {
            set_error("gs_bin_sort: %llu instances exceed capacity %lld", (unsigned long long)I, (long long)capacity);
            return GS_ERR_CAPACITY;
        }
        if (I == 0) return GS_OK;
        I_grid = (uint32_t)I;
    } else {
        if (capacity == 0) {
            k_duplicate<<<1, 32, 0, s>>>(0, 0, n, offs, perm, sv, mean2d, radius, nullptr, nullptr,
                                         n_instances_dev, err);
            count_launches();
            return cuda_status(cudaGetLastError(), "gs_bin_sort: count");
        }
        I_dev = offs + n;
        I_grid = (uint32_t)capacity;
    }

    // 3. duplicate, then stable sort by global tile id
    uint32_t* tk[2] = {U32(L.tk0), U32(L.tk1)};
    uint32_t* tv[2] = {U32(L.tv0), U32(L.tv1)};
    k_duplicate<<<cdiv((int64_t)I_grid, 256), 256, 0, s>>>((uint32_t)I, capacity, n, offs, perm, sv, mean2d, radius,
                                                            tk[0], tv[0], graph ? n_instances_dev : nullptr, err);
    count_launches();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e, "gs_bin_sort: duplicate");
    int tile_bits = 1;
    while ((1ll << tile_bits) < ntiles) ++tile_bits;
    if ((e = radix_sort(tk, tv, I_grid, I_dev, tile_bits, rs, &which, s)) != cudaSuccess)
        return cuda_status(e, "gs_bin_sort: tile sort");
    k_finalize<<<cdiv((int64_t)I_grid, 256), 256, 0, s>>>(I_grid, I_dev, tk[which], tv[which], depth, keys_sorted,
                                                         ids_sorted, tile_ranges);
    count_launches();
    return cuda_status(cudaGetLastError(), "gs_bin_sort: finalize");
}

}  // namespace gs
