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
//
// Every radix pass is one launch.  The digit histograms of all passes are
// counted up front by the kernel that produces the keys (the counts of an LSD
// pass do not depend on the order the previous pass leaves), and each block
// finds where its digits go among the blocks before it by decoupled
// look-back: blocks take tile numbers from an atomic ticket in the order they
// start, publish their per-digit counts, then add up their predecessors'
// published counts until one carries an inclusive prefix.  A block only waits
// for blocks that started before it, so the waits always end; each is still
// bounded in time and sets the timeout bit of the error word if it gives up.
// The scan of instance counts in depth order is done the same way inside the
// duplication kernel, so the whole stage is
//   memset, count, 4 depth passes, duplicate, ceil(bits / 8) tile passes, finalize.
#include <algorithm>

#include "internal.h"
#include "tight.cuh"

namespace gs {
namespace {

constexpr int kThreads = 256;
constexpr uint32_t kSmallPass = 1u << 20;  // passes up to this size use 1024-item tiles, larger ones 4096
constexpr int kDupItems = 1;                // items per thread of the duplication kernel
constexpr int kDupTile = kThreads * kDupItems;
constexpr int kMaxPasses = 8;               // 4 depth passes + up to 4 tile-id passes
constexpr uint64_t kLookbackLimitNs = 2000000000ull;

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
inline int pass_items(uint64_t n) { return n <= kSmallPass ? 4 : 16; }
// Most radix tiles a pass over at most m items can have.
inline int64_t radix_tiles_max(int64_t m) {
    return std::max(cdiv(std::min<int64_t>(m, kSmallPass), kThreads * 4), cdiv(m, kThreads * pass_items(m)));
}

// ---------------------------------------------------------- block helpers --

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

// ------------------------------------------------------ look-back status --
//
// A status word holds a tag in bits [56, 64) and a count in bits [0, 56).
// Pass p publishes tag 2p + 1 (this block's own count) and then 2p + 2 (the
// inclusive prefix up to and including this block); any other tag (zero after
// the clear, or a value an earlier pass left in the same word) means "not yet".

constexpr uint64_t kValMask = (uint64_t(1) << 56) - 1;

__device__ __forceinline__ void st_status(unsigned long long* p, uint32_t tag, uint64_t v) {
    const unsigned long long w = ((unsigned long long)tag << 56) | (v & kValMask);
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}
__device__ __forceinline__ unsigned long long ld_status(const unsigned long long* p) {
    unsigned long long w;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
    return w;
}

// Sum of the counts of tiles [0, tile) for one digit, walking back from
// tile - 1 until an inclusive prefix is found.  Eight predecessors are read
// per round trip; the ready ones nearest to this tile are consumed, up to the
// first inclusive prefix.
__device__ __forceinline__ uint64_t lookback_serial(const unsigned long long* status, int64_t tile, int stride,
                                                    int d, uint32_t tag_agg, unsigned* err) {
    constexpr int W = 8;
    uint64_t prefix = 0, t0 = 0;
    int64_t j = tile - 1;
    while (j >= 0) {
        unsigned long long w[W];
#pragma unroll
        for (int q = 0; q < W; ++q)
            w[q] = j - q >= 0 ? ld_status(status + (size_t)(j - q) * stride + d)
                              : ((unsigned long long)(tag_agg + 1) << 56);  // before tile 0: 0
        int used = 0;
        bool done = false, blocked = false;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            if (done || blocked) continue;
            const uint32_t tag = (uint32_t)(w[q] >> 56);
            if (tag == tag_agg || tag == tag_agg + 1) {
                prefix += w[q] & kValMask;
                ++used;
                done = tag == tag_agg + 1;
            } else {
                blocked = true;
            }
        }
        if (done) break;
        j -= used;
        if (blocked) {
            const uint64_t now = globaltimer_ns();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > kLookbackLimitNs) {
                atomicOr(err, kErrTimeout);
                break;
            }
        }
    }
    return prefix;
}

// The same for a single count per tile, by one warp over windows of 32
// predecessors (lane l reads tile j - l).  Every lane returns the prefix.
__device__ __forceinline__ uint64_t lookback_warp(const unsigned long long* status, int64_t tile, uint32_t tag_agg,
                                                  unsigned* err) {
    const int lane = threadIdx.x & 31;
    uint64_t prefix = 0, t0 = 0;
    int64_t j = tile - 1;
    while (j >= 0) {
        const int64_t jj = j - lane;
        const unsigned long long w =
            jj >= 0 ? ld_status(status + jj) : ((unsigned long long)(tag_agg + 1) << 56);  // before tile 0: 0
        const uint32_t tag = (uint32_t)(w >> 56);
        const unsigned inc = __ballot_sync(0xffffffffu, tag == tag_agg + 1);
        const unsigned notready = __ballot_sync(0xffffffffu, tag != tag_agg && tag != tag_agg + 1);
        const int first_inc = inc ? __ffs(inc) - 1 : 32;
        const unsigned needed = first_inc == 32 ? 0xffffffffu : (0xffffffffu >> (31 - first_inc));
        if (notready & needed) {
            const uint64_t now = globaltimer_ns();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > kLookbackLimitNs) {
                if (lane == 0) atomicOr(err, kErrTimeout);
                break;
            }
            continue;
        }
        uint64_t v = lane <= first_inc ? (uint64_t)(w & kValMask) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        prefix += v;
        if (first_inc < 32) break;
        j -= 32;
    }
    return prefix;
}

// The lanes of the warp whose digit equals this lane's, among the valid lanes
// (an invalid lane gets only itself).  FULL: one ballot per bit of the 8-bit
// digit, a cost that does not grow with the number of distinct digits in the
// warp (random digits: up to 32); otherwise __match_any_sync, cheap when the
// digit has only a few significant bits (the last pass over a short key).
template <bool FULL>
__device__ __forceinline__ unsigned digit_peers(uint32_t d, bool valid) {
    const unsigned lane_bit = 1u << (threadIdx.x & 31);
    if constexpr (!FULL) return __match_any_sync(0xffffffffu, valid ? d : 0x100u + (threadIdx.x & 31));
    unsigned m = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const bool bit = (d >> b) & 1u;
        const unsigned bal = __ballot_sync(0xffffffffu, bit);
        m &= bit ? bal : ~bal;
    }
    return valid ? m : lane_bit;
}

// s_h[bin] += 1 for every active lane, one atomic per distinct bin in the warp
// (digits of nearby keys often agree, and same-address shared atomics serialise).
__device__ __forceinline__ void hist_add(uint32_t* s_h, uint32_t bin) {
    const unsigned peers = __match_any_sync(__activemask(), bin);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&s_h[bin], (uint32_t)__popc(peers));
}

// Item count of a pass: the host value, or min(*n_dev, host value) in graph mode.
__device__ __forceinline__ uint32_t pass_count(uint32_t n_host, const uint64_t* n_dev) {
    if (n_dev == nullptr) return n_host;
    const uint64_t v = *n_dev;
    return v < n_host ? (uint32_t)v : n_host;
}

// ------------------------------------------------------------ radix pass --

// One stable pass on bits [shift, shift + 8).  The block takes the next tile
// of TILE items from the ticket; warp w owns the contiguous items
// [w * 32 ITEMS, (w + 1) * 32 ITEMS) walked in rounds of 32, so lane order is
// input order, and each item's rank among equal digits comes from the lanes
// with the same digit (digit_peers; FULL: ballots, for digits of more than
// 4 significant bits).  Items are placed in shared memory in digit order, then
// written so that consecutive threads write consecutive addresses of each
// digit's run.  hist holds the pass's global digit counts.
template <int ITEMS, bool FULL>
__global__ void __launch_bounds__(kThreads, 4) k_onesweep(const uint32_t* __restrict__ kin,
                                                       const uint32_t* __restrict__ vin, uint32_t n_host,
                                                       const uint64_t* __restrict__ n_dev, int shift, int pass_id,
                                                       const uint32_t* __restrict__ hist, uint32_t* tickets,
                                                       unsigned long long* status, uint32_t* __restrict__ kout,
                                                       uint32_t* __restrict__ vout, unsigned* err) {
    constexpr int TILE = kThreads * ITEMS;
    __shared__ uint32_t s_w[kThreads / 32][256];  // per-warp digit counts, then local bases
    __shared__ uint32_t s_dbase[256];              // block-local start of each digit's run
    __shared__ uint32_t s_goff[256];               // global start of each digit's run
    __shared__ uint32_t s_warp[kThreads / 32 + 1];
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_key[TILE], s_val[TILE];
    const uint32_t n = pass_count(n_host, n_dev);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = atomicAdd(&tickets[pass_id], 1u);
    for (int i = threadIdx.x; i < (kThreads / 32) * 256; i += kThreads) (&s_w[0][0])[i] = 0;
    __syncthreads();
    const uint32_t tile = s_tile;
    const int64_t bbase = (int64_t)tile * TILE;
    if (bbase >= n) return;  // uniform over the block; no later tile is needed either
    const int cnt = (int)((int64_t)n - bbase < TILE ? (int64_t)n - bbase : TILE);
    const int wbase = warp * (ITEMS * 32);
    uint32_t k[ITEMS], v[ITEMS];
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
        const int i = wbase + r * 32 + lane;
        k[r] = i < cnt ? kin[bbase + i] : 0u;
        v[r] = i < cnt ? vin[bbase + i] : 0u;
    }
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
        const bool valid = wbase + r * 32 + lane < cnt;
        const uint32_t d = (k[r] >> shift) & 0xFFu;
        const unsigned peers = digit_peers<FULL>(d, valid);
        if (valid && (peers & lt) == 0) s_w[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        const int d = threadIdx.x;
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) c += s_w[w][d];
        unsigned long long* mine = status + (size_t)tile * 256 + d;
        const uint32_t tag_agg = 2u * pass_id + 1u;
        st_status(mine, tile == 0 ? tag_agg + 1 : tag_agg, c);  // publish first, successors may be waiting
        uint32_t total;
        const uint32_t db = block_excl_scan<uint32_t, kThreads>(c, total, s_warp);
        const uint32_t gstart = block_excl_scan<uint32_t, kThreads>(hist[d], total, s_warp);
        uint32_t prefix = 0;
        if (tile > 0) {
            prefix = (uint32_t)lookback_serial(status, tile, 256, d, tag_agg, err);
            st_status(mine, tag_agg + 1, prefix + c);
        }
        s_dbase[d] = db;
        s_goff[d] = gstart + prefix;
        uint32_t run = db;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) {
            const uint32_t cw = s_w[w][d];
            s_w[w][d] = run;
            run += cw;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
        const bool valid = wbase + r * 32 + lane < cnt;
        const uint32_t d = (k[r] >> shift) & 0xFFu;
        const unsigned peers = digit_peers<FULL>(d, valid);
        uint32_t pos = 0;
        if (valid) pos = s_w[warp][d] + __popc(peers & lt);
        __syncwarp();
        if (valid) {
            s_key[pos] = k[r];
            s_val[pos] = v[r];
            if ((peers & lt) == 0) s_w[warp][d] += __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += kThreads) {
        const uint32_t key = s_key[i];
        const uint32_t d = (key >> shift) & 0xFFu;
        const uint32_t g = s_goff[d] + (uint32_t)i - s_dbase[d];
        if (g < n) {  // always, unless a look-back gave up (timeout bit set)
            kout[g] = key;
            vout[g] = s_val[i];
        }
    }
}

struct PassScratch {
    const uint32_t* hist;  // [kMaxPasses][256] digit counts
    uint32_t* tickets;     // [kMaxPasses]
    unsigned long long* status;
    unsigned* err;
};

// Stable LSD sort of (k[0], v[0]) on bits [0, bits) with pass ids
// first_pass, first_pass + 1, ...; the result ends in buffer *which.  n_host
// sizes the grid; in graph mode the passes sort min(*n_dev, n_host) items.
cudaError_t radix_sort(uint32_t* k[2], uint32_t* v[2], uint32_t n_host, const uint64_t* n_dev, int bits,
                       int first_pass, const PassScratch& ps, int* which, cudaStream_t s) {
    int cur = 0;
    const int items = pass_items(n_host);
    const int nblk = (int)cdiv(n_host, (int64_t)kThreads * items);
    for (int p = 0, shift = 0; shift < bits; ++p, shift += 8) {
        const int id = first_pass + p;
        // ballots unless the digit has at most 4 significant bits (16 values: match_any is cheaper);
        // the ballot of an unused high bit is the same for every lane
        const bool full = bits - shift > 4;
        auto kern = items == 4 ? (full ? k_onesweep<4, true> : k_onesweep<4, false>)
                               : (full ? k_onesweep<16, true> : k_onesweep<16, false>);
        kern<<<nblk, kThreads, 0, s>>>(k[cur], v[cur], n_host, n_dev, shift, id, ps.hist + 256 * id, ps.tickets,
                                       ps.status, k[cur ^ 1], v[cur ^ 1], ps.err);
        count_launches();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        cur ^= 1;
    }
    *which = cur;
    return cudaSuccess;
}

// ------------------------------------------------------ duplicate/finalize --

// ----------------------------------------------- opacity-aware membership --
//
// With sv.conic and sv.power_min set, tiles are kept by the rule of tight.cuh.
__device__ __forceinline__ TightRows item_tight_rows(const SortViews& sv, const float2* mean2d, uint32_t item) {
    const float2 m = mean2d[item];
    const uint32_t g = item - (item / (uint32_t)sv.n_per_view) * (uint32_t)sv.n_per_view;
    return tight_rows(m.x, m.y, sv.conic[3 * (size_t)item], sv.conic[3 * (size_t)item + 1],
                      sv.conic[3 * (size_t)item + 2], sv.power_min[g]);
}

// Per item: its tile count and depth key; the depth keys' four digit
// histograms (pass ids 0..3).  Also clears the tile ranges and the look-back
// status words for this call.  Each thread takes ITEMS items, strided by the
// block size, with all loads issued before any use.  TIGHT: opacity-aware
// counts, one O(1) run per rectangle row.
constexpr int kCountItems = 4, kCountItemsTight = 2;
template <bool TIGHT, int ITEMS>
__global__ void __launch_bounds__(kThreads) k_count(int n_items, const __grid_constant__ SortViews sv,
                                                    const float2* __restrict__ mean2d,
                                                    const int* __restrict__ radius, const float* __restrict__ depth,
                                                    uint32_t* __restrict__ cnt, uint32_t* __restrict__ dkey,
                                                    uint32_t* __restrict__ dval, uint32_t* __restrict__ hist,
                                                    uint4* __restrict__ clear, size_t clear_n,
                                                    uint32_t* __restrict__ ranges, size_t ranges_n) {
    __shared__ uint32_t s_h[4 * 256];
    for (int i = threadIdx.x; i < 4 * 256; i += kThreads) s_h[i] = 0;
    const int64_t base = (int64_t)blockIdx.x * (kThreads * ITEMS) + threadIdx.x;
    float2 m[ITEMS];
    int r[ITEMS];
    uint32_t key[ITEMS];
#pragma unroll
    for (int q = 0; q < ITEMS; ++q) {
        const int64_t i = base + q * kThreads;
        const bool ok = i < n_items;
        m[q] = ok ? mean2d[i] : make_float2(0.f, 0.f);
        r[q] = ok ? radius[i] : 0;
        key[q] = ok ? __float_as_uint(depth[i]) : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < ITEMS; ++q) {
        const int64_t i = base + q * kThreads;
        if (i >= n_items) continue;
        const ViewDesc& vd = sv.views[(int)i / sv.n_per_view];
        int x0, x1, y0, y1;
        uint32_t c = 0;
        if (tile_rect(m[q].x, m[q].y, r[q], vd.W, vd.H, x0, x1, y0, y1)) {
            if constexpr (TIGHT) {
                const TightRows t = item_tight_rows(sv, mean2d, (uint32_t)i);
                for (int y = y0; y <= y1; ++y) {
                    int f, l;
                    tight_row(t, y, x0, x1, f, l);
                    c += (uint32_t)max(l - f + 1, 0);
                }
            } else {
                c = (uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1));
            }
        }
        cnt[i] = c;
        dkey[i] = key[q];
        dval[i] = (uint32_t)i;
#pragma unroll
        for (int p = 0; p < 4; ++p) hist_add(s_h, p * 256 + ((key[q] >> (8 * p)) & 0xFFu));
    }
    const size_t stride = (size_t)gridDim.x * kThreads;
    const uint4 z = make_uint4(0, 0, 0, 0);
    for (size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x; i < clear_n; i += stride) clear[i] = z;
    for (size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x; i < ranges_n; i += stride) ranges[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * 256; i += kThreads)
        if (s_h[i]) atomicAdd(&hist[i], s_h[i]);
}

// Digit histograms of the tile ids [a, a + w) of one rectangle row, by runs:
// a run inside one aligned block of 256 ids has constant digits 1..3, and its
// digit-0 values form a contiguous range, added to the difference array s_d0
// (the histogram of digit 0 is its prefix sum).
__device__ __forceinline__ void row_hist(uint32_t a, uint32_t w, int passes, int* s_d0, uint32_t* s_h) {
    while (w > 0) {
        const uint32_t lo = a & 0xFFu, len = min(w, 256u - lo);
        atomicAdd(&s_d0[lo], 1);
        atomicSub(&s_d0[lo + len], 1);
        for (int p = 1; p < passes; ++p) atomicAdd(&s_h[(p - 1) * 256 + ((a >> (8 * p)) & 0xFFu)], len);
        a += len;
        w -= len;
    }
}

// Duplication in depth order with the scan of instance counts folded in.
// Tile t (from the ticket) holds the depth-ordered items
// [t * kDupTile, (t + 1) * kDupTile) in kDupItems rounds of 256; the tile's
// instance offset comes from decoupled look-back over the tiles before it.
// Each item's instances are its rectangle's tiles (TIGHT: each row's run of
// tiles that meet the opacity-aware rule), row-major, at [offset, offset +
// count).  Full rectangles: each warp writes its items of at most 32
// instances as one flat, coalesced sequence, then each bigger item with the
// whole warp.  TIGHT: one thread per item, an item of more than 32 instances
// by the whole warp.
// Writes stop at `limit`; the total goes to *total and, in graph
// mode, to *count_out, with kErrCapacity raised when it exceeds the capacity.
// The digit histograms of the written instances' tile ids go to hist
// (tile_passes of them), so a truncated list still sorts into a permutation
// of what was written.
template <bool TIGHT>
__global__ void __launch_bounds__(kThreads) k_duplicate(int n_items, const uint32_t* __restrict__ perm,
                                                        const uint32_t* __restrict__ cnt,
                                                        const __grid_constant__ SortViews sv,
                                                        const float2* __restrict__ mean2d,
                                                        const int* __restrict__ radius, uint64_t limit,
                                                        int tile_passes, uint32_t* tickets,
                                                        unsigned long long* status, uint32_t* __restrict__ tkey,
                                                        uint32_t* __restrict__ tval, uint32_t* __restrict__ hist,
                                                        uint64_t* __restrict__ total, int64_t* __restrict__ count_out,
                                                        unsigned* err) {
    __shared__ uint64_t s_warp[kThreads / 32 + 1];
    __shared__ uint64_t s_prefix;
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_h[3 * 256];  // digits 1..3
    __shared__ int s_d0[257];          // digit 0, as a difference array
    __shared__ int s_warp_i[kThreads / 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = atomicAdd(&tickets[kMaxPasses], 1u);
    for (int i = threadIdx.x; i < 3 * 256; i += kThreads) s_h[i] = 0;
    for (int i = threadIdx.x; i < 257; i += kThreads) s_d0[i] = 0;
    __syncthreads();
    const uint32_t tile = s_tile;
    const int64_t base = (int64_t)tile * kDupTile;
    if (base >= n_items) return;

    uint32_t item[kDupItems], c[kDupItems];
    uint64_t local[kDupItems];
    uint64_t tile_sum = 0;
#pragma unroll
    for (int r = 0; r < kDupItems; ++r) {
        const int64_t k = base + r * kThreads + threadIdx.x;
        item[r] = k < n_items ? perm[k] : 0u;
        c[r] = k < n_items ? cnt[item[r]] : 0u;
        uint64_t rt;
        local[r] = tile_sum + block_excl_scan<uint64_t, kThreads>((uint64_t)c[r], rt, s_warp);
        tile_sum += rt;
    }
    unsigned long long* mine = status + tile;
    if (warp == 0) {
        if (lane == 0) st_status(mine, tile == 0 ? 2u : 1u, tile_sum);
        uint64_t prefix = 0;
        if (tile > 0) {
            prefix = lookback_warp(status, tile, 1u, err);
            if (lane == 0) st_status(mine, 2u, prefix + tile_sum);
        }
        if (lane == 0) {
            s_prefix = prefix;
            if (base + kDupTile >= n_items) {  // the last tile: the total
                const uint64_t all = prefix + tile_sum;
                *total = all;
                if (count_out != nullptr) {
                    *count_out = (int64_t)all;
                    if (all > limit) atomicOr(err, kErrCapacity);
                }
            }
        }
    }
    __syncthreads();
    const uint64_t prefix = s_prefix;

    if constexpr (!TIGHT) {
#pragma unroll
    for (int r = 0; r < kDupItems; ++r) {
        uint32_t w = 1, h = 0, tile0 = 0, tx = 0;
        if (c[r] > 0) {
            const ViewDesc& vd = sv.views[item[r] / (uint32_t)sv.n_per_view];
            int x0, x1, y0, y1;
            const float2 m = mean2d[item[r]];
            tile_rect(m.x, m.y, radius[item[r]], vd.W, vd.H, x0, x1, y0, y1);
            w = (uint32_t)(x1 - x0 + 1);
            h = (uint32_t)(y1 - y0 + 1);
            tx = (uint32_t)vd.tiles_x;
            tile0 = (uint32_t)vd.tile_begin + (uint32_t)y0 * tx + (uint32_t)x0;
        }
        const uint64_t off = prefix + local[r];
        // written: all of the item's instances unless the capacity cuts it
        const uint32_t nw = off >= limit ? 0u : (uint32_t)min((uint64_t)c[r], limit - off);
        const bool big = c[r] > 32;
        if (!big)
            for (uint32_t y = 0; y * w < nw; ++y) row_hist(tile0 + y * tx, min(w, nw - y * w), tile_passes, s_d0, s_h);
        // Items of at most 32 instances, flat and coalesced: the warp walks the
        // concatenation of their ranges (offsets exs, compacted over these items)
        // 32 positions at a time; position j belongs to the last lane whose
        // range starts at or before j (a lane without such an item shares its
        // start with the next lane).
        const uint32_t cs = big ? 0u : c[r];
        uint32_t incl = cs;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        const uint32_t exs = incl - cs, tot_s = __shfl_sync(0xffffffffu, incl, 31);
        for (uint32_t j0 = 0; j0 < tot_s; j0 += 32) {
            const uint32_t j = j0 + lane;
            int k = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (__shfl_sync(0xffffffffu, exs, k + step) <= j) k += step;
            const uint32_t q = j - __shfl_sync(0xffffffffu, exs, k);
            const uint64_t p = __shfl_sync(0xffffffffu, off, k) + q;
            const uint32_t kw = __shfl_sync(0xffffffffu, w, k);  // 1 for a lane without instances
            const uint32_t kt = __shfl_sync(0xffffffffu, tile0, k) + (q / kw) * __shfl_sync(0xffffffffu, tx, k) + q % kw;
            const uint32_t ki = __shfl_sync(0xffffffffu, item[r], k);
            if (j < tot_s && p < limit) {
                tkey[p] = kt;
                tval[p] = ki;
            }
        }
        unsigned bigs = __ballot_sync(0xffffffffu, big);
        while (bigs) {  // a bigger item: the whole warp, one row's histogram per lane, the instances flat
            const int src = __ffs(bigs) - 1;
            bigs &= bigs - 1;
            const uint32_t bi = __shfl_sync(0xffffffffu, item[r], src), bnw = __shfl_sync(0xffffffffu, nw, src);
            const uint32_t bw = __shfl_sync(0xffffffffu, w, src), bt0 = __shfl_sync(0xffffffffu, tile0, src);
            const uint32_t btx = __shfl_sync(0xffffffffu, tx, src), bh = __shfl_sync(0xffffffffu, h, src);
            const uint64_t boff = __shfl_sync(0xffffffffu, off, src);
            for (uint32_t y = lane; y < bh && y * bw < bnw; y += 32)
                row_hist(bt0 + y * btx, min(bw, bnw - y * bw), tile_passes, s_d0, s_h);
            for (uint32_t j = lane; j < bnw; j += 32) {
                tkey[boff + j] = bt0 + (j / bw) * btx + j % bw;
                tval[boff + j] = bi;
            }
        }
    }
    } else {
#pragma unroll
    for (int r = 0; r < kDupItems; ++r) {
        int x0 = 0, x1 = -1, y0 = 0, y1 = -1;
        uint32_t rowbase = 0, tx = 0;
        TightRows t{};
        if (c[r] > 0) {
            const ViewDesc& vd = sv.views[item[r] / (uint32_t)sv.n_per_view];
            const float2 m = mean2d[item[r]];
            tile_rect(m.x, m.y, radius[item[r]], vd.W, vd.H, x0, x1, y0, y1);
            tx = (uint32_t)vd.tiles_x;
            rowbase = (uint32_t)vd.tile_begin;
            t = item_tight_rows(sv, mean2d, item[r]);
        }
        const uint64_t off = prefix + local[r];
        const bool big = c[r] > 32;
        if (c[r] > 0 && !big) {
            uint64_t pos = off;
            for (int y = y0; y <= y1 && pos < limit; ++y) {
                int f, l;
                tight_row(t, y, x0, x1, f, l);
                if (f > l) continue;
                const uint32_t t0 = rowbase + (uint32_t)y * tx + (uint32_t)f;
                const uint32_t len = (uint32_t)(l - f + 1);
                const uint32_t nw = (uint32_t)min((uint64_t)len, limit - pos);  // written (capacity)
                for (uint32_t j = 0; j < nw; ++j) {
                    tkey[pos + j] = t0 + j;
                    tval[pos + j] = item[r];
                }
                row_hist(t0, nw, tile_passes, s_d0, s_h);
                pos += len;
            }
        }
        unsigned bigs = __ballot_sync(0xffffffffu, big);
        while (bigs) {  // the whole warp, 32 rows at a time
            const int src = __ffs(bigs) - 1;
            bigs &= bigs - 1;
            const uint32_t bi = __shfl_sync(0xffffffffu, item[r], src);
            const int bx0 = __shfl_sync(0xffffffffu, x0, src), bx1 = __shfl_sync(0xffffffffu, x1, src);
            const int by0 = __shfl_sync(0xffffffffu, y0, src), by1 = __shfl_sync(0xffffffffu, y1, src);
            const uint32_t btx = __shfl_sync(0xffffffffu, tx, src), brb = __shfl_sync(0xffffffffu, rowbase, src);
            uint64_t pos = __shfl_sync(0xffffffffu, off, src);
            TightRows bt;
            bt.mode = __shfl_sync(0xffffffffu, t.mode, src);
            bt.mx = __shfl_sync(0xffffffffu, t.mx, src);
            bt.my = __shfl_sync(0xffffffffu, t.my, src);
            bt.nB = __shfl_sync(0xffffffffu, t.nB, src);
            bt.det = __shfl_sync(0xffffffffu, t.det, src);
            bt.Atau = __shfl_sync(0xffffffffu, t.Atau, src);
            bt.rA = __shfl_sync(0xffffffffu, t.rA, src);
            bt.ymax = __shfl_sync(0xffffffffu, t.ymax, src);
            bt.dyr = __shfl_sync(0xffffffffu, t.dyr, src);
            for (int yb = by0; yb <= by1 && pos < limit; yb += 32) {
                // lane k: row yb + k's run, its offset among the 32 rows' instances and its histogram
                int f = 0, l = -1;
                if (yb + lane <= by1) tight_row(bt, yb + lane, bx0, bx1, f, l);
                const uint32_t len = (uint32_t)max(l - f + 1, 0);
                uint32_t incl = len;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
                    if (lane >= d) incl += v;
                }
                const uint32_t excl = incl - len, rows_total = __shfl_sync(0xffffffffu, incl, 31);
                const uint32_t t0 = brb + (uint32_t)(yb + lane) * btx + (uint32_t)f;  // used where len > 0
                const uint64_t rpos = pos + excl;
                if (len > 0 && rpos < limit)
                    row_hist(t0, (uint32_t)min((uint64_t)len, limit - rpos), tile_passes, s_d0, s_h);
                // the instances flat: element j belongs to the last row whose offset is <= j
                const uint32_t nw = (uint32_t)min((uint64_t)rows_total, limit - pos);
                for (uint32_t j0 = 0; j0 < nw; j0 += 32) {
                    const uint32_t j = j0 + lane;
                    int k = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1)
                        if (__shfl_sync(0xffffffffu, excl, k + step) <= j) k += step;
                    const uint32_t kt0 = __shfl_sync(0xffffffffu, t0, k), kex = __shfl_sync(0xffffffffu, excl, k);
                    if (j < nw) {
                        tkey[pos + j] = kt0 + (j - kex);
                        tval[pos + j] = bi;
                    }
                }
                pos += rows_total;
            }
        }
    }
    }
    __syncthreads();
    {
        int tot;
        const int v = s_d0[threadIdx.x];
        const int d0 = block_excl_scan<int, kThreads>(v, tot, s_warp_i) + v;  // count of digit-0 value threadIdx.x
        if (d0) atomicAdd(&hist[threadIdx.x], (uint32_t)d0);
    }
    for (int i = threadIdx.x; i < (tile_passes - 1) * 256; i += kThreads)
        if (s_h[i]) atomicAdd(&hist[256 + i], s_h[i]);
}

// Sorted keys (if asked for), ids and tile ranges.  Tile ids and item indices are checked
// against their bounds: after a look-back that gave up (timeout bit set) the
// passes can leave stale entries, which become item 0 and no range.
__global__ void k_finalize(uint32_t I_host, const uint64_t* __restrict__ I_dev, const uint32_t* __restrict__ tkey,
                           const uint32_t* __restrict__ tval, const float* __restrict__ depth, uint32_t n_items,
                           uint32_t num_tiles, uint64_t* __restrict__ keys_sorted, uint32_t* __restrict__ ids_sorted,
                           uint32_t* __restrict__ ranges) {
    const uint32_t I = pass_count(I_host, I_dev);
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= I) return;
    const uint32_t t = tkey[i];
    const uint32_t g = tval[i] < n_items ? tval[i] : 0u;
    if (keys_sorted != nullptr) keys_sorted[i] = ((uint64_t)t << 32) | __float_as_uint(depth[g]);
    ids_sorted[i] = g;
    if (t >= num_tiles) return;
    if (i == 0 || tkey[i - 1] != t) ranges[2 * t] = i;
    if (i == I - 1 || tkey[i + 1] != t) ranges[2 * t + 1] = i + 1;
}

// Workspace: per-item arrays, a header cleared by one memset (digit
// histograms, tickets, total), the look-back status words (cleared by
// k_count), and the instance key/value double buffers.
struct Layout {
    size_t cnt, dk0, dk1, dv0, dv1, hdr, hist, tickets, total, hdr_bytes, status, status_bytes, tk0, tk1, tv0, tv1,
        total_bytes;
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
    L.hdr = o;
    L.hist = take(4 * 256 * kMaxPasses);
    L.tickets = take(4 * (kMaxPasses + 1));
    L.total = take(8);
    L.hdr_bytes = o - L.hdr;
    // status words: 256 per radix tile (the largest tile count of either sort)
    // plus one per duplication tile
    const size_t radix_tiles = (size_t)std::max(radix_tiles_max((int64_t)N), radix_tiles_max((int64_t)C));
    L.status = take(8 * (256 * radix_tiles + (size_t)cdiv((int64_t)N, kDupTile)));
    L.status_bytes = o - L.status;  // a multiple of 256
    L.tk0 = take(4 * C);
    L.tk1 = take(4 * C);
    L.tv0 = take(4 * C);
    L.tv1 = take(4 * C);
    L.total_bytes = o;
    return L;
}

}  // namespace

namespace {
// power_min[g] = ln(1 / (255 o_g)) - kTightMargin: the exponent a splat must reach
// for alpha = o exp(power) >= 1/255, lowered by a margin that covers the
// exponent error of the blend variants (the split tensor-core ones are <= 1e-3);
// +inf for o below the blend's FP32 threshold 1/255 (alpha <= o never reaches
// it; o equal to it still passes where the exponent is 0).
constexpr float kTightMargin = 2e-3f;
__global__ void k_alpha_power_min(int n, const float* __restrict__ opacity, float* __restrict__ out) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const float o = opacity[g];
    out[g] = o >= 1.0f / 255.0f ? -logf(255.0f * o) - kTightMargin : INFINITY;
}
}  // namespace

cudaError_t launch_alpha_power_min(int n, const float* opacity, float* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_alpha_power_min<<<(n + 255) / 256, 256, 0, s>>>(n, opacity, out);
    count_launches();
    return cudaGetLastError();
}

size_t bin_sort_workspace_bytes(int n_items, int64_t capacity, int /*num_tiles*/) {
    return make_layout(n_items, capacity).total_bytes;
}

gs_status bin_sort_run(const SortViews& sv, const float* mean2d_f, const int* radius, const float* depth,
                       int64_t capacity, void* ws, size_t /*ws_bytes*/, uint64_t* keys_sorted, uint32_t* ids_sorted,
                       uint32_t* tile_ranges, int64_t* n_instances_host, int64_t* n_instances_dev, cudaStream_t s) {
    const int ntiles = sv.total_tiles;
    const int n = sv.num_views * sv.n_per_view;  // items
    const bool graph = n_instances_host == nullptr;
    cudaError_t e;
    if (!graph) *n_instances_host = 0;
    if (n == 0) {
        if ((e = cudaMemsetAsync(tile_ranges, 0, sizeof(uint32_t) * 2 * (size_t)ntiles, s)) != cudaSuccess)
            return cuda_status(e, "gs_bin_sort: clear ranges");
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
    uint32_t* hist = U32(L.hist);
    uint32_t* tickets = U32(L.tickets);
    uint64_t* total = reinterpret_cast<uint64_t*>(base + L.total);
    unsigned long long* status = reinterpret_cast<unsigned long long*>(base + L.status);
    const int64_t radix_status_words = (int64_t)(L.status_bytes / 8) - cdiv(n, kDupTile);
    unsigned long long* dup_status = status + radix_status_words;
    const PassScratch ps{hist, tickets, status, err};

    // 1. counts, depth keys and their digit histograms; clears
    if ((e = cudaMemsetAsync(base + L.hdr, 0, L.hdr_bytes, s)) != cudaSuccess)
        return cuda_status(e, "gs_bin_sort: clear header");
    const bool tight = sv.conic != nullptr;
    if (tight)
        k_count<true, kCountItemsTight><<<(int)cdiv(n, kThreads * kCountItemsTight), kThreads, 0, s>>>(
            n, sv, mean2d, radius, depth, U32(L.cnt), U32(L.dk0), U32(L.dv0), hist, reinterpret_cast<uint4*>(status),
            L.status_bytes / 16, tile_ranges, 2 * (size_t)ntiles);
    else
        k_count<false, kCountItems><<<(int)cdiv(n, kThreads * kCountItems), kThreads, 0, s>>>(
            n, sv, mean2d, radius, depth, U32(L.cnt), U32(L.dk0), U32(L.dv0), hist, reinterpret_cast<uint4*>(status),
            L.status_bytes / 16, tile_ranges, 2 * (size_t)ntiles);
    count_launches();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e, "gs_bin_sort: count");

    // 2. depth sort of all items (pass ids 0..3)
    uint32_t* dk[2] = {U32(L.dk0), U32(L.dk1)};
    uint32_t* dv[2] = {U32(L.dv0), U32(L.dv1)};
    int which = 0;
    if ((e = radix_sort(dk, dv, (uint32_t)n, nullptr, 32, 0, ps, &which, s)) != cudaSuccess)
        return cuda_status(e, "gs_bin_sort: depth sort");
    const uint32_t* perm = dv[which];

    // 3. duplicate in depth order (pass ids 4.. for the tile-id histograms)
    int tile_bits = 1;
    while ((1ll << tile_bits) < ntiles) ++tile_bits;
    const int tile_passes = (tile_bits + 7) / 8;
    uint32_t* tk[2] = {U32(L.tk0), U32(L.tk1)};
    uint32_t* tv[2] = {U32(L.tv0), U32(L.tv1)};
    auto dup = tight ? k_duplicate<true> : k_duplicate<false>;
    dup<<<(int)cdiv(n, kDupTile), kThreads, 0, s>>>(n, perm, U32(L.cnt), sv, mean2d, radius, (uint64_t)capacity,
                                                    tile_passes, tickets, dup_status, tk[0], tv[0], hist + 256 * 4,
                                                    total, graph ? n_instances_dev : nullptr, err);
    count_launches();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e, "gs_bin_sort: duplicate");

    uint32_t I_grid = 0;  // items the remaining kernels are launched for
    const uint64_t* I_dev = nullptr;
    if (!graph) {
        uint64_t I = 0;
        if ((e = cudaMemcpyAsync(&I, total, sizeof(uint64_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
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
        if (capacity == 0) return GS_OK;
        I_dev = total;
        I_grid = (uint32_t)capacity;
    }

    // 4. stable sort by global tile id, then keys, ids and ranges
    if ((e = radix_sort(tk, tv, I_grid, I_dev, tile_bits, 4, ps, &which, s)) != cudaSuccess)
        return cuda_status(e, "gs_bin_sort: tile sort");
    k_finalize<<<(int)cdiv((int64_t)I_grid, 256), 256, 0, s>>>(I_grid, I_dev, tk[which], tv[which], depth,
                                                               (uint32_t)n, (uint32_t)ntiles, keys_sorted,
                                                               ids_sorted, tile_ranges);
    count_launches();
    return cuda_status(cudaGetLastError(), "gs_bin_sort: finalize");
}

}  // namespace gs
