// Duplication and sorting stages (Sec. 2.1 (b), (c)).
//
// The result equals a stable sort of (tile << 32 | depth_bits) keys emitted in
// Gaussian order, i.e. every tile's list ordered by (depth bits, Gaussian
// index).  It is produced without sorting the instances themselves:
//   1. stable LSD radix sort of the N items by depth bits (32-bit keys);
//   2. coarse duplication in that depth order: one (supertile, item) pair
//      per supertile (4 x 4 tiles) holding at least one of the item's
//      instances (about an eighth of the instances), with the pair's 16-bit
//      mask of those instances, and the count of all instances;
//   3. stable LSD radix sort of those pairs by supertile id, so each
//      supertile's items are contiguous and in depth order;
//   4. the instances of each tile counted from the pairs' masks, a scan over
//      the tiles gives every tile's range, and one block per supertile walks
//      its pairs writing each instance's id once, at its tile's next
//      position: a stable per-tile compaction, so every list keeps the depth
//      (then index) order of step 1.
// Each instance is written once (4 bytes of id, plus its key if asked for)
// instead of being duplicated and moved by a radix pass per 8 bits of tile id.
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
// The scan of coarse counts in depth order is done the same way inside the
// duplication kernel, so the whole stage is
//   memset, keys, 4 depth passes, coarse duplicate, ceil(bits / 8) supertile
//   passes, tile counts, tile scan, fine write.
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
// warp (random digits: up to 32); otherwise __match_any_sync, the cheaper when
// the digit has at most 4 significant bits (the last pass over a short key).
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

// s_h[bin] += 1 for every active lane: one atomic when the lanes agree on the
// bin (the high digits of nearby keys usually do, and same-address shared
// atomics serialise), else one per lane.
__device__ __forceinline__ void hist_add(uint32_t* s_h, uint32_t bin) {
    const unsigned act = __activemask();
    const int first = __ffs(act) - 1;
    const uint32_t b0 = __shfl_sync(act, bin, first);
    if (__all_sync(act, bin == b0)) {
        if ((int)(threadIdx.x & 31) == first) atomicAdd(&s_h[bin], (uint32_t)__popc(act));
    } else {
        atomicAdd(&s_h[bin], 1u);
    }
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
// 4 significant bits).  The ranking runs once: it keeps each item's rank among
// its warp's items of the same digit, so placing an item needs only its warp's
// start of the digit.  Items are placed in shared memory in digit order, then
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
    // persistent: the block takes tiles until the pass is done (a tile's
    // look-back waits only on tiles ticketed before it, which blocks are
    // already processing)
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&tickets[pass_id], 1u);
        for (int i = threadIdx.x; i < (kThreads / 32) * 256; i += kThreads) (&s_w[0][0])[i] = 0;
        __syncthreads();
        const uint32_t tile = s_tile;
        const int64_t bbase = (int64_t)tile * TILE;
        if (bbase >= n) return;  // uniform over the block; no later tile is needed either
        const int cnt = (int)((int64_t)n - bbase < TILE ? (int64_t)n - bbase : TILE);
        const int wbase = warp * (ITEMS * 32);
        uint32_t k[ITEMS];
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
            const int i = wbase + r * 32 + lane;
            k[r] = i < cnt ? kin[bbase + i] : 0u;
        }
        const unsigned lt = (1u << lane) - 1u;
        // each item's rank among the warp's items with its digit (input order),
        // 16 bits per item: the warp's running count before this round plus the
        // lower lanes of the round with the same digit
        uint32_t rank[(ITEMS + 1) / 2];
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
            const bool valid = wbase + r * 32 + lane < cnt;
            const uint32_t d = (k[r] >> shift) & 0xFFu;
            const unsigned peers = digit_peers<FULL>(d, valid);
            const uint32_t before = valid ? s_w[warp][d] : 0u;
            __syncwarp();
            if (valid && (peers & lt) == 0) s_w[warp][d] = before + __popc(peers);
            __syncwarp();
            const uint32_t rk = before + __popc(peers & lt);
            if (r & 1)
                rank[r >> 1] |= rk << 16;
            else
                rank[r >> 1] = rk;
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
        // the values are needed only from here on (fewer registers live across the look-back)
        uint32_t v[ITEMS];
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
            const int i = wbase + r * 32 + lane;
            v[r] = i < cnt ? vin[bbase + i] : 0u;
        }
        __syncthreads();
        // s_w[w][d] now holds warp w's block-local start of digit d
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
            if (wbase + r * 32 + lane < cnt) {
                const uint32_t d = (k[r] >> shift) & 0xFFu;
                const uint32_t pos = s_w[warp][d] + ((rank[r >> 1] >> (16 * (r & 1))) & 0xFFFFu);
                s_key[pos] = k[r];
                s_val[pos] = v[r];
            }
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
        __syncthreads();  // shared memory is reused by the next tile
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
    int dev = 0, sms = 0;
    cudaError_t ea = cudaGetDevice(&dev);
    if (ea == cudaSuccess) ea = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (ea != cudaSuccess) return ea;
    // persistent blocks: at most 4 per SM (a graph-mode grid sized for the capacity would
    // otherwise start many blocks that only find the pass done)
    const int nblk = (int)std::min<int64_t>(cdiv(n_host, (int64_t)kThreads * items), 4 * (int64_t)sms);
    for (int p = 0, shift = 0; shift < bits; ++p, shift += 8) {
        const int id = first_pass + p;
        // ballots unless the digit has at most 4 significant bits (match_any is cheaper then)
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

// ------------------------------------------------------------ supertiles --
//
// A supertile is 4 x 4 tiles of one view.  Within one supertile row an item's
// supertiles are the union of [f / 4, l / 4] over the runs [f, l] of its (at
// most 4) tile rows there: up to 4 intervals, merged after a sorting network
// on their starts (registers only).  Every supertile counted holds at least
// one of the item's instances.
constexpr int kSuper = 4;

struct Iv {
    int lo, hi;  // empty: lo > hi (lo = INT_MAX sorts last)
};
__device__ __forceinline__ void iv_swap(Iv& a, Iv& b) {
    if (b.lo < a.lo) {
        const Iv t = a;
        a = b;
        b = t;
    }
}
// emit(lo, hi) for each maximal interval of the union; returns its size
template <class F>
__device__ __forceinline__ int iv_union4(Iv a, Iv b, Iv c, Iv d, F emit) {
    iv_swap(a, b);
    iv_swap(c, d);
    iv_swap(a, c);
    iv_swap(b, d);
    iv_swap(b, c);
    if (a.lo > a.hi) return 0;
    int n = 0, clo = a.lo, chi = a.hi;
    auto step = [&](const Iv& x) {
        if (x.lo > x.hi) return;
        if (x.lo <= chi + 1) {
            chi = max(chi, x.hi);
        } else {
            emit(clo, chi);
            n += chi - clo + 1;
            clo = x.lo;
            chi = x.hi;
        }
    };
    step(b);
    step(c);
    step(d);
    emit(clo, chi);
    return n + chi - clo + 1;
}

// The four tile-row runs of one supertile row (f > l: none).
struct Runs4 {
    int f[kSuper], l[kSuper];
};

// The 16-bit mask of supertile column sx within a supertile row's runs: bit
// 4 k + c for tile (4 sx + c) of the row's k-th tile row.
__device__ __forceinline__ uint32_t runs_mask(const Runs4& rr, int sx) {
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < kSuper; ++k) {
        const int a = max(rr.f[k], sx * kSuper), b = min(rr.l[k], sx * kSuper + kSuper - 1);
        if (a <= b) m |= ((1u << (b - a + 1)) - 1u) << (k * kSuper + a - sx * kSuper);
    }
    return m;
}

// The four tile-row runs of supertile row sy within the rectangle [x0, x1] x
// [y0, y1], and in *fine their instance count.
template <bool TIGHT>
__device__ __forceinline__ Runs4 row_runs(const TightRows& t, int sy, int x0, int x1, int y0, int y1,
                                          uint32_t* fine) {
    Runs4 rr;
#pragma unroll
    for (int k = 0; k < kSuper; ++k) {
        const int y = sy * kSuper + k;
        int f = 1, l = 0;
        if (y >= y0 && y <= y1) {
            if constexpr (TIGHT) {
                tight_row(t, y, x0, x1, f, l);
            } else {
                f = x0;
                l = x1;
            }
        }
        rr.f[k] = f;
        rr.l[k] = l;
        if (f <= l) *fine += (uint32_t)(l - f + 1);
    }
    return rr;
}

// The supertile columns holding an instance of the runs rr (emit(lo, hi) per
// maximal interval, in increasing order); returns their count.
template <class F>
__device__ __forceinline__ int runs_union(const Runs4& rr, F emit) {
    Iv r[kSuper];
#pragma unroll
    for (int k = 0; k < kSuper; ++k)
        r[k] = rr.f[k] <= rr.l[k] ? Iv{rr.f[k] / kSuper, rr.l[k] / kSuper} : Iv{0x7fffffff, -1};
    return iv_union4(r[0], r[1], r[2], r[3], emit);
}

// Deals the work units of a warp's items (lane l's item has units[l] of
// them: its supertile rows) out to the lanes, 32 per round, in lane-then-unit
// order, so that every lane evaluates one supertile row whatever the spread
// of the items' heights.  body(active, src, u, f) runs on every lane each
// round: src is the lane whose item the unit belongs to, u the unit's index
// within that item, f its index among the warp's units; active is false on
// the idle lanes of the last round.
template <class F>
__device__ __forceinline__ void warp_units(uint32_t units, F body) {
    const int lane = threadIdx.x & 31;
    uint32_t incl = units;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += v;
    }
    const uint32_t excl = incl - units, total = __shfl_sync(0xffffffffu, incl, 31);
    for (uint32_t r0 = 0; r0 < total; r0 += 32) {
        const uint32_t f = r0 + (uint32_t)lane;
        // the last lane whose first unit is at or before f (the first units are nondecreasing)
        int src = 0;
        uint32_t start = 0;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            const uint32_t v = __shfl_sync(0xffffffffu, excl, src + d);
            if (v <= f) {
                src += d;
                start = v;
            }
        }
        body(f < total, src, f - start, f);
    }
}

__device__ __forceinline__ TightRows shfl_rows(const TightRows& t, int src) {
    TightRows b;
    b.mode = __shfl_sync(0xffffffffu, t.mode, src);
    b.mx = __shfl_sync(0xffffffffu, t.mx, src);
    b.my = __shfl_sync(0xffffffffu, t.my, src);
    b.nB = __shfl_sync(0xffffffffu, t.nB, src);
    b.det = __shfl_sync(0xffffffffu, t.det, src);
    b.Atau = __shfl_sync(0xffffffffu, t.Atau, src);
    b.rA = __shfl_sync(0xffffffffu, t.rA, src);
    b.ymax = __shfl_sync(0xffffffffu, t.ymax, src);
    b.dyr = __shfl_sync(0xffffffffu, t.dyr, src);
    return b;
}

// Per item: its depth key and index (the depth sort's input) and the keys'
// four digit histograms (pass ids 0..3).  Also clears the tile ranges and the
// look-back status words of the depth sort (clear) and of the duplication
// (clear2).
constexpr int kKeyItems = 4;
__global__ void __launch_bounds__(kThreads) k_keys(int n_items, const float* __restrict__ depth,
                                                   uint32_t* __restrict__ dkey, uint32_t* __restrict__ dval,
                                                   uint32_t* __restrict__ hist, uint4* __restrict__ clear,
                                                   size_t clear_n, unsigned long long* __restrict__ clear2,
                                                   size_t clear2_n, uint32_t* __restrict__ ranges, size_t ranges_n) {
    __shared__ uint32_t s_h[4 * 256];
    for (int i = threadIdx.x; i < 4 * 256; i += kThreads) s_h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * (kThreads * kKeyItems) + threadIdx.x;
    uint32_t key[kKeyItems];
#pragma unroll
    for (int q = 0; q < kKeyItems; ++q) {
        const int64_t i = base + q * kThreads;
        key[q] = i < n_items ? __float_as_uint(depth[i]) : 0u;
    }
#pragma unroll
    for (int q = 0; q < kKeyItems; ++q) {
        const int64_t i = base + q * kThreads;
        if (i < n_items) {
            dkey[i] = key[q];
            dval[i] = (uint32_t)i;
#pragma unroll
            for (int p = 0; p < 4; ++p) hist_add(s_h, p * 256 + ((key[q] >> (8 * p)) & 0xFFu));
        }
    }
    const size_t stride = (size_t)gridDim.x * kThreads;
    const uint4 z = make_uint4(0, 0, 0, 0);
    for (size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x; i < clear_n; i += stride) clear[i] = z;
    for (size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x; i < clear2_n; i += stride) clear2[i] = 0ull;
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

// Digit histograms of one tile id (the wide-row path: one id per lane).
__device__ __forceinline__ void key_hist(uint32_t a, int passes, int* s_d0, uint32_t* s_h) {
    atomicAdd(&s_d0[a & 0xFFu], 1);
    atomicSub(&s_d0[(a & 0xFFu) + 1], 1);
    for (int p = 1; p < passes; ++p) hist_add(s_h, (p - 1) * 256 + ((a >> (8 * p)) & 0xFFu));
}

// A unit's runs in four words (16 bits per end; an empty run as (1, 0)).
__device__ __forceinline__ uint4 pack_runs(const Runs4& rr) {
    uint32_t w[kSuper];
#pragma unroll
    for (int k = 0; k < kSuper; ++k)
        w[k] = rr.f[k] <= rr.l[k] ? ((uint32_t)rr.f[k] | ((uint32_t)rr.l[k] << 16)) : 1u;
    return make_uint4(w[0], w[1], w[2], w[3]);
}
__device__ __forceinline__ Runs4 unpack_runs(uint4 v) {
    const uint32_t w[kSuper] = {v.x, v.y, v.z, v.w};
    Runs4 rr;
#pragma unroll
    for (int k = 0; k < kSuper; ++k) {
        rr.f[k] = (int)(w[k] & 0xFFFFu);
        rr.l[k] = (int)(w[k] >> 16);
    }
    return rr;
}

// Coarse duplication in depth order, with the supertile counts and their scan
// folded in.  Tile t (from the ticket) holds the depth-ordered items
// [t * kDupTile, (t + 1) * kDupTile).  Each warp deals its items' supertile
// rows out to its lanes (warp_units) and evaluates every row's tile runs once,
// keeping them in shared memory (the first kStashUnits of each warp; later
// ones are evaluated again when written): the items' supertile counts and the
// instance count, added into *fine_total.  The tile's pair count goes out for
// the decoupled look-back over the tiles before it.  Each item then emits one
// (global supertile id, item) pair per supertile it touches, supertile rows in
// order, placed by a warp scan of the rows' pair counts; a row of more than
// kWideRow supertiles is emitted by the whole warp, one supertile column per
// lane.  A tile of at most kStagePairs pairs emits them into shared memory
// before its look-back (so the predecessors' prefixes are usually there by
// then) and copies them out with consecutive threads on consecutive pairs; a
// larger tile looks back first and writes them directly.  With `pack` the
// key's high half holds the pair's 16-bit tile mask (runs_mask).  Writes stop
// at `limit`; the pair total goes to *total.  The digit histograms of the
// written pairs' supertile ids go to hist (passes of them), so a truncated
// list still sorts into a permutation of what was written.  With coarse_tile
// > 0 the block also clears the look-back status words (256 per radix tile,
// at radix_status) of the pair sort's tiles that start within its pairs
// (below `limit`), and the blocks together zero st_zero[0, st_n).
constexpr uint32_t kWideRow = 8;
constexpr uint32_t kStashUnits = 128;  // per warp
constexpr uint32_t kStagePairs = 2048;
template <bool TIGHT>
__global__ void __launch_bounds__(kThreads) k_dup_coarse(int n_items, const uint32_t* __restrict__ perm,
                                                         const __grid_constant__ SortViews sv,
                                                         const float2* __restrict__ mean2d,
                                                         const int* __restrict__ radius, uint64_t limit, int passes,
                                                         bool pack, uint32_t* tickets, unsigned long long* status,
                                                         uint32_t* __restrict__ ckey, uint32_t* __restrict__ cval,
                                                         uint32_t* __restrict__ hist, uint64_t* __restrict__ total,
                                                         unsigned long long* __restrict__ fine_total,
                                                         unsigned long long* __restrict__ radix_status,
                                                         uint32_t coarse_tile, uint32_t* __restrict__ st_zero,
                                                         int st_n, unsigned* err) {
    __shared__ uint64_t s_warp[kThreads / 32 + 1];
    __shared__ uint64_t s_prefix;
    __shared__ unsigned long long s_fine;
    if (st_zero != nullptr)  // the supertile counters of k_pair_masks
        for (int i = blockIdx.x * kThreads + threadIdx.x; i < st_n; i += gridDim.x * kThreads) st_zero[i] = 0;
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_h[3 * 256];  // digits 1..3
    __shared__ int s_d0[257];          // digit 0, as a difference array
    __shared__ int s_warp_i[kThreads / 32 + 1];
    __shared__ uint32_t s_c[kThreads];  // per lane: its item's supertile count
    __shared__ uint4 s_runs[(kThreads / 32) * kStashUnits];
    __shared__ uint8_t s_n[(kThreads / 32) * kStashUnits];
    __shared__ uint32_t s_pk[kStagePairs], s_pv[kStagePairs];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        s_tile = atomicAdd(&tickets[kMaxPasses], 1u);
        s_fine = 0;
    }
    for (int i = threadIdx.x; i < 3 * 256; i += kThreads) s_h[i] = 0;
    for (int i = threadIdx.x; i < 257; i += kThreads) s_d0[i] = 0;
    __syncthreads();
    const uint32_t tile = s_tile;
    const int64_t base = (int64_t)tile * kDupTile;
    if (base >= n_items) return;

    const int64_t k = base + threadIdx.x;
    const uint32_t item = k < n_items ? perm[k] : 0u;
    int x0 = 0, x1 = -1, y0 = 0, y1 = -1, stx = 0, stb = 0;
    bool vis = false;
    TightRows t{};
    if (k < n_items) {
        const int v = (int)(item / (uint32_t)sv.n_per_view);
        const ViewDesc& vd = sv.views[v];
        const float2 m = mean2d[item];
        vis = tile_rect(m.x, m.y, radius[item], vd.W, vd.H, x0, x1, y0, y1);
        stx = sv.st_x[v];
        stb = sv.st_begin[v];
        if constexpr (TIGHT)
            if (vis) t = item_tight_rows(sv, mean2d, item);
    }
    const uint32_t units = vis ? (uint32_t)(y1 / kSuper - y0 / kSuper + 1) : 0u;
    uint4* stash = s_runs + warp * kStashUnits;
    uint8_t* stash_n = s_n + warp * kStashUnits;
    const int wlane0 = threadIdx.x & ~31;

    // every unit's runs once: the items' supertile counts and the instance count
    s_c[threadIdx.x] = 0;
    __syncwarp();
    uint32_t fine = 0;
    warp_units(units, [&](bool act, int src, uint32_t u, uint32_t f) {
        const int bx0 = __shfl_sync(0xffffffffu, x0, src), bx1 = __shfl_sync(0xffffffffu, x1, src);
        const int by0 = __shfl_sync(0xffffffffu, y0, src), by1 = __shfl_sync(0xffffffffu, y1, src);
        TightRows bt{};
        if constexpr (TIGHT) bt = shfl_rows(t, src);
        if (act) {
            const Runs4 rr = row_runs<TIGHT>(bt, by0 / kSuper + (int)u, bx0, bx1, by0, by1, &fine);
            const int n = runs_union(rr, [](int, int) {});
            atomicAdd(&s_c[wlane0 + src], (uint32_t)n);
            if (f < kStashUnits) {
                stash[f] = pack_runs(rr);
                stash_n[f] = (uint8_t)min(n, 255);
            }
        }
    });
    __syncwarp();
    const uint32_t c = s_c[threadIdx.x];
    if (fine) atomicAdd(&s_fine, (unsigned long long)fine);

    uint64_t tile_sum;
    const uint64_t local = block_excl_scan<uint64_t, kThreads>((uint64_t)c, tile_sum, s_warp);
    unsigned long long* mine = status + tile;
    const bool staged = tile_sum <= kStagePairs;  // uniform over the block
    if (warp == 0 && lane == 0) st_status(mine, tile == 0 ? 2u : 1u, tile_sum);
    // the tile's offset among all pairs: the look-back, then the clears that need it
    auto resolve = [&]() {
        if (warp == 0) {
            uint64_t prefix = 0;
            if (tile > 0) {
                prefix = lookback_warp(status, tile, 1u, err);
                if (lane == 0) st_status(mine, 2u, prefix + tile_sum);
            }
            if (lane == 0) {
                s_prefix = prefix;
                if (base + kDupTile >= n_items) *total = prefix + tile_sum;  // the last tile: the total
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && s_fine) atomicAdd(fine_total, s_fine);
        if (coarse_tile > 0) {
            // the sort takes at most `limit` pairs: its tiles start below it
            const uint64_t lo = s_prefix, hi = min(s_prefix + tile_sum, limit);
            for (uint64_t ct = (lo + coarse_tile - 1) / coarse_tile; ct * coarse_tile < hi; ++ct)
                radix_status[ct * 256 + threadIdx.x] = 0ull;
        }
    };
    if (!staged) resolve();
    const uint64_t gbase = staged ? 0 : s_prefix;  // where block offset 0 goes
    // one pair at block offset p: staged, or written below `limit` (histograms counted)
    auto put = [&](uint64_t p, uint32_t key, uint32_t val) {
        if (staged) {
            s_pk[p] = key;
            s_pv[p] = val;
        } else if (gbase + p < limit) {
            ckey[gbase + p] = key;
            cval[gbase + p] = val;
        }
    };

    uint64_t p_warp = __shfl_sync(0xffffffffu, local, 0);  // the warp's pairs start at its lane 0's item
    const unsigned lt = (1u << lane) - 1u;
    warp_units(units, [&](bool act, int src, uint32_t u, uint32_t f) {
        const int bx0 = __shfl_sync(0xffffffffu, x0, src), bx1 = __shfl_sync(0xffffffffu, x1, src);
        const int by0 = __shfl_sync(0xffffffffu, y0, src), by1 = __shfl_sync(0xffffffffu, y1, src);
        const int bstx = __shfl_sync(0xffffffffu, stx, src), bstb = __shfl_sync(0xffffffffu, stb, src);
        const uint32_t bi = __shfl_sync(0xffffffffu, item, src);
        const int sy = by0 / kSuper + (int)u;
        const bool again = act && f >= kStashUnits;  // beyond the stash: evaluated again
        TightRows bt{};
        if constexpr (TIGHT)
            if (__any_sync(0xffffffffu, again)) bt = shfl_rows(t, src);
        Runs4 rr{};
        uint32_t n = 0;
        if (act) {
            if (again) {
                uint32_t fine2 = 0;
                rr = row_runs<TIGHT>(bt, sy, bx0, bx1, by0, by1, &fine2);
                n = (uint32_t)runs_union(rr, [](int, int) {});
            } else {
                rr = unpack_runs(stash[f]);
                n = stash_n[f];
                if (n == 255) n = (uint32_t)runs_union(rr, [](int, int) {});
            }
        }
        uint32_t incl = n;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += v;
        }
        uint64_t p = p_warp + (incl - n);
        p_warp += __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t krow = (uint32_t)bstb + (uint32_t)sy * (uint32_t)bstx;  // the row's supertile 0
        const bool wide = n > kWideRow;
        if (act && !wide)
            runs_union(rr, [&](int lo, int hi) {
                const uint32_t len = (uint32_t)(hi - lo + 1);
                for (uint32_t j = 0; j < len; ++j)
                    put(p + j, (krow + (uint32_t)lo + j) | (pack ? runs_mask(rr, lo + (int)j) << 16 : 0u), bi);
                if (!staged && gbase + p < limit)
                    row_hist(krow + (uint32_t)lo, (uint32_t)min((uint64_t)len, limit - (gbase + p)), passes, s_d0,
                             s_h);
                p += len;
            });
        unsigned wides = __ballot_sync(0xffffffffu, act && wide);
        while (wides) {  // a wide row: the whole warp, supertile column lo + j on lane j
            const int w = __ffs(wides) - 1;
            wides &= wides - 1;
            Runs4 wr;
#pragma unroll
            for (int q = 0; q < kSuper; ++q) {
                wr.f[q] = __shfl_sync(0xffffffffu, rr.f[q], w);
                wr.l[q] = __shfl_sync(0xffffffffu, rr.l[q], w);
            }
            uint64_t wp = __shfl_sync(0xffffffffu, p, w);
            const uint32_t wk = __shfl_sync(0xffffffffu, krow, w), wi = __shfl_sync(0xffffffffu, bi, w);
            int lo = 0x7fffffff, hi = -1;
#pragma unroll
            for (int q = 0; q < kSuper; ++q)
                if (wr.f[q] <= wr.l[q]) {
                    lo = min(lo, wr.f[q] / kSuper);
                    hi = max(hi, wr.l[q] / kSuper);
                }
            for (int sx0 = lo; sx0 <= hi; sx0 += 32) {
                const int sx = sx0 + lane;
                const uint32_t m = sx <= hi ? runs_mask(wr, sx) : 0u;
                const unsigned nz = __ballot_sync(0xffffffffu, m != 0u);
                const uint64_t q = wp + (uint64_t)__popc(nz & lt);
                if (m != 0u) {
                    put(q, (wk + (uint32_t)sx) | (pack ? m << 16 : 0u), wi);
                    if (!staged && gbase + q < limit) key_hist(wk + (uint32_t)sx, passes, s_d0, s_h);
                }
                wp += (uint64_t)__popc(nz);
            }
        }
    });
    if (staged) {
        resolve();  // (its barrier also orders the staging before the copy)
        const uint64_t g0 = s_prefix;
        for (uint32_t i = threadIdx.x; i < (uint32_t)tile_sum; i += kThreads) {
            if (g0 + i >= limit) break;
            const uint32_t key = s_pk[i];
            ckey[g0 + i] = key;
            cval[g0 + i] = s_pv[i];
            key_hist(pack ? key & 0xFFFFu : key, passes, s_d0, s_h);
        }
    }
    __syncthreads();
    {
        int tot;
        const int v = s_d0[threadIdx.x];
        const int d0 = block_excl_scan<int, kThreads>(v, tot, s_warp_i) + v;  // count of digit-0 value threadIdx.x
        if (d0) atomicAdd(&hist[threadIdx.x], (uint32_t)d0);
    }
    for (int i = threadIdx.x; i < (passes - 1) * 256; i += kThreads)
        if (s_h[i]) atomicAdd(&hist[256 + i], s_h[i]);
}

// First position of key >= want in keys[0, n), ascending in (key & kmask).
__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t* __restrict__ keys, uint32_t n, uint32_t want,
                                                    uint32_t kmask) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if ((keys[mid] & kmask) < want) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// The 16-bit mask of an item's instances in the supertile whose first tile
// is (cx0, cy0): bit 4 r + c for tile (cx0 + c, cy0 + r).  The same rule as
// the counts (tile_rect, then tight_row per row with the item's whole
// rectangle), clipped to the supertile.
template <bool TIGHT>
__device__ __forceinline__ uint32_t supertile_mask(const SortViews& sv, const float2* mean2d, const int* radius,
                                                   uint32_t item, const ViewDesc& vd, int cx0, int cy0) {
    const float2 m = mean2d[item];
    int x0, x1, y0, y1;
    if (!tile_rect(m.x, m.y, radius[item], vd.W, vd.H, x0, x1, y0, y1)) return 0u;
    const int a0 = max(x0, cx0), a1 = min(x1, cx0 + kSuper - 1);
    if (a0 > a1) return 0u;
    TightRows t{};
    if constexpr (TIGHT) t = item_tight_rows(sv, mean2d, item);
    uint32_t mask = 0;
#pragma unroll
    for (int r = 0; r < kSuper; ++r) {
        const int y = cy0 + r;
        if (y < y0 || y > y1) continue;
        int f = x0, l = x1;
        if constexpr (TIGHT) tight_row(t, y, x0, x1, f, l);
        f = max(f, a0);
        l = min(l, a1);
        if (f <= l) mask |= ((1u << (l - f + 1)) - 1u) << (r * kSuper + f - cx0);
    }
    return mask;
}

// The instance counts of the supertile's tiles, added into ranges[2 t + 1]
// (cleared by k_keys), from the sorted pairs' 16-bit tile masks: the
// duplication packed them above the supertile id (`pack`), else they are
// computed here and stored to masks[].  Each warp takes segments of
// kPairSeg consecutive pairs; the pairs are sorted by supertile, so a warp's
// 32 pairs mostly share one, and while they do the warp counts each tile's
// bits with four lane reductions (bit j of every mask spread to its own byte)
// into lane j's count, adding it to ranges with one atomic per tile when the
// supertile changes.  32 pairs of several supertiles: one atomic per group
// of equal supertiles and tile.  With st_count (zeroed by k_dup_coarse), each
// supertile's total is added there as well.
constexpr uint32_t kPairSeg = 512;
template <bool TIGHT>
__global__ void __launch_bounds__(kThreads) k_pair_masks(const __grid_constant__ SortViews sv,
                                                         const float2* __restrict__ mean2d,
                                                         const int* __restrict__ radius,
                                                         const uint32_t* __restrict__ ckey,
                                                         const uint32_t* __restrict__ cval, uint32_t n_host,
                                                         const uint64_t* __restrict__ n_dev, uint32_t n_items,
                                                         bool pack, uint16_t* __restrict__ masks,
                                                         uint32_t* __restrict__ ranges, uint32_t* st_count) {
    const uint32_t Ic = pass_count(n_host, n_dev);
    const int lane = threadIdx.x & 31;
    // tile j of supertile key (global id) as a global tile index
    auto tile_of = [&](uint32_t key, int j) -> size_t {
        int v = 0;
        while (v + 1 < sv.num_views && sv.st_begin[v + 1] <= (int)key) ++v;
        const int ls = (int)key - sv.st_begin[v];
        const ViewDesc& vd = sv.views[v];
        return (size_t)vd.tile_begin + (size_t)((ls / sv.st_x[v]) * kSuper + (j >> 2)) * vd.tiles_x +
               (size_t)((ls % sv.st_x[v]) * kSuper + (j & 3));
    };
    const uint64_t warp_id = ((uint64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const uint64_t warps = ((uint64_t)gridDim.x * kThreads) >> 5;
    for (uint64_t s0 = warp_id * kPairSeg; s0 < Ic; s0 += warps * kPairSeg) {
        const uint64_t s1 = min(s0 + (uint64_t)kPairSeg, (uint64_t)Ic);
        uint32_t cur = 0xffffffffu;  // the supertile being counted (warp-uniform)
        uint32_t acc = 0;            // lane j < 16: its count of tile j
        auto flush = [&]() {
            if (cur != 0xffffffffu && lane < 16 && acc) atomicAdd(&ranges[2 * tile_of(cur, lane) + 1], acc);
            if (st_count != nullptr) {  // the supertile's total
                const uint32_t all = __reduce_add_sync(0xffffffffu, lane < 16 ? acc : 0u);
                if (cur != 0xffffffffu && lane == 0 && all) atomicAdd(&st_count[cur], all);
            }
            acc = 0;
        };
        for (uint64_t b = s0; b < s1; b += 32) {
            const uint64_t e = b + (uint64_t)lane;
            uint32_t key = 0xffffffffu, m = 0;
            if (e < s1) {
                key = ckey[e];
                if (pack) {
                    m = key >> 16;
                    key &= 0xFFFFu;
                } else {
                    int v = 0;
                    while (v + 1 < sv.num_views && sv.st_begin[v + 1] <= (int)key) ++v;
                    const int ls = (int)key - sv.st_begin[v];
                    const uint32_t it = cval[e];
                    m = it < n_items ? supertile_mask<TIGHT>(sv, mean2d, radius, it, sv.views[v],
                                                             (ls % sv.st_x[v]) * kSuper, (ls / sv.st_x[v]) * kSuper)
                                     : 0u;
                    masks[e] = (uint16_t)m;
                }
            }
            const uint32_t k0 = __shfl_sync(0xffffffffu, key, 0);  // lane 0 always holds a pair
            if (!__all_sync(0xffffffffu, key == k0 || e >= s1)) {
                // pairs of several supertiles: one atomic per group and tile
                flush();
                cur = 0xffffffffu;
                const unsigned peers = __match_any_sync(0xffffffffu, key);
                const bool leader = lane == __ffs(peers) - 1 && key != 0xffffffffu;
                uint32_t all = 0;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const unsigned bj = __ballot_sync(0xffffffffu, (m >> j) & 1u) & peers;
                    if (leader && bj) atomicAdd(&ranges[2 * tile_of(key, j) + 1], (uint32_t)__popc(bj));
                    all += (uint32_t)__popc(bj);
                }
                if (st_count != nullptr && leader && all) atomicAdd(&st_count[key], all);
                continue;
            }
            if (k0 != cur) {
                flush();
                cur = k0;
            }
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                // bits 4w .. 4w + 3 of the mask to bytes 0..3, summed over the warp (<= 32 each)
                const uint32_t spread = (((m >> (4 * w)) & 0xFu) * 0x00204081u) & 0x01010101u;
                const uint32_t sum = __reduce_add_sync(0xffffffffu, spread);
                if ((lane >> 2) == w) acc += (sum >> (8 * (lane & 3))) & 0xFFu;
            }
        }
        flush();
    }
}

// One block per supertile s (st_order[blockIdx], the largest first, when
// given), after k_tile_scan: its items are the sorted pairs [cs, ce) with
// key s; every instance's id (and key) goes to its tile's next position, in
// item order, from the pairs' tile masks (in the key's high half when kmask
// is 0xFFFF, else in masks[]).  Rounds of kFineRound pairs, the next round's
// loads in flight during the current one: warp w owns tiles w and w + 8 and
// walks the round's pairs 32 at a time, one ballot per group giving each
// pair's place in the tile's run and the run's length, into a shared-memory
// stage of the tile's ids; it then writes the run with consecutive lanes on
// consecutive ids.
constexpr int kFineThreads = 256, kFineRound = 512;
__global__ void __launch_bounds__(kFineThreads) k_fine(const __grid_constant__ SortViews sv,
                                                       const float* __restrict__ depth,
                                                       const uint32_t* __restrict__ ckey,
                                                       const uint32_t* __restrict__ cval, uint32_t n_host,
                                                       const uint64_t* __restrict__ n_dev, uint32_t kmask,
                                                       const uint16_t* __restrict__ masks,
                                                       const uint32_t* __restrict__ ranges,
                                                       const uint32_t* __restrict__ st_order,
                                                       uint32_t* __restrict__ ids_out, uint64_t* __restrict__ keys_out) {
    constexpr int PT = kFineRound / kFineThreads;  // pairs each thread loads
    constexpr int TW = 16 / (kFineThreads / 32);  // tiles per warp
    __shared__ uint32_t s_rng[2];
    __shared__ uint32_t s_beg[16], s_end[16], s_run[16];
    __shared__ uint16_t s_mask[kFineRound];
    __shared__ uint32_t s_item[kFineRound];
    __shared__ uint32_t s_out[16][kFineRound];
    const int s = st_order != nullptr ? (int)st_order[blockIdx.x] : (int)blockIdx.x;  // largest first
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    int v = 0;
    while (v + 1 < sv.num_views && sv.st_begin[v + 1] <= s) ++v;
    const ViewDesc& vd = sv.views[v];
    const int ls = s - sv.st_begin[v];
    const int cx0 = (ls % sv.st_x[v]) * kSuper, cy0 = (ls / sv.st_x[v]) * kSuper;
    const int tx = vd.tiles_x, ty = tiles_y(vd.H);
    const uint32_t Ic = pass_count(n_host, n_dev);
    if (threadIdx.x < 2) s_rng[threadIdx.x] = lower_bound_u32(ckey, Ic, (uint32_t)s + threadIdx.x, kmask);
    if (threadIdx.x < 16) {
        const int c = cx0 + (threadIdx.x & 3), r = cy0 + (threadIdx.x >> 2);
        const bool ok = c < tx && r < ty;
        const uint32_t gt = (uint32_t)vd.tile_begin + (uint32_t)r * (uint32_t)tx + (uint32_t)c;
        s_run[threadIdx.x] = 0;
        s_beg[threadIdx.x] = ok ? ranges[2 * gt] : 0u;
        s_end[threadIdx.x] = ok ? ranges[2 * gt + 1] : 0u;
    }
    __syncthreads();
    const uint32_t cs = s_rng[0], ce = s_rng[1];
    if (cs >= ce) return;
    const bool packed = kmask == 0xFFFFu;
    uint32_t mk[PT], it[PT];
    auto fetch = [&](uint32_t r0) {
#pragma unroll
        for (int i = 0; i < PT; ++i) {
            const uint32_t e = r0 + (uint32_t)(i * kFineThreads + threadIdx.x);
            mk[i] = e < ce ? (packed ? ckey[e] >> 16 : (uint32_t)masks[e]) : 0u;
            it[i] = e < ce ? cval[e] : 0u;
        }
    };
    fetch(cs);
    for (uint32_t r0 = cs; r0 < ce; r0 += kFineRound) {
#pragma unroll
        for (int i = 0; i < PT; ++i) {
            s_mask[i * kFineThreads + threadIdx.x] = (uint16_t)mk[i];
            s_item[i * kFineThreads + threadIdx.x] = it[i];
        }
        if (r0 + kFineRound < ce) fetch(r0 + kFineRound);
        __syncthreads();
        const int ng = (int)((min(ce - r0, (uint32_t)kFineRound) + 31) / 32);  // groups of 32 pairs in the round
#pragma unroll
        for (int h = 0; h < TW; ++h) {
            const int t = warp + h * (kFineThreads / 32);
            uint32_t n_t = 0;
            for (int g = 0; g < ng; ++g) {
                const int i = 32 * g + lane;
                const bool in = (s_mask[i] >> t) & 1u;
                const unsigned b = __ballot_sync(0xffffffffu, in);
                if (in) s_out[t][n_t + (uint32_t)__popc(b & lt)] = s_item[i];
                n_t += (uint32_t)__popc(b);
            }
            __syncwarp();
            const uint64_t p0 = (uint64_t)s_beg[t] + s_run[t];
            const uint64_t end = s_end[t];
            const uint64_t dkey = keys_out != nullptr
                                      ? (uint64_t)((uint32_t)vd.tile_begin + (uint32_t)(cy0 + (t >> 2)) * (uint32_t)tx +
                                                   (uint32_t)(cx0 + (t & 3))) << 32
                                      : 0ull;
            for (uint32_t k = lane; k < n_t; k += 32) {
                const uint64_t p = p0 + k;
                if (p < end) {
                    const uint32_t g = s_out[t][k];
                    ids_out[p] = g;
                    if (keys_out != nullptr) keys_out[p] = dkey | __float_as_uint(depth[g]);
                }
            }
            __syncwarp();
            if (lane == 0) s_run[t] += n_t;  // this warp's tile alone
        }
        __syncthreads();  // the round's masks and items are replaced next
    }
}

// Tile ranges from the per-tile counts in ranges[2 t + 1]: an exclusive scan
// over all tiles (one block), each bound clamped to the capacity.  With
// st_order: the supertiles in decreasing order of their instance counts
// (st_count, from k_pair_masks), by octave buckets
// (st_order, total_st entries), so that the fine writes start the longest
// supertiles first (the order within a bucket is arbitrary; the output does
// not depend on it).  Graph mode: the instance count (fine_total, from
// k_dup_coarse) to *count_out, and the capacity bit when it exceeds the
// capacity.
constexpr int kScanThreads = 1024;
constexpr int kStBuckets = 33;  // 0: empty, b: counts in [2^(b-1), 2^b)
__device__ __forceinline__ int octave(uint32_t x) { return x == 0 ? 0 : 32 - __clz(x); }
__global__ void __launch_bounds__(kScanThreads) k_tile_scan(const __grid_constant__ SortViews sv, int num_tiles,
                                                            uint32_t* __restrict__ ranges, uint64_t cap,
                                                            const unsigned long long* fine_total,
                                                            int64_t* count_out, const uint32_t* st_count,
                                                            uint32_t* __restrict__ st_order, unsigned* err) {
    constexpr int PER = 4;                       // consecutive tiles per thread and round
    constexpr int R = kScanThreads * PER;        // tiles per round
    __shared__ uint64_t s_warp[kScanThreads / 32 + 1];
    __shared__ uint32_t s_bk[kStBuckets];
    __shared__ uint32_t s_a[R + R / 32], s_b[R + R / 32];  // counts, then begins and ends (padded)
    auto at = [](int i) { return i + (i >> 5); };
    const int nst = sv.total_st;
    if (threadIdx.x < kStBuckets) s_bk[threadIdx.x] = 0;
    uint64_t run = 0;
    for (int64_t b = 0; b < num_tiles; b += R) {
        // the round's counts, consecutive threads on consecutive tiles
        for (int i = threadIdx.x; i < R; i += kScanThreads)
            s_a[at(i)] = b + i < num_tiles ? ranges[2 * (b + i) + 1] : 0u;
        __syncthreads();
        uint32_t c[PER];
        uint64_t sum = 0;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            c[k] = s_a[at(threadIdx.x * PER + k)];
            sum += c[k];
        }
        uint64_t tot;
        uint64_t pre = run + block_excl_scan<uint64_t, kScanThreads>(sum, tot, s_warp);
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = threadIdx.x * PER + k;
            s_a[at(i)] = (uint32_t)(c[k] > 0 ? min(pre, cap) : 0);
            s_b[at(i)] = (uint32_t)(c[k] > 0 ? min(pre + c[k], cap) : 0);
            pre += c[k];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < R; i += kScanThreads)
            if (b + i < num_tiles) {
                ranges[2 * (b + i)] = s_a[at(i)];
                ranges[2 * (b + i) + 1] = s_b[at(i)];
            }
        __syncthreads();  // s_a is reloaded next round
        run += tot;
    }
    if (st_order != nullptr) {
        __syncthreads();
        for (int i = threadIdx.x; i < nst; i += kScanThreads) atomicAdd(&s_bk[octave(__ldcg(st_count + i))], 1u);
        __syncthreads();
        if (threadIdx.x == 0) {  // bucket starts, the largest octave first
            uint32_t acc = 0;
            for (int k = kStBuckets - 1; k >= 0; --k) {
                const uint32_t n = s_bk[k];
                s_bk[k] = acc;
                acc += n;
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nst; i += kScanThreads)
            st_order[atomicAdd(&s_bk[octave(__ldcg(st_count + i))], 1u)] = (uint32_t)i;
    }
    if (threadIdx.x == 0 && count_out != nullptr) {
        const uint64_t all = *fine_total;
        *count_out = (int64_t)all;
        if (all > cap) atomicOr(err, kErrCapacity);
    }
}

// Workspace: per-item arrays, a header cleared by one memset (digit
// histograms, tickets, counts), the look-back status words (cleared by
// k_keys), and the pair key/value double buffers.
struct Layout {
    size_t dk0, dk1, dv0, dv1, hdr, hist, tickets, total, ctotal, hdr_bytes, status, status_bytes, tk0, tk1, tv0,
        tv1, total_bytes;
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
    L.dk0 = take(4 * N);
    L.dk1 = take(4 * N);
    L.dv0 = take(4 * N);
    L.dv1 = take(4 * N);
    L.hdr = o;
    L.hist = take(4 * 256 * kMaxPasses);
    L.tickets = take(4 * (kMaxPasses + 1));
    L.total = take(16);  // instances, then supertile pairs (k_dup_coarse)
    L.ctotal = L.total + 8;
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

    // supertiles of every view
    SortViews sv2 = sv;
    {
        int st = 0;
        for (int v = 0; v < sv.num_views; ++v) {
            sv2.st_begin[v] = st;
            sv2.st_x[v] = (int)cdiv(sv.views[v].tiles_x, kSuper);
            st += sv2.st_x[v] * (int)cdiv(tiles_y(sv.views[v].H), kSuper);
        }
        sv2.total_st = st;
    }
    uint64_t* ctotal = reinterpret_cast<uint64_t*>(base + L.ctotal);

    // 1. depth keys and their digit histograms; clears
    if ((e = cudaMemsetAsync(base + L.hdr, 0, L.hdr_bytes, s)) != cudaSuccess)
        return cuda_status(e, "gs_bin_sort: clear header");
    const bool tight = sv.conic != nullptr;
    unsigned long long* fine_total = reinterpret_cast<unsigned long long*>(total);
    // status words: the depth sort's here; the pair sort's by the duplication (graph mode) or a
    // memset sized by the pair count (synchronising mode)
    const size_t depth_status_words = 256 * (size_t)radix_tiles_max(n);
    k_keys<<<(int)cdiv(n, kThreads * kKeyItems), kThreads, 0, s>>>(
        n, depth, U32(L.dk0), U32(L.dv0), hist, reinterpret_cast<uint4*>(status), depth_status_words / 2, dup_status,
        (size_t)cdiv(n, kDupTile), tile_ranges, 2 * (size_t)ntiles);
    count_launches();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e, "gs_bin_sort: keys");

    // 2. depth sort of all items (pass ids 0..3)
    uint32_t* dk[2] = {U32(L.dk0), U32(L.dk1)};
    uint32_t* dv[2] = {U32(L.dv0), U32(L.dv1)};
    int which = 0;
    if ((e = radix_sort(dk, dv, (uint32_t)n, nullptr, 32, 0, ps, &which, s)) != cudaSuccess)
        return cuda_status(e, "gs_bin_sort: depth sort");
    const uint32_t* perm = dv[which];

    // 3. supertile pairs in depth order, the instance count (pass ids 4.. for the supertile-id histograms)
    int st_bits = 1;
    while ((1ll << st_bits) < sv2.total_st) ++st_bits;
    const int st_passes = (st_bits + 7) / 8;
    uint32_t* ck[2] = {U32(L.tk0), U32(L.tk1)};
    uint32_t* cv[2] = {U32(L.tv0), U32(L.tv1)};
    // up to 2^16 supertiles the pairs' tile masks ride in the key's high half
    const bool pack = st_bits <= 16;
    auto dup = tight ? k_dup_coarse<true> : k_dup_coarse<false>;
    const uint32_t coarse_tile = graph ? (uint32_t)(kThreads * pass_items((uint64_t)capacity)) : 0u;
    // per-supertile instance counts and their order, largest first, in the depth keys'
    // buffers (free once the depth sort is done), when they fit
    const int nst = sv2.total_st;
    uint32_t* st_count = nst <= n ? dk[0] : nullptr;
    uint32_t* st_order = nst <= n ? dk[1] : nullptr;
    if ((e = record_kernel_event(GS_KERNEL_DUPLICATE, false, s)) != cudaSuccess)
        return cuda_status(e, "gs_bin_sort: kernel event");
    dup<<<(int)cdiv(n, kDupTile), kThreads, 0, s>>>(n, perm, sv2, mean2d, radius, (uint64_t)capacity, st_passes,
                                                    pack, tickets, dup_status, ck[0], cv[0], hist + 256 * 4, ctotal,
                                                    fine_total, status, coarse_tile, st_count, nst, err);
    count_launches();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e, "gs_bin_sort: duplicate");
    if ((e = record_kernel_event(GS_KERNEL_DUPLICATE, true, s)) != cudaSuccess)
        return cuda_status(e, "gs_bin_sort: kernel event");

    // synchronising mode: the instance and pair counts, before any further work
    uint32_t I_grid = 0;  // pairs the later kernels are sized for
    if (!graph) {
        uint64_t counts[2] = {0, 0};  // instances, supertile pairs (adjacent in the header)
        if ((e = cudaMemcpyAsync(counts, total, sizeof(counts), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return cuda_status(e, "gs_bin_sort: read count");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_status(e, "gs_bin_sort: synchronize");
        *n_instances_host = (int64_t)counts[0];
        if ((int64_t)counts[0] > capacity) {
            set_error("gs_bin_sort: %llu instances exceed capacity %lld", (unsigned long long)counts[0],
                      (long long)capacity);
            return GS_ERR_CAPACITY;
        }
        if (counts[0] == 0) return GS_OK;  // k_keys cleared the ranges
        I_grid = (uint32_t)counts[1];
        if ((e = cudaMemsetAsync(status, 0, 8 * 256 * (size_t)radix_tiles_max(I_grid), s)) != cudaSuccess)
            return cuda_status(e, "gs_bin_sort: clear pair-sort status");
    } else {
        if (capacity == 0) {
            k_tile_scan<<<1, kScanThreads, 0, s>>>(sv2, 0, tile_ranges, 0, fine_total, n_instances_dev, nullptr,
                                                   nullptr, err);
            count_launches();
            return cuda_status(cudaGetLastError(), "gs_bin_sort: count");
        }
        I_grid = (uint32_t)capacity;
    }

    // 4. stable sort of the pairs by supertile id: each supertile's items contiguous, in depth order
    if ((e = radix_sort(ck, cv, I_grid, ctotal, st_bits, 4, ps, &which, s)) != cudaSuccess)
        return cuda_status(e, "gs_bin_sort: supertile sort");

    // 5. per-tile counts, tile ranges, then every instance's id at its place
    // the pairs' tile masks go to the free half of the pair buffers (2 bytes per pair)
    uint16_t* masks = reinterpret_cast<uint16_t*>(ck[which ^ 1]);
    auto pair_masks = tight ? k_pair_masks<true> : k_pair_masks<false>;
    int pair_grid = 0;  // at most 8 blocks per SM, each warp taking segments of kPairSeg pairs
    {
        int dev = 0, sms = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return cuda_status(e, "gs_bin_sort: device");
        pair_grid = 8 * sms;
    }
    pair_masks<<<(int)std::min<int64_t>(pair_grid, cdiv(I_grid, (int64_t)kPairSeg * (kThreads / 32))), kThreads, 0,
                 s>>>(
        sv2, mean2d, radius, ck[which], cv[which], I_grid, ctotal, (uint32_t)n, pack, masks, tile_ranges, st_count);
    count_launches();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e, "gs_bin_sort: tile counts");
    k_tile_scan<<<1, kScanThreads, 0, s>>>(sv2, ntiles, tile_ranges, (uint64_t)capacity, fine_total,
                                           graph ? n_instances_dev : nullptr, st_count, st_order, err);
    count_launches();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e, "gs_bin_sort: tile ranges");
    k_fine<<<nst, kFineThreads, 0, s>>>(sv2, depth, ck[which], cv[which], I_grid, ctotal,
                                        pack ? 0xFFFFu : 0xFFFFFFFFu, masks, tile_ranges, st_order, ids_sorted,
                                        keys_sorted);
    count_launches();
    return cuda_status(cudaGetLastError(), "gs_bin_sort: write lists");
}

}  // namespace gs
