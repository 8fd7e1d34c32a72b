// segsort.cu -- stable segmented radix sort (local sort of Sec. 5/6 and, over
// bucket ranges, the local merge).
//
// Design for sm_103a:
//  * A segment of at most 14336 keys is sorted by one CTA on chip: its keys are
//    read from HBM once into shared memory; a counting pass on a 10-bit digit
//    that interpolates the segment's [min, max] key range splits them into
//    1024 groups in key order; every key's final slot is its group's start plus
//    the number of keys of its group below it in (key, input position) order;
//    the keys are written once (16 B of HBM traffic per key).  Three CTA shapes
//    by segment size (128, 256, 512 threads).  A segment whose largest group is
//    above kTinyGroup keys (heavy duplicates, skew) goes to a stable LSD kernel
//    (8-bit digit passes over a 16-bit index permutation).
//  * A larger segment takes one read pass for statistics (digit counts and the
//    OR/AND of its keys) and one stable scatter on its first-split
//    digit (its top varying byte, or an interpolation of the key range the
//    caller bounds): the statistics pass counts every 4096-key tile's digits,
//    a scan turns the counts into each tile's destination offsets, and every
//    tile ranks its keys in shared memory (ballot peer masks with a payload,
//    one shared atomic per key for keys alone) and writes them out.  The 256 sub-buckets are then sorted the same way (on chip
//    when small, recursively otherwise), so a uniform 64-bit input costs
//    8 + 16 + 16 B of HBM traffic per key instead of the 136 B of eight LSD
//    passes.  A segment whose keys are all equal is copied straight to the
//    output by its scatter pass.
#include "segsort.cuh"

#include <algorithm>
#include <atomic>

namespace hss {

__host__ __device__ static inline uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }
static inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Process-wide tuning (hss_set_tuning).
static std::atomic<uint32_t> g_chip_max{(uint32_t)kC1Cap};
static std::atomic<uint32_t> g_child_interp{0u};
static std::atomic<uint32_t> g_child_keys{384u};
static std::atomic<uint32_t> g_pack_keys{1024u};
static std::atomic<uint32_t> g_splitters{0u};
static std::atomic<uint32_t> g_scatter{0u};

int set_tuning(const hss_tuning* t) {
    if (!t) {
        g_chip_max = (uint32_t)kC1Cap;
        g_child_interp = 0u;
        g_child_keys = 384u;
        g_pack_keys = 1024u;
        g_splitters = 0u;
        g_scatter = 0u;
        return HSS_OK;
    }
    const uint32_t cm = t->chip_max_keys ? t->chip_max_keys : (uint32_t)kC1Cap;
    const uint32_t ck = t->child_bucket_keys ? t->child_bucket_keys : 384u;
    const uint32_t pk = t->pack_keys ? t->pack_keys : 1024u;
    if ((cm != (uint32_t)kC1Cap && cm != (uint32_t)kSmallCap) || t->child_interp > 1u || ck < 128u || ck > 4096u ||
        pk > 4096u || t->first_split > 1u || t->split_scatter > 1u)
        return HSS_ERR_INVALID;
    for (uint32_t r : t->reserved)
        if (r) return HSS_ERR_INVALID;
    g_chip_max = cm;
    g_child_interp = t->child_interp;
    g_child_keys = ck;
    g_pack_keys = pk;
    g_splitters = t->first_split;
    g_scatter = t->split_scatter;
    return HSS_OK;
}
void get_tuning(hss_tuning* t) {
    *t = hss_tuning{};
    t->chip_max_keys = g_chip_max;
    t->child_interp = g_child_interp;
    t->child_bucket_keys = g_child_keys;
    t->pack_keys = g_pack_keys;
    t->first_split = g_splitters;
    t->split_scatter = g_scatter;
}

// Large segments of a level hold more than kC1Cap keys (keys alone split above
// the middle on-chip class), so a level has at most N / (kC1Cap + 1) of them.
static uint64_t max_large_of(uint64_t N) { return std::max<uint64_t>(1, N / (kC1Cap + 1)); }

struct WsDims {
    uint64_t ml, list, tiles;
};
static WsDims ws_dims(uint64_t N, uint64_t nseg) {
    WsDims d;
    d.ml = max_large_of(N);
    d.list = std::max<uint64_t>(nseg, d.ml * kRadix);
    d.tiles = ceil_div(std::max<uint64_t>(N, 1), kOsTile) + d.ml + 1;
    return d;
}

size_t segsort_ws_bytes(uint64_t N, uint64_t nseg) {
    const WsDims d = ws_dims(N, nseg);
    size_t b = 0;
    b += align_up((d.list + 1) * 4, 256) + align_up(d.list * 4, 256);  // tile_start, large_id
    b += align_up(d.tiles * 4, 256);                                  // tile_seg
    b += align_up(d.ml * 4, 256);                                     // large_seg
    b += align_up(d.tiles * 2 * kRadix * 2, 256);                     // tile_hist
    b += align_up(d.tiles, 256);                                      // tile_skew
    b += align_up(std::min(nseg, d.ml) * kRadix * 8, 256);           // spl_tab
    b += align_up(std::min(nseg, d.ml), 256);                        // spl_mode
    b += 2 * align_up(d.ml * 8, 256);                                 // vor, vand
    b += 4 * align_up(d.ml * 4, 256);                                 // msd_shift x2, spec, direct
    b += 2 * align_up(d.ml * 8, 256);                                 // msd_base, msd_mult
    b += 4 * align_up(d.ml * kRadix * 8, 256);                        // sub_lo/hi x2
    b += 6 * align_up(d.ml * kRadix * 8, 256);                        // cmin/cmax/cmult x2
    b += align_up(d.ml * 8 * 4, 256) + align_up(d.ml * 4, 256);       // large_mask, any_large
    b += align_up(d.tiles * kRadix * 4, 256);                         // tile_off
    b += align_up(64 * 4, 256);                                       // counters
    b += 8 * align_up(d.list * 4, 256);                               // class lists, fallback, slow lists
    b += align_up(8 * (d.list / 1024 + 2) * 4, 256);                  // blk
    return b;
}

SegSortWs segsort_ws_carve(void* base, uint64_t N, uint64_t nseg, uint32_t* err) {
    const WsDims d = ws_dims(N, nseg);
    SegSortWs w;
    w.max_large = d.ml;
    w.max_list = d.list;
    w.max_tiles = d.tiles;
    char* p = (char*)base;
    auto take = [&](size_t bytes) { void* r = p; p += align_up(bytes, 256); return r; };
    w.tile_start = (uint32_t*)take((d.list + 1) * 4);
    w.large_id = (uint32_t*)take(d.list * 4);
    w.tile_seg = (uint32_t*)take(d.tiles * 4);
    w.large_seg = (uint32_t*)take(d.ml * 4);
    w.tile_hist = (uint16_t*)take(d.tiles * 2 * kRadix * 2);
    w.tile_skew = (uint8_t*)take(d.tiles);
    w.max_spl = std::min(nseg, d.ml);
    w.spl_tab = (uint64_t*)take(w.max_spl * kRadix * 8);
    w.spl_mode = (uint8_t*)take(w.max_spl);
    w.vor = (unsigned long long*)take(d.ml * 8);
    w.vand = (unsigned long long*)take(d.ml * 8);
    w.msd_shift[0] = (uint32_t*)take(d.ml * 4);
    w.msd_shift[1] = (uint32_t*)take(d.ml * 4);
    w.spec = (uint32_t*)take(d.ml * 4);
    w.direct = (uint32_t*)take(d.ml * 4);
    w.msd_base = (uint64_t*)take(d.ml * 8);
    w.msd_mult = (uint64_t*)take(d.ml * 8);
    for (int i = 0; i < 2; ++i) {
        w.sub_lo[i] = (uint64_t*)take(d.ml * kRadix * 8);
        w.sub_hi[i] = (uint64_t*)take(d.ml * kRadix * 8);
        w.cmin[i] = (uint64_t*)take(d.ml * kRadix * 8);
        w.cmax[i] = (uint64_t*)take(d.ml * kRadix * 8);
        w.cmult[i] = (uint64_t*)take(d.ml * kRadix * 8);
    }
    w.large_mask = (uint32_t*)take(d.ml * 8 * 4);
    w.any_large = (uint32_t*)take(d.ml * 4);
    w.tile_off = (uint32_t*)take(d.tiles * kRadix * 4);
    w.counters = (uint32_t*)take(64 * 4);
    for (int i = 0; i < 3; ++i) w.list[i] = (uint32_t*)take(d.list * 4);
    w.fb_list = (uint32_t*)take(d.list * 4);
    w.slow_list = (uint32_t*)take(d.list * 4);
    for (int i = 0; i < 3; ++i) w.slow_keys[i] = (uint32_t*)take(d.list * 4);
    w.blk = (uint32_t*)take(8 * (d.list / 1024 + 2) * 4);
    w.err = err;
    return w;
}

// Digit of the first split of a segment: an 8-bit window of the key, or (mult
// != 0) a linear interpolation of the segment's key range onto 0..255.
__device__ __forceinline__ uint32_t split_digit(uint64_t key, int shift, uint64_t base, uint64_t mult) {
    if (mult) return min((uint32_t)__umul64hi(key - base, mult), 255u);
    return (uint32_t)((key >> shift) - base) & 255u;
}

// Multiplier m of an interpolating digit mulhi(x - lo, m) of a key range of
// width `range` onto 0..R-1: about (R-1) 2^64 / range, in single precision.
// Any m keeps the digit monotone in the key (callers clamp it to R-1); this
// one spreads the range evenly.  (Double precision is far slower here and
// buys nothing.)
__device__ __forceinline__ uint64_t interp_mult(uint64_t range, uint32_t R) {
    if (range < (uint64_t)R) return 0ull;
    return __float2ull_rz((float)(R - 1) * 18446744073709551616.0f / (float)range);
}
// The same for 32-bit offsets: mulhi(x - lo, m) onto 0..R-1.
__device__ __forceinline__ uint32_t interp_mult32(uint32_t range, uint32_t R) {
    if (range < R) return 0u;
    return __float2uint_rz((float)(R - 1) * 4294967296.0f / (float)range);
}

// ---------------------------------------------------------------------------
// Exclusive scan of 256 shared values by a CTA of T threads (T >= 64).
// ---------------------------------------------------------------------------
template <int T>
__device__ __forceinline__ void scan256_smem(const uint32_t* in, uint32_t* out, uint32_t* s_warp) {
    constexpr int U = T < kRadix ? T : kRadix;
    constexpr int K = kRadix / U;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    uint32_t loc[K];
    uint32_t sum = 0;
    if (tid < U) {
#pragma unroll
        for (int k = 0; k < K; ++k) { loc[k] = in[tid * K + k]; sum += loc[k]; }
    }
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31 && tid < U) s_warp[w] = x;
    __syncthreads();
    if (tid < U) {
        uint32_t run = x - sum;
        for (int i = 0; i < w; ++i) run += s_warp[i];
#pragma unroll
        for (int k = 0; k < K; ++k) { out[tid * K + k] = run; run += loc[k]; }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Peer mask of an 8-bit digit inside a warp, from eight ballots: the lanes
// whose digit equals this lane's.  Lanes with valid == false match nobody and
// are matched by nobody.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t warp_peers8(uint32_t d, bool valid) {
    uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int b = 0; b < kRadixBits; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t m = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? m : ~m;
    }
    return valid ? peers : 0u;
}

// ---------------------------------------------------------------------------
// Stable block ranking of 8-bit digits, in three steps:
//   1. counts: every warp counts its digits into its own 256 shared counters
//      (fire-and-forget shared atomics, no dependency chain);
//   2. offsets: the counts become absolute bases start[d] + (earlier warps'
//      counts of d), plus the tile totals;
//   3. ranks: per item, the lanes holding the same digit (ballot peer mask)
//      take consecutive slots: the highest such lane adds their number to the
//      warp's base for that digit and broadcasts the old value.
// Items are warp-striped: item i of lane l in warp w is element
// w*32*ITEMS + i*32 + l, so (w, i, l) order is element order and the ranks are
// stable.  Shared atomics issued by one warp in program order are applied in
// that order, which the running bases of step 3 rely on.  `between` runs after
// step 2.
// ---------------------------------------------------------------------------
struct NoOp { __device__ void operator()() const {} };

template <int WARPS, int ITEMS, typename DigitOf, typename Between>
__device__ __forceinline__ void block_rank(DigitOf digit_of, uint32_t count, uint32_t (&rank)[ITEMS],
                                           uint32_t* s_cnt /*[WARPS*256]*/, uint32_t* s_total, uint32_t* s_start,
                                           uint32_t* s_warp, Between between) {
    constexpr int T = WARPS * 32;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t wfirst = (uint32_t)w * 32 * ITEMS;  // element of the warp's first item slot
    for (int i = tid; i < WARPS * kRadix; i += T) s_cnt[i] = 0;
    __syncthreads();
    uint32_t* c = s_cnt + w * kRadix;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if (wfirst + i * 32 >= count) break;  // the rest of this warp's slots are empty
        const uint32_t d = digit_of(i);
        if (d < kRadix) atomicAdd(&c[d], 1u);
    }
    __syncthreads();
    for (int d = tid; d < kRadix; d += T) {
        uint32_t run = 0;
        for (int ww = 0; ww < WARPS; ++ww) {
            const uint32_t x = s_cnt[ww * kRadix + d];
            s_cnt[ww * kRadix + d] = run;
            run += x;
        }
        s_total[d] = run;
    }
    __syncthreads();
    scan256_smem<T>(s_total, s_start, s_warp);
    for (int d = tid; d < kRadix; d += T) {
        const uint32_t st = s_start[d];
        for (int ww = 0; ww < WARPS; ++ww) s_cnt[ww * kRadix + d] += st;
    }
    __syncthreads();
    between();
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if (wfirst + i * 32 >= count) break;
        const uint32_t d = digit_of(i);
        const bool valid = d < kRadix;
        const uint32_t peers = warp_peers8(d & 255u, valid);
        const int leader = valid ? 31 - __clz(peers) : lane;
        uint32_t base = 0;
        if (valid && lane == leader) base = atomicAdd(&c[d], (uint32_t)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        rank[i] = base + __popc(peers & lt);
    }
}

// ---------------------------------------------------------------------------
// On-chip sort of segments with min_n < n <= max_n keys (n <= CAP), taken
// from `list` (compact ids, count at *nlist) or, when list is null, from all
// nseg segments.  The keys are read once into shared memory.  One counting
// pass on a 10-bit digit (the segment's key range interpolated onto 1024
// groups) splits them into groups that come in key order; inside a group the
// atomics leave an arbitrary order, and each key's final slot is its group's
// start plus the number of keys of the group below it in (key, input
// position) order -- a total order, so the result is the stable sort.
// Groups larger than kTinyGroup are not ranked that way: when every such
// group holds one key value (heavy duplicates), its members only need input
// order, which two ordered warp passes over the positions give; a segment
// with a larger group of distinct keys is left to the stable LSD kernel below
// (appended to the fallback list).
// ---------------------------------------------------------------------------
constexpr int kChipRadix = 1024;  // groups of the on-chip counting pass
constexpr int kMaxBig = 64;       // groups above kTinyGroup keys that one segment may hold
constexpr uint32_t kMixedMax = 256;  // a big group of distinct keys up to this size is ranked on chip

// Exclusive scan of NV shared values in place by a CTA of T threads.
template <int T, int NV>
__device__ __forceinline__ void scan_smem_inplace(uint32_t* v, uint32_t* s_warp) {
    constexpr int K = NV / T;
    static_assert(NV % T == 0, "scan size");
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    uint32_t loc[K];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) { loc[k] = v[tid * K + k]; sum += loc[k]; }
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    uint32_t run = x - sum;
    for (int i = 0; i < w; ++i) run += s_warp[i];
#pragma unroll
    for (int k = 0; k < K; ++k) { v[tid * K + k] = run; run += loc[k]; }
    __syncthreads();
}

// Write a sorted segment: keys from shared memory in the order `order`, and
// the payload gathered from the segment's input payload.  The output may be
// the input itself (every second level of the recursion sorts its small
// buckets in place), so every payload value is gathered into registers before
// the barrier and stored after it, and the on-chip kernels take their key and
// payload buffers without __restrict__: with it the compiler may move the
// gathers past the stores.
template <bool PAY, int THREADS, int CAP>
__device__ __forceinline__ void write_sorted(uint64_t* kout, uint32_t* pout, const uint32_t* pin, uint64_t base,
                                             uint32_t n, const uint64_t* s_keys, const uint16_t* order, uint64_t flip_out) {
    const int tid = threadIdx.x;
    if (PAY) {
        constexpr int PER = (CAP + THREADS - 1) / THREADS;
        uint32_t pv[PER];
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const uint32_t j = tid + i * THREADS;
            pv[i] = j < n ? pin[base + order[j]] : 0u;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const uint32_t j = tid + i * THREADS;
            if (j < n) pout[base + j] = pv[i];
        }
    }
    for (uint32_t j = tid; j < n; j += THREADS) kout[base + j] = s_keys[order[j]] ^ flip_out;
    __syncthreads();
}

// Groups of the counting pass by size class: about two keys per group for
// the smallest segments (a smaller scan per segment), 1024 groups above that
// (clustered keys in larger segments would otherwise crowd one group).
template <int CAP>
constexpr int chip_radix() { return CAP <= kC0Cap ? 512 : kChipRadix; }

// The largest class re-splits crowded groups on chip (see k_small_msd).
template <int CAP>
constexpr bool chip_resplit() { return CAP > kC1Cap; }

template <int THREADS, int CAP>
constexpr size_t msd_sort_smem() {
    return (size_t)CAP * 8 + 3 * (size_t)CAP * 2 + 2 * (chip_radix<CAP>() + 1) * 4 + 32 * 4 + 2 * 32 * 8 +
           (size_t)(THREADS / 32) * kMaxBig * 4 + kMaxBig * 4 + chip_radix<CAP>() + 64 +
           (chip_resplit<CAP>() ? (size_t)(chip_radix<CAP>() + 1) * 4 + kMaxBig * 2 : 0);
}

template <bool PAY, int THREADS, int CAP>
__global__ __launch_bounds__(THREADS) void k_small_msd(
    const uint64_t* kin, uint64_t* kout, const uint32_t* pin, uint32_t* pout, const uint64_t* __restrict__ seg_lo,
    const uint64_t* __restrict__ seg_hi, const uint32_t* __restrict__ list, const uint32_t* __restrict__ nlist,
    uint64_t nseg, uint32_t min_n,
    uint32_t max_n, uint64_t flip_in, uint64_t flip_out, uint32_t* __restrict__ fb_list, uint32_t* __restrict__ fb_count) {
    constexpr int WARPS = THREADS / 32;
    constexpr int R = chip_radix<CAP>();
    // Mixed big groups are ranked on chip in the two smaller classes (up to
    // kMixedMax keys).  The largest class, where big groups come from
    // clustered keys, re-splits each one by a second counting pass that
    // interpolates the group's own key range; a segment with a sub-group
    // still above kTinyGroup keys goes to the LSD kernel.
    constexpr bool kMixed = CAP <= kC1Cap;
    constexpr bool kResplit = chip_resplit<CAP>();
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* s_keys = (uint64_t*)smem;                        // CAP u64
    uint16_t* s_grp = (uint16_t*)(s_keys + CAP);               // CAP u16: positions grouped by digit
    uint16_t* s_out = s_grp + CAP;                             // CAP u16: positions in sorted order
    uint16_t* s_dig = s_out + CAP;                             // CAP u16: digit of each position
    uint32_t* s_start = (uint32_t*)(s_dig + CAP);              // R+1: counts, then group starts
    uint32_t* s_run = s_start + (R + 1);              // R+1: running write positions
    uint32_t* s_warp = s_run + (R + 1);               // 32
    uint64_t* s_red = (uint64_t*)(((uintptr_t)(s_warp + 32) + 7) & ~(uintptr_t)7);  // 2*32
    uint32_t* s_wcnt = (uint32_t*)(s_red + 64);                 // WARPS*kMaxBig: per-warp counts of the big groups
    uint32_t* s_misc = s_wcnt + WARPS * kMaxBig;                // [0] big groups, [1] a mixed group above kMixedMax
    uint32_t* s_mixed = s_misc + 2;                             // kMaxBig: the big group holds distinct keys
    uint8_t* s_bigid = (uint8_t*)(s_mixed + kMaxBig);           // R: index of a big group, 0xff otherwise
    uint32_t* s_h2 = (uint32_t*)(s_bigid + R);                  // R+1 (kResplit): sub-group starts
    uint16_t* s_bigd = (uint16_t*)(s_h2 + R + 1);               // kMaxBig (kResplit): digit of each big group

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint64_t count = list ? (uint64_t)*nlist : nseg;
    for (uint64_t k = blockIdx.x; k < count; k += gridDim.x) {
        const uint64_t s = list ? (uint64_t)list[k] : k;
        const uint64_t base = seg_lo[s];
        const uint64_t n64 = seg_hi[s] - base;
        if (n64 <= min_n || n64 > max_n) continue;  // uniform per CTA
        const uint32_t n = (uint32_t)n64;
        uint64_t kmin = ~0ull, kmax = 0;
        for (uint32_t j = tid; j < n; j += THREADS) {
            const uint64_t key = kin[base + j] ^ flip_in;
            s_keys[j] = key;
            kmin = min(kmin, key);
            kmax = max(kmax, key);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            kmin = min(kmin, (uint64_t)__shfl_xor_sync(0xffffffffu, kmin, o));
            kmax = max(kmax, (uint64_t)__shfl_xor_sync(0xffffffffu, kmax, o));
        }
        if (lane == 0) { s_red[w] = kmin; s_red[32 + w] = kmax; }
        for (int d = tid; d < R; d += THREADS) s_start[d] = 0;
        if (tid == 0) { s_misc[0] = 0; s_misc[1] = 0; }
        __syncthreads();
        {
            uint64_t a = ~0ull, b = 0;
            for (int i = 0; i < WARPS; ++i) { a = min(a, s_red[i]); b = max(b, s_red[32 + i]); }
            kmin = a;
            kmax = b;
        }
        if (kmin == kmax) {  // all keys equal: already in order
            for (uint32_t j = tid; j < n; j += THREADS) {
                kout[base + j] = s_keys[j] ^ flip_out;
                if (PAY) pout[base + j] = pin[base + j];
            }
            __syncthreads();
            continue;
        }
        // Counting pass on a 10-bit digit: the key range [kmin, kmax]
        // interpolated onto 0..1023, monotone in the key (a plain offset when
        // the range is narrower than 1024).  The groups come in key order; the
        // atomics leave an arbitrary order inside a group, and each key's final
        // slot is its group's start plus the number of keys of the group below
        // it in (key, input position) order -- a total order, so the result is
        // the stable sort.  Any monotone digit gives the same result, so the
        // multiplier only needs to be about 1023 * 2^64 / range.
        const uint64_t range = kmax - kmin;
        const uint64_t mult = interp_mult(range, (uint32_t)R);
        for (uint32_t e = tid; e < n; e += THREADS) {
            const uint64_t off = s_keys[e] - kmin;
            const uint32_t d = mult ? min((uint32_t)__umul64hi(off, mult), (uint32_t)R - 1) : (uint32_t)off;
            s_dig[e] = (uint16_t)d;
            atomicAdd(&s_start[d], 1u);
        }
        __syncthreads();
        uint32_t mx = 0;
        for (int d = tid; d < R; d += THREADS) mx = max(mx, s_start[d]);
        mx = __reduce_max_sync(0xffffffffu, mx);
        scan_smem_inplace<THREADS, R>(s_start, s_warp);
        if (lane == 0) s_warp[w] = mx;
        for (int d = tid; d < R; d += THREADS) s_run[d] = s_start[d];
        if (tid == 0) s_start[R] = n;
        __syncthreads();
        mx = 0;
        for (int i = 0; i < WARPS; ++i) mx = max(mx, s_warp[i]);
        const bool big = mx > (uint32_t)kTinyGroup;  // uniform per CTA
        if (big) {
            for (int d = tid; d < R; d += THREADS) {
                uint8_t id = 0xff;
                if (s_start[d + 1] - s_start[d] > (uint32_t)kTinyGroup) {
                    const uint32_t i = atomicAdd(&s_misc[0], 1u);
                    if (kResplit && i < (uint32_t)kMaxBig) s_bigd[i] = (uint16_t)d;
                    id = (uint8_t)min(i, 255u);
                }
                s_bigid[d] = id;
            }
            if (kMixed || kResplit)
                for (int g = tid; g < kMaxBig; g += THREADS) s_mixed[g] = 0u;
            __syncthreads();
            if (s_misc[0] > (uint32_t)kMaxBig) {  // too many big groups: the LSD kernel takes this segment
                if (tid == 0) fb_list[atomicAdd(fb_count, 1u)] = (uint32_t)s;
                __syncthreads();
                continue;
            }
        }
        for (uint32_t e = tid; e < n; e += THREADS) s_grp[atomicAdd(&s_run[s_dig[e]], 1u)] = (uint16_t)e;
        __syncthreads();
        for (uint32_t q = tid; q < n; q += THREADS) {
            const uint16_t x = s_grp[q];
            const uint64_t kx = s_keys[x];
            const uint32_t d = s_dig[x];
            const uint32_t a = s_start[d], b = s_start[d + 1];
            if (b - a > (uint32_t)kTinyGroup) {  // big group: only check whether it holds one key value
                if (kx != s_keys[s_grp[a]]) {
                    if (kResplit) {
                        s_mixed[s_bigid[d]] = 2u;  // re-split below
                    } else {
                        if (kMixed) s_mixed[s_bigid[d]] = 1u;
                        if (!kMixed || b - a > kMixedMax) s_misc[1] = 1u;
                    }
                }
                continue;
            }
            uint32_t r = 0;
            for (uint32_t g = a; g < b; ++g) {
                const uint16_t y = s_grp[g];
                const uint64_t ky = s_keys[y];
                r += (ky < kx || (ky == kx && y < x)) ? 1u : 0u;
            }
            s_out[a + r] = x;
        }
        __syncthreads();
        if (big && kResplit) {
            // Re-split every big group of distinct keys, one at a time by the
            // whole CTA: a counting pass on a digit interpolating the group's
            // own key range (any monotone digit keeps the order), positions
            // scattered by sub-group into the group's slots of s_out, then
            // each key ranked inside its sub-group by (key, input position)
            // into s_grp and copied back to s_out.
            const uint32_t nbig = s_misc[0];
            for (uint32_t g = 0; g < nbig; ++g) {
                if (s_mixed[g] != 2u) continue;  // uniform: read after a barrier
                const uint32_t dg = s_bigd[g];
                const uint32_t a = s_start[dg], b = s_start[dg + 1];
                uint64_t gmin = ~0ull, gmax = 0;
                for (uint32_t q = a + tid; q < b; q += THREADS) {
                    const uint64_t kq = s_keys[s_grp[q]];
                    gmin = min(gmin, kq);
                    gmax = max(gmax, kq);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    gmin = min(gmin, (uint64_t)__shfl_xor_sync(0xffffffffu, gmin, o));
                    gmax = max(gmax, (uint64_t)__shfl_xor_sync(0xffffffffu, gmax, o));
                }
                if (lane == 0) { s_red[w] = gmin; s_red[32 + w] = gmax; }
                for (int i = tid; i < R; i += THREADS) s_h2[i] = 0u;
                __syncthreads();
                for (int i = 0; i < WARPS; ++i) { gmin = min(gmin, s_red[i]); gmax = max(gmax, s_red[32 + i]); }
                const uint64_t r2 = gmax - gmin;
                const uint64_t m2 = interp_mult(r2, (uint32_t)R);
                auto dig2 = [&](uint64_t kq) -> uint32_t {
                    const uint64_t off = kq - gmin;
                    return m2 ? min((uint32_t)__umul64hi(off, m2), (uint32_t)R - 1) : (uint32_t)off;
                };
                for (uint32_t q = a + tid; q < b; q += THREADS) atomicAdd(&s_h2[dig2(s_keys[s_grp[q]])], 1u);
                __syncthreads();
                for (int i = tid; i < R; i += THREADS)
                    if (s_h2[i] > (uint32_t)kTinyGroup) s_misc[1] = 1u;  // still crowded: LSD kernel
                scan_smem_inplace<THREADS, R>(s_h2, s_warp);        // ends with a barrier
                if (s_misc[1]) break;                               // uniform
                for (int i = tid; i < R; i += THREADS) s_run[i] = s_h2[i];
                if (tid == 0) s_h2[R] = b - a;
                __syncthreads();
                for (uint32_t q = a + tid; q < b; q += THREADS) {
                    const uint16_t x = s_grp[q];
                    s_out[a + atomicAdd(&s_run[dig2(s_keys[x])], 1u)] = x;
                }
                __syncthreads();
                for (uint32_t q = a + tid; q < b; q += THREADS) {
                    const uint16_t x = s_out[q];
                    const uint64_t kx = s_keys[x];
                    const uint32_t d2 = dig2(kx);
                    const uint32_t lo2 = a + s_h2[d2], hi2 = a + s_h2[d2 + 1];
                    uint32_t r = 0;
                    for (uint32_t q2 = lo2; q2 < hi2; ++q2) {
                        const uint16_t y = s_out[q2];
                        const uint64_t ky = s_keys[y];
                        r += (ky < kx || (ky == kx && y < x)) ? 1u : 0u;
                    }
                    s_grp[lo2 + r] = x;
                }
                __syncthreads();
                for (uint32_t q = a + tid; q < b; q += THREADS) s_out[q] = s_grp[q];
                __syncthreads();
            }
        }
        if (big) {
            if (s_misc[1]) {  // a large group of distinct keys: the LSD kernel takes this segment
                if (tid == 0) fb_list[atomicAdd(fb_count, 1u)] = (uint32_t)s;
                __syncthreads();
                continue;
            }
            // Big groups of distinct keys (at most kMixedMax): the same rank by
            // (key, input position), quadratic in the group size.
            for (uint32_t q = tid; kMixed && q < n; q += THREADS) {
                const uint16_t x = s_grp[q];
                const uint32_t d = s_dig[x];
                const uint32_t a = s_start[d], b = s_start[d + 1];
                if (b - a <= (uint32_t)kTinyGroup || !s_mixed[s_bigid[d]]) continue;
                const uint64_t kx = s_keys[x];
                uint32_t r = 0;
                for (uint32_t g = a; g < b; ++g) {
                    const uint16_t y = s_grp[g];
                    const uint64_t ky = s_keys[y];
                    r += (ky < kx || (ky == kx && y < x)) ? 1u : 0u;
                }
                s_out[a + r] = x;
            }
            // Members of each big group in input order: warp w walks the
            // positions [w*C, (w+1)*C) in order; pass A counts the members of
            // every big group per warp, a scan over the warps turns the counts
            // into starts, and pass B places each member at its group's start
            // plus the members before it.
            const uint32_t nbig = s_misc[0];
            const uint32_t C = ((n + WARPS - 1) / WARPS + 31) / 32 * 32;
            const uint32_t lo = min(n, (uint32_t)w * C), hi = min(n, lo + C);
            const uint32_t lt = (1u << lane) - 1u;
            uint32_t* wc = s_wcnt + w * kMaxBig;
            for (uint32_t b = lane; b < nbig; b += 32) wc[b] = 0;
            __syncwarp();
            for (uint32_t p0 = lo; p0 < hi; p0 += 32) {
                const uint32_t e = p0 + lane;
                uint32_t g = e < hi ? (uint32_t)s_bigid[s_dig[e]] : 0xffu;
                if ((kMixed || kResplit) && g != 0xffu && s_mixed[g]) g = 0xffu;  // ranked above
                const bool valid = g != 0xffu;
                const uint32_t peers = __match_any_sync(0xffffffffu, valid ? g : 0x100u + lane);
                if (valid && (peers & lt) == 0u) wc[g] += (uint32_t)__popc(peers);
                __syncwarp();
            }
            __syncthreads();
            for (uint32_t b = tid; b < nbig; b += THREADS) {
                uint32_t run = 0;
                for (int v = 0; v < WARPS; ++v) {
                    const uint32_t c = s_wcnt[v * kMaxBig + b];
                    s_wcnt[v * kMaxBig + b] = run;
                    run += c;
                }
            }
            __syncthreads();
            for (uint32_t p0 = lo; p0 < hi; p0 += 32) {
                const uint32_t e = p0 + lane;
                const uint32_t d = e < hi ? (uint32_t)s_dig[e] : 0u;
                uint32_t g = e < hi ? (uint32_t)s_bigid[d] : 0xffu;
                if ((kMixed || kResplit) && g != 0xffu && s_mixed[g]) g = 0xffu;  // ranked above
                const bool valid = g != 0xffu;
                const uint32_t peers = __match_any_sync(0xffffffffu, valid ? g : 0x100u + lane);
                const uint32_t before = valid ? wc[g] : 0u;
                __syncwarp();
                if (valid) {
                    s_out[s_start[d] + before + (uint32_t)__popc(peers & lt)] = (uint16_t)e;
                    if ((peers & lt) == 0u) wc[g] = before + (uint32_t)__popc(peers);
                }
                __syncwarp();
            }
            __syncthreads();
        }
        write_sorted<PAY, THREADS, CAP>(kout, pout, pin, base, n, s_keys, s_out, flip_out);
    }
}

// ---------------------------------------------------------------------------
// The same on-chip sort for segments of up to CAP = THREADS * ITEMS keys
// (ITEMS <= 16) with the keys, digits and group slots held in registers:
// one counting pass on the 10-bit digit, a scatter that stores each key and
// its input position at its group slot, and a rank only for keys whose group
// holds more than one key (a singleton's slot is its final position).  About
// half the shared-memory traffic of k_small_msd.  A segment with a group
// larger than kTinyGroup is appended to slow_list for k_small_msd.  It runs
// the middle size class (up to 4096 keys, 256 threads); for the smallest
// class the shared-memory kernel measured faster (more CTAs per SM).
// ---------------------------------------------------------------------------
template <int CAP>
constexpr size_t reg_sort_smem() {
    return (size_t)CAP * 8 + (size_t)CAP * 2 + 2 * (kChipRadix + 1) * 4 + 32 * 4 + 2 * 32 * 8 + 64;
}

template <bool PAY, int THREADS, int CAP>
__global__ __launch_bounds__(THREADS) void k_small_reg(
    const uint64_t* kin, uint64_t* kout, const uint32_t* pin, uint32_t* pout, const uint64_t* __restrict__ seg_lo,
    const uint64_t* __restrict__ seg_hi, const uint32_t* __restrict__ list, const uint32_t* __restrict__ nlist,
    uint64_t nseg, uint32_t min_n, uint32_t max_n, uint64_t flip_in, uint64_t flip_out,
    uint32_t* __restrict__ slow_list, uint32_t* __restrict__ slow_count) {
    constexpr int ITEMS = CAP / THREADS;
    static_assert(CAP % THREADS == 0 && ITEMS <= 16 && CAP <= 4096 && kChipRadix <= 4096, "register sort shape");
    constexpr int WARPS = THREADS / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* s_key = (uint64_t*)smem;                     // CAP: keys by group slot, then in final order
    uint16_t* s_idx = (uint16_t*)(s_key + CAP);            // CAP: their input positions
    uint32_t* s_start = (uint32_t*)(s_idx + CAP);          // kChipRadix+1: counts, then group starts
    uint32_t* s_run = s_start + (kChipRadix + 1);          // kChipRadix+1: running slots
    uint32_t* s_warp = s_run + (kChipRadix + 1);           // 32
    uint64_t* s_red = (uint64_t*)(((uintptr_t)(s_warp + 32) + 7) & ~(uintptr_t)7);  // 2*32

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint64_t count = list ? (uint64_t)*nlist : nseg;
    for (uint64_t k = blockIdx.x; k < count; k += gridDim.x) {
        const uint64_t s = list ? (uint64_t)list[k] : k;
        const uint64_t base = seg_lo[s];
        const uint64_t n64 = seg_hi[s] - base;
        if (n64 <= min_n || n64 > max_n) continue;  // uniform per CTA
        const uint32_t n = (uint32_t)n64;
        uint64_t key[ITEMS];
        uint64_t kmin = ~0ull, kmax = 0;
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t e = tid + i * THREADS;
            key[i] = e < n ? kin[base + e] ^ flip_in : 0ull;
            if (e < n) { kmin = min(kmin, key[i]); kmax = max(kmax, key[i]); }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            kmin = min(kmin, (uint64_t)__shfl_xor_sync(0xffffffffu, kmin, o));
            kmax = max(kmax, (uint64_t)__shfl_xor_sync(0xffffffffu, kmax, o));
        }
        if (lane == 0) { s_red[w] = kmin; s_red[32 + w] = kmax; }
        for (int d = tid; d < kChipRadix; d += THREADS) s_start[d] = 0;
        __syncthreads();
        {
            uint64_t a = ~0ull, b = 0;
            for (int i = 0; i < WARPS; ++i) { a = min(a, s_red[i]); b = max(b, s_red[32 + i]); }
            kmin = a;
            kmax = b;
        }
        if (kmin == kmax) {  // all keys equal: already in order
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const uint32_t e = tid + i * THREADS;
                if (e < n) {
                    kout[base + e] = key[i] ^ flip_out;
                    if (PAY) pout[base + e] = pin[base + e];
                }
            }
            __syncthreads();
            continue;
        }
        const uint64_t range = kmax - kmin;
        const uint64_t mult = interp_mult(range, (uint32_t)kChipRadix);
        uint32_t dp[ITEMS];  // digit in bits 0..11, group slot from bit 12
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t e = tid + i * THREADS;
            dp[i] = 0;
            if (e < n) {
                const uint64_t off = key[i] - kmin;
                const uint32_t d = mult ? min((uint32_t)__umul64hi(off, mult), (uint32_t)kChipRadix - 1) : (uint32_t)off;
                dp[i] = d;
                atomicAdd(&s_start[d], 1u);
            }
        }
        __syncthreads();
        uint32_t mx = 0;
        for (int d = tid; d < kChipRadix; d += THREADS) mx = max(mx, s_start[d]);
        mx = __reduce_max_sync(0xffffffffu, mx);
        scan_smem_inplace<THREADS, kChipRadix>(s_start, s_warp);
        if (lane == 0) s_warp[w] = mx;
        for (int d = tid; d < kChipRadix; d += THREADS) s_run[d] = s_start[d];
        if (tid == 0) s_start[kChipRadix] = n;
        __syncthreads();
        mx = 0;
        for (int i = 0; i < WARPS; ++i) mx = max(mx, s_warp[i]);
        if (mx > (uint32_t)kTinyGroup) {  // skewed: the shared-memory kernel takes this segment
            if (tid == 0) slow_list[atomicAdd(slow_count, 1u)] = (uint32_t)s;
            __syncthreads();
            continue;
        }
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t e = tid + i * THREADS;
            if (e < n) {
                const uint32_t slot = atomicAdd(&s_run[dp[i]], 1u);
                s_key[slot] = key[i];
                s_idx[slot] = (uint16_t)e;
                dp[i] |= slot << 12;
            }
        }
        __syncthreads();
        // Final position: the group start plus the keys of the group below
        // this one in (key, input position) order; a singleton keeps its slot.
        uint32_t fin[ITEMS];
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t e = tid + i * THREADS;
            fin[i] = dp[i] >> 12;
            if (e < n) {
                const uint32_t d = dp[i] & 4095u;
                const uint32_t a = s_start[d], b = s_start[d + 1];
                if (b - a > 1u) {
                    uint32_t r = 0;
                    for (uint32_t g = a; g < b; ++g) {
                        const uint64_t ky = s_key[g];
                        r += (ky < key[i] || (ky == key[i] && s_idx[g] < e)) ? 1u : 0u;
                    }
                    fin[i] = a + r;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t e = tid + i * THREADS;
            if (e < n && fin[i] != (dp[i] >> 12)) {
                s_key[fin[i]] = key[i];
                if (PAY) s_idx[fin[i]] = (uint16_t)e;
            }
        }
        __syncthreads();
        if (PAY) {  // the output may be the input: gather every payload first
            uint32_t pv[ITEMS];
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const uint32_t j = tid + i * THREADS;
                pv[i] = j < n ? pin[base + s_idx[j]] : 0u;
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const uint32_t j = tid + i * THREADS;
                if (j < n) pout[base + j] = pv[i];
            }
        }
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t j = tid + i * THREADS;
            if (j < n) kout[base + j] = s_key[j] ^ flip_out;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Keys alone, on chip, segments of up to CAP = THREADS * ITEMS keys held in
// registers.  Equal keys are indistinguishable, so no input order has to be
// kept.  A counting pass on a digit interpolating the segment's key range (R
// groups, monotone in the key) hands every key a slot in its group through
// one shared counter, and the keys are scattered into group order; since the
// groups come in key order, what is left is the order inside each group:
// a key of a small group counts the group's keys below it (the keys stay in
// registers, so the only shared-memory traffic is the group's few keys), and
// a large group holding distinct keys is sorted by the CTA (a segment with
// more than kKeysMixedMax of them goes to slow_list for the shared-memory
// kernel).  The digit has about as many values as the segment has keys, so
// most groups hold one key.
// With PREFETCH the segments move between HBM and shared memory by bulk
// asynchronous copies (the TMA engine): one thread copies the next segment of
// the list into a staging buffer while the current one is sorted, and copies
// each sorted segment out of shared memory, so the threads issue no load or
// store per key.  A bulk copy needs 16-byte aligned addresses, so a segment's
// first key (when its address is 8 mod 16) and its last key (when one is left
// over) travel by 8-byte copies, and the keys sit in shared memory one slot
// further on in that case (key j at buffer[j + head]).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// One arrival that also announces `bytes` of bulk copies completing on bar.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// Bounded wait for the phase of the given parity to complete; false when the
// limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t it = 0; it < (1u << 20); ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void bulk_load(void* sdst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(sdst)),
                 "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(gdst), "r"(smem_u32(ssrc)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}
// The issuing thread's bulk stores have read their shared-memory source.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
// Shared-memory writes of this thread become visible to bulk copies.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

template <int CAP, int R, bool PREFETCH>
constexpr size_t keys_sort_smem() {
    return (size_t)(CAP + 2) * 8 * (PREFETCH ? 2 : 1) + (size_t)(R + 1) * 4 + 32 * 4 + 2 * 32 * 8 + 64 + (size_t)R +
           16;
}

// Mixed large groups sorted in place by the CTA per segment (more go to the
// shared-memory kernel).
constexpr int kKeysMixedMax = 8;

// In-place ascending sort of base[SI(a + i)], i in [0, m), by the whole CTA
// (SI: the caller's index map): a bitonic network over
// the next power of two P >= m in the form whose comparators all put the
// smaller key at the lower index (the first step of every merge compares
// mirrored positions), so that positions past m act as +infinity and are
// never touched.  Ends with a barrier.
template <int THREADS, typename Index>
__device__ __forceinline__ void cta_bitonic_sort(uint64_t* base, uint32_t a, uint32_t m, Index SI) {
    auto s = [&](uint32_t i) -> uint64_t& { return base[SI(a + i)]; };
    uint32_t P = 1;
    while (P < m) P <<= 1;
    for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t t = threadIdx.x; t < (P >> 1); t += THREADS) {
                uint32_t i, l;
                if (j == (k >> 1)) {  // mirrored pairs of each k-block
                    const uint32_t blk = t / j, r = t - blk * j;
                    i = blk * k + r;
                    l = blk * k + k - 1 - r;
                } else {
                    i = (t / j) * 2 * j + (t % j);
                    l = i + j;
                }
                if (l < m) {
                    const uint64_t x = s(i), y = s(l);
                    if (y < x) { s(i) = y; s(l) = x; }
                }
            }
            __syncthreads();
        }
    }
}

// CTAs per SM the register budget must allow: the small classes live on
// many buckets in flight per SM (their keys are prefetched while the
// previous bucket is sorted).
template <int THREADS>
constexpr int keys_min_blocks() { return THREADS <= 128 ? 8 : (THREADS <= 256 ? 3 : 1); }

// A digit monotone in off that spreads keys over many binary orders of
// magnitude: the position e of off's leading one, counted from e_lo (32
// positions e_lo .. e_lo + 31), followed by the M = log2(R) - 5 bits below
// the leading one; offsets below 2^e_lo (zero included) take digit 0.
template <int R>
__device__ __forceinline__ uint32_t log_digit(uint64_t off, int e_lo) {
    constexpr int M = (R >= 4096) ? 7 : (R >= 2048 ? 6 : (R >= 1024 ? 5 : 4));
    static_assert(32 * (1 << M) <= R, "log digit width");
    if (off == 0ull) return 0u;
    const int e = 63 - __clzll((long long)off);
    if (e < e_lo) return 0u;
    const uint32_t mant = e >= M ? (uint32_t)(off >> (e - M)) & ((1u << M) - 1u)
                                 : (uint32_t)(off << (M - e)) & ((1u << M) - 1u);
    return ((uint32_t)(e - e_lo) << M) | mant;
}

template <int THREADS, int CAP, int R, bool PREFETCH>
__global__ __launch_bounds__(THREADS, keys_min_blocks<THREADS>()) void k_small_keys(
    const uint64_t* kin, uint64_t* kout, const uint64_t* __restrict__ seg_lo, const uint64_t* __restrict__ seg_hi,
    const uint32_t* __restrict__ list, const uint32_t* __restrict__ nlist, uint64_t nseg, uint32_t min_n,
    uint32_t max_n, uint64_t flip_in, uint64_t flip_out, uint32_t* __restrict__ slow_list,
    uint32_t* __restrict__ slow_count, uint32_t* __restrict__ err) {
    constexpr int ITEMS = CAP / THREADS;
    constexpr int WARPS = THREADS / 32;
    static_assert(CAP % THREADS == 0 && R % THREADS == 0 && R <= 4096 && CAP <= 16384 && WARPS <= 16 &&
                      THREADS >= 64,
                  "keys sort shape");
    // dp[i]: digit in bits 0..11, slot in its group from bit 12
    constexpr uint32_t kDigitMask = 4095u, kSlotShift = 12, kSlotMask = 16383u;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* s_key = (uint64_t*)smem;                                              // CAP + 2
    uint64_t* s_stage = s_key + (CAP + 2);                                          // CAP + 2 (PREFETCH)
    uint32_t* s_start = (uint32_t*)(s_stage + (PREFETCH ? CAP + 2 : 0));            // R + 1
    uint32_t* s_warp = s_start + (R + 1);                                           // 32
    uint64_t* s_red = (uint64_t*)(((uintptr_t)(s_warp + 32) + 7) & ~(uintptr_t)7);  // 2 * 32
    uint32_t* s_flag = (uint32_t*)(s_red + 64);  // [0] mixed large groups, [1..kKeysMixedMax] their digits
    uint8_t* s_mark = (uint8_t*)(s_flag + 16);   // R: the group is large and holds distinct keys
    uint64_t* s_bar = (uint64_t*)(((uintptr_t)(s_mark + R) + 7) & ~(uintptr_t)7);  // staging buffer full

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint64_t count = list ? (uint64_t)*nlist : nseg;
    for (int d = tid; d < R; d += THREADS) s_mark[d] = 0;
    if (PREFETCH && tid == 0) mbar_init(s_bar, 1u);
    __syncthreads();
    // Segment descriptors travel one iteration ahead in registers: the loads
    // of the next segment's list entry and bounds are issued at the top of an
    // iteration and first used after its first barrier, so their latency
    // hides behind the current segment's work.
    struct Desc {
        uint64_t base;
        uint32_t n;
        bool ok;  // exists and belongs to this class
    };
    auto load_desc = [&](uint64_t k) -> Desc {
        Desc d{0ull, 0u, false};
        if (k < count) {
            const uint64_t s = list ? (uint64_t)list[k] : k;
            const uint64_t b = seg_lo[s], n = seg_hi[s] - b;
            d.base = b;
            d.n = (uint32_t)n;
            d.ok = n > min_n && n <= max_n && n > 0;
        }
        return d;
    };
    // 1 when the segment's first key sits at an address that is 8 mod 16.
    auto head_of = [](const uint64_t* p) -> uint32_t { return (uint32_t)(((uintptr_t)p >> 3) & 1u); };
    uint32_t phase = 0;  // parity of the staging buffer's next completion
    auto prefetch = [&](const Desc& d) {  // copy a segment into the staging buffer
        if (!d.ok) return;  // uniform
        const uint64_t* g = kin + d.base;
        const uint32_t hd = head_of(g), m = ((d.n - hd) >> 1) << 1;
        if (tid == 0) {
            mbar_arrive_expect_tx(s_bar, m * 8u);
            if (m) bulk_load(s_stage + 2 * hd, g + hd, m * 8u, s_bar);
        }
        if (hd && tid == 1) cp_async8(&s_stage[1], g);
        if (hd + m < d.n && tid == 2) cp_async8(&s_stage[d.n - 1 + hd], g + d.n - 1);
        cp_async_commit();
    };
    Desc nxt = load_desc(blockIdx.x);
    if (PREFETCH) prefetch(nxt);
    for (uint64_t k = blockIdx.x; k < count; k += gridDim.x) {
        const Desc cur = nxt;
        nxt = load_desc(k + gridDim.x);
        if (!cur.ok) {  // uniform per CTA; such a segment was never prefetched
            if (PREFETCH) prefetch(nxt);
            continue;
        }
        const uint64_t s = list ? (uint64_t)list[k] : k;
        const uint64_t base = cur.base;
        const uint32_t n = cur.n;
        uint32_t sh = 0;  // key j of the segment at src[j + sh]
        if (PREFETCH) {
            cp_async_wait_all();
            const bool late = !mbar_wait(s_bar, phase);
            phase ^= 1u;
            if (__syncthreads_or(late)) {  // uniform; not expected: a bulk copy that never landed
                if (tid == 0) atomicOr(err, kDevErrTimeout);
                break;
            }
            sh = head_of(kin + base);
        }
        const uint64_t* src = PREFETCH ? s_stage : kin + base;
        // The sorted keys: key j at s_key[j + ho], so that the part written
        // back by a bulk copy starts on a 16-byte boundary.
        const uint32_t ho = PREFETCH ? head_of(kout + base) : 0u;
        uint64_t* sk = s_key + ho;
        // Items past the segment are skipped by a uniform break (n is the
        // same for the whole CTA), so a short segment costs no predicated work.
        uint64_t key[ITEMS];
        uint32_t hmin = ~0u, hmax = 0u;
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            if ((uint32_t)(i * THREADS) >= n) break;
            const uint32_t e = tid + i * THREADS;
            key[i] = e < n ? src[e + sh] ^ flip_in : 0ull;
            const uint32_t h = (uint32_t)(key[i] >> 32);
            if (e < n) { hmin = min(hmin, h); hmax = max(hmax, h); }
        }
        hmin = __reduce_min_sync(0xffffffffu, hmin);
        hmax = __reduce_max_sync(0xffffffffu, hmax);
        if (lane == 0) { s_warp[w] = hmin; s_warp[WARPS + w] = hmax; }
        for (int d = tid; d < R; d += THREADS) s_start[d] = 0;
        if (tid == 0) s_flag[0] = 0;
        __syncthreads();
        if (PREFETCH) prefetch(nxt);  // the staging buffer has been read
        hmin = ~0u; hmax = 0u;
#pragma unroll
        for (int i = 0; i < WARPS; ++i) { hmin = min(hmin, s_warp[i]); hmax = max(hmax, s_warp[WARPS + i]); }
        // Digit: the high 32 key bits interpolated onto R groups when they
        // spread over at least 8 R values (the common case, 32-bit work);
        // else the whole 64-bit key range.  Either is monotone in the key.
        const bool hi_mode = hmax - hmin >= 8u * (uint32_t)R;
        uint64_t kmin = 0, mult64 = 0;
        uint32_t mult32 = 0;
        if (hi_mode) {
            mult32 = interp_mult32(hmax - hmin, (uint32_t)R);
        } else {
            uint64_t lo = ~0ull, hi = 0ull;
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                if ((uint32_t)(i * THREADS) >= n) break;
                if (tid + i * THREADS < n) { lo = min(lo, key[i]); hi = max(hi, key[i]); }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lo = min(lo, (uint64_t)__shfl_xor_sync(0xffffffffu, lo, o));
                hi = max(hi, (uint64_t)__shfl_xor_sync(0xffffffffu, hi, o));
            }
            if (lane == 0) { s_red[w] = lo; s_red[32 + w] = hi; }
            __syncthreads();
            lo = ~0ull; hi = 0ull;
            for (int i = 0; i < WARPS; ++i) { lo = min(lo, s_red[i]); hi = max(hi, s_red[32 + i]); }
            if (lo == hi) {  // all keys equal
#pragma unroll
                for (int i = 0; i < ITEMS; ++i) {
                    if ((uint32_t)(i * THREADS) >= n) break;
                    const uint32_t e = tid + i * THREADS;
                    if (e < n) kout[base + e] = key[i] ^ flip_out;
                }
                __syncthreads();
                continue;
            }
            kmin = lo;
            mult64 = interp_mult(hi - lo, (uint32_t)R);
        }
        uint32_t dp[ITEMS];
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            if ((uint32_t)(i * THREADS) >= n) break;
            const uint32_t e = tid + i * THREADS;
            uint32_t d = (uint32_t)R;  // past the segment
            if (e < n) {
                if (hi_mode) {
                    d = min(__umulhi((uint32_t)(key[i] >> 32) - hmin, mult32), (uint32_t)R - 1);
                } else {
                    const uint64_t off = key[i] - kmin;
                    d = mult64 ? min((uint32_t)__umul64hi(off, mult64), (uint32_t)R - 1) : (uint32_t)off;
                }
            }
            if (d < (uint32_t)R) {
                dp[i] = d | (atomicAdd(&s_start[d], 1u) << kSlotShift);
            }
        }
        // The previous segment's bulk store has read s_key before the
        // scatter below overwrites it (ordered by the scan's barriers).
        if (PREFETCH && tid == 0) bulk_wait_read();
        __syncthreads();
        uint32_t mx = 0;
        for (int d = tid; d < R; d += THREADS) mx = max(mx, s_start[d]);
        mx = __reduce_max_sync(0xffffffffu, mx);
        scan_smem_inplace<THREADS, R>(s_start, s_warp);
        if (lane == 0) s_warp[w] = mx;
        if (tid == 0) s_start[R] = n;
        __syncthreads();
        mx = 0;
#pragma unroll
        for (int i = 0; i < WARPS; ++i) mx = max(mx, s_warp[i]);
        // scatter into group order
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            if ((uint32_t)(i * THREADS) >= n) break;
            const uint32_t e = tid + i * THREADS;
            if (e < n) sk[s_start[dp[i] & kDigitMask] + (dp[i] >> kSlotShift)] = key[i];
        }
        __syncthreads();
        if (mx >= (uint32_t)kTinyGroup) {
            // A large group is fine as it is if it holds a single value;
            // the few that hold distinct keys are sorted in place by the CTA
            // (a segment with more goes to the shared-memory kernel).
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                if ((uint32_t)(i * THREADS) >= n) break;
                if (tid + i * THREADS >= n) continue;
                const uint32_t d = dp[i] & kDigitMask;
                const uint32_t a = s_start[d];
                if (s_start[d + 1] - a >= (uint32_t)kTinyGroup && sk[a] != sk[a + ((dp[i] >> kSlotShift) & kSlotMask)])
                    s_mark[d] = 1u;
            }
            __syncthreads();
            for (int d = tid; d < R; d += THREADS) {
                if (s_mark[d]) {
                    s_mark[d] = 0;
                    const uint32_t q = atomicAdd(&s_flag[0], 1u);
                    if (q < (uint32_t)kKeysMixedMax) s_flag[1 + q] = (uint32_t)d;
                }
            }
            __syncthreads();
            uint32_t nmixed = s_flag[0];
            if (nmixed > (uint32_t)kKeysMixedMax) {  // uniform
                // Keys spread over many binary orders of magnitude (lognormal
                // ones, say) crowd the lowest groups of the linear digit: count
                // and scatter once more on the logarithmic digit (log_digit of
                // key - min, also monotone in the key), the keys re-read from
                // the input, which is untouched until this segment is written.
                const uint64_t* g = kin + base;
                uint64_t lo = ~0ull, hi = 0ull;
                for (uint32_t j = tid; j < n; j += THREADS) {
                    const uint64_t k = g[j] ^ flip_in;
                    lo = min(lo, k);
                    hi = max(hi, k);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    lo = min(lo, (uint64_t)__shfl_xor_sync(0xffffffffu, lo, o));
                    hi = max(hi, (uint64_t)__shfl_xor_sync(0xffffffffu, hi, o));
                }
                if (lane == 0) { s_red[w] = lo; s_red[32 + w] = hi; }
                for (int d = tid; d < R; d += THREADS) s_start[d] = 0;
                __syncthreads();
                lo = ~0ull;
                hi = 0ull;
                for (int i = 0; i < WARPS; ++i) { lo = min(lo, s_red[i]); hi = max(hi, s_red[32 + i]); }
                // the 32 binary orders of magnitude below the range's top
                const int e_lo = max(0, (63 - __clzll((long long)(hi - lo))) - 31);
#pragma unroll
                for (int i = 0; i < ITEMS; ++i) {
                    if ((uint32_t)(i * THREADS) >= n) break;
                    const uint32_t e = tid + i * THREADS;
                    if (e < n) {
                        const uint32_t d = log_digit<R>((g[e] ^ flip_in) - lo, e_lo);
                        dp[i] = d | (atomicAdd(&s_start[d], 1u) << kSlotShift);
                    }
                }
                __syncthreads();
                uint32_t m2 = 0;
                for (int d = tid; d < R; d += THREADS) m2 = max(m2, s_start[d]);
                m2 = __reduce_max_sync(0xffffffffu, m2);
                scan_smem_inplace<THREADS, R>(s_start, s_warp);
                if (lane == 0) s_warp[w] = m2;
                if (tid == 0) { s_start[R] = n; s_flag[0] = 0; }
                __syncthreads();
                mx = 0;
#pragma unroll
                for (int i = 0; i < WARPS; ++i) mx = max(mx, s_warp[i]);
#pragma unroll
                for (int i = 0; i < ITEMS; ++i) {
                    if ((uint32_t)(i * THREADS) >= n) break;
                    const uint32_t e = tid + i * THREADS;
                    if (e < n) sk[s_start[dp[i] & kDigitMask] + (dp[i] >> kSlotShift)] = g[e] ^ flip_in;
                }
                __syncthreads();
                if (mx >= (uint32_t)kTinyGroup) {
#pragma unroll
                    for (int i = 0; i < ITEMS; ++i) {
                        if ((uint32_t)(i * THREADS) >= n) break;
                        if (tid + i * THREADS >= n) continue;
                        const uint32_t d = dp[i] & kDigitMask;
                        const uint32_t a = s_start[d];
                        if (s_start[d + 1] - a >= (uint32_t)kTinyGroup &&
                            sk[a] != sk[a + ((dp[i] >> kSlotShift) & kSlotMask)])
                            s_mark[d] = 1u;
                    }
                    __syncthreads();
                    for (int d = tid; d < R; d += THREADS) {
                        if (s_mark[d]) {
                            s_mark[d] = 0;
                            const uint32_t q = atomicAdd(&s_flag[0], 1u);
                            if (q < (uint32_t)kKeysMixedMax) s_flag[1 + q] = (uint32_t)d;
                        }
                    }
                    __syncthreads();
                }
                nmixed = s_flag[0];
                if (nmixed > (uint32_t)kKeysMixedMax) {  // the log digit crowds too
                    if (tid == 0) slow_list[atomicAdd(slow_count, 1u)] = (uint32_t)s;
                    __syncthreads();
                    continue;
                }
            }
            for (uint32_t q = 0; q < nmixed; ++q) {
                const uint32_t d = s_flag[1 + q];
                const uint32_t a = s_start[d];
                cta_bitonic_sort<THREADS>(sk, a, s_start[d + 1] - a, [](uint32_t i) { return i; });
            }
        }
        if (mx > 1u) {
            // Every group of 2..kTinyGroup-1 keys is sorted in place by the
            // thread owning it (each thread owns G consecutive groups; the
            // groups hold a few keys, nearly in order); a large group holding
            // one value needs nothing.  The groups come in key order, so when
            // a thread's groups hold few keys in all, one insertion sort over
            // their whole range does it.
            constexpr int G = R / THREADS;
            const uint32_t ga = s_start[tid * G], gb = s_start[tid * G + G];
            if (gb - ga < (uint32_t)kTinyGroup) {
                for (uint32_t j = ga + 1; j < gb; ++j) {
                    const uint64_t x = sk[j];
                    uint32_t i = j;
                    while (i > ga) {
                        const uint64_t y = sk[i - 1];
                        if (y <= x) break;
                        sk[i] = y;
                        --i;
                    }
                    sk[i] = x;
                }
            } else {
                for (int g = tid * G; g < tid * G + G; ++g) {
                    const uint32_t a = s_start[g], b = s_start[g + 1];
                    if (b - a < 2u || b - a >= (uint32_t)kTinyGroup) continue;
                    for (uint32_t j = a + 1; j < b; ++j) {
                        const uint64_t x = sk[j];
                        uint32_t i = j;
                        while (i > a) {
                            const uint64_t y = sk[i - 1];
                            if (y <= x) break;
                            sk[i] = y;
                            --i;
                        }
                        sk[i] = x;
                    }
                }
            }
            __syncthreads();
        }
        uint64_t* dst = kout + base;
        if (PREFETCH) {
            if (flip_out) {  // uniform: signed keys back from order-preserving bits
                for (uint32_t j = tid; j < n; j += THREADS) sk[j] ^= flip_out;
                __syncthreads();
            }
            // One bulk copy writes the 16-byte aligned middle; the first and
            // last key go by plain stores when they fall outside it.
            const uint32_t m = ((n - ho) >> 1) << 1;
            if (ho && tid == 1) dst[0] = sk[0];
            if (ho + m < n && tid == 2) dst[n - 1] = sk[n - 1];
            fence_async_smem();
            __syncthreads();
            if (tid == 0 && m) bulk_store(dst + ho, s_key + 2 * ho, m * 8u);
        } else {
            for (uint32_t j = tid; j < n; j += THREADS) dst[j] = sk[j] ^ flip_out;
            __syncthreads();
        }
    }
    if (PREFETCH) {
        cp_async_wait_all();
        if (tid == 0) bulk_wait_all();
    }
}

// ---------------------------------------------------------------------------
// Stable LSD sort on chip of the segments in the fallback list (at most
// kSmallCap keys each): 8-bit digit passes over a 16-bit index permutation,
// skipping digits that are constant over the segment.
// ---------------------------------------------------------------------------
template <int THREADS, int ITEMS>
constexpr size_t lsd_sort_smem() {
    return (size_t)THREADS * ITEMS * 8 + 2 * (size_t)THREADS * ITEMS * 2 + (size_t)(THREADS / 32) * kRadix * 4 +
           2 * kRadix * 4 + 32 * 4 + 2 * 32 * 8;
}

template <bool PAY, int THREADS, int ITEMS>
__global__ __launch_bounds__(THREADS, 1) void k_small_lsd(
    const uint64_t* kin, uint64_t* kout, const uint32_t* pin, uint32_t* pout, const uint64_t* __restrict__ seg_lo,
    const uint64_t* __restrict__ seg_hi, const uint32_t* __restrict__ list, const uint32_t* __restrict__ nlist,
    uint64_t flip_in, uint64_t flip_out) {
    constexpr int WARPS = THREADS / 32;
    constexpr int CAP = THREADS * ITEMS;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* s_keys = (uint64_t*)smem;                        // CAP u64
    uint16_t* s_idx0 = (uint16_t*)(s_keys + CAP);              // CAP u16
    uint16_t* s_idx1 = s_idx0 + CAP;                           // CAP u16
    uint32_t* s_cnt = (uint32_t*)(s_idx1 + CAP);               // WARPS*256
    uint32_t* s_total = s_cnt + WARPS * kRadix;                // 256
    uint32_t* s_start = s_total + kRadix;                      // 256
    uint32_t* s_warp = s_start + kRadix;                       // 32
    uint64_t* s_red = (uint64_t*)(s_warp + 32);                // 2*32

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint64_t count = *nlist;
    const uint32_t wbase = w * 32 * ITEMS + lane;
    const uint32_t wfirst = (uint32_t)w * 32 * ITEMS;
    for (uint64_t k = blockIdx.x; k < count; k += gridDim.x) {
        const uint64_t s = list[k];
        const uint64_t base = seg_lo[s];
        const uint64_t n64 = seg_hi[s] - base;
        if (n64 == 0 || n64 > (uint64_t)CAP) continue;
        const uint32_t n = (uint32_t)n64;
        uint64_t vor = 0, vand = ~0ull;
        for (uint32_t j = tid; j < n; j += THREADS) {
            const uint64_t key = kin[base + j] ^ flip_in;
            s_keys[j] = key;
            s_idx0[j] = (uint16_t)j;
            vor |= key;
            vand &= key;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vor |= __shfl_xor_sync(0xffffffffu, vor, o);
            vand &= __shfl_xor_sync(0xffffffffu, vand, o);
        }
        if (lane == 0) { s_red[w] = vor; s_red[32 + w] = vand; }
        __syncthreads();
        uint64_t vary;
        {
            uint64_t a = 0, b = ~0ull;
            for (int i = 0; i < WARPS; ++i) { a |= s_red[i]; b &= s_red[32 + i]; }
            vary = a ^ b;
        }
        uint16_t* cur = s_idx0;
        uint16_t* nxt = s_idx1;
        for (int pass = 0; pass < 8; ++pass) {
            const int shift = 8 * pass;
            if (((vary >> shift) & 255u) == 0u) continue;  // digit constant: identity pass
            uint32_t idx[ITEMS], rank[ITEMS];
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) idx[i] = (wbase + i * 32 < n) ? cur[wbase + i * 32] : 0u;
            auto digit_of = [&](int i) -> uint32_t {
                return (wbase + i * 32 < n) ? ((uint32_t)(s_keys[idx[i]] >> shift) & 255u) : (uint32_t)kRadix;
            };
            block_rank<WARPS, ITEMS>(digit_of, n, rank, s_cnt, s_total, s_start, s_warp, NoOp());
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                if (wfirst + i * 32 >= n) break;
                if (wbase + i * 32 < n && rank[i] < n) nxt[rank[i]] = (uint16_t)idx[i];
            }
            __syncthreads();
            uint16_t* t = cur; cur = nxt; nxt = t;
        }
        write_sorted<PAY, THREADS, CAP>(kout, pout, pin, base, n, s_keys, cur, flip_out);
    }
}

// ---------------------------------------------------------------------------
// Planning of one level, as a three-step scan over chunks of 1024 segments:
// compact lists of the segments of each on-chip size class, compact ids and
// tiles of the segments above the on-chip capacity.
// counters[16..18] = class sizes, [19] = #large, [20] = #tiles,
// [22..23] = keys in large segments.
// ---------------------------------------------------------------------------
struct PlanV {
    uint32_t c[5];  // classes 0..2, large, tiles
    unsigned long long keys;
};

// chip_max: the largest segment sorted on chip at this level (kSmallCap, or
// kC1Cap to split larger ones again instead of the largest on-chip class).
__device__ __forceinline__ PlanV plan_item(const uint64_t* seg_lo, const uint64_t* seg_hi, uint64_t nseg, uint64_t s,
                                           uint32_t chip_max) {
    PlanV v = {{0, 0, 0, 0, 0}, 0ull};
    if (s < nseg) {
        const uint64_t n = seg_hi[s] - seg_lo[s];
        if (n == 0) {
        } else if (n <= (uint64_t)kC0Cap) {
            v.c[0] = 1;
        } else if (n <= (uint64_t)kC1Cap) {
            v.c[1] = 1;
        } else if (n <= (uint64_t)chip_max) {
            v.c[2] = 1;
        } else if (n >= kMaxSegKeys) {
            // too large for the split's 30-bit counts: left unsorted, reported by k_plan_write
        } else {
            v.c[3] = 1;
            v.c[4] = (uint32_t)ceil_div(n, kOsTile);
            v.keys = n;
        }
    }
    return v;
}

// Inclusive scan of PlanV over the CTA; returns the totals in tot.
__device__ __forceinline__ void plan_scan(PlanV& v, PlanV& tot) {
    __shared__ uint32_t s_c[5][32];
    __shared__ unsigned long long s_k[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, v.c[i], o);
            if (lane >= o) v.c[i] += y;
        }
        const unsigned long long yk = __shfl_up_sync(0xffffffffu, v.keys, o);
        if (lane >= o) v.keys += yk;
    }
    if (lane == 31) {
#pragma unroll
        for (int i = 0; i < 5; ++i) s_c[i][w] = v.c[i];
        s_k[w] = v.keys;
    }
    __syncthreads();
    tot = PlanV{{0, 0, 0, 0, 0}, 0ull};
    for (int j = 0; j < nw; ++j) {
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            if (j < w) v.c[i] += s_c[i][j];
            tot.c[i] += s_c[i][j];
        }
        if (j < w) v.keys += s_k[j];
        tot.keys += s_k[j];
    }
    __syncthreads();
}

__device__ __forceinline__ void blk_store(uint32_t* blk, uint32_t i, const PlanV& v) {
    uint32_t* b = blk + 8 * (uint64_t)i;
#pragma unroll
    for (int k = 0; k < 5; ++k) b[k] = v.c[k];
    *(unsigned long long*)(b + 6) = v.keys;
}
__device__ __forceinline__ PlanV blk_load(const uint32_t* blk, uint32_t i) {
    const uint32_t* b = blk + 8 * (uint64_t)i;
    PlanV v;
#pragma unroll
    for (int k = 0; k < 5; ++k) v.c[k] = b[k];
    v.keys = *(const unsigned long long*)(b + 6);
    return v;
}

__global__ __launch_bounds__(1024) void k_plan_count(const uint64_t* __restrict__ seg_lo, const uint64_t* __restrict__ seg_hi,
                                                     uint64_t nseg, uint32_t* __restrict__ blk, uint32_t chip_max) {
    PlanV v = plan_item(seg_lo, seg_hi, nseg, (uint64_t)blockIdx.x * 1024 + threadIdx.x, chip_max), tot;
    plan_scan(v, tot);
    if (threadIdx.x == 0) blk_store(blk, blockIdx.x, tot);
}

// Exclusive scan of the chunk totals (one CTA), totals into counters.
__global__ __launch_bounds__(1024) void k_plan_scan(uint32_t nblk, uint32_t* __restrict__ blk, uint32_t* __restrict__ counters,
                                                    volatile uint32_t* host_counts) {
    PlanV carry = {{0, 0, 0, 0, 0}, 0ull};
    for (uint32_t base = 0; base < nblk; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        PlanV v = i < nblk ? blk_load(blk, i) : PlanV{{0, 0, 0, 0, 0}, 0ull};
        const PlanV v0 = v;
        PlanV tot;
        plan_scan(v, tot);
        if (i < nblk) {
            PlanV ex;
#pragma unroll
            for (int k = 0; k < 5; ++k) ex.c[k] = carry.c[k] + v.c[k] - v0.c[k];
            ex.keys = carry.keys + v.keys - v0.keys;
            blk_store(blk, i, ex);
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) carry.c[k] += tot.c[k];
        carry.keys += tot.keys;
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < 5; ++k) counters[16 + k] = carry.c[k];
        *(unsigned long long*)(counters + 22) = carry.keys;
        if (host_counts) {  // the same eight words for the host, in mapped pinned memory
            for (int k = 0; k < 5; ++k) host_counts[k] = carry.c[k];
            host_counts[5] = 0;
            host_counts[6] = (uint32_t)carry.keys;
            host_counts[7] = (uint32_t)(carry.keys >> 32);
        }
        counters[24] = 0;  // fallback list of this level's on-chip sorts
        counters[25] = 0;  // segments the register kernels leave to the shared-memory kernel
        counters[26] = 0;  // ... and the keys-only kernels, per size class
        counters[27] = 0;
        counters[28] = 0;
    }
}

__global__ __launch_bounds__(1024) void k_plan_write(const uint64_t* __restrict__ seg_lo, const uint64_t* __restrict__ seg_hi,
                                                     uint64_t nseg, const uint32_t* __restrict__ blk,
                                                     const uint32_t* __restrict__ counters, uint32_t* __restrict__ tile_start,
                                                     uint32_t* __restrict__ large_id, uint32_t* __restrict__ large_seg,
                                                     uint32_t* __restrict__ list0, uint32_t* __restrict__ list1,
                                                     uint32_t* __restrict__ list2, uint32_t* __restrict__ err,
                                                     uint32_t* __restrict__ tile_seg, uint32_t chip_max) {
    const uint64_t s = (uint64_t)blockIdx.x * 1024 + threadIdx.x;
    const PlanV item = plan_item(seg_lo, seg_hi, nseg, s, chip_max);
    if (s < nseg && seg_hi[s] - seg_lo[s] >= kMaxSegKeys) atomicOr(err, kDevErrSize);
    PlanV v = item, tot;
    plan_scan(v, tot);
    const PlanV off = blk_load(blk, blockIdx.x);
    if (s < nseg) {
        tile_start[s] = off.c[4] + v.c[4] - item.c[4];
        large_id[s] = 0xffffffffu;
        if (item.c[0]) list0[off.c[0] + v.c[0] - 1] = (uint32_t)s;
        if (item.c[1]) list1[off.c[1] + v.c[1] - 1] = (uint32_t)s;
        if (item.c[2]) list2[off.c[2] + v.c[2] - 1] = (uint32_t)s;
        if (item.c[3]) {
            const uint32_t id = off.c[3] + v.c[3] - 1;
            large_id[s] = id;
            large_seg[id] = (uint32_t)s;
            const uint32_t t0 = off.c[4] + v.c[4] - item.c[4];
            for (uint32_t u = 0; u < item.c[4]; ++u) tile_seg[t0 + u] = (uint32_t)s;
        }
    }
    if (s == nseg) tile_start[nseg] = counters[20];
}

// ---------------------------------------------------------------------------
// Statistics of the large segments, per tile of kOsTile keys: the digit
// histogram of the tile (on a speculative window, or on the interpolating
// hint) and the OR/AND of the segment's keys, in one read.  One CTA per tile.
// From these the split pass gets every tile's destination offsets by a scan
// (k_msd_prep) instead of a look-back across the tiles of its segment.
// ---------------------------------------------------------------------------
// msd_shift flag: the split interpolated the key range (no byte is fixed in
// its sub-buckets).
constexpr uint32_t kShiftInterp = 0x100u;
// msd_shift flag: the split's digit is the bucket among 255 sampled splitters.
constexpr uint32_t kShiftSplit = 0x200u;

// Bucket of key k among the 255 sorted splitters spl[0..254]: the number of
// splitters <= k (0..255), by eight halvings without branches.  Monotone in
// the key, so it serves as a digit of the split.
__device__ __forceinline__ uint32_t splitter_digit(const uint64_t* spl, uint64_t k) {
    uint32_t i = 0;
#pragma unroll
    for (uint32_t step = 128; step > 0; step >>= 1)
        if (spl[i + step - 1] <= k) i += step;
    return i;
}

// Splitters of the first split of a segment with skewed keys (Gaussian
// clusters, heavy duplicates), where the top varying byte would leave most of
// the segment in a few buckets and cost another level: one CTA per segment
// split at this level draws 2048 keys at evenly spaced positions; when the
// busiest value of the sample's top varying byte holds more than 4x its
// share (32 of 2048), it sorts the sample and keeps every 8th key as the 255
// splitters (spl_mode 1), else the byte split stays (spl_mode 0).
constexpr int kSplSample = 2048;
__global__ __launch_bounds__(256) void k_seg_sample(const uint64_t* __restrict__ kin, const uint64_t* __restrict__ seg_lo,
                                                    const uint64_t* __restrict__ seg_hi,
                                                    const uint32_t* __restrict__ large_seg,
                                                    const uint32_t* __restrict__ counters, uint64_t flip_in,
                                                    uint64_t* __restrict__ spl_tab, uint8_t* __restrict__ spl_mode) {
    __shared__ uint64_t s_k[kSplSample];
    __shared__ uint32_t s_h[kRadix];
    __shared__ unsigned long long s_or[8], s_and[8];
    const uint32_t id = blockIdx.x;
    if (id >= counters[19]) return;  // uniform
    const uint32_t s = large_seg[id];
    const uint64_t lo = seg_lo[s], n = seg_hi[s] - lo;
    const int tid = threadIdx.x;
    s_h[tid] = 0;
    unsigned long long o = 0, an = ~0ull;
    for (int i = tid; i < kSplSample; i += 256) {
        const uint64_t pos = (uint64_t)(((unsigned __int128)(2 * i + 1) * n) / (2 * kSplSample));
        const uint64_t k = kin[lo + pos] ^ flip_in;
        s_k[i] = k;
        o |= k;
        an &= k;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        o |= __shfl_xor_sync(0xffffffffu, o, off);
        an &= __shfl_xor_sync(0xffffffffu, an, off);
    }
    if ((tid & 31) == 0) { s_or[tid >> 5] = o; s_and[tid >> 5] = an; }
    __syncthreads();
    unsigned long long vo = 0, va = ~0ull;
    for (int i = 0; i < 8; ++i) { vo |= s_or[i]; va &= s_and[i]; }
    const unsigned long long vary = vo ^ va;
    if (vary == 0ull) {  // uniform: a single value in the sample
        if (tid == 0) spl_mode[id] = 0u;
        return;
    }
    const int sh = 8 * (int)((uint32_t)(63 - __clzll((long long)vary)) >> 3);
    for (int i = tid; i < kSplSample; i += 256) atomicAdd(&s_h[(uint32_t)(s_k[i] >> sh) & 255u], 1u);
    __syncthreads();
    const int crowded = __syncthreads_or(s_h[tid] > 4u * (kSplSample / kRadix));
    if (!crowded) {
        if (tid == 0) spl_mode[id] = 0u;
        return;
    }
    cta_bitonic_sort<256>(s_k, 0u, (uint32_t)kSplSample, [](uint32_t i) { return i; });
    uint64_t* spl = spl_tab + (uint64_t)id * kRadix;
    for (int i = tid; i < kRadix - 1; i += 256) spl[i] = s_k[(i + 1) * (kSplSample / kRadix) - 1];
    if (tid == 0) {
        spl[kRadix - 1] = ~0ull;
        spl_mode[id] = 1u;
    }
}

__device__ __forceinline__ int spec_window(const uint32_t* __restrict__ prev_shift, uint32_t s) {
    // the byte below the parent split's window (a sub-bucket's keys agree on
    // that window and above); the top byte at the first level
    if (!prev_shift) return 7;
    const uint32_t ps = prev_shift[s >> 8];
    return (ps & (kShiftInterp | kShiftSplit)) ? 7 : (ps >= 8 ? (int)(ps >> 3) - 1 : 0);
}

// A tile is skewed when one digit holds more than an eighth of it: the
// split then gives the lanes of a warp that share lane 0's digit their slots
// with one atomic (sorted runs of equal keys hit one counter otherwise).
// Called by all 256 threads with their digit's count.
__device__ __forceinline__ void tile_skew_flag(uint32_t count, uint8_t* __restrict__ tile_skew, uint32_t t) {
    const bool big = count > (uint32_t)(kOsTile / 8);
    const int any = __syncthreads_or(big);
    if (threadIdx.x == 0) tile_skew[t] = any ? 1u : 0u;
}

template <bool SPL>
__global__ __launch_bounds__(256) void k_tile_stats(const uint64_t* __restrict__ kin, const uint64_t* __restrict__ seg_lo,
                                                    const uint64_t* __restrict__ seg_hi, uint64_t nseg,
                                                    const uint32_t* __restrict__ tile_start,
                                                    const uint32_t* __restrict__ tile_seg,
                                                    const uint32_t* __restrict__ large_id, uint16_t* __restrict__ tile_hist,
                                                    uint8_t* __restrict__ tile_skew,
                                                    unsigned long long* __restrict__ vor, unsigned long long* __restrict__ vand,
                                                    const uint64_t* __restrict__ hint_lo, const uint64_t* __restrict__ hint_mult,
                                                    const uint64_t* __restrict__ hint_hi,
                                                    const uint32_t* __restrict__ prev_shift, uint32_t* __restrict__ spec_out,
                                                    uint64_t flip_in, const uint64_t* __restrict__ spl_tab,
                                                    const uint8_t* __restrict__ spl_mode) {
    __shared__ uint32_t s_h[kRadix];
    __shared__ unsigned long long s_or[8], s_and[8];
    __shared__ uint64_t s_spl[kRadix];
    const uint32_t t = blockIdx.x;
    if (t >= tile_start[nseg]) return;  // uniform
    s_h[threadIdx.x] = 0;
    const uint32_t s = tile_seg[t], id = large_id[s];
    const bool bysplit = SPL && spl_mode[id];  // uniform per CTA
    if (bysplit) s_spl[threadIdx.x] = spl_tab[(uint64_t)id * kRadix + threadIdx.x];
    __syncthreads();
    const uint64_t lo = seg_lo[s], n = seg_hi[s] - lo;
    const uint32_t ti = t - tile_start[s];
    const uint64_t a = (uint64_t)ti * kOsTile, b = min(n, a + kOsTile);
    const bool win = hint_lo != nullptr;
    const int spec = spec_window(prev_shift, s);
    if (ti == 0 && threadIdx.x == 0) spec_out[id] = (uint32_t)spec;
    if (win && hint_hi && hint_hi[s] == hint_lo[s]) {
        // every key of the segment equals the one the parent's split saw: no read
        if (threadIdx.x == 0) {
            atomicOr(&vor[id], (unsigned long long)hint_lo[s]);
            atomicAnd(&vand[id], (unsigned long long)hint_lo[s]);
        }
        tile_hist[(uint64_t)t * (2 * kRadix) + threadIdx.x] = (uint16_t)(threadIdx.x == 0 ? b - a : 0);
        if (threadIdx.x == 0) tile_skew[t] = 1u;
        return;
    }
    const uint64_t hb = win ? hint_lo[s] : 0ull;
    const uint64_t hm = win ? hint_mult[s] : 0ull;
    const int sh = 8 * spec;
    unsigned long long o = 0, an = ~0ull;
#pragma unroll 4
    for (uint64_t e = a + threadIdx.x; e < b; e += 256) {
        const uint64_t k = kin[lo + e] ^ flip_in;
        o |= k;
        an &= k;
        const uint32_t d =
            bysplit ? splitter_digit(s_spl, k) : (win ? split_digit(k, 0, hb, hm) : (uint32_t)(k >> sh) & 255u);
        atomicAdd(&s_h[d], 1u);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        o |= __shfl_xor_sync(0xffffffffu, o, off);
        an &= __shfl_xor_sync(0xffffffffu, an, off);
    }
    if ((threadIdx.x & 31) == 0) { s_or[threadIdx.x >> 5] = o; s_and[threadIdx.x >> 5] = an; }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long x = 0, y = ~0ull;
        for (int i = 0; i < 8; ++i) { x |= s_or[i]; y &= s_and[i]; }
        atomicOr(&vor[id], x);
        atomicAnd(&vand[id], y);
    }
    tile_hist[(uint64_t)t * (2 * kRadix) + threadIdx.x] = (uint16_t)s_h[threadIdx.x];
    tile_skew_flag(s_h[threadIdx.x], tile_skew, t);
}

// Recount of the tiles of segments whose top varying byte (from the OR/AND of
// the statistics pass) is not the speculative one: the histogram of that byte
// into the tile's second row.  Other CTAs return at once.
__global__ __launch_bounds__(256) void k_tile_recount(const uint64_t* __restrict__ kin, const uint64_t* __restrict__ seg_lo,
                                                      const uint64_t* __restrict__ seg_hi, uint64_t nseg,
                                                      const uint32_t* __restrict__ tile_start,
                                                      const uint32_t* __restrict__ tile_seg,
                                                      const uint32_t* __restrict__ large_id, uint16_t* __restrict__ tile_hist,
                                                      uint8_t* __restrict__ tile_skew, const uint8_t* __restrict__ spl_mode,
                                                      const unsigned long long* __restrict__ vor,
                                                      const unsigned long long* __restrict__ vand,
                                                      const uint32_t* __restrict__ spec, uint64_t flip_in) {
    // A grid of a few CTAs per SM walks the tiles: most levels recount few
    // or none, and a CTA per tile would cost a launch of tens of thousands of
    // CTAs that all return at once.
    __shared__ uint32_t s_h[kRadix];
    const uint32_t total = tile_start[nseg];
    for (uint32_t t = blockIdx.x; t < total; t += gridDim.x) {  // uniform per CTA
        const uint32_t s = tile_seg[t], id = large_id[s];
        if (spl_mode && spl_mode[id]) continue;  // the statistics pass counted the splitter buckets
        const unsigned long long vary = vor[id] ^ vand[id];
        if (vary == 0ull) continue;
        const uint32_t w = (uint32_t)(63 - __clzll((long long)vary)) >> 3;
        if (w == spec[id]) continue;
        s_h[threadIdx.x] = 0;
        __syncthreads();
        const uint64_t lo = seg_lo[s], n = seg_hi[s] - lo;
        const uint64_t a = (uint64_t)(t - tile_start[s]) * kOsTile, b = min(n, a + kOsTile);
        const int sh = 8 * (int)w;
#pragma unroll 4
        for (uint64_t e = a + threadIdx.x; e < b; e += 256)
            atomicAdd(&s_h[(uint32_t)((kin[lo + e] ^ flip_in) >> sh) & 255u], 1u);
        __syncthreads();
        tile_hist[(uint64_t)t * (2 * kRadix) + kRadix + threadIdx.x] = (uint16_t)s_h[threadIdx.x];
        tile_skew_flag(s_h[threadIdx.x], tile_skew, t);  // ends with a barrier
    }
}

// Per large segment (thread d = digit d): the split window, the digit totals
// (summed over the segment's tile histograms), their exclusive offsets, the
// bounds of the 256 sub-buckets (empty when the keys are all equal), and the
// destination of every tile's digit-d keys: the digit's offset plus the
// digit-d keys of the segment's earlier tiles.
__global__ __launch_bounds__(256) void k_msd_prep(const uint64_t* __restrict__ seg_lo, const uint32_t* __restrict__ large_seg,
                                                  const uint32_t* __restrict__ counters,
                                                  const uint32_t* __restrict__ tile_start,
                                                  const uint16_t* __restrict__ tile_hist,
                                                  const unsigned long long* __restrict__ vor,
                                                  const unsigned long long* __restrict__ vand, const uint64_t* __restrict__ hint_lo,
                                                  const uint64_t* __restrict__ hint_mult, uint64_t* __restrict__ msd_base,
                                                  uint64_t* __restrict__ msd_mult, uint32_t* __restrict__ msd_shift,
                                                  const uint32_t* __restrict__ spec, uint32_t* __restrict__ direct,
                                                  uint64_t* __restrict__ sub_lo, uint64_t* __restrict__ sub_hi,
                                                  uint32_t* __restrict__ tile_off, uint32_t chip_max,
                                                  uint32_t* __restrict__ large_mask, uint32_t* __restrict__ any_large,
                                                  uint64_t* __restrict__ cmin, uint64_t* __restrict__ cmax,
                                                  uint32_t level_chip_max, uint32_t pack_keys,
                                                  const uint8_t* __restrict__ spl_mode) {
    __shared__ uint32_t s_c[kRadix], s_x[kRadix + 1], s_warp[32], s_end[kRadix];
    __shared__ uint16_t s_jump[8][kRadix + 1];  // packing: 2^i packs ahead of each sub-bucket
    __shared__ uint32_t s_big[8];               // packing: sub-buckets split again, one bit each
    __shared__ uint8_t s_first[kRadix];         // packing: the sub-bucket starts a pack
    const uint32_t id = blockIdx.x;
    if (id >= counters[19]) return;
    const uint32_t s = large_seg[id];
    const uint64_t lo = seg_lo[s];
    const unsigned long long vary = vor[id] ^ vand[id];
    uint32_t shift = 0, row;
    uint64_t base = 0, mult = 0;
    if (hint_lo) {
        base = hint_lo[s];
        mult = hint_mult[s];
        row = 0;
    } else {
        const uint32_t w = vary ? (uint32_t)(63 - __clzll((long long)vary)) >> 3 : spec[id];
        shift = 8 * w;
        row = w == spec[id] ? 0u : 1u;
    }
    const bool bysplit = spl_mode && spl_mode[id];
    if (bysplit) row = 0;
    const bool dir = vary == 0ull;
    const uint32_t d = threadIdx.x;
    const uint32_t t0 = tile_start[s], t1 = tile_start[s + 1];
    const uint16_t* h = tile_hist + row * kRadix + d;
    uint32_t total = 0;
    for (uint32_t t = t0; t < t1; ++t) total += h[(uint64_t)t * (2 * kRadix)];
    s_c[d] = total;
    __syncthreads();
    scan256_smem<256>(s_c, s_x, s_warp);
    const uint32_t x = s_x[d];
    // Packing: runs of consecutive sub-buckets sorted on chip (each at most
    // level_chip_max keys) are merged greedily into packs of at most
    // pack_keys keys; the keys of consecutive sub-buckets are in order
    // between them, so the next level sorting a pack as one segment sorts
    // each.  s_end[d]: end offset of the pack that starts at sub-bucket d,
    // or ~0 when d belongs to an earlier pack (it becomes empty).  Sub-buckets
    // split again stand alone.
    // Nothing to pack unless two neighbouring sub-buckets fit one pack
    // (uniform keys: none do, and the serial walk below is skipped).
    const bool pair_fits = d + 1 < (uint32_t)kRadix && total + s_c[d + 1] <= pack_keys && total + s_c[d + 1] > 0u;
    const bool packable = __syncthreads_or(pair_fits) != 0;
    if (packable) {  // uniform per CTA
        // The greedy walk over the sub-buckets in order (a sub-bucket split
        // again stands alone; otherwise a pack takes sub-buckets while they
        // add up to at most pack_keys), computed in parallel: next[d], the
        // sub-bucket after the pack that would start at d, by a bit search
        // and a binary search; the packs reachable from sub-bucket 0 by
        // pointer doubling (thread m finds the m-th pack's start).
        const bool big = total > level_chip_max;
        const uint32_t bal = __ballot_sync(0xffffffffu, big);
        if ((d & 31) == 0) s_big[d >> 5] = bal;
        if (d == 0) s_x[kRadix] = s_x[kRadix - 1] + s_c[kRadix - 1];
        __syncthreads();
        uint32_t nxt;
        if (big) {
            nxt = d + 1;
        } else {
            uint32_t fb = kRadix;  // the first sub-bucket after d split again
            for (uint32_t wd = (d + 1) >> 5; wd < 8; ++wd) {
                const uint32_t m = s_big[wd] & (wd == ((d + 1) >> 5) ? ~0u << ((d + 1) & 31) : ~0u);
                if ((d + 1) < (uint32_t)kRadix && m) { fb = wd * 32 + (uint32_t)(__ffs(m) - 1); break; }
            }
            // the first j > d whose keys would take the pack past pack_keys:
            // the first m >= d + 2 with s_x[m] > s_x[d] + pack_keys, j = m - 1
            const uint32_t lim = x + pack_keys;
            uint32_t lo = d + 2, hi = kRadix + 1;  // search m in [lo, hi)
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (s_x[mid] > lim) hi = mid; else lo = mid + 1;
            }
            const uint32_t fs = lo <= (uint32_t)kRadix ? lo - 1 : (uint32_t)kRadix;
            nxt = min(fb, fs);
        }
        s_jump[0][d] = (uint16_t)nxt;
        if (d == 0) s_jump[0][kRadix] = (uint16_t)kRadix;
        s_first[d] = 0;
        __syncthreads();
        for (int i = 1; i < 8; ++i) {
            const uint32_t a = s_jump[i - 1][d];
            s_jump[i][d] = a < (uint32_t)kRadix ? s_jump[i - 1][a] : (uint16_t)kRadix;
            if (d == 0) s_jump[i][kRadix] = (uint16_t)kRadix;
            __syncthreads();
        }
        uint32_t pos = 0;  // start of pack number d
        for (int i = 0; i < 8 && pos < (uint32_t)kRadix; ++i)
            if ((d >> i) & 1u) pos = s_jump[i][pos];
        if (pos < (uint32_t)kRadix) s_first[pos] = 1;
        __syncthreads();
        s_end[d] = s_first[d] ? s_x[nxt] : ~0u;
    }
    if (!packable) s_end[d] = x + total;
    __syncthreads();
    const uint32_t pend = s_end[d];
    sub_lo[(uint64_t)id * kRadix + d] = dir ? lo : lo + x;
    sub_hi[(uint64_t)id * kRadix + d] = dir ? lo : lo + (pend == ~0u ? x : pend);
    // sub-buckets that the next level splits again: the split pass gathers
    // their smallest and largest key
    const bool large = !dir && total > chip_max;  // chip_max = ~0: nothing gathered
    const uint32_t bal = __ballot_sync(0xffffffffu, large);
    if ((d & 31) == 0) large_mask[(uint64_t)id * 8 + (d >> 5)] = bal;
    if (d == 0) any_large[id] = 0u;
    cmin[(uint64_t)id * kRadix + d] = ~0ull;
    cmax[(uint64_t)id * kRadix + d] = 0ull;
    __syncthreads();
    if (bal && (d & 31) == 0) atomicOr(&any_large[id], 1u);
    uint32_t run = x;
    for (uint32_t t = t0; t < t1; ++t) {
        tile_off[(uint64_t)t * kRadix + d] = run;
        run += h[(uint64_t)t * (2 * kRadix)];
    }
    if (d == 0) {
        msd_shift[id] = shift | (hint_lo ? kShiftInterp : 0u) | (bysplit ? kShiftSplit : 0u);
        msd_base[id] = base;
        msd_mult[id] = mult;
        direct[id] = dir ? 1u : 0u;
    }
}

// ---------------------------------------------------------------------------
// The split pass: stable scatter of every large segment on its window, one
// CTA per tile of every large segment, each tile to the offsets k_msd_prep
// assigned it.
// ---------------------------------------------------------------------------
struct SplitArgs {
    const uint64_t* kin;
    uint64_t* kout;      // next level
    uint64_t* kfinal;    // output (segments whose keys are all equal)
    const uint32_t* pin;
    uint32_t* pout;
    uint32_t* pfinal;
    const uint64_t* seg_lo;
    const uint64_t* seg_hi;
    uint64_t nseg;
    const uint32_t* tile_start;
    const uint32_t* tile_seg;
    const uint32_t* large_id;
    const uint32_t* tile_off;  // [tile][256] destination of the tile's digit-d keys, relative to the segment
    const uint8_t* tile_skew;  // [tile] one digit holds more than an eighth of the tile
    const uint64_t* spl_tab;   // [large id][256] sampled splitters (segments split with kShiftSplit)
    const uint32_t* msd_shift;
    const uint64_t* msd_base;
    const uint64_t* msd_mult;
    const uint32_t* direct;
    const uint32_t* large_mask;  // [large id][8] sub-buckets that the next level splits again
    const uint32_t* any_large;
    uint64_t* cmin;              // their smallest and largest key (atomics)
    uint64_t* cmax;
    uint32_t* err;
    uint64_t flip_in;
    uint64_t flip_out;
    uint32_t scatter;  // 1: tiles that gather no key ranges write each key straight to its run
};

// The tile's shape: keys alone 256 threads x 16 keys (four CTAs per SM);
// with a payload 512 threads x 8 (two per SM), whose stable ranking then
// fits 64 registers without spilling.
template <bool PAY>
constexpr int split_threads() { return PAY ? 512 : 256; }

template <bool PAY, bool SPL>
__global__ __launch_bounds__(split_threads<PAY>(), PAY ? 2 : 4) void k_split(const SplitArgs A) {
    constexpr int kThreads = split_threads<PAY>();
    constexpr int kWarps = kThreads / 32;
    constexpr int kItems = kOsTile / kThreads;
    extern __shared__ __align__(16) unsigned char os_smem[];
    uint64_t* s_keys = (uint64_t*)os_smem;             // kOsTile keys
    uint32_t* s_pay = (uint32_t*)(s_keys + kOsTile);   // kOsTile payloads (PAY)
    uint8_t* s_dg = (uint8_t*)(s_pay + (PAY ? kOsTile : 0));  // kOsTile digits of the staged keys
    __shared__ uint32_t s_hist[PAY ? kWarps * kRadix : 1];
    __shared__ uint32_t s_total[kRadix], s_start[kRadix];
    __shared__ uint64_t s_gbase[kRadix];
    __shared__ uint32_t s_warp[32];
    __shared__ uint64_t s_mn[kRadix], s_mx[kRadix];
    __shared__ uint64_t s_spl[kRadix];
    __shared__ uint32_t s_mask[8];

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t total_tiles = A.tile_start[A.nseg];
    const uint32_t t = blockIdx.x;
    if (t >= total_tiles) return;  // uniform
    const uint32_t s = A.tile_seg[t];
    const uint32_t id = A.large_id[s];
    const uint64_t seg_base = A.seg_lo[s];
    const uint64_t seg_n = A.seg_hi[s] - seg_base;
    const uint32_t ti = t - A.tile_start[s];
    const uint64_t tile_lo = (uint64_t)ti * kOsTile;
    const uint32_t count = (uint32_t)min((uint64_t)kOsTile, seg_n - tile_lo);
    const int shift = (int)(A.msd_shift[id] & 0xffu);
    const uint64_t dbase = A.msd_base[id];
    const uint64_t dmult = A.msd_mult[id];
    // SPL: this level's segments may split on sampled splitters (uniform per CTA)
    const bool bysplit = SPL && (A.msd_shift[id] & kShiftSplit) != 0u;
    const bool dir = A.direct[id] != 0u;
    uint64_t* kout = dir ? A.kfinal : A.kout;
    uint32_t* pout = dir ? A.pfinal : A.pout;
    const uint64_t flip_out = dir ? A.flip_out : 0ull;
    // A segment of one key value already in place in the output (every
    // second level reads the output buffer) needs no copy at all.
    if (dir && A.kin == A.kfinal && flip_out == 0ull && (!PAY || A.pin == A.pfinal)) return;
    const bool gather = A.any_large[id] != 0u;  // some sub-bucket is split again: note its key range
    if (gather) {
        if (tid < kRadix) { s_mn[tid] = ~0ull; s_mx[tid] = 0ull; }
        if (tid < 8) s_mask[tid] = A.large_mask[(uint64_t)id * 8 + tid];
    }
    if (bysplit) {
        if (tid < kRadix) s_spl[tid] = A.spl_tab[(uint64_t)id * kRadix + tid];
        __syncthreads();
    }
    auto dig = [&](uint64_t k) -> uint32_t {
        return bysplit ? splitter_digit(s_spl, k) : split_digit(k, shift, dbase, dmult);
    };

    uint64_t key[kItems];
    uint32_t pay[kItems];
    uint32_t rank[kItems];
    const uint32_t wbase = w * 32 * kItems + lane;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const uint32_t e = wbase + i * 32;
        if (e < count) {
            key[i] = A.kin[seg_base + tile_lo + e] ^ A.flip_in;
            if (PAY) pay[i] = A.pin[seg_base + tile_lo + e];
        } else {
            key[i] = 0;
            if (PAY) pay[i] = 0;
        }
    }
    if constexpr (PAY) {
        // Each key's digit once, byte-packed in four registers.
        uint32_t dpk[kItems / 4];
#pragma unroll
        for (int i = 0; i < kItems / 4; ++i) dpk[i] = 0;
#pragma unroll
        for (int i = 0; i < kItems; ++i)
            dpk[i >> 2] |= dig(key[i]) << (8 * (i & 3));
        auto digit_of = [&](int i) -> uint32_t {
            return (wbase + i * 32 < count) ? (dpk[i >> 2] >> (8 * (i & 3))) & 255u : (uint32_t)kRadix;
        };
        block_rank<kWarps, kItems>(digit_of, count, rank, s_hist, s_total, s_start, s_warp, NoOp());
        if (A.scatter && !gather) {  // uniform per CTA
            // The stable tile rank less the digit's tile start is the key's
            // place in its digit's run: write it there.
            if (tid < kRadix)
                s_gbase[tid] = seg_base + (uint64_t)A.tile_off[(uint64_t)t * kRadix + tid] - (uint64_t)s_start[tid];
            __syncthreads();
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                if (wbase + i * 32 < count) {
                    const uint64_t dst = s_gbase[(dpk[i >> 2] >> (8 * (i & 3))) & 255u] + rank[i];
                    if (dst - seg_base >= seg_n) {  // never taken when the digit offsets are consistent
                        atomicOr(A.err, kDevErrBounds);
                        continue;
                    }
                    kout[dst] = key[i] ^ flip_out;
                    pout[dst] = pay[i];
                }
            }
            return;
        }
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            if (wbase + i * 32 < count) {
                s_keys[rank[i]] = key[i];
                s_dg[rank[i]] = (uint8_t)((dpk[i >> 2] >> (8 * (i & 3))) & 255u);
                s_pay[rank[i]] = pay[i];
            }
        }
    } else {
        // Keys alone: equal keys are indistinguishable, so the order of a
        // digit's keys inside the tile is free and one shared counter per
        // digit hands out the slots (one atomic per key instead of the
        // ballot ranking the payload path needs for stability).  rank[i]
        // holds the digit and, from bit 8, the key's slot.  (Aggregating the
        // lanes of a warp that share a digit with a match instruction costs
        // more than it saves, even on heavily duplicated keys.)
        const bool direct = A.scatter && !gather;  // uniform per CTA
        for (int d = tid; d < kRadix; d += kThreads) {
            s_total[d] = 0;
            // direct: digit d's keys of this tile start here in the output
            if (direct) s_gbase[d] = seg_base + (uint64_t)A.tile_off[(uint64_t)t * kRadix + d];
        }
        __syncthreads();
        if (direct) {
            // Each key goes straight to the slot its digit's counter hands
            // out; nothing is staged, so no further barrier.
            const bool skew = A.tile_skew[t] != 0;
            const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                const uint32_t d = wbase + i * 32 < count ? dig(key[i]) : (uint32_t)kRadix;
                uint32_t slot = 0;
                if (skew) {
                    const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
                    const uint32_t eq = __ballot_sync(0xffffffffu, d == d0);
                    uint32_t b0 = 0;
                    if (lane == 0 && d0 < (uint32_t)kRadix) b0 = atomicAdd(&s_total[d0], (uint32_t)__popc(eq));
                    b0 = __shfl_sync(0xffffffffu, b0, 0);
                    if (d < (uint32_t)kRadix) slot = d == d0 ? b0 + (uint32_t)__popc(eq & lt_mask) : atomicAdd(&s_total[d], 1u);
                } else if (d < (uint32_t)kRadix) {
                    slot = atomicAdd(&s_total[d], 1u);
                }
                if (d < (uint32_t)kRadix) {
                    const uint64_t dst = s_gbase[d] + slot;
                    if (dst - seg_base >= seg_n) {  // never taken when the digit offsets are consistent
                        atomicOr(A.err, kDevErrBounds);
                        continue;
                    }
                    kout[dst] = key[i] ^ flip_out;
                }
            }
            return;
        }
        if (A.tile_skew[t]) {  // uniform per CTA: see tile_skew_flag
            const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                const uint32_t d =
                    wbase + i * 32 < count ? dig(key[i]) : (uint32_t)kRadix;
                const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
                const uint32_t eq = __ballot_sync(0xffffffffu, d == d0);
                uint32_t b0 = 0;
                if (lane == 0 && d0 < (uint32_t)kRadix) b0 = atomicAdd(&s_total[d0], (uint32_t)__popc(eq));
                b0 = __shfl_sync(0xffffffffu, b0, 0);
                if (d < (uint32_t)kRadix)
                    rank[i] = d | ((d == d0 ? b0 + (uint32_t)__popc(eq & lt_mask) : atomicAdd(&s_total[d], 1u)) << 8);
            }
        } else {
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                if (wbase + i * 32 < count) {
                    const uint32_t d = dig(key[i]);
                    rank[i] = d | (atomicAdd(&s_total[d], 1u) << 8);
                }
            }
        }
        __syncthreads();
        scan256_smem<kThreads>(s_total, s_start, s_warp);
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            if (wbase + i * 32 < count) {
                const uint32_t d = rank[i] & 255u;
                const uint32_t pos = s_start[d] + (rank[i] >> 8);
                s_keys[pos] = key[i];
                s_dg[pos] = (uint8_t)d;
            }
        }
    }

    // The tile's digit-d keys go to the offsets the statistics scan assigned
    // to this tile (digit offset plus the earlier tiles' digit-d keys).
    if (tid < kRadix)
        s_gbase[tid] = seg_base + (uint64_t)A.tile_off[(uint64_t)t * kRadix + tid] - (uint64_t)s_start[tid];
    __syncthreads();
    for (uint32_t j = tid; j < count; j += kThreads) {
        const uint64_t k = s_keys[j];
        const uint32_t d = s_dg[j];
        const uint64_t dst = s_gbase[d] + j;
        if (dst - seg_base >= seg_n) {  // never taken when the digit offsets are consistent
            atomicOr(A.err, kDevErrBounds);
            continue;
        }
        kout[dst] = k ^ flip_out;
        if (PAY) pout[dst] = s_pay[j];
    }
    if (gather) {  // uniform per CTA
        // Smallest and largest key of every sub-bucket the next level splits
        // again (its digit range there).  The staged keys come in digit runs,
        // so a warp usually reduces one run and issues one atomic pair.
        for (uint32_t j0 = (uint32_t)w * 32; j0 < count; j0 += kThreads) {
            const uint32_t j = j0 + lane;
            const bool v = j < count;
            const uint64_t k = v ? s_keys[j] : 0ull;
            const uint32_t d = v ? (uint32_t)s_dg[j] : 0x1ffu;
            const bool flagged = v && ((s_mask[d >> 5] >> (d & 31)) & 1u);
            const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
            if (__all_sync(0xffffffffu, d == d0)) {
                if (flagged) {  // the whole warp: one digit
                    uint64_t mn = k, mx = k;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        mn = min(mn, (uint64_t)__shfl_xor_sync(0xffffffffu, mn, o));
                        mx = max(mx, (uint64_t)__shfl_xor_sync(0xffffffffu, mx, o));
                    }
                    if (lane == 0) {
                        if (mn < s_mn[d]) atomicMin((unsigned long long*)&s_mn[d], (unsigned long long)mn);
                        if (mx > s_mx[d]) atomicMax((unsigned long long*)&s_mx[d], (unsigned long long)mx);
                    }
                }
            } else if (flagged) {
                if (k < s_mn[d]) atomicMin((unsigned long long*)&s_mn[d], (unsigned long long)k);
                if (k > s_mx[d]) atomicMax((unsigned long long*)&s_mx[d], (unsigned long long)k);
            }
        }
        __syncthreads();
        if (tid < kRadix && ((s_mask[tid >> 5] >> (tid & 31)) & 1u) && s_mx[tid] >= s_mn[tid]) {
            atomicMin((unsigned long long*)&A.cmin[(uint64_t)id * kRadix + tid], (unsigned long long)s_mn[tid]);
            atomicMax((unsigned long long*)&A.cmax[(uint64_t)id * kRadix + tid], (unsigned long long)s_mx[tid]);
        }
    }
}

// The digit of the next split of every sub-bucket that will be split again:
// its own key range [min, max] interpolated onto 2^b sub-buckets, b chosen so
// that they hold about `target` keys on average; a sub-bucket of one key
// value keeps multiplier 0.  An interpolated split into 2^b sub-buckets
// narrows the key range by a factor 2^b - 1 >= 2^(b-1) whatever the keys, so
// b is at least ceil(B / levels) + 1 for a range of B bits and `levels`
// levels left before the depth limit (one kept for the copy of single-valued
// sub-buckets): clustered keys with a few outliers then still end within the
// limit (each level keeps B / levels from growing).
__global__ void k_child_hints(uint32_t n_children, const uint64_t* __restrict__ sub_lo, const uint64_t* __restrict__ sub_hi,
                              const uint64_t* __restrict__ cmin, const uint64_t* __restrict__ cmax,
                              uint64_t* __restrict__ cmult, uint32_t chip_max, uint32_t target, uint32_t child_depth) {
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_children) return;
    const uint64_t n = sub_hi[c] - sub_lo[c];
    if (n <= chip_max) return;
    const uint64_t lo = cmin[c], hi = cmax[c];
    if (hi < lo) return;  // no key seen (cannot happen for a non-empty sub-bucket)
    const uint32_t want = (uint32_t)min((n + target - 1) / target, (uint64_t)kRadix);  // sub-buckets wanted
    uint32_t b = 1;
    while (b < 8 && (1u << b) < want) ++b;
    const int levels = kMaxDepth - (int)child_depth - 1;
    const uint32_t B = hi > lo ? 64u - (uint32_t)__clzll((long long)(hi - lo)) : 0u;
    const uint32_t b_min = levels >= 1 ? min(8u, (B + (uint32_t)levels - 1u) / (uint32_t)levels + 1u) : 8u;
    b = max(b, b_min);
    cmult[c] = interp_mult(hi - lo, 1u << b);
}

__global__ void k_even_offsets(uint64_t* __restrict__ seg_off, uint64_t N, uint64_t p) {
    const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s <= p) seg_off[s] = (uint64_t)(((unsigned __int128)s * N) / p);
}

cudaError_t fill_even_offsets(uint64_t* d_seg_off, uint64_t N, uint64_t p, cudaStream_t st) {
    const uint64_t n = p + 1;
    HSS_LAUNCH(k_even_offsets, (unsigned)ceil_div(n, 256), 256, 0, st, d_seg_off, N, p);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Host driver.
// ---------------------------------------------------------------------------
static int num_sms() { return device_sm_count(); }

template <bool PAY, int THREADS, int CAP>
static cudaError_t launch_small(const uint64_t* in, uint64_t* out, const uint32_t* pin, uint32_t* pout,
                                const uint64_t* seg_lo, const uint64_t* seg_hi, const uint32_t* list,
                                const uint32_t* nlist, uint64_t count, uint64_t nseg, uint32_t min_n, uint32_t max_n,
                                uint64_t fin, uint64_t fout, const SegSortWs& ws, cudaStream_t st) {
    constexpr size_t smem = msd_sort_smem<THREADS, CAP>();
    {
        const cudaError_t e = ensure_func_attrs((const void*)k_small_msd<PAY, THREADS, CAP>, (int)smem, 100);
        if (e != cudaSuccess) return e;
    }
    const int per_sm = resident_ctas((const void*)k_small_msd<PAY, THREADS, CAP>, THREADS, smem);
    const uint64_t grid = std::min<uint64_t>(count, (uint64_t)num_sms() * per_sm * 4);
    if (grid == 0) return cudaSuccess;
    HSS_LAUNCH((k_small_msd<PAY, THREADS, CAP>), (unsigned)grid, THREADS, smem, st, in, out, pin, pout, seg_lo, seg_hi,
               list, nlist, nseg, min_n, max_n, fin, fout, ws.fb_list, ws.counters + 24);
    return cudaGetLastError();
}

template <bool PAY, int THREADS, int CAP>
static cudaError_t launch_small_reg(const uint64_t* in, uint64_t* out, const uint32_t* pin, uint32_t* pout,
                                    const uint64_t* seg_lo, const uint64_t* seg_hi, const uint32_t* list,
                                    const uint32_t* nlist, uint64_t count, uint64_t nseg, uint32_t min_n, uint32_t max_n,
                                    uint64_t fin, uint64_t fout, const SegSortWs& ws, cudaStream_t st) {
    constexpr size_t smem = reg_sort_smem<CAP>();
    {
        const cudaError_t e = ensure_func_attrs((const void*)k_small_reg<PAY, THREADS, CAP>, (int)smem, 100);
        if (e != cudaSuccess) return e;
    }
    const int per_sm = resident_ctas((const void*)k_small_reg<PAY, THREADS, CAP>, THREADS, smem);
    const uint64_t grid = std::min<uint64_t>(count, (uint64_t)num_sms() * per_sm * 4);
    if (grid == 0) return cudaSuccess;
    HSS_LAUNCH((k_small_reg<PAY, THREADS, CAP>), (unsigned)grid, THREADS, smem, st, in, out, pin, pout, seg_lo, seg_hi,
               list, nlist, nseg, min_n, max_n, fin, fout, ws.slow_list, ws.counters + 25);
    return cudaGetLastError();
}

template <int THREADS, int CAP, int R, bool PREFETCH>
static cudaError_t launch_keys(const uint64_t* in, uint64_t* out, const uint64_t* seg_lo, const uint64_t* seg_hi,
                               const uint32_t* list, const uint32_t* nlist, uint64_t count, uint64_t nseg,
                               uint32_t min_n, uint32_t max_n, uint64_t fin, uint64_t fout, uint32_t* slow,
                               uint32_t* slow_count, uint32_t* err, cudaStream_t st) {
    constexpr size_t smem = keys_sort_smem<CAP, R, PREFETCH>();
    const void* fn = (const void*)k_small_keys<THREADS, CAP, R, PREFETCH>;
    {
        // all of L1 as shared memory: the CTAs per SM are limited by their buffers
        const cudaError_t e = ensure_func_attrs(fn, (int)smem, 100);
        if (e != cudaSuccess) return e;
    }
    const int per_sm = resident_ctas(fn, THREADS, smem);
    // With prefetching every CTA walks several segments of the list.
    const uint64_t grid = std::min<uint64_t>(count, (uint64_t)num_sms() * per_sm * (PREFETCH ? 1 : 4));
    if (grid == 0) return cudaSuccess;
    HSS_LAUNCH((k_small_keys<THREADS, CAP, R, PREFETCH>), (unsigned)grid, THREADS, smem, st, in, out, seg_lo, seg_hi,
               list, nlist, nseg, min_n, max_n, fin, fout, slow, slow_count, err);
    return cudaGetLastError();
}

// The stable LSD kernel over this level's fallback list (length on the device).
template <bool PAY>
// max_entries bounds the list on the host (the segments that could have
// been appended): a CTA per entry at most, since each launch of this kernel
// reconfigures the SMs for its large shared-memory tile.
static cudaError_t launch_fallback(const uint64_t* in, uint64_t* out, const uint32_t* pin, uint32_t* pout,
                                   const uint64_t* seg_lo, const uint64_t* seg_hi, uint64_t fin, uint64_t fout,
                                   const SegSortWs& ws, cudaStream_t st, uint64_t max_entries) {
    constexpr size_t smem = lsd_sort_smem<kC2Threads, kC2Items>();
    {
        const cudaError_t e = ensure_func_attrs((const void*)k_small_lsd<PAY, kC2Threads, kC2Items>, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const uint64_t grid = std::min<uint64_t>((uint64_t)num_sms(), max_entries);
    if (grid == 0) return cudaSuccess;
    HSS_LAUNCH((k_small_lsd<PAY, kC2Threads, kC2Items>), (unsigned)grid, kC2Threads, smem, st, in, out, pin, pout,
               seg_lo, seg_hi, ws.fb_list, ws.counters + 24, fin, fout);
    return cudaGetLastError();
}

struct Level {
    const uint64_t* in;
    const uint32_t* pin;
    const uint64_t* seg_lo;
    const uint64_t* seg_hi;
    uint64_t nseg;
    uint64_t flip_in;
    const uint64_t* hint_lo;
    const uint64_t* hint_mult;
    int depth;
    const uint64_t* hint_hi = nullptr;  // largest key of each segment, when known
};

// This thread's mapped pinned buffer for the planning counts (allocated once
// per thread; null if the allocation fails, and then the counts are copied).
struct MappedCounts {
    volatile uint32_t* host = nullptr;
    uint32_t* dev = nullptr;
    bool tried = false;
};
static thread_local MappedCounts t_counts;

static void mapped_counts(volatile uint32_t** host, uint32_t** dev) {
    if (!t_counts.tried) {
        t_counts.tried = true;
        void* p = nullptr;
        if (cudaHostAlloc(&p, 64, cudaHostAllocMapped | cudaHostAllocPortable) == cudaSuccess) {
            void* dp = nullptr;
            if (cudaHostGetDevicePointer(&dp, p, 0) == cudaSuccess) {
                t_counts.host = (volatile uint32_t*)p;
                t_counts.dev = (uint32_t*)dp;
            } else {
                (void)cudaGetLastError();
                cudaFreeHost(p);
            }
        } else {
            (void)cudaGetLastError();
        }
    }
    *host = t_counts.host;
    *dev = t_counts.dev;
}

template <bool PAY>
static cudaError_t segsort_t(const uint64_t* src, uint64_t* dst, uint64_t* tmp, const uint32_t* psrc, uint32_t* pdst,
                             uint32_t* ptmp, uint64_t N, uint64_t nseg, const uint64_t* d_seg_off, bool flip_in,
                             bool flip_out, const SegSortWs& ws, cudaStream_t st, SegSortTiming* timing,
                             const uint64_t* hint_lo, const uint64_t* hint_mult) {
    if (N == 0 || nseg == 0) return cudaSuccess;
    const uint64_t fout = flip_out ? kSignBit : 0ull;
    const uint32_t tune_chip_max = g_chip_max.load();
    const bool child_interp = g_child_interp.load() != 0u;
    const uint32_t child_keys = g_child_keys.load();
    const uint32_t pack_keys = g_pack_keys.load();
    const bool use_splitters = g_splitters.load() != 0u;
    const uint32_t scatter = g_scatter.load();
    volatile uint32_t* mapped = nullptr;  // host view of the planning counts
    uint32_t* mapped_dev = nullptr;        // the kernel's view
    if (ws.mapped_counts) mapped_counts(&mapped, &mapped_dev);
    cudaError_t e;
    Level L{src, psrc, d_seg_off, d_seg_off + 1, nseg, flip_in ? kSignBit : 0ull, hint_lo, hint_mult, 0};
    if (N <= (uint64_t)kSmallCap) {
        // No segment can exceed the on-chip capacity: sort every segment in
        // its class without planning (and without a host round trip).
        if ((e = cudaMemsetAsync(ws.counters + 24, 0, 8, st)) != cudaSuccess) return e;
        if ((e = launch_small<PAY, kC0Threads, kC0Cap>(L.in, dst, L.pin, pdst, L.seg_lo, L.seg_hi, nullptr, nullptr, nseg,
                                                       nseg, 0u, (uint32_t)kC0Cap, L.flip_in, fout, ws, st)) !=
            cudaSuccess)
            return e;
        if (N > (uint64_t)kC0Cap &&
            (e = launch_small_reg<PAY, kC1Threads, kC1Cap>(L.in, dst, L.pin, pdst, L.seg_lo, L.seg_hi, nullptr, nullptr,
                                                           nseg, nseg, (uint32_t)kC0Cap, (uint32_t)kC1Cap, L.flip_in,
                                                           fout, ws, st)) != cudaSuccess)
            return e;
        if ((e = launch_small<PAY, kC1Threads, kC1Cap>(L.in, dst, L.pin, pdst, L.seg_lo, L.seg_hi, ws.slow_list,
                                                       ws.counters + 25, nseg, nseg, 0u, (uint32_t)kC1Cap, L.flip_in,
                                                       fout, ws, st)) != cudaSuccess)
            return e;
        if (N > (uint64_t)kC1Cap &&
            (e = launch_small<PAY, kC2Threads, kSmallCap>(L.in, dst, L.pin, pdst, L.seg_lo, L.seg_hi, nullptr, nullptr,
                                                          nseg, nseg, (uint32_t)kC1Cap, (uint32_t)kSmallCap, L.flip_in,
                                                          fout, ws, st)) != cudaSuccess)
            return e;
        return launch_fallback<PAY>(L.in, dst, L.pin, pdst, L.seg_lo, L.seg_hi, L.flip_in, fout, ws, st, nseg);
    }
    for (;;) {
        if (L.nseg > ws.max_list) return cudaErrorInvalidValue;
        const uint32_t nblk = (uint32_t)ceil_div(L.nseg + 1, 1024);
        // By default a segment above the middle on-chip class is split again
        // (into buckets of about a thousand keys that the small classes sort)
        // rather than sorted by the largest class (tuning.chip_max_keys).
        const uint32_t chip_max = tune_chip_max;
        HSS_LAUNCH(k_plan_count, nblk, 1024, 0, st, L.seg_lo, L.seg_hi, L.nseg, ws.blk, chip_max);
        HSS_LAUNCH(k_plan_scan, 1, 1024, 0, st, nblk, ws.blk, ws.counters, mapped_dev);
        HSS_LAUNCH(k_plan_write, nblk, 1024, 0, st, L.seg_lo, L.seg_hi, L.nseg, ws.blk, ws.counters, ws.tile_start,
                   ws.large_id, ws.large_seg, ws.list[0], ws.list[1], ws.list[2], ws.err, ws.tile_seg, chip_max);
        uint32_t hc[8];
        if (!mapped && (e = cudaMemcpyAsync(hc, ws.counters + 16, sizeof(hc), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        if (mapped)
            for (int k = 0; k < 8; ++k) hc[k] = mapped[k];
        const uint32_t n_large = hc[3], tiles = hc[4];
        const uint64_t keys_large = (uint64_t)hc[6] | ((uint64_t)hc[7] << 32);
        // Segments of this level that fit on chip: straight to the output.
        if (!PAY) {
            // keys alone: the register kernels first, their leftovers to the
            // shared-memory kernel of the same class
            const uint32_t* lists[3] = {ws.list[0], ws.list[1], ws.list[2]};
            for (int c = 0; c < 3; ++c) {
                if (!hc[c]) continue;
                const uint32_t lo_n = c == 0 ? 0u : (c == 1 ? (uint32_t)kC0Cap : (uint32_t)kC1Cap);
                const uint32_t hi_n = c == 0 ? (uint32_t)kC0Cap : (c == 1 ? (uint32_t)kC1Cap : (uint32_t)kSmallCap);
                uint32_t* slow = ws.slow_keys[c];
                uint32_t* slow_n = ws.counters + 26 + c;
                if (c == 0)
                    e = launch_keys<kC0Threads, kC0Cap, 512, true>(L.in, dst, L.seg_lo, L.seg_hi, lists[c], ws.counters + 16,
                                                            hc[c], L.nseg, lo_n, hi_n, L.flip_in, fout, slow, slow_n, ws.err, st);
                else if (c == 1)
                    e = launch_keys<kC1Threads, kC1Cap, 2048, true>(L.in, dst, L.seg_lo, L.seg_hi, lists[c], ws.counters + 17,
                                                            hc[c], L.nseg, lo_n, hi_n, L.flip_in, fout, slow, slow_n, ws.err, st);
                else
                    e = launch_keys<kC2Threads, kSmallCap, 4096, false>(L.in, dst, L.seg_lo, L.seg_hi, lists[c],
                                                               ws.counters + 18, hc[c], L.nseg, lo_n, hi_n, L.flip_in,
                                                               fout, slow, slow_n, ws.err, st);
                if (e != cudaSuccess) return e;
                if (c == 0)
                    e = launch_small<PAY, kC0Threads, kC0Cap>(L.in, dst, L.pin, pdst, L.seg_lo, L.seg_hi, slow, slow_n,
                                                              hc[c], L.nseg, lo_n, hi_n, L.flip_in, fout, ws, st);
                else if (c == 1)
                    e = launch_small<PAY, kC1Threads, kC1Cap>(L.in, dst, L.pin, pdst, L.seg_lo, L.seg_hi, slow, slow_n,
                                                              hc[c], L.nseg, lo_n, hi_n, L.flip_in, fout, ws, st);
                else
                    e = launch_small<PAY, kC2Threads, kSmallCap>(L.in, dst, L.pin, pdst, L.seg_lo, L.seg_hi, slow,
                                                                 slow_n, hc[c], L.nseg, lo_n, hi_n, L.flip_in, fout,
                                                                 ws, st);
                if (e != cudaSuccess) return e;
            }
        }
        if (PAY && hc[0] && (e = launch_small<PAY, kC0Threads, kC0Cap>(L.in, dst, L.pin, pdst, L.seg_lo, L.seg_hi, ws.list[0],
                                                                ws.counters + 16, hc[0], L.nseg, 0u, (uint32_t)kC0Cap,
                                                                L.flip_in, fout, ws, st)) != cudaSuccess)
            return e;
        if (PAY && hc[1] && (e = launch_small_reg<PAY, kC1Threads, kC1Cap>(L.in, dst, L.pin, pdst, L.seg_lo, L.seg_hi,
                                                                    ws.list[1], ws.counters + 17, hc[1], L.nseg,
                                                                    (uint32_t)kC0Cap, (uint32_t)kC1Cap, L.flip_in, fout,
                                                                    ws, st)) != cudaSuccess)
            return e;
        if (PAY && hc[1] &&
            (e = launch_small<PAY, kC1Threads, kC1Cap>(L.in, dst, L.pin, pdst, L.seg_lo, L.seg_hi, ws.slow_list,
                                                       ws.counters + 25, hc[1], L.nseg, 0u, (uint32_t)kC1Cap, L.flip_in,
                                                       fout, ws, st)) != cudaSuccess)
            return e;
        if (PAY && hc[2] && (e = launch_small<PAY, kC2Threads, kSmallCap>(L.in, dst, L.pin, pdst, L.seg_lo, L.seg_hi,
                                                                   ws.list[2], ws.counters + 18, hc[2], L.nseg,
                                                                   (uint32_t)kC1Cap, (uint32_t)kSmallCap, L.flip_in, fout,
                                                                   ws, st)) != cudaSuccess)
            return e;
        if ((hc[0] || hc[1] || hc[2]) &&
            (e = launch_fallback<PAY>(L.in, dst, L.pin, pdst, L.seg_lo, L.seg_hi, L.flip_in, fout, ws, st,
                                      (uint64_t)hc[0] + hc[1] + hc[2])) != cudaSuccess)
            return e;
        if (n_large == 0) return cudaSuccess;
        if (n_large > ws.max_large || tiles > ws.max_tiles || L.depth >= kMaxDepth) return cudaErrorInvalidValue;
        // Statistics per tile, the split window and every tile's offsets.
        if ((e = cudaMemsetAsync(ws.vor, 0, (size_t)n_large * 8, st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(ws.vand, 0xff, (size_t)n_large * 8, st)) != cudaSuccess) return e;
        const int buf = L.depth & 1;
        const uint32_t* prev_shift = L.depth > 0 ? ws.msd_shift[buf ^ 1] : nullptr;
        // The first split of a level-0 segment may take sampled splitters
        // (skewed keys); later levels and hinted splits keep their digits.
        const bool bysplit_level = use_splitters && L.depth == 0 && !L.hint_lo && n_large <= ws.max_spl;
        if (bysplit_level)
            HSS_LAUNCH(k_seg_sample, n_large, 256, 0, st, L.in, L.seg_lo, L.seg_hi, ws.large_seg, ws.counters, L.flip_in,
                       ws.spl_tab, ws.spl_mode);
        if (bysplit_level)
            HSS_LAUNCH(k_tile_stats<true>, tiles, 256, 0, st, L.in, L.seg_lo, L.seg_hi, L.nseg, ws.tile_start, ws.tile_seg,
                       ws.large_id, ws.tile_hist, ws.tile_skew, ws.vor, ws.vand, L.hint_lo, L.hint_mult, L.hint_hi,
                       prev_shift, ws.spec, L.flip_in, ws.spl_tab, ws.spl_mode);
        else
            HSS_LAUNCH(k_tile_stats<false>, tiles, 256, 0, st, L.in, L.seg_lo, L.seg_hi, L.nseg, ws.tile_start, ws.tile_seg,
                       ws.large_id, ws.tile_hist, ws.tile_skew, ws.vor, ws.vand, L.hint_lo, L.hint_mult, L.hint_hi,
                       prev_shift, ws.spec, L.flip_in, nullptr, nullptr);
        if (!L.hint_lo)
            HSS_LAUNCH(k_tile_recount, (unsigned)std::min<uint64_t>(tiles, (uint64_t)num_sms() * 8), 256, 0, st, L.in,
                       L.seg_lo, L.seg_hi, L.nseg, ws.tile_start, ws.tile_seg, ws.large_id,
                       ws.tile_hist, ws.tile_skew, bysplit_level ? ws.spl_mode : nullptr, ws.vor, ws.vand, ws.spec,
                       L.flip_in);
        HSS_LAUNCH(k_msd_prep, n_large, 256, 0, st, L.seg_lo, ws.large_seg, ws.counters, ws.tile_start, ws.tile_hist,
                   ws.vor, ws.vand, L.hint_lo, L.hint_mult, ws.msd_base, ws.msd_mult, ws.msd_shift[buf], ws.spec,
                   ws.direct, ws.sub_lo[buf], ws.sub_hi[buf], ws.tile_off, child_interp ? chip_max : 0xffffffffu,
                   ws.large_mask, ws.any_large, ws.cmin[buf], ws.cmax[buf], chip_max,
                   // sampled-splitter sub-buckets (about 256 keys, unevenly wide) pack at most 256 keys
                   std::min(bysplit_level ? std::min(pack_keys, 256u) : pack_keys, chip_max),
                   bysplit_level ? ws.spl_mode : nullptr);
        // The split pass: level buffers alternate tmp, dst, tmp, ... after src.
        uint64_t* next = (L.depth & 1) ? dst : tmp;
        uint32_t* pnext = PAY ? ((L.depth & 1) ? pdst : ptmp) : nullptr;
        SplitArgs A;
        A.kin = L.in; A.kout = next; A.kfinal = dst;
        A.pin = L.pin; A.pout = pnext; A.pfinal = pdst;
        A.seg_lo = L.seg_lo; A.seg_hi = L.seg_hi; A.nseg = L.nseg;
        A.tile_start = ws.tile_start; A.tile_seg = ws.tile_seg; A.large_id = ws.large_id;
        A.tile_off = ws.tile_off; A.tile_skew = ws.tile_skew; A.spl_tab = ws.spl_tab; A.msd_shift = ws.msd_shift[buf]; A.msd_base = ws.msd_base; A.msd_mult = ws.msd_mult;
        A.direct = ws.direct;
        A.large_mask = ws.large_mask; A.any_large = ws.any_large; A.cmin = ws.cmin[buf]; A.cmax = ws.cmax[buf];
        A.err = ws.err;
        A.scatter = scatter;
        A.flip_in = L.flip_in; A.flip_out = fout;
        const size_t smem = (size_t)kOsTile * 9 + (PAY ? (size_t)kOsTile * 4 : 0);
        // all of L1 as shared memory: the CTAs per SM are limited by their tiles
        const void* split_fn = bysplit_level ? (const void*)k_split<PAY, true> : (const void*)k_split<PAY, false>;
        if ((e = ensure_func_attrs(split_fn, (int)smem, 100)) != cudaSuccess) return e;
        const bool timed = timing && timing->enabled && timing->n < 16;
        if (timed) {
            cudaEventCreate(&timing->ev[timing->n][0]);
            cudaEventCreate(&timing->ev[timing->n][1]);
            cudaEventRecord(timing->ev[timing->n][0], st);
        }
        if (bysplit_level)
            HSS_LAUNCH((k_split<PAY, true>), tiles, split_threads<PAY>(), smem, st, A);
        else
            HSS_LAUNCH((k_split<PAY, false>), tiles, split_threads<PAY>(), smem, st, A);
        if (timed) {
            cudaEventRecord(timing->ev[timing->n][1], st);
            timing->keys[timing->n] = keys_large;
            timing->n += 1;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // Next level: the 256 sub-buckets of every large segment; those split
        // again interpolate their own key range (gathered by the split).
        const uint32_t nch = n_large * kRadix;
        if (child_interp) {
            HSS_LAUNCH(k_child_hints, (nch + 255) / 256, 256, 0, st, nch, ws.sub_lo[buf], ws.sub_hi[buf], ws.cmin[buf],
                       ws.cmax[buf], ws.cmult[buf], chip_max, child_keys, (uint32_t)L.depth + 1u);
            L = Level{next, pnext, ws.sub_lo[buf], ws.sub_hi[buf], (uint64_t)n_large * kRadix, 0ull, ws.cmin[buf],
                      ws.cmult[buf], L.depth + 1, ws.cmax[buf]};
        } else {
            L = Level{next, pnext, ws.sub_lo[buf], ws.sub_hi[buf], (uint64_t)n_large * kRadix, 0ull, nullptr, nullptr,
                      L.depth + 1};
        }
    }
}

cudaError_t segsort(const uint64_t* src, uint64_t* dst, uint64_t* tmp, const uint32_t* psrc, uint32_t* pdst,
                    uint32_t* ptmp, uint64_t N, uint64_t nseg, const uint64_t* d_seg_off, bool flip_in, bool flip_out,
                    const SegSortWs& ws, cudaStream_t st, SegSortTiming* timing, const uint64_t* hint_lo,
                    const uint64_t* hint_mult) {
    if (psrc)
        return segsort_t<true>(src, dst, tmp, psrc, pdst, ptmp, N, nseg, d_seg_off, flip_in, flip_out, ws, st, timing,
                               hint_lo, hint_mult);
    return segsort_t<false>(src, dst, tmp, nullptr, nullptr, nullptr, N, nseg, d_seg_off, flip_in, flip_out, ws, st,
                            timing, hint_lo, hint_mult);
}

}  // namespace hss
