// segsort.cu -- stable segmented LSD radix sort (local sort of Sec. 5/6 and,
// over bucket ranges, the local merge).
//
// Design for sm_103a:
//  * Small segments (<= 16384 keys): one 1024-thread CTA loads the whole
//    segment into shared memory once, runs the 8-bit digit passes on chip over
//    a 16-bit index permutation (the keys stay put), skips digits that are
//    constant over the segment, and writes the sorted keys once: 16 B of HBM
//    traffic per key.
//  * Large segments: a digit-histogram pass (8 B/key) followed by eight
//    one-sweep digit passes (16 B/key each).  Each 4096-key tile ranks its keys
//    in shared memory (warp match + per-warp counters), publishes its digit
//    counts and chains the per-segment exclusive prefix by decoupled look-back
//    over the tiles of the same segment, then scatters from shared memory so
//    that runs of equal digits are written contiguously.
#include "segsort.cuh"

#include <algorithm>

namespace hss {

constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagPre = 1u << 31;
constexpr uint32_t kCountMask = (1u << 30) - 1u;

__host__ __device__ static inline uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }
static inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

size_t segsort_ws_bytes(uint64_t N, uint64_t nseg) {
    const uint64_t max_tiles = ceil_div(N, kOsTile) + nseg + 1;
    size_t b = 0;
    b += align_up(nseg * kPasses * kRadix * sizeof(uint32_t), 256);
    b += align_up((nseg + 1) * sizeof(uint32_t), 256);
    b += align_up(2 * max_tiles * kRadix * sizeof(uint32_t), 256);
    b += align_up(64 * sizeof(uint32_t), 256);
    return b;
}

SegSortWs segsort_ws_carve(void* base, uint64_t N, uint64_t nseg, uint32_t* err) {
    SegSortWs w;
    w.max_tiles = ceil_div(N, kOsTile) + nseg + 1;
    char* p = (char*)base;
    w.digit_off = (uint32_t*)p; p += align_up(nseg * kPasses * kRadix * sizeof(uint32_t), 256);
    w.tile_start = (uint32_t*)p; p += align_up((nseg + 1) * sizeof(uint32_t), 256);
    w.status = (uint32_t*)p; p += align_up(2 * w.max_tiles * kRadix * sizeof(uint32_t), 256);
    w.counters = (uint32_t*)p; p += align_up(64 * sizeof(uint32_t), 256);
    w.err = err;
    return w;
}

// ---------------------------------------------------------------------------
// Block-wide exclusive scan of 256 values held one per thread by threads
// 0..255 (the caller guarantees blockDim >= 256).  Returns the exclusive
// prefix for threads < 256.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t scan256_exclusive(uint32_t v, uint32_t* s_warp /*[8]*/) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    uint32_t x = v;
    if (tid < 256) {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[w] = x;
    }
    __syncthreads();
    uint32_t add = 0;
    if (tid < 256) {
        for (int i = 0; i < w; ++i) add += s_warp[i];
    }
    __syncthreads();
    return add + x - v;
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
//   2. offsets: thread d turns the counts into absolute bases
//      start[d] + sum of earlier warps' counts of d, and the tile totals;
//   3. ranks: per item, the lanes holding the same digit (ballot peer mask)
//      take consecutive slots: the highest such lane adds their number to the
//      warp's base for that digit and broadcasts the old value.
// Items are warp-striped: item i of lane l in warp w is element
// w*32*ITEMS + i*32 + l, so (w, i, l) order is element order and the ranks are
// stable.  Shared atomics issued by one warp in program order are applied in
// that order, which the running bases of step 3 rely on.
// `between` runs after step 2 (used to publish the look-back aggregate).
// ---------------------------------------------------------------------------
struct NoOp { __device__ void operator()() const {} };

template <int WARPS, int ITEMS, typename DigitOf, typename Between>
__device__ __forceinline__ void block_rank(DigitOf digit_of, uint32_t (&rank)[ITEMS], uint32_t* s_cnt /*[WARPS*256]*/,
                                           uint32_t* s_total, uint32_t* s_start, uint32_t* s_warp, Between between) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int i = tid; i < WARPS * kRadix; i += WARPS * 32) s_cnt[i] = 0;
    __syncthreads();
    uint32_t* c = s_cnt + w * kRadix;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t d = digit_of(i);
        if (d < kRadix) atomicAdd(&c[d], 1u);
    }
    __syncthreads();
    uint32_t tot = 0;
    if (tid < kRadix) {
        uint32_t run = 0;
        for (int ww = 0; ww < WARPS; ++ww) {
            const uint32_t x = s_cnt[ww * kRadix + tid];
            s_cnt[ww * kRadix + tid] = run;
            run += x;
        }
        tot = run;
        s_total[tid] = tot;
    }
    const uint32_t ex = scan256_exclusive(tot, s_warp);
    if (tid < kRadix) {
        s_start[tid] = ex;
        for (int ww = 0; ww < WARPS; ++ww) s_cnt[ww * kRadix + tid] += ex;
    }
    __syncthreads();
    between();
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
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
// Planning: tiles of the large segments.
// ---------------------------------------------------------------------------
__global__ void k_seg_plan(const uint64_t* __restrict__ seg_off, uint64_t nseg, uint32_t* __restrict__ tile_start,
                           uint32_t* __restrict__ counters) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_carry;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) s_carry = 0;
    if (tid < 64) counters[tid] = 0;
    __syncthreads();
    for (uint64_t base = 0; base < nseg; base += blockDim.x) {
        const uint64_t s = base + tid;
        uint32_t nt = 0;
        if (s < nseg) {
            const uint64_t n = seg_off[s + 1] - seg_off[s];
            nt = n > (uint64_t)kSmallCap ? (uint32_t)ceil_div(n, kOsTile) : 0u;
        }
        uint32_t x = nt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[w] = x;
        __syncthreads();
        uint32_t add = s_carry;
        for (int i = 0; i < w; ++i) add += s_warp[i];
        if (s < nseg) tile_start[s] = add + x - nt;
        __syncthreads();
        if (tid == blockDim.x - 1) s_carry = add + x;
        __syncthreads();
    }
    if (tid == 0) tile_start[nseg] = s_carry;
}

__device__ __forceinline__ uint32_t find_tile_segment(const uint32_t* __restrict__ tile_start, uint64_t nseg, uint32_t t) {
    // largest s with tile_start[s] <= t (segments with no tiles share a start value)
    uint64_t lo = 0, hi = nseg;  // answer in [lo, hi)
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        if (tile_start[mid] <= t) lo = mid; else hi = mid;
    }
    return (uint32_t)lo;
}

// ---------------------------------------------------------------------------
// Digit histograms of the large segments: all 8 digit positions in one read.
// Grid (nseg, split); CTA (s, k) counts the k-th share of segment s's tiles.
// ---------------------------------------------------------------------------
__global__ __launch_bounds__(256) void k_digit_hist(const uint64_t* __restrict__ kin, const uint64_t* __restrict__ seg_off,
                                                    uint32_t* __restrict__ digit_off, uint32_t split, uint64_t flip_in) {
    __shared__ uint32_t s_h[kPasses * kRadix];
    const uint64_t s = blockIdx.x;
    const uint64_t lo = seg_off[s], n = seg_off[s + 1] - lo;
    if (n <= (uint64_t)kSmallCap) return;
    const uint64_t per = ceil_div(ceil_div(n, kOsTile), split) * kOsTile;
    const uint64_t a = (uint64_t)blockIdx.y * per;
    if (a >= n) return;
    const uint64_t b = min(n, a + per);
    for (int i = threadIdx.x; i < kPasses * kRadix; i += blockDim.x) s_h[i] = 0;
    __syncthreads();
    for (uint64_t e = a + threadIdx.x; e < b; e += blockDim.x) {
        const uint64_t k = kin[lo + e] ^ flip_in;
#pragma unroll
        for (int p = 0; p < kPasses; ++p) atomicAdd(&s_h[p * kRadix + ((k >> (8 * p)) & 255u)], 1u);
    }
    __syncthreads();
    uint32_t* g = digit_off + s * (kPasses * kRadix);
    for (int i = threadIdx.x; i < kPasses * kRadix; i += blockDim.x) {
        const uint32_t c = s_h[i];
        if (c) atomicAdd(&g[i], c);
    }
}

// In place: counts -> exclusive offsets, per (segment, pass).
__global__ __launch_bounds__(256) void k_digit_scan(const uint64_t* __restrict__ seg_off, uint32_t* __restrict__ digit_off) {
    __shared__ uint32_t s_warp[8];
    const uint64_t s = blockIdx.x;
    const uint64_t n = seg_off[s + 1] - seg_off[s];
    if (n <= (uint64_t)kSmallCap) return;
    uint32_t* g = digit_off + s * (kPasses * kRadix) + blockIdx.y * kRadix;
    const uint32_t v = g[threadIdx.x];
    const uint32_t ex = scan256_exclusive(v, s_warp);
    g[threadIdx.x] = ex;
}

// ---------------------------------------------------------------------------
// One digit pass of the one-sweep radix sort over the tiles of all large
// segments.
// ---------------------------------------------------------------------------
template <bool PAY>
__global__ __launch_bounds__(kOsThreads, 3) void k_onesweep(
    const uint64_t* __restrict__ kin, uint64_t* __restrict__ kout,
    const uint32_t* __restrict__ pin, uint32_t* __restrict__ pout,
    const uint64_t* __restrict__ seg_off, const uint32_t* __restrict__ tile_start, uint64_t nseg,
    const uint32_t* __restrict__ digit_off, uint32_t* __restrict__ status, uint64_t max_tiles,
    uint32_t* __restrict__ counters, uint32_t* __restrict__ err, int pass, uint64_t flip_in, uint64_t flip_out) {
    extern __shared__ __align__(16) unsigned char os_smem[];
    uint64_t* s_keys = (uint64_t*)os_smem;                 // kOsTile keys
    uint32_t* s_pay = (uint32_t*)(s_keys + kOsTile);       // kOsTile payloads (PAY)
    __shared__ uint32_t s_hist[kOsWarps * kRadix];
    __shared__ uint32_t s_total[kRadix], s_start[kRadix];
    __shared__ uint64_t s_gbase[kRadix];
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_tile, s_seg;

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t total_tiles = tile_start[nseg];
    if (tid == 0) {
        const uint32_t t = atomicAdd(&counters[pass], 1u);
        s_tile = t;
        s_seg = t < total_tiles ? find_tile_segment(tile_start, nseg, t) : 0u;
    }
    __syncthreads();
    const uint32_t t = s_tile;
    if (t >= total_tiles) return;
    const uint32_t s = s_seg;
    const uint64_t seg_base = seg_off[s];
    const uint64_t seg_n = seg_off[s + 1] - seg_base;
    const uint32_t ti = t - tile_start[s];
    const uint64_t tile_lo = (uint64_t)ti * kOsTile;
    const uint32_t count = (uint32_t)min((uint64_t)kOsTile, seg_n - tile_lo);
    const int shift = 8 * pass;

    uint64_t key[kOsItems];
    uint32_t pay[kOsItems];
    uint32_t rank[kOsItems];
    const uint32_t wbase = w * 32 * kOsItems + lane;
#pragma unroll
    for (int i = 0; i < kOsItems; ++i) {
        const uint32_t e = wbase + i * 32;
        if (e < count) {
            key[i] = kin[seg_base + tile_lo + e] ^ flip_in;
            if (PAY) pay[i] = pin[seg_base + tile_lo + e];
        } else {
            key[i] = 0;
            if (PAY) pay[i] = 0;
        }
    }
    auto digit_of = [&](int i) -> uint32_t {
        return (wbase + i * 32 < count) ? ((uint32_t)(key[i] >> shift) & 255u) : (uint32_t)kRadix;
    };

    // Publish this tile's digit counts as soon as they are known, so the next
    // tile's look-back does not wait for our ranking.
    uint32_t* cur = status + (uint64_t)(pass & 1) * max_tiles * kRadix;
    uint32_t* nxt = status + (uint64_t)((pass + 1) & 1) * max_tiles * kRadix;
    auto publish = [&]() {
        if (tid < kRadix) st_relaxed(&cur[(uint64_t)t * kRadix + tid], (ti == 0 ? kFlagPre : kFlagAgg) | s_total[tid]);
    };
    block_rank<kOsWarps, kOsItems>(digit_of, rank, s_hist, s_total, s_start, s_warp, publish);
#pragma unroll
    for (int i = 0; i < kOsItems; ++i) {
        if (wbase + i * 32 < count) {
            s_keys[rank[i]] = key[i];
            if (PAY) s_pay[rank[i]] = pay[i];
        }
    }

    // Decoupled look-back over the earlier tiles of this segment: thread d
    // owns digit d.
    if (tid < kRadix) {
        const uint32_t d = tid;
        const uint32_t cnt = s_total[d];
        uint32_t excl = 0;
        if (ti != 0) {
            const uint64_t first = tile_start[s];
            uint64_t tt = t - 1;
            for (;;) {
                uint32_t v;
                uint32_t it = 0;
                while (((v = ld_relaxed(&cur[tt * kRadix + d])) & (kFlagAgg | kFlagPre)) == 0u) {
                    if (++it > kSpinLimit) {
                        atomicOr(err, kDevErrTimeout);
                        v = kFlagPre;
                        break;
                    }
                    __nanosleep(64);
                }
                excl += v & kCountMask;
                if (v & kFlagPre) break;
                if (tt == first) {  // the first tile always publishes a prefix
                    atomicOr(err, kDevErrBounds);
                    break;
                }
                --tt;
            }
            st_relaxed(&cur[(uint64_t)t * kRadix + d], kFlagPre | (excl + cnt));
        }
        const uint32_t goff = digit_off[((uint64_t)s * kPasses + pass) * kRadix + d];
        s_gbase[d] = seg_base + (uint64_t)goff + (uint64_t)excl - (uint64_t)s_start[d];
        nxt[(uint64_t)t * kRadix + d] = 0u;  // ready for the pass after this one
    }
    __syncthreads();
    for (uint32_t j = tid; j < count; j += kOsThreads) {
        const uint64_t k = s_keys[j];
        const uint32_t d = (uint32_t)(k >> shift) & 255u;
        const uint64_t dst = s_gbase[d] + j;
        if (dst - seg_base >= seg_n) {  // never taken when the digit offsets are consistent
            atomicOr(err, kDevErrBounds);
            continue;
        }
        kout[dst] = k ^ flip_out;
        if (PAY) pout[dst] = s_pay[j];
    }
}

// ---------------------------------------------------------------------------
// Small segments: one CTA, whole segment on chip.
// ---------------------------------------------------------------------------
template <bool PAY>
__global__ __launch_bounds__(kSmThreads, 1) void k_small_sort(
    const uint64_t* __restrict__ kin, uint64_t* __restrict__ kout,
    const uint32_t* __restrict__ pin, uint32_t* __restrict__ pout,
    const uint64_t* __restrict__ seg_off, uint64_t nseg, uint64_t flip_in, uint64_t flip_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* s_keys = (uint64_t*)smem;                                   // kSmallCap u64
    uint16_t* s_idx0 = (uint16_t*)(s_keys + kSmallCap);                   // kSmallCap u16
    uint16_t* s_idx1 = s_idx0 + kSmallCap;                                // kSmallCap u16
    uint32_t* s_hist = (uint32_t*)(s_idx1 + kSmallCap);                   // kSmWarps*256 u32
    uint32_t* s_total = s_hist + kSmWarps * kRadix;                       // 256
    uint32_t* s_start = s_total + kRadix;                                 // 256
    uint32_t* s_warp = s_start + kRadix;                                  // 32
    uint64_t* s_red = (uint64_t*)(s_warp + 32);                           // 2*32 u64

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (uint64_t s = blockIdx.x; s < nseg; s += gridDim.x) {
        const uint64_t base = seg_off[s];
        const uint32_t n = (uint32_t)(seg_off[s + 1] - base);
        if (n == 0 || seg_off[s + 1] - base > (uint64_t)kSmallCap) continue;  // uniform per CTA
        uint64_t vor = 0, vand = ~0ull;
        for (uint32_t j = tid; j < n; j += kSmThreads) {
            const uint64_t k = kin[base + j] ^ flip_in;
            s_keys[j] = k;
            s_idx0[j] = (uint16_t)j;
            vor |= k; vand &= k;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vor |= __shfl_xor_sync(0xffffffffu, vor, o);
            vand &= __shfl_xor_sync(0xffffffffu, vand, o);
        }
        if (lane == 0) { s_red[w] = vor; s_red[32 + w] = vand; }
        __syncthreads();
        uint64_t vary = 0;
        {
            uint64_t a = 0, b = ~0ull;
            for (int i = 0; i < kSmWarps; ++i) { a |= s_red[i]; b &= s_red[32 + i]; }
            vary = a ^ b;  // bits that differ between some two keys
        }
        uint16_t* cur = s_idx0;
        uint16_t* nxt = s_idx1;
        for (int pass = 0; pass < kPasses; ++pass) {
            const int shift = 8 * pass;
            if (((vary >> shift) & 255u) == 0u) continue;  // digit constant: identity pass
            uint32_t rank[kSmItems], idx[kSmItems];
            const uint32_t wbase = w * 32 * kSmItems + lane;
#pragma unroll
            for (int i = 0; i < kSmItems; ++i) idx[i] = (wbase + i * 32 < n) ? cur[wbase + i * 32] : 0u;
            auto digit_of = [&](int i) -> uint32_t {
                return (wbase + i * 32 < n) ? ((uint32_t)(s_keys[idx[i]] >> shift) & 255u) : (uint32_t)kRadix;
            };
            block_rank<kSmWarps, kSmItems>(digit_of, rank, s_hist, s_total, s_start, s_warp, NoOp());
#pragma unroll
            for (int i = 0; i < kSmItems; ++i)
                if (wbase + i * 32 < n && rank[i] < n) nxt[rank[i]] = (uint16_t)idx[i];
            __syncthreads();
            uint16_t* t = cur; cur = nxt; nxt = t;
        }
        for (uint32_t j = tid; j < n; j += kSmThreads) {
            const uint32_t src = cur[j];
            kout[base + j] = s_keys[src] ^ flip_out;
            if (PAY) pout[base + j] = pin[base + src];
        }
        __syncthreads();
    }
}

static size_t small_sort_smem() {
    return (size_t)kSmallCap * 8 + 2 * (size_t)kSmallCap * 2 + (size_t)kSmWarps * kRadix * 4 + 2 * kRadix * 4 + 32 * 4 +
           64 * 8;
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

template <bool PAY>
static cudaError_t segsort_t(const uint64_t* src, uint64_t* dst, uint64_t* tmp,
                             const uint32_t* psrc, uint32_t* pdst, uint32_t* ptmp,
                             uint64_t N, uint64_t nseg, const uint64_t* d_seg_off,
                             bool flip_in, bool flip_out, const SegSortWs& ws, cudaStream_t st,
                             SegSortTiming* timing) {
    if (N == 0 || nseg == 0) return cudaSuccess;
    const uint64_t fin = flip_in ? kSignBit : 0ull, fout = flip_out ? kSignBit : 0ull;
    cudaError_t e;
    // Small segments: on chip, straight from src to dst.
    {
        static bool attr_set[2] = {false, false};
        const size_t smem = small_sort_smem();
        if (!attr_set[PAY ? 1 : 0]) {
            e = cudaFuncSetAttribute(k_small_sort<PAY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr_set[PAY ? 1 : 0] = true;
        }
        int dev = 0, nsm = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const uint64_t grid = std::min<uint64_t>(nseg, (uint64_t)nsm * 64);
        HSS_LAUNCH(k_small_sort<PAY>, (unsigned)grid, kSmThreads, smem, st, src, dst, psrc, pdst, d_seg_off, nseg, fin, fout);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // Large segments: histogram + 8 one-sweep passes.
    if (N <= (uint64_t)kSmallCap) return cudaSuccess;  // no segment can be large
    HSS_LAUNCH(k_seg_plan, 1, 1024, 0, st, d_seg_off, nseg, ws.tile_start, ws.counters);
    if ((e = cudaMemsetAsync(ws.digit_off, 0, nseg * kPasses * kRadix * sizeof(uint32_t), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ws.status, 0, ws.max_tiles * kRadix * sizeof(uint32_t), st)) != cudaSuccess) return e;
    {
        // enough CTAs for several waves over the device
        const uint64_t approx_tiles = ceil_div(N, kOsTile);
        uint64_t split = std::max<uint64_t>(1, std::min<uint64_t>(64, ceil_div(approx_tiles, std::max<uint64_t>(nseg, 1) * 16)));
        dim3 g((unsigned)nseg, (unsigned)split);
        HSS_LAUNCH(k_digit_hist, g, 256, 0, st, src, d_seg_off, ws.digit_off, (uint32_t)split, fin);
        dim3 g2((unsigned)nseg, kPasses);
        HSS_LAUNCH(k_digit_scan, g2, 256, 0, st, d_seg_off, ws.digit_off);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const uint64_t grid = ws.max_tiles;  // upper bound; extra CTAs exit at once
    const size_t os_smem = (size_t)kOsTile * 8 + (PAY ? (size_t)kOsTile * 4 : 0);
    {
        static bool os_attr[2] = {false, false};
        if (!os_attr[PAY ? 1 : 0]) {
            e = cudaFuncSetAttribute(k_onesweep<PAY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)os_smem);
            if (e != cudaSuccess) return e;
            os_attr[PAY ? 1 : 0] = true;
        }
    }
    const bool timed = timing && timing->enabled && timing->n < 8;
    if (timed) {
        cudaEventCreate(&timing->ev[timing->n][0]);
        cudaEventCreate(&timing->ev[timing->n][1]);
        cudaEventRecord(timing->ev[timing->n][0], st);
    }
    for (int pass = 0; pass < kPasses; ++pass) {
        // pass writes: even -> tmp, odd -> dst; the last (odd) pass lands in dst
        const uint64_t* in = pass == 0 ? src : ((pass & 1) ? tmp : dst);
        uint64_t* out = (pass & 1) ? dst : tmp;
        const uint32_t* pin = PAY ? (pass == 0 ? psrc : ((pass & 1) ? ptmp : pdst)) : nullptr;
        uint32_t* pout = PAY ? ((pass & 1) ? pdst : ptmp) : nullptr;
        HSS_LAUNCH(k_onesweep<PAY>, (unsigned)grid, kOsThreads, os_smem, st, in, out, pin, pout, d_seg_off, ws.tile_start, nseg,
                   ws.digit_off, ws.status, ws.max_tiles, ws.counters, ws.err, pass, pass == 0 ? fin : 0ull,
                   pass == kPasses - 1 ? fout : 0ull);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (timed) {
        cudaEventRecord(timing->ev[timing->n][1], st);
        timing->launches[timing->n] = kPasses;
        timing->n += 1;
    }
    return cudaSuccess;
}

cudaError_t segsort(const uint64_t* src, uint64_t* dst, uint64_t* tmp,
                    const uint32_t* psrc, uint32_t* pdst, uint32_t* ptmp,
                    uint64_t N, uint64_t nseg, const uint64_t* d_seg_off,
                    bool flip_in, bool flip_out, const SegSortWs& ws, cudaStream_t st,
                    SegSortTiming* timing) {
    if (psrc) return segsort_t<true>(src, dst, tmp, psrc, pdst, ptmp, N, nseg, d_seg_off, flip_in, flip_out, ws, st, timing);
    return segsort_t<false>(src, dst, tmp, nullptr, nullptr, nullptr, N, nseg, d_seg_off, flip_in, flip_out, ws, st, timing);
}

}  // namespace hss
