// rounds_dev.cuh -- device helpers of the splitter rounds shared by the
// single-job kernels (rounds.cu) and the batched ones (batch.cu).
#pragma once

#include "hss_internal.cuh"

namespace hss {

// ---------------------------------------------------------------------------
// Block scans (blockDim a multiple of 32, at most 1024).
// ---------------------------------------------------------------------------
template <typename T, typename Op>
__device__ __forceinline__ T warp_incl_scan(T x, Op op) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x = op(x, y);
    }
    return x;
}

// Inclusive block scan with identity `id`; returns the inclusive value and
// sets `total`.  Uses s_warp[32] of T.
template <typename T, typename Op>
__device__ __forceinline__ T block_incl_scan(T v, T id, Op op, T* s_warp, T& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T x = warp_incl_scan(v, op);
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (w == 0) {
        T y = lane < nw ? s_warp[lane] : id;
        y = warp_incl_scan(y, op);
        s_warp[lane] = y;
    }
    __syncthreads();
    T r = w > 0 ? op(s_warp[w - 1], x) : x;
    total = s_warp[nw - 1];
    __syncthreads();
    return r;
}

struct AddU32 { __device__ uint32_t operator()(uint32_t a, uint32_t b) const { return a + b; } };
struct AddU64 { __device__ uint64_t operator()(uint64_t a, uint64_t b) const { return a + b; } };
struct MaxI32 { __device__ int32_t operator()(int32_t a, int32_t b) const { return a > b ? a : b; } };

__device__ __forceinline__ uint64_t ideal_rank(uint64_t i1, uint64_t N, uint64_t p) {
    return (uint64_t)(((unsigned __int128)i1 * N) / p);  // t_i for splitter number i1 (1-based)
}

// Count of keys in a[0..n) below key: strict (<) or not (<=), branch-free.
__device__ __forceinline__ uint32_t count_below(const uint64_t* __restrict__ a, uint32_t n, uint64_t key, bool strict) {
    uint32_t base = 0;
    while (n > 0) {
        const uint32_t half = n >> 1;
        const uint64_t v = a[base + half];
        const bool go = strict ? (v < key) : (v <= key);
        base = go ? base + half + 1 : base;
        n = go ? n - half - 1 : half;
    }
    return base;
}

// Improve L/U of one splitter with a ranked cut c (Sec. 4.2.2 step 3): L is
// the cut of largest rank <= t, U the cut of smallest rank >= t, equal ranks
// keeping the smaller cut; cl/cu record the probe index that changed them.
__device__ __forceinline__ void offer(DCut& L, DCut& U, int32_t& cl, int32_t& cu, uint64_t t, const DCut& c, int32_t k) {
    if (c.rank <= t && (c.rank > L.rank || (c.rank == L.rank && cut_less(c, L)))) { L = c; cl = k; }
    if (c.rank >= t && (c.rank < U.rank || (c.rank == U.rank && cut_less(c, U)))) { U = c; cu = k; }
}

struct IntervalsOut {
    uint64_t gamma, T;
    uint32_t nint, unresolved, take_all;
};

// Resolved flags, distinct unresolved intervals (their representative
// splitters into int_rep), |gamma| and the next threshold of one job, by one
// CTA of up to 1024 threads walking the splitters in chunks.  The outputs are
// valid in thread 0.
// With int_T non-null, every distinct interval u also gets the threshold of
// the equal-per-interval schedule: probability (s p / nint) / its length.
__device__ __forceinline__ void intervals_body(uint32_t S, uint64_t N, uint32_t p, uint64_t tol, float oversample,
                                               const DCut* __restrict__ Lcut, const DCut* __restrict__ Ucut,
                                               uint32_t* __restrict__ res, uint32_t* __restrict__ int_rep,
                                               IntervalsOut& out, uint64_t* __restrict__ int_T = nullptr,
                                               uint32_t* __restrict__ int_all = nullptr) {
    __shared__ uint32_t s_u32[32];
    __shared__ int32_t s_i32[32];
    __shared__ uint64_t s_u64[32];
    uint32_t carry_heads = 0, carry_f = 0, carry_unres = 0;
    int32_t carry_max = -1;
    uint64_t gamma = 0;
    for (uint32_t base = 0; base < S; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const bool valid = i < S;
        uint32_t head = 0, unres = 0;
        uint64_t glen = 0;
        if (valid) {
            const DCut L = Lcut[i], U = Ucut[i];
            const uint64_t t = ideal_rank(i + 1, N, p);
            const bool r = (t - L.rank) <= tol || (U.rank - t) <= tol;
            res[i] = r ? 1u : 0u;
            unres = r ? 0u : 1u;
            head = (i == 0) || !(cut_equal(L, Lcut[i - 1]) && cut_equal(U, Ucut[i - 1]));
            glen = U.rank - L.rank - (L.kind == kMember ? 1u : 0u);
        }
        uint32_t tot;
        const uint32_t heads_incl = block_incl_scan<uint32_t>(head, 0u, AddU32(), s_u32, tot) + carry_heads;
        carry_heads += tot;
        const int32_t rid = (int32_t)heads_incl - 1;
        int32_t mtot;
        const int32_t mv = unres ? rid : -1;
        int32_t mincl = block_incl_scan<int32_t>(mv, -1, MaxI32(), s_i32, mtot);
        mincl = mincl > carry_max ? mincl : carry_max;
        int32_t mexcl = __shfl_up_sync(0xffffffffu, mincl, 1);
        // lane 0 needs the previous warp's last value
        __shared__ int32_t s_last[32];
        if ((threadIdx.x & 31) == 31) s_last[threadIdx.x >> 5] = mincl;
        __syncthreads();
        if ((threadIdx.x & 31) == 0) mexcl = (threadIdx.x == 0) ? carry_max : s_last[(threadIdx.x >> 5) - 1];
        __syncthreads();
        carry_max = carry_max > mtot ? carry_max : mtot;
        const uint32_t f = (valid && unres && mexcl != rid) ? 1u : 0u;
        uint32_t ftot;
        const uint32_t fincl = block_incl_scan<uint32_t>(f, 0u, AddU32(), s_u32, ftot);
        if (f) int_rep[carry_f + fincl - 1] = i;
        carry_f += ftot;
        uint32_t utot;
        block_incl_scan<uint32_t>(unres, 0u, AddU32(), s_u32, utot);
        carry_unres += utot;
        uint64_t gtot;
        block_incl_scan<uint64_t>(f ? glen : 0ull, 0ull, AddU64(), s_u64, gtot);
        gamma += gtot;
    }
    if (int_T) {
        __syncthreads();  // int_rep is complete
        const double per_int = carry_f ? ((double)oversample * (double)p) / (double)carry_f : 0.0;
        for (uint32_t u = threadIdx.x; u < carry_f; u += blockDim.x) {
            const uint32_t rep = int_rep[u];
            const DCut L = Lcut[rep], U = Ucut[rep];
            const uint64_t len = U.rank - L.rank - (L.kind == kMember ? 1u : 0u);
            const double q = len ? per_int / (double)len : 1.0;
            if (q >= 1.0) { int_all[u] = 1u; int_T[u] = 0ull; }
            else { int_all[u] = 0u; int_T[u] = (uint64_t)floor(ldexp(q, 64)); }
        }
    }
    if (threadIdx.x == 0) {
        out.gamma = gamma;
        out.nint = carry_f;
        out.unresolved = carry_unres;
        double q = gamma == 0 ? 1.0 : ((double)oversample * (double)p) / (double)gamma;
        if (q >= 1.0) {
            out.take_all = 1u;
            out.T = 0ull;
        } else {
            out.take_all = 0u;
            out.T = (uint64_t)floor(ldexp(q, 64));
        }
    }
}

// ---------------------------------------------------------------------------
// Sampling helpers.
// ---------------------------------------------------------------------------
constexpr int kIntChunk = 2048;
constexpr int kSampThreads = 256;

// Fill the interval ranges of segment s for intervals [u0, u0+nu) and the
// exclusive prefix of their position-pair counts.  Returns the pair total.
__device__ __forceinline__ uint32_t load_seg_intervals(uint32_t s, uint32_t n_s, uint32_t S, uint32_t u0, uint32_t nu,
                                       const uint32_t* __restrict__ Lpos, const uint32_t* __restrict__ Upos,
                                       const DCut* __restrict__ Lcut, const uint32_t* __restrict__ int_rep,
                                       uint32_t* s_a, uint32_t* s_b, uint32_t* s_pre, uint32_t* s_warp) {
    constexpr int kPer = kIntChunk / kSampThreads;
    uint32_t loc[kPer];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const uint32_t u = threadIdx.x * kPer + k;
        uint32_t np = 0;
        if (u < nu) {
            const uint32_t rep = int_rep[u0 + u];
            const DCut L = Lcut[rep];
            uint32_t a = Lpos[(uint64_t)s * S + rep];
            if (L.kind == kMember && (uint32_t)L.seg == s) a += 1;
            uint32_t b = Upos[(uint64_t)s * S + rep];
            if (b > n_s) b = n_s;  // defensive: a range never leaves its segment
            s_a[u] = a;
            s_b[u] = b;
            np = b > a ? ((b - 1) >> 1) - (a >> 1) + 1 : 0u;
        }
        loc[k] = sum;
        sum += np;
    }
    uint32_t tot;
    const uint32_t incl = block_incl_scan<uint32_t>(sum, 0u, AddU32(), s_warp, tot);
    const uint32_t ex = incl - sum;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const uint32_t u = threadIdx.x * kPer + k;
        if (u < nu) s_pre[u] = ex + loc[k];
    }
    if (threadIdx.x == 0) s_pre[nu] = tot;
    __syncthreads();
    return tot;
}

__device__ __forceinline__ uint32_t find_interval(const uint32_t* s_pre, uint32_t nu, uint32_t f) {
    uint32_t lo = 0, hi = nu;  // last u with s_pre[u] <= f
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s_pre[mid] <= f) lo = mid; else hi = mid;
    }
    return lo;
}

// Visit the pairs f in [0, P) of one interval chunk, body(u, f) with u the
// interval of pair f.  Each thread takes a contiguous block of pairs, so one
// search finds the interval of its first pair and the others follow by a
// forward walk over the (non-decreasing) interval starts.
template <class Body>
__device__ __forceinline__ void for_each_pair(const uint32_t* s_pre, uint32_t nu, uint32_t P, Body body) {
    const uint32_t per = (P + kSampThreads - 1) / kSampThreads;
    const uint32_t f0 = min(P, threadIdx.x * per), f1 = min(P, f0 + per);
    if (f0 >= f1) return;
    uint32_t u = find_interval(s_pre, nu, f0);
    for (uint32_t f = f0; f < f1; ++f) {
        while (u + 1 < nu && s_pre[u + 1] <= f) ++u;
        body(u, f);
    }
}

}  // namespace hss
