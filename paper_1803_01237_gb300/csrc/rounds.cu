// rounds.cu -- splitter determination of HSS (Sec. 4.2.2) on one GB300.
//
// The p processors are the p locally sorted segments of one device array.
// One round:
//   sample   every key strictly inside a distinct unresolved splitter
//            interval is kept with probability q = min(1, s p/|gamma|) by
//            comparing its Philox4x32-10 word with T = floor(q 2^64); the
//            draw needs only (segment, position, round), so keys are read
//            only for the keys that are kept.  A CTA per segment walks the
//            interval ranges of its segment, marks a bitmap and counts; a
//            second pass writes the kept keys in (segment, position) order.
//   sort     the probes, stably by key (the segmented radix sort with one
//            segment), i.e. in (key, segment, position) tag order.
//   histogram the exact global rank of every probe: for every segment a
//            branch-free binary search confined to the probe's interval,
//            giving also the per-segment counts the next round and the
//            exchange need.
//   update   L_i / U_i move to the best-ranked probe at or below / at or above
//            t_i = floor(iN/p); a splitter resolves when one of them is within
//            tol = floor(N eps/(2p)) of t_i; the distinct unresolved intervals,
//            |gamma| and the next threshold are computed on the device.
// The host reads one small status record per round.
#include "rounds.cuh"
#include "rounds_dev.cuh"

#include <cmath>
#include <algorithm>
#include <mutex>
#include <vector>

namespace hss {

// Probe count argument meaning "read it from the control record" (the
// device-driven loop, where the host does not know a round's sample size).
constexpr uint64_t kZFromCtl = ~0ull;

static inline uint64_t cdiv(uint64_t a, uint64_t b) { return (a + b - 1) / b; }
static inline size_t aup(size_t x) { return (x + 255) / 256 * 256; }

uint64_t sample_capacity(uint64_t N, uint64_t p, float oversample) {
    const double want = std::ceil(2.0 * (double)oversample * (double)p) + 4096.0;
    uint64_t cap = (uint64_t)std::min<double>(want, (double)std::max<uint64_t>(N, 1));
    return std::max<uint64_t>(cap, 1);
}

size_t rounds_ws_bytes(uint64_t N, uint64_t p, uint64_t cap, uint64_t nb) {
    const uint64_t NB = nb ? nb : p;
    const uint64_t S = NB > 0 ? NB - 1 : 0;
    const uint64_t S1 = std::max<uint64_t>(S, 1);
    size_t b = 0;
    b += aup(sizeof(RoundCtl));
    b += 2 * aup(S1 * sizeof(DCut));
    b += 2 * aup(p * S1 * sizeof(uint32_t));
    b += 6 * aup(S1 * sizeof(uint32_t));
    b += aup(S1 * sizeof(uint64_t)) + aup(S1 * sizeof(uint32_t));  // int_T, int_all
    b += aup((N / 32 + 2) * sizeof(uint32_t));
    b += aup(p * sizeof(uint32_t)) + aup((p + 1) * sizeof(uint32_t));
    b += 3 * aup(cap * sizeof(uint64_t));      // skey, skey_sorted, stmp
    b += 5 * aup(cap * sizeof(uint32_t));      // sseg, sspos, siota, sperm, ptmp
    b += aup(cap * sizeof(uint64_t)) * 2;      // pkey, prank
    b += 3 * aup(cap * sizeof(uint32_t));      // pseg, pspos, pint
    b += aup(p * cap * sizeof(uint32_t));      // probe_pos
    b += aup(S1 * sizeof(uint64_t)) + aup(S1 * sizeof(uint32_t));  // fin_okey, fin_kind
    b += 2 * aup(p * sizeof(uint64_t));                             // bucket_lo, bucket_mult
    b += aup(2 * sizeof(uint64_t));                                 // key_range
    b += segsort_ws_bytes(cap, 1);
    return b;
}

RoundWs rounds_ws_carve(void* base, uint64_t N, uint64_t p, uint64_t cap, uint32_t* err, uint64_t nb) {
    const uint64_t NB = nb ? nb : p;
    const uint64_t S = NB > 0 ? NB - 1 : 0;
    const uint64_t S1 = std::max<uint64_t>(S, 1);
    RoundWs w;
    char* q = (char*)base;
    auto take = [&](size_t bytes) { void* r = q; q += aup(bytes); return r; };
    w.ctl = (RoundCtl*)take(sizeof(RoundCtl));
    w.Lcut = (DCut*)take(S1 * sizeof(DCut));
    w.Ucut = (DCut*)take(S1 * sizeof(DCut));
    w.Lpos = (uint32_t*)take(p * S1 * sizeof(uint32_t));
    w.Upos = (uint32_t*)take(p * S1 * sizeof(uint32_t));
    w.res = (uint32_t*)take(S1 * sizeof(uint32_t));
    w.chgL = (int32_t*)take(S1 * sizeof(uint32_t));
    w.chgU = (int32_t*)take(S1 * sizeof(uint32_t));
    w.choose_u = (uint32_t*)take(S1 * sizeof(uint32_t));
    w.int_rep = (uint32_t*)take(S1 * sizeof(uint32_t));
    w.int_T = (uint64_t*)take(S1 * sizeof(uint64_t));
    w.int_all = (uint32_t*)take(S1 * sizeof(uint32_t));
    take(S1 * sizeof(uint32_t));
    w.bitmap = (uint32_t*)take((N / 32 + 2) * sizeof(uint32_t));
    w.seg_cnt = (uint32_t*)take(p * sizeof(uint32_t));
    w.seg_cnt_off = (uint32_t*)take((p + 1) * sizeof(uint32_t));
    w.skey = (uint64_t*)take(cap * sizeof(uint64_t));
    w.skey_sorted = (uint64_t*)take(cap * sizeof(uint64_t));
    w.stmp = (uint64_t*)take(cap * sizeof(uint64_t));
    w.sseg = (uint32_t*)take(cap * sizeof(uint32_t));
    w.sspos = (uint32_t*)take(cap * sizeof(uint32_t));
    w.siota = (uint32_t*)take(cap * sizeof(uint32_t));
    w.sperm = (uint32_t*)take(cap * sizeof(uint32_t));
    w.ptmp = (uint32_t*)take(cap * sizeof(uint32_t));
    w.pkey = (uint64_t*)take(cap * sizeof(uint64_t));
    w.prank = (uint64_t*)take(cap * sizeof(uint64_t));
    w.pseg = (int32_t*)take(cap * sizeof(uint32_t));
    w.pspos = (uint32_t*)take(cap * sizeof(uint32_t));
    w.pint = (uint32_t*)take(cap * sizeof(uint32_t));
    w.probe_pos = (uint32_t*)take(p * cap * sizeof(uint32_t));
    w.fin_okey = (uint64_t*)take(S1 * sizeof(uint64_t));
    w.fin_kind = (uint32_t*)take(S1 * sizeof(uint32_t));
    w.bucket_lo = (uint64_t*)take(p * sizeof(uint64_t));
    w.bucket_mult = (uint64_t*)take(p * sizeof(uint64_t));
    w.key_range = (uint64_t*)take(2 * sizeof(uint64_t));
    w.sws = segsort_ws_carve(q, cap, 1, err);
    w.cap = cap;
    return w;
}

// ---------------------------------------------------------------------------
// Initial state: every splitter interval is (-inf, +inf).
// ---------------------------------------------------------------------------
__global__ void k_rounds_init(const uint64_t* __restrict__ seg_off, uint32_t S, uint64_t N, DCut* Lcut, DCut* Ucut,
                              uint32_t* Lpos, uint32_t* Upos) {
    const uint64_t s = blockIdx.x;
    const uint32_t i = blockIdx.y * blockDim.x + threadIdx.x;
    if (i >= S) return;
    const uint32_t n = (uint32_t)(seg_off[s + 1] - seg_off[s]);
    Lpos[s * S + i] = 0;
    Upos[s * S + i] = n;
    if (s == 0) {
        DCut a; a.okey = 0; a.seg = -2; a.spos = 0; a.rank = 0; a.kind = kNegInf; a.pad = 0;
        DCut b; b.okey = 0; b.seg = -3; b.spos = 0; b.rank = N; b.kind = kPosInf; b.pad = 0;
        Lcut[i] = a;
        Ucut[i] = b;
    }
}

// ---------------------------------------------------------------------------
// Resolved flags, distinct unresolved intervals, |gamma| and the threshold.
// One CTA of 1024 threads walks the splitters in chunks.
// ---------------------------------------------------------------------------
// schedule THEORY: the next round's threshold comes from the host (T_ovr,
// all_ovr); EQUAL: per-interval thresholds into int_T / int_all.
__global__ __launch_bounds__(1024) void k_intervals(uint32_t S, uint64_t N, uint32_t p, uint64_t tol, float oversample,
                                                    const DCut* __restrict__ Lcut, const DCut* __restrict__ Ucut,
                                                    uint32_t* __restrict__ res, uint32_t* __restrict__ int_rep,
                                                    RoundCtl* ctl, uint32_t schedule, uint64_t T_ovr, uint32_t all_ovr,
                                                    uint64_t* __restrict__ int_T, uint32_t* __restrict__ int_all) {
    IntervalsOut o;
    const bool equal = schedule == HSS_SCHEDULE_EQUAL;
    intervals_body(S, N, p, tol, oversample, Lcut, Ucut, res, int_rep, o, equal ? int_T : nullptr,
                   equal ? int_all : nullptr);
    if (threadIdx.x == 0) {
        ctl->gamma = o.gamma;
        ctl->nint = o.nint;
        ctl->unresolved = o.unresolved;
        const bool theory = schedule == HSS_SCHEDULE_THEORY;
        ctl->take_all = theory ? all_ovr : o.take_all;
        ctl->T = theory ? T_ovr : o.T;
    }
}

// ---------------------------------------------------------------------------
// Sampling.
// ---------------------------------------------------------------------------
// Round-j Bernoulli marks of segment blockIdx.x (Sec. 4.2.2 step 4, Sec. 6):
// every key of an unresolved interval draws its Philox word and is kept when
// the word is below the round's threshold.  gridDim.y CTAs share a segment,
// each taking an equal share of its position pairs; each thread walks a
// contiguous run of pairs two at a time (two independent Philox chains in
// flight) and the CTA adds its count to seg_cnt[s] (zeroed before the round).
// Philox4x32-10 of the counters (m, seg, round, 0) for one (seed, seg,
// round): the round keys and the parts of the first two rounds that do not
// depend on m are computed once, so a word pair costs 18 of the 20
// multiplies and none of the key additions.  Same words as sample_words.
struct PairDraw {
    uint32_t k0[10], k1[10];  // round keys
    uint32_t c0_1, c1_1;      // words 0 and 1 after round 1 (independent of m)
    uint32_t lo0_2, hi0_2;    // M0 x (word 0 after round 1), used in round 2
    __device__ __forceinline__ void init(uint64_t seed, uint32_t seg, uint32_t round) {
        const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u, M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
        uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
#pragma unroll
        for (int r = 0; r < 10; ++r) { k0[r] = a; k1[r] = b; a += W0; b += W1; }
        // round 1 on (m, seg, round, 0): the M1 product and the new word 0
        // involve only seg and round
        const uint32_t lo1 = M1 * round, hi1 = __umulhi(M1, round);
        c0_1 = hi1 ^ seg ^ k0[0];
        c1_1 = lo1;
        lo0_2 = M0 * c0_1;
        hi0_2 = __umulhi(M0, c0_1);
    }
    __device__ __forceinline__ void words(uint32_t m, uint64_t& even, uint64_t& odd) const {
        const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
        // round 1: only the M0 x m product varies
        const uint32_t lo0 = M0 * m, hi0 = __umulhi(M0, m);
        uint32_t c2 = hi0 ^ k1[0];  // ^ word 3 (0)
        uint32_t c3 = lo0;
        uint32_t c0 = c0_1, c1 = c1_1;
        // round 2: the M0 product is known
        {
            const uint32_t l1 = M1 * c2, h1 = __umulhi(M1, c2);
            const uint32_t n0 = h1 ^ c1 ^ k0[1];
            const uint32_t n2 = hi0_2 ^ c3 ^ k1[1];
            c0 = n0; c1 = l1; c2 = n2; c3 = lo0_2;
        }
#pragma unroll
        for (int r = 2; r < 10; ++r) {
            const uint32_t l0 = M0 * c0, h0 = __umulhi(M0, c0);
            const uint32_t l1 = M1 * c2, h1 = __umulhi(M1, c2);
            const uint32_t n0 = h1 ^ c1 ^ k0[r];
            const uint32_t n2 = h0 ^ c3 ^ k1[r];
            c0 = n0; c1 = l1; c2 = n2; c3 = l0;
        }
        even = ((uint64_t)c1 << 32) | c0;
        odd = ((uint64_t)c3 << 32) | c2;
    }
};

__device__ __forceinline__ void mark_pair(uint32_t a, uint32_t b, uint32_t m, uint64_t w0, uint64_t w1, uint64_t Tu,
                                          bool all_u, uint64_t base, uint32_t* __restrict__ bitmap, uint32_t& cnt) {
    const uint32_t p0 = 2 * m, p1 = 2 * m + 1;
    if (p0 >= a && p0 < b && (all_u || w0 < Tu)) {
        const uint64_t g = base + p0;
        atomicOr(&bitmap[g >> 5], 1u << (g & 31));
        ++cnt;
    }
    if (p1 >= a && p1 < b && (all_u || w1 < Tu)) {
        const uint64_t g = base + p1;
        atomicOr(&bitmap[g >> 5], 1u << (g & 31));
        ++cnt;
    }
}

__global__ __launch_bounds__(kSampThreads, 4) void k_sample_mark(
    const uint64_t* __restrict__ seg_off, uint32_t S, const uint32_t* __restrict__ Lpos, const uint32_t* __restrict__ Upos,
    const DCut* __restrict__ Lcut, const uint32_t* __restrict__ int_rep, const RoundCtl* __restrict__ ctl,
    uint64_t seed, uint32_t round, uint32_t* __restrict__ bitmap, uint32_t* __restrict__ seg_cnt,
    const uint64_t* __restrict__ int_T, const uint32_t* __restrict__ int_all) {
    __shared__ uint32_t s_a[kIntChunk], s_b[kIntChunk], s_pre[kIntChunk + 1];
    __shared__ uint32_t s_warp[32];
    const uint32_t s = blockIdx.x;
    const uint64_t base = seg_off[s];
    if (round == 0) {  // device-driven loop: the next round and the seed come from the control record
        round = ctl->round + 1;
        seed = ctl->seed;
    }
    const uint32_t nint = ctl->nint;
    const uint64_t T = ctl->T;
    const bool take_all = ctl->take_all != 0;
    PairDraw pd;
    pd.init(seed, s, round);
    uint32_t cnt = 0;
    for (uint32_t u0 = 0; u0 < nint; u0 += kIntChunk) {
        const uint32_t nu = min((uint32_t)kIntChunk, nint - u0);
        const uint32_t P = load_seg_intervals(s, (uint32_t)(seg_off[s + 1] - base), S, u0, nu, Lpos, Upos, Lcut, int_rep,
                                              s_a, s_b, s_pre, s_warp);
        // this CTA's share of the pairs, then each thread's run of it
        const uint32_t F0 = (uint32_t)(((uint64_t)P * blockIdx.y) / gridDim.y);
        const uint32_t F1 = (uint32_t)(((uint64_t)P * (blockIdx.y + 1)) / gridDim.y);
        const uint32_t per = (F1 - F0 + kSampThreads - 1) / kSampThreads;
        const uint32_t f0 = min(F1, F0 + threadIdx.x * per), f1 = min(F1, f0 + per);
        if (f0 < f1) {
            uint32_t u = find_interval(s_pre, nu, f0);
            auto thr = [&](uint32_t uu, uint64_t& Tu, bool& all_u) {
                Tu = T;
                all_u = take_all;
                if (int_T) {  // equal-per-interval schedule
                    Tu = int_T[u0 + uu];
                    all_u = int_all[u0 + uu] != 0u;
                }
            };
            uint32_t f = f0;
            for (; f + 1 < f1; f += 2) {
                while (u + 1 < nu && s_pre[u + 1] <= f) ++u;
                uint32_t v = u;
                while (v + 1 < nu && s_pre[v + 1] <= f + 1) ++v;
                const uint32_t m0 = (s_a[u] >> 1) + (f - s_pre[u]);
                const uint32_t m1 = (s_a[v] >> 1) + (f + 1 - s_pre[v]);
                uint64_t x0, x1, y0, y1;
                pd.words(m0, x0, x1);
                pd.words(m1, y0, y1);
                uint64_t Tu, Tv;
                bool au, av;
                thr(u, Tu, au);
                thr(v, Tv, av);
                mark_pair(s_a[u], s_b[u], m0, x0, x1, Tu, au, base, bitmap, cnt);
                mark_pair(s_a[v], s_b[v], m1, y0, y1, Tv, av, base, bitmap, cnt);
                u = v;
            }
            if (f < f1) {
                while (u + 1 < nu && s_pre[u + 1] <= f) ++u;
                const uint32_t m0 = (s_a[u] >> 1) + (f - s_pre[u]);
                uint64_t x0, x1, Tu;
                bool au;
                pd.words(m0, x0, x1);
                thr(u, Tu, au);
                mark_pair(s_a[u], s_b[u], m0, x0, x1, Tu, au, base, bitmap, cnt);
            }
        }
        __syncthreads();
    }
    uint32_t tot;
    block_incl_scan<uint32_t>(cnt, 0u, AddU32(), s_warp, tot);
    if (threadIdx.x == 0 && tot) atomicAdd(&seg_cnt[s], tot);
}

// CTAs per segment of the marking pass: about 16K position pairs each in a
// round that samples whole segments, at most 8 (each one reads the
// segment's intervals).
static unsigned mark_chunks(uint64_t N, uint32_t p) {
    const uint64_t pairs = (N / std::max<uint32_t>(p, 1) + 1) / 2;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(8, pairs / 16384));
}

__global__ __launch_bounds__(1024) void k_count_scan(const uint32_t* __restrict__ seg_cnt, uint32_t p, uint32_t* __restrict__ seg_cnt_off,
                                                     uint64_t cap, RoundCtl* ctl) {
    __shared__ uint32_t s_warp[32];
    uint64_t carry = 0;
    for (uint32_t base = 0; base < p; base += blockDim.x) {
        const uint32_t s = base + threadIdx.x;
        const uint32_t v = s < p ? seg_cnt[s] : 0u;
        uint32_t tot;
        const uint32_t incl = block_incl_scan<uint32_t>(v, 0u, AddU32(), s_warp, tot);
        if (s < p) seg_cnt_off[s] = (uint32_t)(carry + incl - v < 0xffffffffull ? carry + incl - v : 0xffffffffull);
        carry += tot;
    }
    if (threadIdx.x == 0) {
        seg_cnt_off[p] = (uint32_t)(carry < 0xffffffffull ? carry : 0xffffffffull);
        ctl->Z = carry;
        ctl->seg_off_z[0] = 0;
        ctl->seg_off_z[1] = carry < cap ? carry : cap;
    }
}

// Write the kept keys of each segment, in position order, at the segment's
// offset of the sample buffer.  Kept keys are exactly the set bits of the
// bitmap inside the segment, so the pass scans the segment's bitmap words and
// skips empty runs of them.
__global__ __launch_bounds__(kSampThreads) void k_sample_write(
    const uint64_t* __restrict__ skeys, const uint64_t* __restrict__ seg_off, const uint32_t* __restrict__ bitmap,
    const uint32_t* __restrict__ seg_cnt, const uint32_t* __restrict__ seg_cnt_off, uint64_t cap,
    uint64_t* __restrict__ skey, uint32_t* __restrict__ sseg, uint32_t* __restrict__ sspos, uint32_t* __restrict__ siota) {
    __shared__ uint32_t s_warp[32];
    const uint32_t s = blockIdx.x;
    const uint32_t want = seg_cnt[s];
    if (want == 0) return;
    const uint64_t base = seg_off[s], end = seg_off[s + 1];
    const uint64_t w0 = base >> 5, w1 = (end + 31) >> 5;
    uint64_t out = seg_cnt_off[s];
    uint32_t found = 0;
    for (uint64_t wb = w0; wb < w1 && found < want; wb += kSampThreads) {
        const uint64_t wi = wb + threadIdx.x;
        uint32_t bits = 0;
        if (wi < w1) {
            bits = bitmap[wi];
            const uint64_t g0 = wi << 5;
            if (g0 < base) bits &= ~0u << (uint32_t)(base - g0);               // bits of the previous segment
            if (g0 + 32 > end) bits &= (uint32_t)((1ull << (uint32_t)(end - g0)) - 1ull);  // bits of the next
        }
        if (__syncthreads_count(bits != 0u) == 0) continue;
        const uint32_t c = __popc(bits);
        uint32_t tot;
        const uint32_t incl = block_incl_scan<uint32_t>(c, 0u, AddU32(), s_warp, tot);
        uint64_t o = out + incl - c;
        while (bits) {
            const uint32_t b = __ffs(bits) - 1;
            bits &= bits - 1;
            const uint64_t g = (wi << 5) + b;
            if (o < cap) {
                skey[o] = skeys[g];
                sseg[o] = s;
                sspos[o] = (uint32_t)(g - base);
                siota[o] = (uint32_t)o;
            }
            ++o;
        }
        out += tot;
        found += tot;
    }
}

// ---------------------------------------------------------------------------
// Probes: gather the sorted sample, find each probe's interval.
// ---------------------------------------------------------------------------
__global__ void k_probe_build(uint64_t Z, const uint64_t* __restrict__ skey_sorted, const uint32_t* __restrict__ sperm,
                              const uint32_t* __restrict__ sseg, const uint32_t* __restrict__ sspos,
                              const DCut* __restrict__ Ucut, const uint32_t* __restrict__ int_rep, const RoundCtl* __restrict__ ctl,
                              uint64_t* __restrict__ pkey, int32_t* __restrict__ pseg, uint32_t* __restrict__ pspos,
                              uint32_t* __restrict__ pint, uint64_t* __restrict__ prank) {
    const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (Z == kZFromCtl) Z = ctl->seg_off_z[1];
    if (k >= Z) return;
    const uint32_t j = sperm[k];
    DCut c;
    c.okey = skey_sorted[k]; c.seg = (int32_t)sseg[j]; c.spos = sspos[j]; c.rank = 0; c.kind = kMember; c.pad = 0;
    pkey[k] = c.okey; pseg[k] = c.seg; pspos[k] = c.spos; prank[k] = 0;
    uint32_t lo = 0, hi = ctl->nint;  // first interval whose upper cut lies above the probe
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (cut_less(c, Ucut[int_rep[mid]])) hi = mid; else lo = mid + 1;
    }
    pint[k] = lo;
}

constexpr int kHistSegPerBlock = 64;

__global__ __launch_bounds__(256) void k_histogram(
    const uint64_t* __restrict__ skeys, const uint64_t* __restrict__ seg_off, uint32_t p, uint32_t S,
    const uint32_t* __restrict__ Lpos, const uint32_t* __restrict__ Upos, const uint32_t* __restrict__ int_rep,
    const uint64_t* __restrict__ pkey, const int32_t* __restrict__ pseg, const uint32_t* __restrict__ pspos,
    const uint32_t* __restrict__ pint, uint64_t Z, uint64_t* __restrict__ prank, uint32_t* __restrict__ probe_pos,
    uint64_t cap, uint32_t* __restrict__ err, const RoundCtl* __restrict__ ctl) {
    __shared__ uint64_t s_part[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (Z == kZFromCtl) {  // device-driven loop: this form runs unless the round is staged
        if (ctl->staged) return;
        Z = ctl->seg_off_z[1];
        if ((uint64_t)blockIdx.x * 32 >= Z) return;
    }
    const uint64_t k = (uint64_t)blockIdx.x * 32 + lane;
    const bool valid = k < Z;
    uint64_t key = 0; int32_t seg = 0; uint32_t spos = 0, rep = 0;
    if (valid) { key = pkey[k]; seg = pseg[k]; spos = pspos[k]; rep = int_rep[pint[k]]; }
    uint64_t partial = 0;
#pragma unroll 2
    for (int j = 0; j < kHistSegPerBlock / 8; ++j) {
        const uint32_t s = blockIdx.y * kHistSegPerBlock + j * 8 + w;
        if (valid && s < p) {
            uint32_t pos;
            if ((int32_t)s == seg) {
                pos = spos;
            } else {
                const uint32_t lo = Lpos[(uint64_t)s * S + rep], hi = Upos[(uint64_t)s * S + rep];
                const uint32_t n = (uint32_t)(seg_off[s + 1] - seg_off[s]);
                if (lo <= hi && hi <= n) {
                    pos = lo + count_below(skeys + seg_off[s] + lo, hi - lo, key, (int32_t)s > seg);
                } else {  // inconsistent interval state: record, do not read out of range
                    atomicOr(err, kDevErrBounds);
                    pos = lo;
                }
            }
            probe_pos[(uint64_t)s * cap + k] = pos;
            partial += pos;
        }
    }
    s_part[w][lane] = partial;
    __syncthreads();
    if (w == 0 && valid) {
        uint64_t sum = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) sum += s_part[i][lane];
        atomicAdd((unsigned long long*)&prank[k], (unsigned long long)sum);
    }
}

// The histogram of a round whose probes all share one interval (round 1,
// and the proposal pass: every interval is then the whole key range).  A CTA
// ranks kStgProbes consecutive sorted probes in kStgSegs segments.  In each
// segment their positions lie between the rank of the first probe (strict
// compare) and that of the last (non-strict), so the keys in between are
// staged in shared memory once and every probe is searched there.  Same
// positions as k_histogram; per segment and probe block about one read of
// the keys between the block's first and last probe, instead of one search
// of the whole segment in HBM per probe.
constexpr int kStgThreads = 256;
constexpr int kStgPer = 4;                          // probes per thread
constexpr int kStgProbes = kStgThreads * kStgPer;   // probes per CTA
constexpr int kStgSegs = 32;                        // segments per CTA
constexpr uint32_t kStgCap = 4096;                  // staged keys (32 KB)

__global__ __launch_bounds__(kStgThreads) void k_histogram_staged(
    const uint64_t* __restrict__ skeys, const uint64_t* __restrict__ seg_off, uint32_t p, uint32_t S,
    const uint32_t* __restrict__ Lpos, const uint32_t* __restrict__ Upos, const uint32_t* __restrict__ int_rep,
    const uint64_t* __restrict__ pkey, const int32_t* __restrict__ pseg, const uint32_t* __restrict__ pspos,
    uint64_t Z, uint64_t* __restrict__ prank, uint32_t* __restrict__ probe_pos, uint64_t cap,
    uint32_t* __restrict__ err, const RoundCtl* __restrict__ ctl) {
    __shared__ uint64_t s_keys[kStgCap];
    __shared__ uint32_t s_lo[kStgSegs], s_a[kStgSegs], s_b[kStgSegs], s_ok[kStgSegs];
    if (Z == kZFromCtl) {  // device-driven loop: this form runs only when the round is staged
        if (!ctl->staged) return;
        Z = ctl->seg_off_z[1];
    }
    const uint64_t k0 = (uint64_t)blockIdx.x * kStgProbes;
    if (k0 >= Z) return;
    const uint64_t k1 = min(Z, k0 + (uint64_t)kStgProbes);
    const uint32_t s0 = blockIdx.y * kStgSegs;
    const uint32_t rep = int_rep[0];
    uint64_t key[kStgPer], part[kStgPer];
    int32_t seg[kStgPer];
    uint32_t spos[kStgPer];
#pragma unroll
    for (int u = 0; u < kStgPer; ++u) {
        const uint64_t k = k0 + threadIdx.x + (uint64_t)u * kStgThreads;
        part[u] = 0;
        key[u] = 0; seg[u] = 0; spos[u] = 0;
        if (k < k1) { key[u] = pkey[k]; seg[u] = pseg[k]; spos[u] = pspos[k]; }
    }
    // bounds of the block's probes in each segment, by 2 kStgSegs threads
    if (threadIdx.x < 2 * kStgSegs) {
        const uint32_t i = threadIdx.x >> 1, s = s0 + i;
        if (s < p) {
            const uint32_t n = (uint32_t)(seg_off[s + 1] - seg_off[s]);
            const uint32_t lo = Lpos[(uint64_t)s * S + rep], hi = Upos[(uint64_t)s * S + rep];
            const bool ok = lo <= hi && hi <= n;
            uint32_t v = 0;
            if (ok) {
                const uint64_t* w = skeys + seg_off[s] + lo;
                v = (threadIdx.x & 1) ? count_below(w, hi - lo, pkey[k1 - 1], false)
                                      : count_below(w, hi - lo, pkey[k0], true);
            }
            if (threadIdx.x & 1) {
                s_b[i] = v;
            } else {
                s_a[i] = v;
                s_lo[i] = lo;
                s_ok[i] = ok ? 1u : 0u;
            }
        }
    }
    __syncthreads();
    for (int i = 0; i < kStgSegs; ++i) {
        const uint32_t s = s0 + i;
        if (s >= p) break;  // uniform per CTA
        const uint32_t lo = s_lo[i], a = s_a[i];
        const bool ok = s_ok[i] != 0u;
        const uint32_t m = ok ? s_b[i] - a : 0u;
        const bool staged = m <= kStgCap;
        const uint64_t* w = skeys + seg_off[s] + lo + a;
        if (ok && staged)
            for (uint32_t j = threadIdx.x; j < m; j += kStgThreads) s_keys[j] = w[j];
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kStgPer; ++u) {
            const uint64_t k = k0 + threadIdx.x + (uint64_t)u * kStgThreads;
            if (k >= k1) continue;
            uint32_t pos;
            if ((int32_t)s == seg[u]) pos = spos[u];
            else if (!ok) pos = lo;  // inconsistent interval state: recorded below, nothing read
            else if (staged) pos = lo + a + count_below(s_keys, m, key[u], (int32_t)s > seg[u]);
            else pos = lo + a + count_below(w, m, key[u], (int32_t)s > seg[u]);
            probe_pos[(uint64_t)s * cap + k] = pos;
            part[u] += pos;
        }
        if (!ok && threadIdx.x == 0) atomicOr(err, kDevErrBounds);
        __syncthreads();  // s_keys is rewritten for the next segment
    }
#pragma unroll
    for (int u = 0; u < kStgPer; ++u) {
        const uint64_t k = k0 + threadIdx.x + (uint64_t)u * kStgThreads;
        if (k < k1) atomicAdd((unsigned long long*)&prank[k], (unsigned long long)part[u]);
    }
}

// ---------------------------------------------------------------------------
// Proposed cuts (a learned splitter proposal): non-member cuts (k, -1) that
// sort before every input key equal to k.  They are ranked and offered to the
// splitters like probes before the first round.
// ---------------------------------------------------------------------------
// Before round 1 every splitter's interval is (-inf, +inf), so every cut is
// searched over whole segments: interval 0 with representative splitter 0
// (whose per-segment bounds are still 0 and the segment length), whatever the
// resolved flags say.
__global__ void k_prop_load(const uint64_t* __restrict__ prop, uint32_t nprop, uint64_t flip, uint64_t* __restrict__ okey,
                            RoundCtl* ctl, uint32_t* __restrict__ int_rep) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) { ctl->seg_off_z[0] = 0; ctl->seg_off_z[1] = nprop; int_rep[0] = 0; }
    if (k < nprop) okey[k] = prop[k] ^ flip;
}

__global__ void k_prop_probes(uint32_t nprop, const uint64_t* __restrict__ okey_sorted, uint64_t* __restrict__ pkey,
                              int32_t* __restrict__ pseg, uint32_t* __restrict__ pspos, uint32_t* __restrict__ pint,
                              uint64_t* __restrict__ prank) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nprop) return;
    pkey[k] = okey_sorted[k]; pseg[k] = -1; pspos[k] = 0; prank[k] = 0; pint[k] = 0;
}

// ---------------------------------------------------------------------------
// L/U update of every splitter from the ranked probes.
// ---------------------------------------------------------------------------

// Probes of one launch are all input keys (kind kMember, distinct ranks) or
// all proposed non-member cuts (kind kNonMember), whose ranks may repeat: then
// the best cut of a rank is the first of its run (the smallest tag).
__global__ void k_update(uint32_t S, uint64_t N, uint32_t p, const uint64_t* __restrict__ pkey, const int32_t* __restrict__ pseg,
                         const uint32_t* __restrict__ pspos, const uint64_t* __restrict__ prank, uint64_t Z, int32_t pkind,
                         DCut* __restrict__ Lcut, DCut* __restrict__ Ucut, int32_t* __restrict__ chgL, int32_t* __restrict__ chgU,
                         const RoundCtl* __restrict__ ctl) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S) return;
    if (Z == kZFromCtl) Z = ctl->seg_off_z[1];
    const uint64_t t = ideal_rank(i + 1, N, p);
    uint64_t lo = 0, hi = Z;  // first probe with rank > t
    while (lo < hi) { const uint64_t m = (lo + hi) >> 1; if (prank[m] <= t) lo = m + 1; else hi = m; }
    const uint64_t kgt = lo;
    lo = 0; hi = Z;           // first probe with rank >= t
    while (lo < hi) { const uint64_t m = (lo + hi) >> 1; if (prank[m] < t) lo = m + 1; else hi = m; }
    const uint64_t kge = lo;
    DCut L = Lcut[i], U = Ucut[i];
    int32_t cl = -1, cu = -1;
    auto probe = [&](uint64_t k) {
        DCut c; c.okey = pkey[k]; c.seg = pseg[k]; c.spos = pspos[k]; c.rank = prank[k]; c.kind = pkind; c.pad = 0;
        return c;
    };
    if (kgt > 0) {
        uint64_t kl = kgt - 1;
        if (pkind != kMember) {  // first probe of the run with rank prank[kl]
            const uint64_t r = prank[kl];
            uint64_t a = 0, b = kl;
            while (a < b) { const uint64_t m = (a + b) >> 1; if (prank[m] < r) a = m + 1; else b = m; }
            kl = a;
        }
        offer(L, U, cl, cu, t, probe(kl), (int32_t)kl);
    }
    if (kge < Z) offer(L, U, cl, cu, t, probe(kge), (int32_t)kge);
    Lcut[i] = L; Ucut[i] = U; chgL[i] = cl; chgU[i] = cu;
}

__global__ void k_update_pos(uint32_t S, const int32_t* __restrict__ chgL, const int32_t* __restrict__ chgU,
                             const uint32_t* __restrict__ probe_pos, uint64_t cap, uint32_t* __restrict__ Lpos,
                             uint32_t* __restrict__ Upos) {
    const uint64_t s = blockIdx.x;
    const uint32_t i = blockIdx.y * blockDim.x + threadIdx.x;
    if (i >= S) return;
    const int32_t cl = chgL[i], cu = chgU[i];
    if (cl >= 0) Lpos[s * S + i] = probe_pos[s * cap + (uint32_t)cl];
    if (cu >= 0) Upos[s * S + i] = probe_pos[s * cap + (uint32_t)cu];
}

// ---------------------------------------------------------------------------
// Final splitters (Sec. 4.2.2 step 5): the closer of L_i, U_i (tie -> L_i).
// ---------------------------------------------------------------------------
__global__ void k_finalize(uint32_t S, uint64_t N, uint32_t p, int key_type, const DCut* __restrict__ Lcut,
                           const DCut* __restrict__ Ucut, hss_cut* __restrict__ spl, uint64_t* __restrict__ offsets,
                           uint32_t* __restrict__ choose_u, uint64_t* __restrict__ fin_okey,
                           uint32_t* __restrict__ fin_kind) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) { offsets[0] = 0; offsets[p] = N; }
    if (i >= S) return;
    const uint64_t t = ideal_rank(i + 1, N, p);
    const DCut L = Lcut[i], U = Ucut[i];
    const bool useU = (U.rank - t) < (t - L.rank);
    const DCut c = useU ? U : L;
    hss_cut o;
    const uint64_t flip = key_type == HSS_KEY_I64 ? kSignBit : 0ull;
    if (c.kind == kMember) { o.key = c.okey ^ flip; o.seg = c.seg; o.spos = c.spos; }
    else if (c.kind == kNonMember) { o.key = c.okey ^ flip; o.seg = -1; o.spos = 0; }
    else if (c.kind == kNegInf) { o.key = 0; o.seg = -2; o.spos = 0; }
    else { o.key = 0; o.seg = -3; o.spos = 0; }
    spl[i] = o;
    offsets[i + 1] = c.rank;
    choose_u[i] = useU ? 1u : 0u;
    fin_okey[i] = c.okey;
    fin_kind[i] = (uint32_t)c.kind;
}

// Bucket b holds keys between splitters b and b+1 (sentinels: the ends of the
// key range).  Its first split interpolates that range onto 256 sub-buckets:
// digit = mulhi(key - lo, floor(255 * 2^64 / (hi - lo))), monotone in the key
// and at most 255; a range narrower than 256 uses key - lo itself.
// Smallest and largest key of the whole input: the first and the last key of
// the locally sorted segments.  One block.
__global__ void __launch_bounds__(1024) k_key_range(const uint64_t* __restrict__ skeys,
                                                    const uint64_t* __restrict__ seg_off, uint32_t p,
                                                    uint64_t* __restrict__ range) {
    __shared__ uint64_t s_lo[32], s_hi[32];
    uint64_t lo = ~0ull, hi = 0ull;
    for (uint32_t s = threadIdx.x; s < p; s += blockDim.x) {
        const uint64_t a = seg_off[s], b = seg_off[s + 1];
        if (a < b) {
            lo = min(lo, skeys[a]);
            hi = max(hi, skeys[b - 1]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) { s_lo[w] = lo; s_hi[w] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < nw; ++i) { lo = min(lo, s_lo[i]); hi = max(hi, s_hi[i]); }
        range[0] = lo;
        range[1] = hi;
    }
}

// Interpolation hint of each bucket for the first digit split of the merge:
// the bucket's keys lie between splitters b and b+1, clipped to the input's
// key range, and mulhi(key - lo, mult) maps that interval onto 0..255.
__global__ void k_bucket_hint(uint32_t p, const uint64_t* __restrict__ fin_okey, const uint32_t* __restrict__ fin_kind,
                              const uint64_t* __restrict__ range, uint64_t* __restrict__ lo_out,
                              uint64_t* __restrict__ mult_out) {
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= p) return;
    auto bound = [&](uint32_t i, uint64_t if_none) -> uint64_t {  // splitter number i (1..p-1)
        if (i == 0 || i == p) return if_none;
        const uint32_t k = fin_kind[i - 1];
        if (k == (uint32_t)kNegInf) return 0ull;
        if (k == (uint32_t)kPosInf) return ~0ull;
        return fin_okey[i - 1];
    };
    const uint64_t kmin = range[0], kmax = range[1];
    const uint64_t lo = max(bound(b, 0ull), kmin);
    uint64_t hi = min(bound(b + 1, ~0ull), kmax);
    if (hi < lo) hi = lo;  // empty bucket
    const uint64_t r = hi - lo;
    // mult = 0 selects the plain form ((key >> 0) - lo) & 255 = key - lo
    const uint64_t mult = r < 256 ? 0ull : (uint64_t)(((unsigned __int128)255 << 64) / r);
    lo_out[b] = lo;
    mult_out[b] = mult;
}

cudaError_t bucket_hints(const RoundWs& ws, const uint64_t* skeys, const uint64_t* d_seg_off, uint32_t p,
                         cudaStream_t st, uint32_t nb) {
    const uint32_t NB = nb ? nb : p;
    HSS_LAUNCH(k_key_range, 1, 1024, 0, st, skeys, d_seg_off, p, ws.key_range);
    HSS_LAUNCH(k_bucket_hint, (unsigned)cdiv(NB, 256), 256, 0, st, NB, ws.fin_okey, ws.fin_kind, ws.key_range,
               ws.bucket_lo, ws.bucket_mult);
    return cudaGetLastError();
}

__global__ void k_final_pos(uint32_t S, const uint32_t* __restrict__ choose_u, uint32_t* __restrict__ Lpos,
                            const uint32_t* __restrict__ Upos) {
    const uint64_t s = blockIdx.x;
    const uint32_t i = blockIdx.y * blockDim.x + threadIdx.x;
    if (i >= S) return;
    if (choose_u[i]) Lpos[s * S + i] = Upos[s * S + i];
}

// ---------------------------------------------------------------------------
// The device-driven round loop: the parameters a round reads from the control
// record, and the decision taken before every round (the host loop's test:
// all resolved, the round limit, the sample capacity), which also records the
// round statistics and sets the WHILE condition of the loop's graph.
// ---------------------------------------------------------------------------
__global__ void k_ctl_init(RoundCtl* ctl, uint64_t seed, uint32_t max_rounds) {
    ctl->seed = seed;
    ctl->max_rounds = max_rounds;
    ctl->round = 0;
    ctl->status = HSS_OK;
    ctl->staged = 0;
}

__global__ void k_ctl_record(RoundCtl* ctl, uint32_t rounds, int32_t status, uint64_t last_z) {
    if (threadIdx.x == 0) {
        ctl->round = rounds;
        ctl->status = status;
        (void)last_z;
    }
}

__global__ void k_round_decide(RoundCtl* ctl, uint64_t cap, uint64_t N, uint32_t p, uint32_t hist_mode,
                               cudaGraphConditionalHandle loop) {
    const uint32_t j = ctl->round;  // rounds done
    ctl->hist_unres[j] = ctl->unresolved;
    uint32_t go = 0;
    if (ctl->unresolved == 0) {
    } else if (j >= ctl->max_rounds) {
        ctl->status = HSS_ERR_ROUND_LIMIT;
    } else {
        const uint64_t Z = ctl->Z;
        ctl->hist_Z[j] = Z;
        ctl->hist_gamma[j] = ctl->gamma;
        ctl->round = j + 1;
        if (Z > cap) {
            ctl->status = HSS_ERR_CAPACITY;
        } else {
            // the histogram form of this round, as the host loop chooses it
            const double searches = (double)Z * (double)p * log2((double)N / (double)p + 2.0);
            ctl->staged = (ctl->nint == 1 && hist_mode != kHistProbe &&
                           (hist_mode == kHistStaged || searches >= 8.0 * (double)N)) ? 1u : 0u;
            go = 1;
        }
    }
    cudaGraphSetConditional(loop, go);
}

// ---------------------------------------------------------------------------
// Host driver of the rounds.
// ---------------------------------------------------------------------------
#define HSS_TRY(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return HSS_ERR_CUDA; } while (0)

static void enqueue_sampling(const RoundWs& ws, const uint64_t* d_seg_off, uint64_t N, uint32_t p, uint32_t S,
                             uint64_t seed, uint32_t round, cudaStream_t st, bool per_interval) {
    cudaMemsetAsync(ws.bitmap, 0, (N / 32 + 2) * sizeof(uint32_t), st);
    cudaMemsetAsync(ws.seg_cnt, 0, (size_t)p * sizeof(uint32_t), st);
    // round 1 samples whole segments: several CTAs share each; later rounds
    // sample narrow intervals, one CTA per segment
    HSS_LAUNCH(k_sample_mark, dim3(p, round == 1 ? mark_chunks(N, p) : 1u), kSampThreads, 0, st, d_seg_off, S, ws.Lpos,
               ws.Upos, ws.Lcut, ws.int_rep, ws.ctl, seed, round, ws.bitmap, ws.seg_cnt,
               per_interval ? ws.int_T : nullptr, per_interval ? ws.int_all : nullptr);
    HSS_LAUNCH(k_count_scan, 1, 1024, 0, st, ws.seg_cnt, p, ws.seg_cnt_off, ws.cap, ws.ctl);
}

bool device_loop_possible(uint64_t cap, uint32_t schedule) {
    // the probe sort of a round must run without host planning (one segment
    // of at most the on-chip capacity), and the threshold must come from the
    // device (the k-round schedule computes it on the host with libm)
    return cap <= (uint64_t)kSmallCap && schedule != HSS_SCHEDULE_THEORY;
}

namespace {

// One round of the device-driven loop, enqueued on `st` (captured into the
// body of the loop's graph): write the sample, sort it, build and rank the
// probes, update L/U and their positions, recompute the intervals, sample the
// next round and decide whether it runs.  Every kernel reads the round's
// sample size, seed and histogram form from the control record.
cudaError_t enqueue_device_round(const uint64_t* skeys, const uint64_t* d_seg_off, uint64_t N, uint32_t p, uint32_t NB,
                                 uint64_t tol, float oversample, uint32_t schedule, uint32_t hist_mode, const RoundWs& ws,
                                 cudaGraphConditionalHandle loop, cudaStream_t st) {
    const uint32_t S = NB - 1;
    const unsigned sblk = (unsigned)cdiv(S, 256);
    const uint64_t cap = ws.cap;
    const bool per_interval = schedule == HSS_SCHEDULE_EQUAL;
    HSS_LAUNCH(k_sample_write, p, kSampThreads, 0, st, skeys, d_seg_off, ws.bitmap, ws.seg_cnt, ws.seg_cnt_off, cap, ws.skey,
               ws.sseg, ws.sspos, ws.siota);
    cudaError_t e = segsort(ws.skey, ws.skey_sorted, ws.stmp, ws.siota, ws.sperm, ws.ptmp, cap, 1, ws.ctl->seg_off_z,
                            false, false, ws.sws, st, nullptr);
    if (e != cudaSuccess) return e;
    HSS_LAUNCH(k_probe_build, (unsigned)cdiv(cap, 256), 256, 0, st, kZFromCtl, ws.skey_sorted, ws.sperm, ws.sseg,
               ws.sspos, ws.Ucut, ws.int_rep, ws.ctl, ws.pkey, ws.pseg, ws.pspos, ws.pint, ws.prank);
    HSS_LAUNCH(k_histogram_staged, dim3((unsigned)cdiv(cap, kStgProbes), (unsigned)cdiv(p, kStgSegs)), kStgThreads, 0, st,
               skeys, d_seg_off, p, S, ws.Lpos, ws.Upos, ws.int_rep, ws.pkey, ws.pseg, ws.pspos, kZFromCtl, ws.prank,
               ws.probe_pos, cap, ws.sws.err, ws.ctl);
    HSS_LAUNCH(k_histogram, dim3((unsigned)cdiv(cap, 32), (unsigned)cdiv(p, kHistSegPerBlock)), 256, 0, st, skeys,
               d_seg_off, p, S, ws.Lpos, ws.Upos, ws.int_rep, ws.pkey, ws.pseg, ws.pspos, ws.pint, kZFromCtl, ws.prank,
               ws.probe_pos, cap, ws.sws.err, ws.ctl);
    HSS_LAUNCH(k_update, sblk, 256, 0, st, S, N, NB, ws.pkey, ws.pseg, ws.pspos, ws.prank, kZFromCtl, (int32_t)kMember,
               ws.Lcut, ws.Ucut, ws.chgL, ws.chgU, ws.ctl);
    HSS_LAUNCH(k_update_pos, dim3(p, sblk), 256, 0, st, S, ws.chgL, ws.chgU, ws.probe_pos, cap, ws.Lpos, ws.Upos);
    HSS_LAUNCH(k_intervals, 1, 1024, 0, st, S, N, NB, tol, oversample, ws.Lcut, ws.Ucut, ws.res, ws.int_rep, ws.ctl,
               schedule, 0ull, 0u, ws.int_T, ws.int_all);
    if ((e = cudaMemsetAsync(ws.bitmap, 0, (N / 32 + 2) * sizeof(uint32_t), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ws.seg_cnt, 0, (size_t)p * sizeof(uint32_t), st)) != cudaSuccess) return e;
    HSS_LAUNCH(k_sample_mark, dim3(p, 1u), kSampThreads, 0, st, d_seg_off, S, ws.Lpos, ws.Upos, ws.Lcut, ws.int_rep,
               ws.ctl, 0ull, 0u, ws.bitmap, ws.seg_cnt, per_interval ? ws.int_T : nullptr,
               per_interval ? ws.int_all : nullptr);
    HSS_LAUNCH(k_count_scan, 1, 1024, 0, st, ws.seg_cnt, p, ws.seg_cnt_off, cap, ws.ctl);
    HSS_LAUNCH(k_round_decide, 1, 1, 0, st, ws.ctl, cap, N, p, hist_mode, loop);
    return cudaGetLastError();
}

// Executable graphs of the loop, keyed by what the captured kernels were
// given (the workspace's round state, the sorted keys, the sizes and the
// sampling form); the seed and the round limit travel in the control record.
struct LoopKey {
    int dev;
    const void* ctl;
    const uint64_t* skeys;
    const uint64_t* seg_off;
    uint64_t N, tol, cap;
    uint32_t p, schedule, hist_mode;
    float oversample;
    uint32_t nb;
    bool operator==(const LoopKey& o) const {
        return dev == o.dev && ctl == o.ctl && skeys == o.skeys && seg_off == o.seg_off && N == o.N && tol == o.tol &&
               cap == o.cap && p == o.p && schedule == o.schedule && hist_mode == o.hist_mode &&
               oversample == o.oversample && nb == o.nb;
    }
};
struct LoopGraph {
    LoopKey key;
    cudaGraphExec_t exec;
    uint64_t used;
};
std::mutex g_loop_mu;
std::vector<LoopGraph> g_loops;
uint64_t g_loop_clock = 0;
constexpr size_t kMaxLoopGraphs = 32;
cudaStream_t g_capture_stream[256] = {};
uint32_t g_body_kernels = 0;  // kernels one round of the loop launches

// Shapes seen once without a graph (the adaptive policy builds a shape's
// graph when it comes again).
std::vector<LoopKey> g_seen;
constexpr size_t kMaxSeen = 64;
constexpr int kLoopDeclined = 1;  // loop_graph: no graph yet, drive these rounds from the host

// Build (once per key) the graph: the decision kernel, then WHILE(cond) { round }.
// Unless build_now, a key met for the first time only is remembered and the
// call declines (kLoopDeclined): capturing and instantiating the graph costs
// more than the host round trips of one call, so only shapes that repeat get
// one.
int loop_graph(const LoopKey& k, const uint64_t* skeys, const uint64_t* d_seg_off, uint64_t N, uint32_t p, uint32_t NB,
               uint64_t tol, float oversample, uint32_t schedule, uint32_t hist_mode, const RoundWs& ws,
               bool build_now, cudaGraphExec_t* out) {
    std::lock_guard<std::mutex> lock(g_loop_mu);
    for (auto& g : g_loops)
        if (g.key == k) {
            g.used = ++g_loop_clock;
            *out = g.exec;
            return HSS_OK;
        }
    if (!build_now) {
        bool seen = false;
        for (size_t i = 0; i < g_seen.size(); ++i)
            if (g_seen[i] == k) {
                g_seen.erase(g_seen.begin() + i);
                seen = true;
                break;
            }
        if (!seen) {
            if (g_seen.size() >= kMaxSeen) g_seen.erase(g_seen.begin());
            g_seen.push_back(k);
            return kLoopDeclined;
        }
    }
    if (k.dev < 0 || k.dev >= 256) return HSS_ERR_CUDA;
    cudaStream_t& cs = g_capture_stream[k.dev];
    if (!cs && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return HSS_ERR_CUDA;
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return HSS_ERR_CUDA;
    auto fail = [&]() { cudaGraphDestroy(g); return HSS_ERR_CUDA; };
    cudaGraphConditionalHandle loop;
    if (cudaGraphConditionalHandleCreate(&loop, g, 0, cudaGraphCondAssignDefault) != cudaSuccess) return fail();
    // the decision before round 1
    LaunchCountPause pause;
    if (cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return fail();
    k_round_decide<<<1, 1, 0, cs>>>(ws.ctl, ws.cap, N, p, hist_mode, loop);
    cudaGraph_t tmp = nullptr;
    if (cudaStreamEndCapture(cs, &tmp) != cudaSuccess || tmp != g) return fail();
    cudaGraphNode_t gate = nullptr;
    size_t n = 1;
    if (cudaGraphGetNodes(g, &gate, &n) != cudaSuccess || n != 1) return fail();
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = loop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode = nullptr;
    if (cudaGraphAddNode(&cnode, g, &gate, nullptr, 1, &cp) != cudaSuccess) return fail();
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return fail();
    const uint64_t before = pause.captured();
    const cudaError_t ce = enqueue_device_round(skeys, d_seg_off, N, p, NB, tol, oversample, schedule, hist_mode, ws, loop,
                                                cs);
    g_body_kernels = (uint32_t)(pause.captured() - before);
    tmp = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(cs, &tmp);
    if (ce != cudaSuccess || ee != cudaSuccess) return fail();
    cudaGraphExec_t exec = nullptr;
    if (cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) return fail();
    cudaGraphDestroy(g);
    if (g_loops.size() >= kMaxLoopGraphs) {  // evict the least recently used
        size_t v = 0;
        for (size_t i = 1; i < g_loops.size(); ++i)
            if (g_loops[i].used < g_loops[v].used) v = i;
        cudaGraphExecDestroy(g_loops[v].exec);
        g_loops.erase(g_loops.begin() + v);
    }
    g_loops.push_back(LoopGraph{k, exec, ++g_loop_clock});
    *out = exec;
    return HSS_OK;
}

}  // namespace

uint32_t device_round_kernels() { return g_body_kernels; }

int read_round_result(const RoundWs& ws, RoundResult* out, cudaStream_t st) {
    RoundCtl h;
    if (read_small(&h, ws.ctl, sizeof(h), st) != cudaSuccess) return HSS_ERR_CUDA;
    out->rounds = h.round;
    out->status = h.status;
    for (uint32_t j = 0; j < h.round && j < HSS_MAX_ROUNDS; ++j) {
        out->sample_size[j] = h.hist_Z[j];
        out->gamma[j] = h.hist_gamma[j];
    }
    // unresolved after round j is recorded by the decision before round j+1
    // (or by the last decision); a capacity stop leaves the last one unset
    const uint32_t last = h.status == HSS_ERR_CAPACITY ? (h.round > 0 ? h.round - 1 : 0) : h.round;
    for (uint32_t j = 0; j <= last && j <= HSS_MAX_ROUNDS; ++j) out->unresolved[j] = h.hist_unres[j];
    return h.status;
}

int run_rounds(const uint64_t* skeys, const uint64_t* d_seg_off, uint64_t N, uint32_t p, double eps, uint64_t seed,
               float oversample, uint32_t max_rounds, int key_type, hss_cut* d_splitters, uint64_t* d_offsets,
               const RoundWs& ws, cudaStream_t st, RoundResult* out, const uint64_t* d_prop, uint32_t nprop,
               uint32_t schedule, uint32_t schedule_k, uint32_t hist_mode, uint32_t loop_mode, bool* used_device_loop,
               uint32_t nb) {
    if (used_device_loop) *used_device_loop = false;
    const uint32_t NB = nb ? nb : p;  // buckets: the splitters target ranks i N / NB
    if (NB > p) return HSS_ERR_INVALID;
    const uint32_t S = NB - 1;
    const uint64_t tol = (uint64_t)std::floor(((double)N * eps) / (2.0 * (double)NB));
    const bool per_interval = schedule == HSS_SCHEDULE_EQUAL;
    // The interval pass before sampling round r; under the k-round schedule
    // the host supplies round r's threshold: probability p s_r / N,
    // s_r = (2 ln p / eps)^(min(r,k)/k) (Theorem 4.7), in IEEE double.
    auto intervals = [&](uint32_t r) {
        uint64_t Tq = 0;
        uint32_t allq = 0;
        if (schedule == HSS_SCHEDULE_THEORY) {
            const uint32_t rr = r < schedule_k ? r : schedule_k;
            const double sj = std::pow(2.0 * std::log((double)NB) / eps, (double)rr / (double)schedule_k);
            const double q = ((double)NB * sj) / (double)N;
            if (q >= 1.0) allq = 1u;
            else Tq = (uint64_t)std::floor(std::ldexp(q, 64));
        }
        HSS_LAUNCH(k_intervals, 1, 1024, 0, st, S, N, NB, tol, oversample, ws.Lcut, ws.Ucut, ws.res, ws.int_rep, ws.ctl,
                   schedule, Tq, allq, ws.int_T, ws.int_all);
    };
    // The histogram of Z probes: staged when they share one interval and
    // searching every segment for every probe (Z p log2(N/p) dependent loads)
    // would cost several reads of the keys (the probe-side form otherwise).
    auto histogram = [&](uint64_t Z, uint32_t nint) -> cudaError_t {
        const double searches = (double)Z * (double)p * std::log2((double)N / (double)p + 2.0);
        const bool staged = nint == 1 && hist_mode != kHistProbe &&
                            (hist_mode == kHistStaged || searches >= 8.0 * (double)N);
        if (staged) {
            HSS_LAUNCH(k_histogram_staged, dim3((unsigned)cdiv(Z, kStgProbes), (unsigned)cdiv(p, kStgSegs)), kStgThreads, 0,
                       st, skeys, d_seg_off, p, S, ws.Lpos, ws.Upos, ws.int_rep, ws.pkey, ws.pseg, ws.pspos, Z, ws.prank,
                       ws.probe_pos, ws.cap, ws.sws.err, ws.ctl);
        } else {
            HSS_LAUNCH(k_histogram, dim3((unsigned)cdiv(Z, 32), (unsigned)cdiv(p, kHistSegPerBlock)), 256, 0, st, skeys,
                       d_seg_off, p, S, ws.Lpos, ws.Upos, ws.int_rep, ws.pkey, ws.pseg, ws.pspos, ws.pint, Z, ws.prank,
                       ws.probe_pos, ws.cap, ws.sws.err, ws.ctl);
        }
        return cudaGetLastError();
    };
    HSS_TRY(cudaMemsetAsync(ws.ctl, 0, sizeof(RoundCtl), st));
    if (S == 0) {
        HSS_LAUNCH(k_finalize, 1, 32, 0, st, 0u, N, NB, key_type, ws.Lcut, ws.Ucut, d_splitters, d_offsets, ws.choose_u,
                   ws.fin_okey, ws.fin_kind);
        HSS_TRY(cudaGetLastError());
        out->rounds = 0;
        out->status = HSS_OK;
        return HSS_OK;
    }
    const unsigned sblk = (unsigned)cdiv(S, 256);
    HSS_LAUNCH(k_rounds_init, dim3(p, sblk), 256, 0, st, d_seg_off, S, N, ws.Lcut, ws.Ucut, ws.Lpos, ws.Upos);
    intervals(1);
    if (nprop > 0) {
        // Proposed cuts: sorted, ranked in every segment, offered to L/U.
        if (nprop > ws.cap) return HSS_ERR_INVALID;
        const uint64_t flip = key_type == HSS_KEY_I64 ? kSignBit : 0ull;
        HSS_LAUNCH(k_prop_load, (unsigned)cdiv(nprop, 256), 256, 0, st, d_prop, nprop, flip, ws.skey, ws.ctl, ws.int_rep);
        HSS_TRY(segsort(ws.skey, ws.skey_sorted, ws.stmp, nullptr, nullptr, nullptr, nprop, 1, ws.ctl->seg_off_z, false,
                        false, ws.sws, st, nullptr));
        HSS_LAUNCH(k_prop_probes, (unsigned)cdiv(nprop, 256), 256, 0, st, nprop, ws.skey_sorted, ws.pkey, ws.pseg,
                   ws.pspos, ws.pint, ws.prank);
        HSS_TRY(histogram((uint64_t)nprop, 1u));
        HSS_LAUNCH(k_update, sblk, 256, 0, st, S, N, NB, ws.pkey, ws.pseg, ws.pspos, ws.prank, (uint64_t)nprop,
                   (int32_t)kNonMember, ws.Lcut, ws.Ucut, ws.chgL, ws.chgU, ws.ctl);
        HSS_LAUNCH(k_update_pos, dim3(p, sblk), 256, 0, st, S, ws.chgL, ws.chgU, ws.probe_pos, ws.cap, ws.Lpos, ws.Upos);
        intervals(1);
    }
    cudaGraphExec_t exec = nullptr;
    if (loop_mode != kLoopHost && device_loop_possible(ws.cap, schedule)) {
        // Sampling of round 1 on the stream, then the loop's graph: no host
        // round trip until the caller reads the statistics.
        int dev = 0;
        HSS_TRY(cudaGetDevice(&dev));
        const LoopKey key{dev, ws.ctl, skeys, d_seg_off, N, tol, ws.cap, p, schedule, hist_mode, oversample, NB};
        const int rc = loop_graph(key, skeys, d_seg_off, N, p, NB, tol, oversample, schedule, hist_mode, ws,
                                  loop_mode == kLoopDevice, &exec);
        if (rc != HSS_OK && rc != kLoopDeclined) return rc;
    }
    if (exec) {
        HSS_LAUNCH(k_ctl_init, 1, 1, 0, st, ws.ctl, seed, max_rounds);
        enqueue_sampling(ws, d_seg_off, N, p, S, seed, 1, st, per_interval);
        HSS_TRY(cudaGetLastError());
        HSS_TRY(cudaGraphLaunch(exec, st));
        HSS_LAUNCH(k_finalize, (unsigned)cdiv(S, 256), 256, 0, st, S, N, NB, key_type, ws.Lcut, ws.Ucut, d_splitters,
                   d_offsets, ws.choose_u, ws.fin_okey, ws.fin_kind);
        HSS_LAUNCH(k_final_pos, dim3(p, sblk), 256, 0, st, S, ws.choose_u, ws.Lpos, ws.Upos);
        HSS_TRY(cudaGetLastError());
        if (used_device_loop) *used_device_loop = true;
        return HSS_OK;
    }
    enqueue_sampling(ws, d_seg_off, N, p, S, seed, 1, st, per_interval);
    HSS_TRY(cudaGetLastError());
    RoundCtl h;
    HSS_TRY(read_small(&h, ws.ctl, sizeof(h), st));
    out->unresolved[0] = h.unresolved;
    uint32_t j = 0;
    int status = HSS_OK;
    for (;;) {
        if (h.unresolved == 0) break;
        if (j >= max_rounds) { status = HSS_ERR_ROUND_LIMIT; break; }
        ++j;
        out->sample_size[j - 1] = h.Z;
        out->gamma[j - 1] = h.gamma;
        if (h.Z > ws.cap) { status = HSS_ERR_CAPACITY; break; }
        const uint64_t Z = h.Z;
        HSS_LAUNCH(k_sample_write, p, kSampThreads, 0, st, skeys, d_seg_off, ws.bitmap, ws.seg_cnt, ws.seg_cnt_off, ws.cap,
                   ws.skey, ws.sseg, ws.sspos, ws.siota);
        if (Z > 0) {
            HSS_TRY(segsort(ws.skey, ws.skey_sorted, ws.stmp, ws.siota, ws.sperm, ws.ptmp, Z, 1, ws.ctl->seg_off_z, false,
                            false, ws.sws, st, nullptr));
            HSS_LAUNCH(k_probe_build, (unsigned)cdiv(Z, 256), 256, 0, st, Z, ws.skey_sorted, ws.sperm, ws.sseg, ws.sspos,
                       ws.Ucut, ws.int_rep, ws.ctl, ws.pkey, ws.pseg, ws.pspos, ws.pint, ws.prank);
            HSS_TRY(histogram(Z, h.nint));
            HSS_LAUNCH(k_update, sblk, 256, 0, st, S, N, NB, ws.pkey, ws.pseg, ws.pspos, ws.prank, Z, (int32_t)kMember,
                       ws.Lcut, ws.Ucut, ws.chgL, ws.chgU, ws.ctl);
            HSS_LAUNCH(k_update_pos, dim3(p, sblk), 256, 0, st, S, ws.chgL, ws.chgU, ws.probe_pos, ws.cap, ws.Lpos, ws.Upos);
        }
        intervals(j + 1);
        enqueue_sampling(ws, d_seg_off, N, p, S, seed, j + 1, st, per_interval);
        HSS_TRY(cudaGetLastError());
        HSS_TRY(read_small(&h, ws.ctl, sizeof(h), st));
        out->unresolved[j] = h.unresolved;
    }
    out->rounds = j;
    out->status = status;
    {   // the same record the device-driven loop leaves, for hss_call_stats
        HSS_LAUNCH(k_ctl_record, 1, 64, 0, st, ws.ctl, j, status, out->sample_size[j > 0 ? j - 1 : 0]);
        HSS_TRY(cudaMemcpyAsync(ws.ctl->hist_Z, out->sample_size, sizeof(out->sample_size), cudaMemcpyHostToDevice, st));
        HSS_TRY(cudaMemcpyAsync(ws.ctl->hist_gamma, out->gamma, sizeof(out->gamma), cudaMemcpyHostToDevice, st));
        HSS_TRY(cudaMemcpyAsync(ws.ctl->hist_unres, out->unresolved, sizeof(out->unresolved), cudaMemcpyHostToDevice, st));
    }
    HSS_LAUNCH(k_finalize, (unsigned)cdiv(S, 256), 256, 0, st, S, N, NB, key_type, ws.Lcut, ws.Ucut, d_splitters, d_offsets,
               ws.choose_u, ws.fin_okey, ws.fin_kind);
    HSS_LAUNCH(k_final_pos, dim3(p, sblk), 256, 0, st, S, ws.choose_u, ws.Lpos, ws.Upos);
    HSS_TRY(cudaGetLastError());
    return status;
}

// ---------------------------------------------------------------------------
// Exchange (Sec. 3.1 step 3 / Sec. 6): runs of the sorted segments to their
// buckets.  dst(s, b) = chi(b) + sum_{s' < s} |run(s', b)|.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t bucket_pos(const uint32_t* __restrict__ pos, uint32_t S, uint32_t p, uint64_t s,
                                               uint32_t b, uint32_t n) {
    return b == 0 ? 0u : (b == p ? n : pos[s * S + (b - 1)]);
}

// Column scans of the run lengths: CTA x handles 32 buckets; its 32 warps
// split the segments into 32 groups, sum their group, scan the group sums and
// write the destinations.
__global__ __launch_bounds__(1024) void k_exchange_dst(const uint64_t* __restrict__ seg_off, uint32_t p, uint32_t NB,
                                                       const uint32_t* __restrict__ pos, const uint64_t* __restrict__ offsets,
                                                       uint64_t* __restrict__ dst, uint32_t* err) {
    __shared__ uint64_t s_part[32][33];
    const uint32_t col = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const uint32_t b = blockIdx.x * 32 + col;
    const uint32_t S = NB - 1;
    const uint32_t R = (p + 31) / 32;
    const uint32_t s0 = min(p, grp * R), s1 = min(p, s0 + R);
    uint64_t part = 0;
    if (b < NB) {
        for (uint32_t s = s0; s < s1; ++s) {
            const uint32_t n = (uint32_t)(seg_off[s + 1] - seg_off[s]);
            part += bucket_pos(pos, S, NB, s, b + 1, n) - bucket_pos(pos, S, NB, s, b, n);
        }
    }
    s_part[grp][col] = part;
    __syncthreads();
    if (b >= NB) return;
    uint64_t run = offsets[b];
    for (uint32_t g = 0; g < grp; ++g) run += s_part[g][col];
    for (uint32_t s = s0; s < s1; ++s) {
        const uint32_t n = (uint32_t)(seg_off[s + 1] - seg_off[s]);
        dst[(uint64_t)s * NB + b] = run;
        run += bucket_pos(pos, S, NB, s, b + 1, n) - bucket_pos(pos, S, NB, s, b, n);
    }
    if (s1 == p && s0 < s1 && run != offsets[b + 1]) atomicOr(err, kDevErrBounds);
}

// Largest m in [lo, hi) with bucket_pos(m) <= v, given bucket_pos(lo) <= v,
// by one full warp: each step splits the range into 32 parts and keeps the
// last part whose first position is <= v (a few parallel loads instead of a
// chain of dependent ones).
__device__ __forceinline__ uint32_t warp_last_le(const uint32_t* __restrict__ pos, uint32_t S, uint32_t p, uint64_t s,
                                                 uint32_t n, uint32_t v, uint32_t lo, uint32_t hi) {
    const uint32_t lane = threadIdx.x & 31;
    while (hi - lo > 1) {
        const uint32_t step = (hi - lo + 31) / 32;
        const uint32_t m = lo + lane * step;
        const bool ok = m < hi && bucket_pos(pos, S, p, s, m, n) <= v;
        const uint32_t bal = __ballot_sync(0xffffffffu, ok);  // lane 0 always holds
        const uint32_t last = 31 - __clz(bal);
        lo = lo + last * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

constexpr uint32_t kXchChunk = 8192;
constexpr uint32_t kXchMaxB = 4096;

__global__ __launch_bounds__(256) void k_exchange_copy(const uint64_t* __restrict__ skeys, const uint32_t* __restrict__ spay,
                                                       const uint64_t* __restrict__ seg_off, uint32_t NB,
                                                       const uint32_t* __restrict__ pos, const uint64_t* __restrict__ dst,
                                                       uint64_t* __restrict__ bkeys, uint32_t* __restrict__ bpay, uint64_t N,
                                                       uint32_t* __restrict__ err) {
    __shared__ uint32_t s_bnd[kXchMaxB + 1];
    __shared__ uint32_t s_b0, s_nb;
    const uint64_t s = blockIdx.x;
    const uint32_t S = NB - 1;
    const uint64_t base = seg_off[s];
    const uint32_t n = (uint32_t)(seg_off[s + 1] - base);
    const uint32_t c0 = blockIdx.y * kXchChunk;
    if (c0 >= n) return;
    const uint32_t c1 = min(n, c0 + kXchChunk);
    if (threadIdx.x < 32) {
        // buckets b0..b1 whose runs meet [c0, c1): last b with pos(b) <= c0, last b with pos(b) <= c1-1
        const uint32_t b0 = warp_last_le(pos, S, NB, s, n, c0, 0, NB);
        const uint32_t b1 = warp_last_le(pos, S, NB, s, n, c1 - 1, b0, NB);
        if (threadIdx.x == 0) {
            s_b0 = b0;
            s_nb = b1 - b0 + 1;
        }
    }
    __syncthreads();
    const uint32_t b0 = s_b0, nb = s_nb;
    if (nb <= kXchMaxB) {
        for (uint32_t i = threadIdx.x; i <= nb; i += blockDim.x) s_bnd[i] = bucket_pos(pos, S, NB, s, b0 + i, n);
        __syncthreads();
        // Four keys per thread per step, their loads issued together (memory
        // parallelism); j grows by the CTA width, so the run of j follows
        // from the previous one by a galloping search forward (one compare
        // when runs are about as long as a step, a few when they are short).
        uint32_t lo = 0;
        for (uint32_t j0 = c0 + threadIdx.x; j0 < c1; j0 += 4 * blockDim.x) {
            uint64_t kv[4];
            uint32_t pv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t j = j0 + u * blockDim.x;
                kv[u] = j < c1 ? skeys[base + j] : 0ull;
                pv[u] = (bpay && j < c1) ? spay[base + j] : 0u;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t j = j0 + u * blockDim.x;
                if (j >= c1) break;
                if (lo + 1 < nb && s_bnd[lo + 1] <= j) {  // gallop forward, then bisect
                    uint32_t at = lo + 1, step = 1;
                    while (at + step < nb && s_bnd[at + step] <= j) { at += step; step <<= 1; }
                    uint32_t hi = min(at + step, nb);
                    while (hi - at > 1) { const uint32_t m = (at + hi) >> 1; if (s_bnd[m] <= j) at = m; else hi = m; }
                    lo = at;
                }
                const uint64_t d = dst[s * NB + b0 + lo] + (j - s_bnd[lo]);
                if (d >= N) { atomicOr(err, kDevErrBounds); continue; }
                bkeys[d] = kv[u];
                if (bpay) bpay[d] = pv[u];
            }
        }
    } else {
        for (uint32_t j = c0 + threadIdx.x; j < c1; j += blockDim.x) {
            uint32_t lo = b0, hi = b0 + nb;
            while (hi - lo > 1) { const uint32_t m = (lo + hi) >> 1; if (bucket_pos(pos, S, NB, s, m, n) <= j) lo = m; else hi = m; }
            const uint64_t d = dst[s * NB + lo] + (j - bucket_pos(pos, S, NB, s, lo, n));
            if (d >= N) { atomicOr(err, kDevErrBounds); continue; }
            bkeys[d] = skeys[base + j];
            if (bpay) bpay[d] = spay[base + j];
        }
    }
}

cudaError_t exchange(const uint64_t* skeys, const uint32_t* spay, uint64_t N, uint32_t p, const uint64_t* d_seg_off,
                     const uint32_t* pos, const uint64_t* d_offsets, uint64_t* bkeys, uint32_t* bpay,
                     uint64_t* dst_scratch, uint32_t* err, cudaStream_t st, uint32_t nb) {
    if (N == 0) return cudaSuccess;
    const uint32_t NB = nb ? nb : p;
    HSS_LAUNCH(k_exchange_dst, (unsigned)cdiv(NB, 32), 1024, 0, st, d_seg_off, p, NB, pos, d_offsets, dst_scratch, err);
    const uint64_t maxn = cdiv(N, p) + 1;
    HSS_LAUNCH(k_exchange_copy, dim3(p, (unsigned)cdiv(maxn, kXchChunk)), 256, 0, st, skeys, spay, d_seg_off, NB, pos,
               dst_scratch, bkeys, bpay, N, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Ranks of caller-supplied cuts (hss_rank_cuts).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t seg_count(const uint64_t* __restrict__ a, uint32_t n, uint64_t okey, bool strict, uint64_t flip) {
    uint32_t base = 0;
    while (n > 0) {
        const uint32_t half = n >> 1;
        const uint64_t v = a[base + half] ^ flip;
        const bool go = strict ? (v < okey) : (v <= okey);
        base = go ? base + half + 1 : base;
        n = go ? n - half - 1 : half;
    }
    return base;
}

__global__ __launch_bounds__(256) void k_rank_cuts(const uint64_t* __restrict__ skeys, uint64_t flip, uint64_t N,
                                                   uint32_t p, const hss_cut* __restrict__ cuts, uint32_t ncuts,
                                                   uint64_t* __restrict__ ranks, uint32_t* __restrict__ seg_pos) {
    __shared__ uint64_t s_part[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t k = blockIdx.x * 32 + lane;
    const bool valid = k < ncuts;
    hss_cut c; c.key = 0; c.seg = -2; c.spos = 0;
    if (valid) c = cuts[k];
    const uint64_t okey = c.key ^ flip;
    uint64_t partial = 0;
    for (int j = 0; j < kHistSegPerBlock / 8; ++j) {
        const uint32_t s = blockIdx.y * kHistSegPerBlock + j * 8 + w;
        if (valid && s < p) {
            const uint64_t lo = ideal_rank(s, N, p), hi = ideal_rank(s + 1, N, p);  // segment bounds
            const uint32_t n = (uint32_t)(hi - lo);
            const uint64_t* a = skeys + lo;
            uint32_t pos;
            if (c.seg == -2) pos = 0;
            else if (c.seg == -3) pos = n;
            else if (c.seg == -1) pos = seg_count(a, n, okey, true, flip);
            else if ((int32_t)s < c.seg) pos = seg_count(a, n, okey, false, flip);
            else if ((int32_t)s > c.seg) pos = seg_count(a, n, okey, true, flip);
            else {
                const uint32_t lb = seg_count(a, n, okey, true, flip), ub = seg_count(a, n, okey, false, flip);
                pos = min(max(c.spos, lb), ub);
            }
            if (seg_pos) seg_pos[(uint64_t)s * ncuts + k] = pos;
            partial += pos;
        }
    }
    s_part[w][lane] = partial;
    __syncthreads();
    if (w == 0 && valid) {
        uint64_t sum = 0;
        for (int i = 0; i < 8; ++i) sum += s_part[i][lane];
        atomicAdd((unsigned long long*)&ranks[k], (unsigned long long)sum);
    }
}

cudaError_t rank_cuts(const uint64_t* skeys, int key_type, uint64_t N, uint32_t p,
                      const hss_cut* cuts, uint32_t ncuts, uint64_t* ranks, uint32_t* seg_pos, cudaStream_t st) {
    if (ncuts == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(ranks, 0, ncuts * sizeof(uint64_t), st);
    if (e != cudaSuccess) return e;
    HSS_LAUNCH(k_rank_cuts, dim3((unsigned)cdiv(ncuts, 32), (unsigned)cdiv(p, kHistSegPerBlock)), 256, 0, st, skeys,
               key_type == HSS_KEY_I64 ? kSignBit : 0ull, N, p, cuts, ncuts, ranks, seg_pos);
    return cudaGetLastError();
}

__global__ void k_sample_words(uint64_t seed, uint32_t seg, uint32_t round, uint32_t spos0, uint32_t count, uint64_t* out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint32_t spos = spos0 + i;
    uint64_t w0, w1;
    sample_words(seed, seg, round, spos >> 1, w0, w1);
    out[i] = (spos & 1u) ? w1 : w0;
}

cudaError_t sample_words_launch(uint64_t seed, uint32_t seg, uint32_t round, uint32_t spos0, uint32_t count,
                                uint64_t* out, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    HSS_LAUNCH(k_sample_words, (unsigned)cdiv(count, 256), 256, 0, st, seed, seg, round, spos0, count, out);
    return cudaGetLastError();
}

}  // namespace hss
