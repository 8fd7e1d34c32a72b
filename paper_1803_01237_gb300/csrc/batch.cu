// batch.cu -- many independent HSS sorts in one call (hss_sort_batch,
// hss_partition_batch).
//
// Job j holds keys [koff_j, koff_j + n_j) of one device array (the jobs are
// consecutive) and is split over p_j processors exactly as hss_sort would do
// it alone with seed + j: the same local sort, the same rounds (Sec. 4.2.2),
// the same exchange and merge.  What changes is that every kernel serves all
// jobs at once: the segments of all jobs form one segmented sort, the rounds
// advance in lock step (a job that has resolved its splitters, or failed,
// stops sampling while the others go on), and each round costs a handful of
// launches and one 16-byte host read for the whole batch instead of per job.
//
// Every per-job quantity lives in one slice of a global table: segments from
// sbase_j, splitters from ibase_j, the p x (p-1) per-segment cut positions
// from lbase_j, the p x p exchange destinations from dbase_j, the sample
// slots from cbase_j (capacity cap_j = min(n_j, ceil(2 s p_j) + 4096), as for
// a single call), the p x cap probe positions from ppbase_j and the p + 1
// offsets from obase_j.
#include "hss_internal.cuh"
#include "rounds.cuh"
#include "rounds_dev.cuh"
#include "segsort.cuh"
#include "batch.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace hss {
namespace {

struct BJob {
    uint64_t koff, n;
    uint32_t p, sbase, ibase, pad;
    uint64_t lbase, dbase, cbase, cap, ppbase, tol, seed, obase;
};

struct BCtl {
    uint64_t gamma, T, Z;
    uint32_t take_all, nint, unresolved, active;
};

struct BTotals {
    unsigned long long Zc;  // samples of the jobs that sample this round
    uint32_t active;        // such jobs
    uint32_t pad;
};

inline uint64_t cdivh(uint64_t a, uint64_t b) { return (a + b - 1) / b; }
inline size_t aup(size_t x) { return (x + 255) / 256 * 256; }

__device__ __forceinline__ uint64_t seg_start(const BJob& J, uint32_t s) { return ideal_rank(s, J.n, J.p); }

// ---------------------------------------------------------------------------
// Initial state of every job: intervals (-inf, +inf), whole segments.
// ---------------------------------------------------------------------------
__global__ void kb_init(const BJob* __restrict__ jobs, BCtl* __restrict__ ctl, hss_job_stats* __restrict__ jst,
                        DCut* __restrict__ Lcut, DCut* __restrict__ Ucut, uint32_t* __restrict__ Lpos,
                        uint32_t* __restrict__ Upos) {
    const BJob J = jobs[blockIdx.x];
    const uint32_t S = J.p - 1;
    const uint64_t ent = (uint64_t)J.p * S;
    for (uint64_t e = threadIdx.x; e < ent; e += blockDim.x) {
        const uint32_t s = (uint32_t)(e / S);
        Lpos[J.lbase + e] = 0;
        Upos[J.lbase + e] = (uint32_t)(seg_start(J, s + 1) - seg_start(J, s));
    }
    for (uint32_t i = threadIdx.x; i < S; i += blockDim.x) {
        DCut a; a.okey = 0; a.seg = -2; a.spos = 0; a.rank = 0; a.kind = kNegInf; a.pad = 0;
        DCut b; b.okey = 0; b.seg = -3; b.spos = 0; b.rank = J.n; b.kind = kPosInf; b.pad = 0;
        Lcut[J.ibase + i] = a;
        Ucut[J.ibase + i] = b;
    }
    if (threadIdx.x == 0) {
        BCtl c; c.gamma = 0; c.T = 0; c.Z = 0; c.take_all = 0; c.nint = 0; c.unresolved = 0; c.active = 0;
        ctl[blockIdx.x] = c;
        jst[blockIdx.x].rounds = 0;
        jst[blockIdx.x].status = HSS_OK;
        jst[blockIdx.x].tol = J.tol;
    }
}

// One CTA per job: resolved flags, distinct unresolved intervals, |gamma|,
// next threshold.  A failed job keeps its state.
__global__ __launch_bounds__(1024) void kb_intervals(const BJob* __restrict__ jobs, BCtl* __restrict__ ctl,
                                                     hss_job_stats* __restrict__ jst, const DCut* __restrict__ Lcut,
                                                     const DCut* __restrict__ Ucut, uint32_t* __restrict__ res,
                                                     uint32_t* __restrict__ int_rep, float oversample) {
    const uint32_t j = blockIdx.x;
    const BJob J = jobs[j];
    if (jst[j].status != HSS_OK) return;  // uniform per CTA
    IntervalsOut o;
    intervals_body(J.p - 1, J.n, J.p, J.tol, oversample, Lcut + J.ibase, Ucut + J.ibase, res + J.ibase,
                   int_rep + J.ibase, o);
    if (threadIdx.x == 0) {
        BCtl c = ctl[j];
        c.gamma = o.gamma; c.T = o.T; c.take_all = o.take_all; c.nint = o.nint; c.unresolved = o.unresolved;
        ctl[j] = c;
        const uint32_t r = jst[j].rounds;
        if (r <= HSS_MAX_ROUNDS) jst[j].unresolved[r] = o.unresolved;
    }
}

// Bernoulli draws of one segment of one job (Sec. 4.2.1): as the single-job
// kernel on the job's slices, Philox counter (spos >> 1, local segment,
// round, 0) under the job's seed.
__global__ __launch_bounds__(kSampThreads) void kb_sample_mark(
    const BJob* __restrict__ jobs, const uint32_t* __restrict__ job_of_seg, const BCtl* __restrict__ ctl,
    const hss_job_stats* __restrict__ jst, const uint32_t* __restrict__ Lpos, const uint32_t* __restrict__ Upos,
    const DCut* __restrict__ Lcut, const uint32_t* __restrict__ int_rep, uint32_t round, uint32_t* __restrict__ bitmap,
    uint32_t* __restrict__ seg_cnt) {
    __shared__ uint32_t s_a[kIntChunk], s_b[kIntChunk], s_pre[kIntChunk + 1];
    __shared__ uint32_t s_warp[32];
    const uint32_t g = blockIdx.x;
    const uint32_t j = job_of_seg[g];
    const BJob J = jobs[j];
    const uint32_t nint = ctl[j].nint;
    if (nint == 0 || jst[j].status != HSS_OK) {  // uniform per CTA
        if (threadIdx.x == 0) seg_cnt[g] = 0;
        return;
    }
    const uint32_t s = g - J.sbase, S = J.p - 1;
    const uint64_t base = J.koff + seg_start(J, s);
    const uint32_t n_s = (uint32_t)(seg_start(J, s + 1) - seg_start(J, s));
    const uint64_t T = ctl[j].T;
    const bool take_all = ctl[j].take_all != 0;
    uint32_t cnt = 0;
    for (uint32_t u0 = 0; u0 < nint; u0 += kIntChunk) {
        const uint32_t nu = min((uint32_t)kIntChunk, nint - u0);
        const uint32_t P = load_seg_intervals(s, n_s, S, u0, nu, Lpos + J.lbase, Upos + J.lbase, Lcut + J.ibase,
                                              int_rep + J.ibase, s_a, s_b, s_pre, s_warp);
        for_each_pair(s_pre, nu, P, [&](uint32_t u, uint32_t f) {
            const uint32_t a = s_a[u], b = s_b[u];
            const uint32_t m = (a >> 1) + (f - s_pre[u]);
            uint64_t w0, w1;
            sample_words(J.seed, s, round, m, w0, w1);
            const uint32_t p0 = 2 * m, p1 = 2 * m + 1;
            if (p0 >= a && p0 < b && (take_all || w0 < T)) {
                const uint64_t q = base + p0;
                atomicOr(&bitmap[q >> 5], 1u << (q & 31));
                ++cnt;
            }
            if (p1 >= a && p1 < b && (take_all || w1 < T)) {
                const uint64_t q = base + p1;
                atomicOr(&bitmap[q >> 5], 1u << (q & 31));
                ++cnt;
            }
        });
        __syncthreads();
    }
    uint32_t tot;
    block_incl_scan<uint32_t>(cnt, 0u, AddU32(), s_warp, tot);
    if (threadIdx.x == 0) seg_cnt[g] = tot;
}

// One CTA: exclusive prefix of the segment counts (G), then per job the
// start of a round exactly as the single-job host loop decides it (stop when
// resolved, the round limit, the sample size against the capacity), and the
// offsets of the sampling jobs' samples in the compact sample buffer (zoff).
__global__ __launch_bounds__(1024) void kb_count_scan(uint32_t P_tot, const uint32_t* __restrict__ seg_cnt,
                                                      uint64_t* __restrict__ G, uint32_t njobs,
                                                      const BJob* __restrict__ jobs, BCtl* __restrict__ ctl,
                                                      hss_job_stats* __restrict__ jst, uint32_t max_rounds,
                                                      uint64_t* __restrict__ zoff, BTotals* __restrict__ tot) {
    __shared__ uint64_t s_w64[32];
    __shared__ uint32_t s_w32[32];
    uint64_t carry = 0;
    for (uint32_t b0 = 0; b0 < P_tot; b0 += blockDim.x) {
        const uint32_t g = b0 + threadIdx.x;
        const uint64_t v = g < P_tot ? seg_cnt[g] : 0ull;
        uint64_t t;
        const uint64_t incl = block_incl_scan<uint64_t>(v, 0ull, AddU64(), s_w64, t);
        if (g < P_tot) G[g] = carry + incl - v;
        carry += t;
    }
    if (threadIdx.x == 0) G[P_tot] = carry;
    __syncthreads();
    uint64_t zc_carry = 0;
    uint32_t act_carry = 0;
    for (uint32_t b0 = 0; b0 < njobs; b0 += blockDim.x) {
        const uint32_t j = b0 + threadIdx.x;
        uint64_t zc = 0;
        uint32_t act = 0;
        if (j < njobs) {
            const BJob J = jobs[j];
            BCtl c = ctl[j];
            const uint64_t Z = G[J.sbase + J.p] - G[J.sbase];
            if (jst[j].status == HSS_OK && c.unresolved > 0) {
                if (jst[j].rounds >= max_rounds) {
                    jst[j].status = HSS_ERR_ROUND_LIMIT;
                } else {
                    const uint32_t r = jst[j].rounds;
                    jst[j].sample_size[r] = Z;
                    jst[j].gamma[r] = c.gamma;
                    jst[j].rounds = r + 1;
                    if (Z > J.cap) jst[j].status = HSS_ERR_CAPACITY;
                    else act = 1;
                }
            }
            c.Z = Z;
            c.active = act;
            ctl[j] = c;
            zc = act ? Z : 0;
        }
        uint64_t t;
        const uint64_t incl = block_incl_scan<uint64_t>(zc, 0ull, AddU64(), s_w64, t);
        if (j < njobs) zoff[j] = zc_carry + incl - zc;
        zc_carry += t;
        uint32_t ta;
        block_incl_scan<uint32_t>(act, 0u, AddU32(), s_w32, ta);
        act_carry += ta;
    }
    if (threadIdx.x == 0) {
        zoff[njobs] = zc_carry;
        tot->Zc = zc_carry;
        tot->active = act_carry;
    }
}

// The kept keys of one segment, in position order, into the job's part of
// the compact sample buffer.
__global__ __launch_bounds__(kSampThreads) void kb_sample_write(
    const uint64_t* __restrict__ skeys, const BJob* __restrict__ jobs, const uint32_t* __restrict__ job_of_seg,
    const BCtl* __restrict__ ctl, const uint32_t* __restrict__ bitmap, const uint32_t* __restrict__ seg_cnt,
    const uint64_t* __restrict__ G, const uint64_t* __restrict__ zoff, uint64_t* __restrict__ skey,
    uint32_t* __restrict__ sseg, uint32_t* __restrict__ sspos, uint32_t* __restrict__ siota) {
    __shared__ uint32_t s_warp[32];
    const uint32_t g = blockIdx.x;
    const uint32_t j = job_of_seg[g];
    const uint32_t want = seg_cnt[g];
    if (want == 0 || !ctl[j].active) return;
    const BJob J = jobs[j];
    const uint32_t s = g - J.sbase;
    const uint64_t base = J.koff + seg_start(J, s), end = J.koff + seg_start(J, s + 1);
    const uint64_t w0 = base >> 5, w1 = (end + 31) >> 5;
    uint64_t out = zoff[j] + (G[g] - G[J.sbase]);
    const uint64_t lim = zoff[j + 1];
    uint32_t found = 0;
    for (uint64_t wb = w0; wb < w1 && found < want; wb += kSampThreads) {
        const uint64_t wi = wb + threadIdx.x;
        uint32_t bits = 0;
        if (wi < w1) {
            bits = bitmap[wi];
            const uint64_t g0 = wi << 5;
            if (g0 < base) bits &= ~0u << (uint32_t)(base - g0);
            if (g0 + 32 > end) bits &= (uint32_t)((1ull << (uint32_t)(end - g0)) - 1ull);
        }
        if (__syncthreads_count(bits != 0u) == 0) continue;
        const uint32_t c = __popc(bits);
        uint32_t t;
        const uint32_t incl = block_incl_scan<uint32_t>(c, 0u, AddU32(), s_warp, t);
        uint64_t o = out + incl - c;
        while (bits) {
            const uint32_t b = __ffs(bits) - 1;
            bits &= bits - 1;
            const uint64_t q = (wi << 5) + b;
            if (o < lim) {
                skey[o] = skeys[q];
                sseg[o] = s;
                sspos[o] = (uint32_t)(q - base);
                siota[o] = (uint32_t)o;
            }
            ++o;
        }
        out += t;
        found += t;
    }
}

__device__ __forceinline__ uint32_t job_of_slot(const uint64_t* __restrict__ zoff, uint32_t njobs, uint64_t k) {
    uint32_t lo = 0, hi = njobs;  // last j with zoff[j] <= k
    while (hi - lo > 1) {
        const uint32_t m = (lo + hi) >> 1;
        if (zoff[m] <= k) lo = m; else hi = m;
    }
    return lo;
}

// Probes of every job from its sorted sample: tags and intervals.
__global__ void kb_probe_build(uint64_t Zc, const uint64_t* __restrict__ zoff, uint32_t njobs,
                               const BJob* __restrict__ jobs, const BCtl* __restrict__ ctl,
                               const uint64_t* __restrict__ skey_sorted, const uint32_t* __restrict__ sperm,
                               const uint32_t* __restrict__ sseg, const uint32_t* __restrict__ sspos,
                               const DCut* __restrict__ Ucut, const uint32_t* __restrict__ int_rep,
                               uint64_t* __restrict__ pkey, int32_t* __restrict__ pseg, uint32_t* __restrict__ pspos,
                               uint32_t* __restrict__ pint, uint64_t* __restrict__ prank, uint32_t* __restrict__ pjob) {
    const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Zc) return;
    const uint32_t j = job_of_slot(zoff, njobs, k);
    const BJob J = jobs[j];
    const uint32_t q = sperm[k];
    DCut c;
    c.okey = skey_sorted[k]; c.seg = (int32_t)sseg[q]; c.spos = sspos[q]; c.rank = 0; c.kind = kMember; c.pad = 0;
    pkey[k] = c.okey; pseg[k] = c.seg; pspos[k] = c.spos; prank[k] = 0; pjob[k] = j;
    const DCut* U = Ucut + J.ibase;
    const uint32_t* rep = int_rep + J.ibase;
    uint32_t lo = 0, hi = ctl[j].nint;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (cut_less(c, U[rep[mid]])) hi = mid; else lo = mid + 1;
    }
    pint[k] = lo;
}

// Histogram (Sec. 4.2.2 step 2): every probe against every segment of its
// job, a branch-free search confined to the probe's interval.
constexpr int kBHistSegs = 64;

__global__ __launch_bounds__(256) void kb_histogram(
    const uint64_t* __restrict__ skeys, const BJob* __restrict__ jobs, const uint32_t* __restrict__ pjob,
    const uint64_t* __restrict__ zoff, const uint32_t* __restrict__ Lpos, const uint32_t* __restrict__ Upos,
    const uint32_t* __restrict__ int_rep, const uint64_t* __restrict__ pkey, const int32_t* __restrict__ pseg,
    const uint32_t* __restrict__ pspos, const uint32_t* __restrict__ pint, uint64_t Zc, uint64_t* __restrict__ prank,
    uint32_t* __restrict__ probe_pos, uint32_t* __restrict__ err) {
    __shared__ uint64_t s_part[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint64_t k = (uint64_t)blockIdx.x * 32 + lane;
    const bool valid = k < Zc;
    BJob J;
    uint64_t key = 0, kl = 0;
    int32_t seg = 0;
    uint32_t spos = 0, rep = 0;
    if (valid) {
        const uint32_t j = pjob[k];
        J = jobs[j];
        kl = k - zoff[j];
        key = pkey[k]; seg = pseg[k]; spos = pspos[k]; rep = int_rep[J.ibase + pint[k]];
    } else {
        J.p = 0;
    }
    uint64_t partial = 0;
#pragma unroll 2
    for (int jj = 0; jj < kBHistSegs / 8; ++jj) {
        const uint32_t s = blockIdx.y * kBHistSegs + jj * 8 + w;
        if (valid && s < J.p) {
            const uint32_t S = J.p - 1;
            uint32_t pos;
            if ((int32_t)s == seg) {
                pos = spos;
            } else {
                const uint32_t lo = Lpos[J.lbase + (uint64_t)s * S + rep], hi = Upos[J.lbase + (uint64_t)s * S + rep];
                const uint64_t a = seg_start(J, s);
                const uint32_t n = (uint32_t)(seg_start(J, s + 1) - a);
                if (lo <= hi && hi <= n) {
                    pos = lo + count_below(skeys + J.koff + a + lo, hi - lo, key, (int32_t)s > seg);
                } else {
                    atomicOr(err, kDevErrBounds);
                    pos = lo;
                }
            }
            probe_pos[J.ppbase + (uint64_t)s * J.cap + kl] = pos;
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

// L/U update of every splitter of the sampling jobs from their ranked
// probes.  cl/cu are probe indices local to the job.
__global__ void kb_update(uint32_t S_tot, const BJob* __restrict__ jobs, const uint32_t* __restrict__ job_of_spl,
                          const BCtl* __restrict__ ctl, const uint64_t* __restrict__ zoff,
                          const uint64_t* __restrict__ pkey, const int32_t* __restrict__ pseg,
                          const uint32_t* __restrict__ pspos, const uint64_t* __restrict__ prank,
                          DCut* __restrict__ Lcut, DCut* __restrict__ Ucut, int32_t* __restrict__ chgL,
                          int32_t* __restrict__ chgU) {
    const uint32_t gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= S_tot) return;
    const uint32_t j = job_of_spl[gi];
    int32_t cl = -1, cu = -1;
    if (ctl[j].active) {
        const BJob J = jobs[j];
        const uint32_t i = gi - J.ibase;
        const uint64_t t = ideal_rank(i + 1, J.n, J.p);
        const uint64_t z0 = zoff[j], z1 = zoff[j + 1];
        uint64_t lo = z0, hi = z1;  // first probe with rank > t
        while (lo < hi) { const uint64_t m = (lo + hi) >> 1; if (prank[m] <= t) lo = m + 1; else hi = m; }
        const uint64_t kgt = lo;
        lo = z0; hi = z1;           // first probe with rank >= t
        while (lo < hi) { const uint64_t m = (lo + hi) >> 1; if (prank[m] < t) lo = m + 1; else hi = m; }
        const uint64_t kge = lo;
        DCut L = Lcut[gi], U = Ucut[gi];
        auto probe = [&](uint64_t k) {
            DCut c; c.okey = pkey[k]; c.seg = pseg[k]; c.spos = pspos[k]; c.rank = prank[k]; c.kind = kMember; c.pad = 0;
            return c;
        };
        if (kgt > z0) offer(L, U, cl, cu, t, probe(kgt - 1), (int32_t)(kgt - 1 - z0));
        if (kge < z1) offer(L, U, cl, cu, t, probe(kge), (int32_t)(kge - z0));
        Lcut[gi] = L;
        Ucut[gi] = U;
    }
    chgL[gi] = cl;
    chgU[gi] = cu;
}

// Per-segment positions of the changed cuts (one CTA per sampling job).
__global__ void kb_update_pos(const BJob* __restrict__ jobs, const BCtl* __restrict__ ctl,
                              const int32_t* __restrict__ chgL, const int32_t* __restrict__ chgU,
                              const uint32_t* __restrict__ probe_pos, uint32_t* __restrict__ Lpos,
                              uint32_t* __restrict__ Upos) {
    const uint32_t j = blockIdx.x;
    if (!ctl[j].active) return;
    const BJob J = jobs[j];
    const uint32_t S = J.p - 1;
    const uint64_t ent = (uint64_t)J.p * S;
    for (uint64_t e = threadIdx.x; e < ent; e += blockDim.x) {
        const uint32_t s = (uint32_t)(e / S), i = (uint32_t)(e % S);
        const int32_t cl = chgL[J.ibase + i], cu = chgU[J.ibase + i];
        if (cl >= 0) Lpos[J.lbase + e] = probe_pos[J.ppbase + (uint64_t)s * J.cap + (uint32_t)cl];
        if (cu >= 0) Upos[J.lbase + e] = probe_pos[J.ppbase + (uint64_t)s * J.cap + (uint32_t)cu];
    }
}

// Final splitters (the closer of L_i, U_i; tie -> L_i), offsets relative to
// the job, and the per-segment positions of the chosen cuts.
__global__ void kb_finalize(uint32_t S_tot, const BJob* __restrict__ jobs, const uint32_t* __restrict__ job_of_spl,
                            int key_type, const DCut* __restrict__ Lcut, const DCut* __restrict__ Ucut,
                            hss_cut* __restrict__ spl, uint64_t* __restrict__ offsets, uint32_t* __restrict__ choose_u) {
    const uint32_t gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= S_tot) return;
    const BJob J = jobs[job_of_spl[gi]];
    const uint32_t i = gi - J.ibase;
    const uint64_t t = ideal_rank(i + 1, J.n, J.p);
    const DCut L = Lcut[gi], U = Ucut[gi];
    const bool useU = (U.rank - t) < (t - L.rank);
    const DCut c = useU ? U : L;
    hss_cut o;
    const uint64_t flip = key_type == HSS_KEY_I64 ? kSignBit : 0ull;
    if (c.kind == kMember) { o.key = c.okey ^ flip; o.seg = c.seg; o.spos = c.spos; }
    else if (c.kind == kNonMember) { o.key = c.okey ^ flip; o.seg = -1; o.spos = 0; }
    else if (c.kind == kNegInf) { o.key = 0; o.seg = -2; o.spos = 0; }
    else { o.key = 0; o.seg = -3; o.spos = 0; }
    spl[gi] = o;
    offsets[J.obase + i + 1] = c.rank;
    choose_u[gi] = useU ? 1u : 0u;
}

__global__ void kb_final_pos(const BJob* __restrict__ jobs, const uint32_t* __restrict__ choose_u,
                             uint32_t* __restrict__ Lpos, const uint32_t* __restrict__ Upos,
                             uint64_t* __restrict__ offsets) {
    const BJob J = jobs[blockIdx.x];
    const uint32_t S = J.p - 1;
    if (threadIdx.x == 0) { offsets[J.obase] = 0; offsets[J.obase + J.p] = J.n; }
    const uint64_t ent = (uint64_t)J.p * S;
    for (uint64_t e = threadIdx.x; e < ent; e += blockDim.x) {
        const uint32_t i = (uint32_t)(e % S);
        if (choose_u[J.ibase + i]) Lpos[J.lbase + e] = Upos[J.lbase + e];
    }
}

// ---------------------------------------------------------------------------
// Exchange (Sec. 3.1 step 3) of every job: runs of its sorted segments to its
// buckets, inside the job's own key range.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t bpos(const uint32_t* __restrict__ pos, uint32_t S, uint32_t p, uint32_t s, uint32_t b,
                                         uint32_t n) {
    return b == 0 ? 0u : (b == p ? n : pos[(uint64_t)s * S + (b - 1)]);
}

// CTA (x, j): buckets 32x .. 32x+31 of job j; its 32 warps split the job's
// segments into groups, sum, scan the group sums and write destinations.
__global__ __launch_bounds__(1024) void kb_exchange_dst(const BJob* __restrict__ jobs, const uint32_t* __restrict__ pos,
                                                        const uint64_t* __restrict__ offsets, uint64_t* __restrict__ dst,
                                                        uint32_t* __restrict__ err) {
    __shared__ uint64_t s_part[32][33];
    const BJob J = jobs[blockIdx.y];
    const uint32_t p = J.p;
    if (blockIdx.x * 32 >= p) return;  // uniform per CTA
    const uint32_t col = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const uint32_t b = blockIdx.x * 32 + col;
    const uint32_t S = p - 1;
    const uint32_t R = (p + 31) / 32;
    const uint32_t s0 = min(p, grp * R), s1 = min(p, s0 + R);
    const uint32_t* P = pos + J.lbase;
    uint64_t part = 0;
    if (b < p) {
        for (uint32_t s = s0; s < s1; ++s) {
            const uint32_t n = (uint32_t)(seg_start(J, s + 1) - seg_start(J, s));
            part += bpos(P, S, p, s, b + 1, n) - bpos(P, S, p, s, b, n);
        }
    }
    s_part[grp][col] = part;
    __syncthreads();
    if (b >= p) return;
    const uint64_t* off = offsets + J.obase;
    uint64_t run = J.koff + off[b];
    for (uint32_t g = 0; g < grp; ++g) run += s_part[g][col];
    for (uint32_t s = s0; s < s1; ++s) {
        const uint32_t n = (uint32_t)(seg_start(J, s + 1) - seg_start(J, s));
        dst[J.dbase + (uint64_t)s * p + b] = run;
        run += bpos(P, S, p, s, b + 1, n) - bpos(P, S, p, s, b, n);
    }
    if (s1 == p && s0 < s1 && run != J.koff + off[b + 1]) atomicOr(err, kDevErrBounds);
}

constexpr uint32_t kBXchChunk = 8192;
constexpr uint32_t kBXchMaxB = 2048;

// CTA (g, y): keys [y kBXchChunk, (y + 1) kBXchChunk) of segment g.  The run
// boundaries of the buckets that chunk meets are staged in shared memory;
// each thread moves four keys per step (their loads issued together) and
// finds each key's run by galloping forward from the previous one.
__global__ __launch_bounds__(256) void kb_exchange_copy(const uint64_t* __restrict__ skeys, const uint32_t* __restrict__ spay,
                                                        const BJob* __restrict__ jobs,
                                                        const uint32_t* __restrict__ job_of_seg,
                                                        const uint32_t* __restrict__ pos, const uint64_t* __restrict__ dst,
                                                        uint64_t* __restrict__ bkeys, uint32_t* __restrict__ bpay,
                                                        uint32_t* __restrict__ err) {
    __shared__ uint32_t s_bnd[kBXchMaxB + 1];
    __shared__ uint32_t s_b0, s_nb;
    const uint32_t g = blockIdx.x;
    const BJob J = jobs[job_of_seg[g]];
    const uint32_t s = g - J.sbase, p = J.p, S = p - 1;
    const uint64_t base = J.koff + seg_start(J, s);
    const uint32_t n = (uint32_t)(seg_start(J, s + 1) - seg_start(J, s));
    const uint32_t c0 = blockIdx.y * kBXchChunk;
    if (c0 >= n) return;
    const uint32_t c1 = min(n, c0 + kBXchChunk);
    const uint32_t* P = pos + J.lbase;
    if (threadIdx.x < 32) {  // 32-way warp searches for the buckets meeting [c0, c1)
        auto last_le = [&](uint32_t v, uint32_t lo, uint32_t hi) {
            const uint32_t lane = threadIdx.x & 31;
            while (hi - lo > 1) {
                const uint32_t step = (hi - lo + 31) / 32;
                const uint32_t m = lo + lane * step;
                const bool ok = m < hi && bpos(P, S, p, s, m, n) <= v;
                const uint32_t bal = __ballot_sync(0xffffffffu, ok);
                lo = lo + (31 - __clz(bal)) * step;
                hi = min(hi, lo + step);
            }
            return lo;
        };
        const uint32_t b0 = last_le(c0, 0, p);
        const uint32_t b1 = last_le(c1 - 1, b0, p);
        if (threadIdx.x == 0) {
            s_b0 = b0;
            s_nb = b1 - b0 + 1;
        }
    }
    __syncthreads();
    const uint32_t b0 = s_b0, nb = s_nb;
    const uint64_t lim = J.koff + J.n;
    const uint64_t* D = dst + J.dbase + (uint64_t)s * p;
    if (nb <= kBXchMaxB) {
        for (uint32_t i = threadIdx.x; i <= nb; i += blockDim.x) s_bnd[i] = bpos(P, S, p, s, b0 + i, n);
        __syncthreads();
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
                const uint64_t d = D[b0 + lo] + (j - s_bnd[lo]);
                if (d < J.koff || d >= lim) { atomicOr(err, kDevErrBounds); continue; }
                bkeys[d] = kv[u];
                if (bpay) bpay[d] = pv[u];
            }
        }
    } else {
        for (uint32_t q = c0 + threadIdx.x; q < c1; q += blockDim.x) {
            uint32_t lo = b0, hi = b0 + nb;  // last bucket whose run starts at or before q
            while (hi - lo > 1) { const uint32_t m = (lo + hi) >> 1; if (bpos(P, S, p, s, m, n) <= q) lo = m; else hi = m; }
            const uint64_t d = D[lo] + (q - bpos(P, S, p, s, lo, n));
            if (d < J.koff || d >= lim) { atomicOr(err, kDevErrBounds); continue; }
            bkeys[d] = skeys[base + q];
            if (bpay) bpay[d] = spay[base + q];
        }
    }
}

// Absolute bucket boundaries of all jobs: the segments of the merge.
__global__ void kb_bucket_off(uint32_t P_tot, uint64_t N_tot, const BJob* __restrict__ jobs,
                              const uint32_t* __restrict__ job_of_seg, const uint64_t* __restrict__ offsets,
                              uint64_t* __restrict__ boff) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g > P_tot) return;
    if (g == P_tot) { boff[g] = N_tot; return; }
    const BJob J = jobs[job_of_seg[g]];
    boff[g] = J.koff + offsets[J.obase + (g - J.sbase)];
}

// Key range of every job: the smallest first key and the largest last key
// of its locally sorted segments.
__global__ __launch_bounds__(256) void kb_key_range(const uint64_t* __restrict__ skeys, const BJob* __restrict__ jobs,
                                                    const uint64_t* __restrict__ seg_off, uint64_t* __restrict__ range) {
    __shared__ uint64_t s_lo[8], s_hi[8];
    const BJob J = jobs[blockIdx.x];
    uint64_t lo = ~0ull, hi = 0ull;
    for (uint32_t s = threadIdx.x; s < J.p; s += blockDim.x) {
        const uint64_t a = seg_off[J.sbase + s], b = seg_off[J.sbase + s + 1];
        if (a < b) {
            lo = min(lo, skeys[a]);
            hi = max(hi, skeys[b - 1]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) { s_lo[threadIdx.x >> 5] = lo; s_hi[threadIdx.x >> 5] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) { lo = min(lo, s_lo[w]); hi = max(hi, s_hi[w]); }
        range[2 * (uint64_t)blockIdx.x] = lo;
        range[2 * (uint64_t)blockIdx.x + 1] = hi;
    }
}

// Window of every bucket for the first split of the merge: its keys lie
// between the job's final cuts b and b + 1 (tag order), clipped to the job's
// key range; mulhi(key - lo, mult) maps that interval onto 0..255.
__global__ void kb_bucket_hint(uint32_t P_tot, const BJob* __restrict__ jobs, const uint32_t* __restrict__ job_of_seg,
                               const DCut* __restrict__ Lcut, const DCut* __restrict__ Ucut,
                               const uint32_t* __restrict__ choose_u, const uint64_t* __restrict__ range,
                               uint64_t* __restrict__ lo_out, uint64_t* __restrict__ mult_out) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P_tot) return;
    const uint32_t j = job_of_seg[g];
    const BJob J = jobs[j];
    const uint32_t b = g - J.sbase;
    auto bound = [&](uint32_t i, uint64_t if_none) -> uint64_t {  // cut i (1..p-1) of the job
        if (i == 0 || i == J.p) return if_none;
        const uint32_t gi = J.ibase + i - 1;
        const DCut c = choose_u[gi] ? Ucut[gi] : Lcut[gi];
        if (c.kind == kNegInf) return 0ull;
        if (c.kind == kPosInf) return ~0ull;
        return c.okey;
    };
    const uint64_t lo = max(bound(b, 0ull), range[2 * (uint64_t)j]);
    uint64_t hi = min(bound(b + 1, ~0ull), range[2 * (uint64_t)j + 1]);
    if (hi < lo) hi = lo;  // empty bucket
    const uint64_t r = hi - lo;
    lo_out[g] = lo;
    mult_out[g] = r < 256 ? 0ull : (uint64_t)(((unsigned __int128)255 << 64) / r);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
struct Tables {
    std::vector<BJob> jobs;
    std::vector<uint32_t> job_of_seg, job_of_spl;
    std::vector<uint64_t> seg_off;
    uint64_t N_tot = 0, L_tot = 0, D_tot = 0, C_tot = 0, PP_tot = 0, O_tot = 0;
    uint32_t P_tot = 0, S_tot = 0, max_p = 0, max_seg = 0;
};

int build_tables(const uint64_t* sizes, const uint32_t* ps, uint32_t njobs, const hss_params* prm, Tables& T,
                 const uint64_t* seeds = nullptr) {
    T.jobs.resize(njobs);
    uint64_t koff = 0, lb = 0, db = 0, cb = 0, pp = 0, ob = 0;
    uint32_t sb = 0, ib = 0;
    for (uint32_t j = 0; j < njobs; ++j) {
        const uint64_t n = sizes[j];
        const uint32_t p = ps[j];
        if (p == 0 || p > (1u << 16) || (uint64_t)p > std::max<uint64_t>(n, 1)) return HSS_ERR_INVALID;
        // every segment and every eps-balanced bucket below 2^30 keys
        const double extra = 2.0 * std::floor(((double)n * prm->eps) / (2.0 * (double)p));
        if ((double)((n + p - 1) / p) + extra + 1.0 >= (double)kMaxSegKeys) return HSS_ERR_INVALID;
        BJob& J = T.jobs[j];
        J.koff = koff; J.n = n; J.p = p; J.sbase = sb; J.ibase = ib; J.pad = 0;
        J.lbase = lb; J.dbase = db; J.cbase = cb;
        J.cap = sample_capacity(n, p, prm->oversample);
        J.ppbase = pp;
        J.tol = (uint64_t)std::floor(((double)n * prm->eps) / (2.0 * (double)p));
        J.seed = seeds ? seeds[j] : prm->seed + j;
        J.obase = ob;
        for (uint32_t s = 0; s < p; ++s) {
            T.seg_off.push_back(koff + (uint64_t)(((unsigned __int128)s * n) / p));
            T.job_of_seg.push_back(j);
            const uint64_t len = (uint64_t)(((unsigned __int128)(s + 1) * n) / p) - (uint64_t)(((unsigned __int128)s * n) / p);
            T.max_seg = std::max<uint32_t>(T.max_seg, (uint32_t)len);
        }
        for (uint32_t i = 0; i + 1 < p; ++i) T.job_of_spl.push_back(j);
        koff += n; sb += p; ib += p - 1;
        lb += (uint64_t)p * (p - 1); db += (uint64_t)p * p; cb += J.cap; pp += (uint64_t)p * J.cap; ob += p + 1;
        T.max_p = std::max(T.max_p, p);
    }
    T.seg_off.push_back(koff);
    T.N_tot = koff; T.P_tot = sb; T.S_tot = ib; T.L_tot = lb; T.D_tot = db; T.C_tot = cb; T.PP_tot = pp; T.O_tot = ob;
    return HSS_OK;
}

struct BLayout {
    size_t keysA, keysB, payA, payB, seg_off, err, sws, jobs, jseg, jspl, ctl, jst, tot, Lcut, Ucut, res, chgL, chgU,
        choose_u, int_rep, Lpos, Upos, bitmap, seg_cnt, G, zoff, skey, skey_sorted, stmp, sseg, sspos, siota, sperm,
        ptmp, pkey, prank, pseg, pspos, pint, pjob, probe_pos, dst, boff, hlo, hmult, jrange, sws_s, spl_in, off_in,
        total;
};

BLayout plan_batch(const Tables& T, uint32_t njobs, bool pay, bool sort) {
    BLayout L{};
    size_t o = 0;
    auto take = [&](size_t b) { size_t r = o; o += aup(std::max<size_t>(b, 1)); return r; };
    const uint64_t N1 = std::max<uint64_t>(T.N_tot, 1), C1 = std::max<uint64_t>(T.C_tot, 1);
    const uint64_t S1 = std::max<uint32_t>(T.S_tot, 1);
    L.keysA = take(N1 * 8); L.keysB = take(N1 * 8);
    L.payA = pay ? take(N1 * 4) : 0; L.payB = pay ? take(N1 * 4) : 0;
    L.seg_off = take(((uint64_t)T.P_tot + 1) * 8);
    L.err = take(256);
    L.sws = take(segsort_ws_bytes(N1, T.P_tot));
    L.jobs = take(njobs * sizeof(BJob));
    L.jseg = take((uint64_t)T.P_tot * 4);
    L.jspl = take(S1 * 4);
    L.ctl = take(njobs * sizeof(BCtl));
    L.jst = take(njobs * sizeof(hss_job_stats));
    L.tot = take(sizeof(BTotals));
    L.Lcut = take(S1 * sizeof(DCut)); L.Ucut = take(S1 * sizeof(DCut));
    L.res = take(S1 * 4); L.chgL = take(S1 * 4); L.chgU = take(S1 * 4); L.choose_u = take(S1 * 4); L.int_rep = take(S1 * 4);
    L.Lpos = take(std::max<uint64_t>(T.L_tot, 1) * 4); L.Upos = take(std::max<uint64_t>(T.L_tot, 1) * 4);
    L.bitmap = take((N1 / 32 + 2) * 4);
    L.seg_cnt = take((uint64_t)T.P_tot * 4);
    L.G = take(((uint64_t)T.P_tot + 1) * 8);
    L.zoff = take(((uint64_t)njobs + 1) * 8);
    L.skey = take(C1 * 8); L.skey_sorted = take(C1 * 8); L.stmp = take(C1 * 8);
    L.sseg = take(C1 * 4); L.sspos = take(C1 * 4); L.siota = take(C1 * 4); L.sperm = take(C1 * 4); L.ptmp = take(C1 * 4);
    L.pkey = take(C1 * 8); L.prank = take(C1 * 8);
    L.pseg = take(C1 * 4); L.pspos = take(C1 * 4); L.pint = take(C1 * 4); L.pjob = take(C1 * 4);
    L.probe_pos = take(std::max<uint64_t>(T.PP_tot, 1) * 4);
    L.dst = sort ? take(std::max<uint64_t>(T.D_tot, 1) * 8) : 0;
    L.boff = sort ? take(((uint64_t)T.P_tot + 1) * 8) : 0;
    L.hlo = sort ? take((uint64_t)T.P_tot * 8) : 0;
    L.hmult = sort ? take((uint64_t)T.P_tot * 8) : 0;
    L.jrange = sort ? take((uint64_t)njobs * 16) : 0;
    L.sws_s = take(segsort_ws_bytes(C1, njobs));
    L.total = o;
    return L;
}

template <typename T>
T* at(void* base, size_t off) { return (T*)((char*)base + off); }

#define HSS_BTRY(x) do { if ((x) != cudaSuccess) return HSS_ERR_CUDA; } while (0)

}  // namespace

int run_batch(const void* d_keys, const uint32_t* d_payload, int key_type, const uint64_t* h_sizes, const uint32_t* h_p,
              uint32_t njobs, const hss_params* prm, void* d_keys_out, uint32_t* d_payload_out, hss_cut* d_splitters,
              uint64_t* d_offsets, void* d_work, size_t work_bytes, hss_batch_stats* h_stats,
              hss_job_stats* h_job_stats, cudaStream_t st, bool sort, const BatchExtra& ex) {
    const uint64_t mark = hss_kernel_launch_count();
    if (h_stats) std::memset(h_stats, 0, sizeof(*h_stats));
    if (!prm || !(prm->eps > 0.0) || !(prm->oversample > 0.0f) || njobs == 0 || !h_sizes || !h_p) return HSS_ERR_INVALID;
    if (prm->schedule != HSS_SCHEDULE_PROPORTIONAL) return HSS_ERR_INVALID;
    if (key_type != HSS_KEY_U64 && key_type != HSS_KEY_I64) return HSS_ERR_INVALID;
    Tables T;
    if (build_tables(h_sizes, h_p, njobs, prm, T, ex.seeds) != HSS_OK) return HSS_ERR_INVALID;
    if ((T.N_tot > 0 && !d_keys) || !d_offsets || (T.S_tot > 0 && !d_splitters) || !d_work) return HSS_ERR_INVALID;
    const bool pay = sort && d_payload != nullptr;
    if (sort && ((d_payload == nullptr) != (d_payload_out == nullptr))) return HSS_ERR_INVALID;
    if (sort && T.N_tot > 0 && !d_keys_out) return HSS_ERR_INVALID;
    const BLayout L = plan_batch(T, njobs, pay, sort);
    if (work_bytes < L.total) return HSS_ERR_WORKSPACE;
    const uint32_t max_rounds = prm->max_rounds == 0 ? HSS_MAX_ROUNDS : std::min<uint32_t>(prm->max_rounds, HSS_MAX_ROUNDS);
    const bool i64 = key_type == HSS_KEY_I64;

    uint64_t* keysA = at<uint64_t>(d_work, L.keysA);
    uint64_t* keysB = at<uint64_t>(d_work, L.keysB);
    uint32_t* payA = pay ? at<uint32_t>(d_work, L.payA) : nullptr;
    uint32_t* payB = pay ? at<uint32_t>(d_work, L.payB) : nullptr;
    uint64_t* seg_off = at<uint64_t>(d_work, L.seg_off);
    uint32_t* err = at<uint32_t>(d_work, L.err);
    BJob* jobs = at<BJob>(d_work, L.jobs);
    uint32_t* jseg = at<uint32_t>(d_work, L.jseg);
    uint32_t* jspl = at<uint32_t>(d_work, L.jspl);
    BCtl* ctl = at<BCtl>(d_work, L.ctl);
    hss_job_stats* jst = at<hss_job_stats>(d_work, L.jst);
    BTotals* tot = at<BTotals>(d_work, L.tot);
    DCut* Lcut = at<DCut>(d_work, L.Lcut);
    DCut* Ucut = at<DCut>(d_work, L.Ucut);
    uint32_t* res = at<uint32_t>(d_work, L.res);
    int32_t* chgL = at<int32_t>(d_work, L.chgL);
    int32_t* chgU = at<int32_t>(d_work, L.chgU);
    uint32_t* choose_u = at<uint32_t>(d_work, L.choose_u);
    uint32_t* int_rep = at<uint32_t>(d_work, L.int_rep);
    uint32_t* Lpos = at<uint32_t>(d_work, L.Lpos);
    uint32_t* Upos = at<uint32_t>(d_work, L.Upos);
    uint32_t* bitmap = at<uint32_t>(d_work, L.bitmap);
    uint32_t* seg_cnt = at<uint32_t>(d_work, L.seg_cnt);
    uint64_t* G = at<uint64_t>(d_work, L.G);
    uint64_t* zoff = at<uint64_t>(d_work, L.zoff);
    uint64_t* skey = at<uint64_t>(d_work, L.skey);
    uint64_t* skey_sorted = at<uint64_t>(d_work, L.skey_sorted);
    uint64_t* stmp = at<uint64_t>(d_work, L.stmp);
    uint32_t* sseg = at<uint32_t>(d_work, L.sseg);
    uint32_t* sspos = at<uint32_t>(d_work, L.sspos);
    uint32_t* siota = at<uint32_t>(d_work, L.siota);
    uint32_t* sperm = at<uint32_t>(d_work, L.sperm);
    uint32_t* ptmp = at<uint32_t>(d_work, L.ptmp);
    uint64_t* pkey = at<uint64_t>(d_work, L.pkey);
    uint64_t* prank = at<uint64_t>(d_work, L.prank);
    int32_t* pseg = at<int32_t>(d_work, L.pseg);
    uint32_t* pspos = at<uint32_t>(d_work, L.pspos);
    uint32_t* pint = at<uint32_t>(d_work, L.pint);
    uint32_t* pjob = at<uint32_t>(d_work, L.pjob);
    uint32_t* probe_pos = at<uint32_t>(d_work, L.probe_pos);
    SegSortWs sws = segsort_ws_carve(at<void>(d_work, L.sws), std::max<uint64_t>(T.N_tot, 1), T.P_tot, err);
    SegSortWs sws_s = segsort_ws_carve(at<void>(d_work, L.sws_s), std::max<uint64_t>(T.C_tot, 1), njobs, err);

    // Tables to the device (the host vectors stay alive until the copies end).
    HSS_BTRY(cudaMemsetAsync(err, 0, 256, st));
    HSS_BTRY(cudaMemsetAsync(jst, 0, njobs * sizeof(hss_job_stats), st));
    HSS_BTRY(cudaMemcpyAsync(jobs, T.jobs.data(), njobs * sizeof(BJob), cudaMemcpyHostToDevice, st));
    HSS_BTRY(cudaMemcpyAsync(jseg, T.job_of_seg.data(), (size_t)T.P_tot * 4, cudaMemcpyHostToDevice, st));
    if (T.S_tot) HSS_BTRY(cudaMemcpyAsync(jspl, T.job_of_spl.data(), (size_t)T.S_tot * 4, cudaMemcpyHostToDevice, st));
    HSS_BTRY(cudaMemcpyAsync(seg_off, T.seg_off.data(), ((size_t)T.P_tot + 1) * 8, cudaMemcpyHostToDevice, st));

    float ms[4] = {0, 0, 0, 0};
    TimingEvents<5> tev;
    cudaEvent_t* ev = tev.ev;
    const bool timing = (prm->flags & HSS_FLAG_TIMING) != 0;
    if (timing) {
        tev.create();
        cudaEventRecord(ev[0], st);
    }

    // Local sort of every segment of every job.
    HSS_BTRY(segsort((const uint64_t*)d_keys, keysA, keysB, d_payload, pay ? payA : nullptr, pay ? payB : nullptr, T.N_tot,
                     T.P_tot, seg_off, i64 && !ex.keys_ordered, false, sws, st, nullptr, ex.hint_lo, ex.hint_mult));
    if (timing) cudaEventRecord(ev[1], st);

    // Rounds, all jobs in lock step.
    const float s = prm->oversample;
    const unsigned sblk = (unsigned)cdivh(std::max<uint32_t>(T.S_tot, 1), 256);
    HSS_LAUNCH(kb_init, njobs, 256, 0, st, jobs, ctl, jst, Lcut, Ucut, Lpos, Upos);
    HSS_LAUNCH(kb_intervals, njobs, 1024, 0, st, jobs, ctl, jst, Lcut, Ucut, res, int_rep, s);
    auto sampling = [&](uint32_t round) {
        cudaMemsetAsync(bitmap, 0, (T.N_tot / 32 + 2) * 4, st);
        HSS_LAUNCH(kb_sample_mark, T.P_tot, kSampThreads, 0, st, jobs, jseg, ctl, jst, Lpos, Upos, Lcut, int_rep, round,
                   bitmap, seg_cnt);
        HSS_LAUNCH(kb_count_scan, 1, 1024, 0, st, T.P_tot, seg_cnt, G, njobs, jobs, ctl, jst, max_rounds, zoff, tot);
    };
    sampling(1);
    BTotals h;
    uint32_t round = 0;
    for (;;) {
        HSS_BTRY(cudaGetLastError());
        HSS_BTRY(read_small(&h, tot, sizeof(h), st));
        if (h.active == 0) break;
        ++round;
        const uint64_t Zc = h.Zc;
        HSS_LAUNCH(kb_sample_write, T.P_tot, kSampThreads, 0, st, keysA, jobs, jseg, ctl, bitmap, seg_cnt, G, zoff, skey,
                   sseg, sspos, siota);
        if (Zc > 0) {
            HSS_BTRY(segsort(skey, skey_sorted, stmp, siota, sperm, ptmp, Zc, njobs, zoff, false, false, sws_s, st,
                             nullptr));
            HSS_LAUNCH(kb_probe_build, (unsigned)cdivh(Zc, 256), 256, 0, st, Zc, zoff, njobs, jobs, ctl, skey_sorted, sperm,
                       sseg, sspos, Ucut, int_rep, pkey, pseg, pspos, pint, prank, pjob);
            HSS_LAUNCH(kb_histogram, dim3((unsigned)cdivh(Zc, 32), (unsigned)cdivh(T.max_p, kBHistSegs)), 256, 0, st,
                       keysA, jobs, pjob, zoff, Lpos, Upos, int_rep, pkey, pseg, pspos, pint, Zc, prank, probe_pos, err);
        }
        if (T.S_tot) {
            HSS_LAUNCH(kb_update, sblk, 256, 0, st, T.S_tot, jobs, jspl, ctl, zoff, pkey, pseg, pspos, prank, Lcut, Ucut,
                       chgL, chgU);
            HSS_LAUNCH(kb_update_pos, njobs, 256, 0, st, jobs, ctl, chgL, chgU, probe_pos, Lpos, Upos);
        }
        HSS_LAUNCH(kb_intervals, njobs, 1024, 0, st, jobs, ctl, jst, Lcut, Ucut, res, int_rep, s);
        sampling(round + 1);
    }
    uint64_t* offsets = d_offsets;
    if (T.S_tot)
        HSS_LAUNCH(kb_finalize, sblk, 256, 0, st, T.S_tot, jobs, jspl, key_type, Lcut, Ucut, d_splitters, offsets, choose_u);
    HSS_LAUNCH(kb_final_pos, njobs, 256, 0, st, jobs, choose_u, Lpos, Upos, offsets);
    if (timing) cudaEventRecord(ev[2], st);

    if (sort) {
        uint64_t* dst = at<uint64_t>(d_work, L.dst);
        uint64_t* boff = at<uint64_t>(d_work, L.boff);
        uint64_t* hlo = at<uint64_t>(d_work, L.hlo);
        uint64_t* hmult = at<uint64_t>(d_work, L.hmult);
        uint64_t* jrange = at<uint64_t>(d_work, L.jrange);
        // The merge's first split interpolates each bucket's key window
        // (computed while the locally sorted keys are still in keysA).
        HSS_LAUNCH(kb_key_range, njobs, 256, 0, st, keysA, jobs, seg_off, jrange);
        HSS_LAUNCH(kb_bucket_hint, (unsigned)cdivh(T.P_tot, 256), 256, 0, st, T.P_tot, jobs, jseg, Lcut, Ucut, choose_u,
                   jrange, hlo, hmult);
        if (T.N_tot > 0) {
            HSS_LAUNCH(kb_exchange_dst, dim3((unsigned)cdivh(T.max_p, 32), njobs), 1024, 0, st, jobs, Lpos, offsets, dst,
                       err);
            HSS_LAUNCH(kb_exchange_copy, dim3(T.P_tot, (unsigned)cdivh(std::max<uint32_t>(T.max_seg, 1), kBXchChunk)), 256,
                       0, st, keysA, payA, jobs, jseg, Lpos, dst, keysB, payB, err);
        }
        if (timing) cudaEventRecord(ev[3], st);
        HSS_LAUNCH(kb_bucket_off, (unsigned)cdivh((uint64_t)T.P_tot + 1, 256), 256, 0, st, T.P_tot, T.N_tot, jobs, jseg,
                   offsets, boff);
        HSS_BTRY(segsort(keysB, (uint64_t*)d_keys_out, keysA, payB, d_payload_out, payA, T.N_tot, T.P_tot, boff, false, i64,
                         sws, st, nullptr, hlo, hmult));
        if (timing) cudaEventRecord(ev[4], st);
    }
    HSS_BTRY(cudaGetLastError());

    uint32_t h_err = 0;
    HSS_BTRY(cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, st));
    std::vector<hss_job_stats> js(njobs);
    HSS_BTRY(cudaMemcpyAsync(js.data(), jst, njobs * sizeof(hss_job_stats), cudaMemcpyDeviceToHost, st));
    HSS_BTRY(cudaStreamSynchronize(st));
    int status = HSS_OK;
    if (h_err & kDevErrTimeout) status = HSS_ERR_TIMEOUT;
    else if (h_err & kDevErrSize) status = HSS_ERR_INVALID;
    else if (h_err & kDevErrBounds) status = HSS_ERR_CUDA;
    uint32_t maxr = 0;
    uint64_t samples = 0;
    for (uint32_t j = 0; j < njobs; ++j) {
        maxr = std::max(maxr, js[j].rounds);
        for (uint32_t r = 0; r < js[j].rounds && r < HSS_MAX_ROUNDS; ++r) samples += js[j].sample_size[r];
        if (status == HSS_OK && js[j].status != HSS_OK) status = js[j].status;
    }
    if (h_job_stats) std::memcpy(h_job_stats, js.data(), njobs * sizeof(hss_job_stats));
    if (h_stats) {
        h_stats->njobs = njobs;
        h_stats->max_rounds = maxr;
        h_stats->lockstep_rounds = round;
        h_stats->status = status;
        h_stats->total_samples = samples;
        h_stats->total_keys = T.N_tot;
        h_stats->total_segments = T.P_tot;
        if (timing) {
            cudaEventElapsedTime(&ms[0], ev[0], ev[1]);
            cudaEventElapsedTime(&ms[1], ev[1], ev[2]);
            if (sort) {
                cudaEventElapsedTime(&ms[2], ev[2], ev[3]);
                cudaEventElapsedTime(&ms[3], ev[3], ev[4]);
            }
            for (int k = 0; k < 4; ++k) h_stats->ms_phase[k] = ms[k];
        }
        h_stats->kernel_launches = (uint32_t)(hss_kernel_launch_count() - mark);
    }
    return status;
}

size_t batch_bytes_bound(uint64_t N, uint32_t njobs, uint32_t pj, const hss_params* prm, bool pay) {
    if (!prm || njobs == 0 || pj == 0) return 0;
    // The layout depends on the sizes only through the sample capacities,
    // each at most ceil(2 s p_j) + 4096 whatever the job's size: lay out
    // jobs of equal size and the largest capacity.
    std::vector<uint64_t> sizes(njobs);
    for (uint32_t j = 0; j < njobs; ++j)
        sizes[j] = (uint64_t)(((unsigned __int128)(j + 1) * N) / njobs) - (uint64_t)(((unsigned __int128)j * N) / njobs);
    std::vector<uint32_t> ps(njobs, pj);
    Tables T;
    if (build_tables(sizes.data(), ps.data(), njobs, prm, T) != HSS_OK) return 0;
    const uint64_t cap = (uint64_t)std::ceil(2.0 * (double)prm->oversample * (double)pj) + 4096;
    T.C_tot = cap * njobs;
    T.PP_tot = (uint64_t)pj * cap * njobs;
    return plan_batch(T, njobs, pay, true).total;
}

}  // namespace hss

using namespace hss;

extern "C" {

size_t hss_batch_workspace_bytes(const uint64_t* h_sizes, const uint32_t* h_p, uint32_t njobs, const hss_params* prm,
                                 int key_type, int has_payload, int sort) {
    (void)key_type;
    if (!prm || njobs == 0 || !h_sizes || !h_p) return 0;
    Tables T;
    if (build_tables(h_sizes, h_p, njobs, prm, T) != HSS_OK) return 0;
    return plan_batch(T, njobs, has_payload != 0 && sort != 0, sort != 0).total;
}

int hss_sort_batch(const void* d_keys, const uint32_t* d_payload, int key_type, const uint64_t* h_sizes,
                   const uint32_t* h_p, uint32_t njobs, const hss_params* prm, void* d_keys_out, uint32_t* d_payload_out,
                   hss_cut* d_splitters, uint64_t* d_offsets, void* d_work, size_t work_bytes, hss_batch_stats* h_stats,
                   hss_job_stats* h_job_stats, void* stream) {
    return run_batch(d_keys, d_payload, key_type, h_sizes, h_p, njobs, prm, d_keys_out, d_payload_out, d_splitters,
                     d_offsets, d_work, work_bytes, h_stats, h_job_stats, (cudaStream_t)stream, true, BatchExtra{});
}

int hss_sort_batch_seeded(const void* d_keys, const uint32_t* d_payload, int key_type, const uint64_t* h_sizes,
                          const uint32_t* h_p, const uint64_t* h_seeds, uint32_t njobs, const hss_params* prm,
                          void* d_keys_out, uint32_t* d_payload_out, hss_cut* d_splitters, uint64_t* d_offsets,
                          void* d_work, size_t work_bytes, hss_batch_stats* h_stats, hss_job_stats* h_job_stats,
                          void* stream) {
    BatchExtra ex;
    ex.seeds = h_seeds;
    return run_batch(d_keys, d_payload, key_type, h_sizes, h_p, njobs, prm, d_keys_out, d_payload_out, d_splitters,
                     d_offsets, d_work, work_bytes, h_stats, h_job_stats, (cudaStream_t)stream, true, ex);
}

int hss_partition_batch_seeded(const void* d_keys, int key_type, const uint64_t* h_sizes, const uint32_t* h_p,
                               const uint64_t* h_seeds, uint32_t njobs, const hss_params* prm, hss_cut* d_splitters,
                               uint64_t* d_offsets, void* d_work, size_t work_bytes, hss_batch_stats* h_stats,
                               hss_job_stats* h_job_stats, void* stream) {
    BatchExtra ex;
    ex.seeds = h_seeds;
    return run_batch(d_keys, nullptr, key_type, h_sizes, h_p, njobs, prm, nullptr, nullptr, d_splitters, d_offsets,
                     d_work, work_bytes, h_stats, h_job_stats, (cudaStream_t)stream, false, ex);
}

int hss_partition_batch(const void* d_keys, int key_type, const uint64_t* h_sizes, const uint32_t* h_p, uint32_t njobs,
                        const hss_params* prm, hss_cut* d_splitters, uint64_t* d_offsets, void* d_work,
                        size_t work_bytes, hss_batch_stats* h_stats, hss_job_stats* h_job_stats, void* stream) {
    return run_batch(d_keys, nullptr, key_type, h_sizes, h_p, njobs, prm, nullptr, nullptr, d_splitters, d_offsets,
                     d_work, work_bytes, h_stats, h_job_stats, (cudaStream_t)stream, false, BatchExtra{});
}

}  // extern "C"
