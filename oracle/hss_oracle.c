/*
 * hss_oracle.c -- CPU oracle for Histogram Sort with Sampling (HSS).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, single-threaded
 * restatement of the method of Harsh, Kale and Solomonik, "Histogram Sort
 * with Sampling" (SPAA'19).  It exists to check the CUDA path; only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code, header, table or constant generator with the CUDA library.
 *
 * What it computes, step by step, in the paper's order:
 *   1. Problem statement (Sec. 2): N keys on p processors, processor s holding
 *      the contiguous input range [floor(sN/p), floor((s+1)N/p)).  Splitter i
 *      must have global rank chi(i) inside the target range
 *      T_i = [Ni/p - N eps/(2p), Ni/p + N eps/(2p)].
 *   2. Local sort (Sec. 5, Sec. 6): every processor sorts its keys.  Duplicates
 *      are made distinct by implicit tagging (Sec. 6.1): key k becomes the
 *      triple (k, processor, index).  Because the local sort is stable the
 *      index is the position in the sorted segment (spos), and
 *      (key, seg, spos) order equals (key, global input index) order.
 *   3. Splitter determination with k histogram rounds (Sec. 4.2.2): in round
 *      j every key lying strictly inside an unresolved splitter interval
 *      (L_i, U_i) is sampled independently with probability q_j; the sorted
 *      sample is the probe set; a histogram gives the exact global rank of
 *      every probe; L_i / U_i move to the closest probes below / above the
 *      ideal rank; the loop ends when every splitter has a probe inside its
 *      target range.
 *   4. Final splitters (Sec. 4.2.2 step 5): the seen key ranked closest to
 *      Ni/p.
 *   5. Data exchange (Sec. 3.1 step 3, Sec. 6): bucket b receives, from every
 *      processor, the keys in [S(b), S(b+1)); then each bucket merges its p
 *      sorted runs.
 *
 * Readings where the paper is silent or inconsistent (each one is fixed here
 * and mirrored by the CUDA path):
 *   - Target range half-width: Sec. 2 and Lemma 4.1 use N eps/(2p); the
 *     notation table prints N eps/p.  We use tol = floor(N*eps/(2p)) computed
 *     in IEEE double as ((double)N * eps) / (2.0 * p).
 *   - Ideal rank: t_i = floor(i*N/p), exact integer arithmetic.
 *   - "Rank" of a cut c is the number of keys strictly below it, #{e : e < c}
 *     in tag order; for a key that is itself an input element this is its
 *     0-based position in the global sorted order, matching S(i) = I(chi(i)).
 *   - L_i is the best cut with rank <= t_i, U_i the best with rank >= t_i
 *     (Sec. 4.2.2 step 3 does not say strict or not).  A tie in rank, which
 *     can only happen between an externally proposed non-member cut and a
 *     member, keeps the smaller tag.
 *   - Splitter i is resolved when |rank(L_i)-t_i| <= tol or
 *     |rank(U_i)-t_i| <= tol.  Only unresolved intervals are sampled; L/U of
 *     every splitter keep improving from every probe, as step 5 picks the
 *     closest key "among the keys seen so far".
 *   - Sampling probability: the implementation section draws s/delta samples
 *     per thread, i.e. q_j = s*p/|gamma_{j-1}| (expected s*p probes per round),
 *     capped at 1; s = 5 by default (5p probes per round, Sec. 7.2).  The draw
 *     is u < T with T = floor(q * 2^64) (q < 1) or "take all" (q >= 1).
 *   - The paper names no random number generator.  Each key draws one 64-bit
 *     word from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with
 *     key (seed_lo, seed_hi) and counter (spos>>1, seg, j, 0); an even spos
 *     takes words (x1:x0), an odd spos (x3:x2).
 *   - Final choice: the closer of L_i, U_i to t_i; a tie picks L_i.
 *   - Signed 64-bit keys are ordered by flipping the sign bit.
 *   - Empty processors (p > N) are allowed; Sec. 2 notes the proofs hold for
 *     uneven distributions.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, from the definition in Salmon et al., SC'11 (Sec. 4.2):     */
/* each round multiplies two counter words by fixed 32-bit constants, swaps  */
/* and xors the high halves with the other words and the round key; the key  */
/* is advanced by the Weyl constants between rounds.                         */
/* ------------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ x1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ x3 ^ k1;
        uint32_t n3 = lo0;
        x0 = n0; x1 = n1; x2 = n2; x3 = n3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The 64-bit Bernoulli draw of the key at position spos of sorted segment seg
 * in histogram round j (see the header comment). */
uint64_t oracle_sample_draw(uint64_t seed, uint32_t seg, uint32_t spos, uint32_t round)
{
    uint32_t ctr[4] = { spos >> 1, seg, round, 0u };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t x[4];
    oracle_philox4x32_10(ctr, key, x);
    if ((spos & 1u) == 0u) return ((uint64_t)x[1] << 32) | x[0];
    return ((uint64_t)x[3] << 32) | x[2];
}

/* Threshold T of round j: returns 1 and sets *take_all when q >= 1. */
void oracle_threshold(double oversample, uint32_t p, uint64_t gamma, uint64_t* T, int* take_all)
{
    double q = gamma == 0 ? 1.0 : ((double)oversample * (double)p) / (double)gamma;
    if (q >= 1.0) { *take_all = 1; *T = 0; return; }
    *take_all = 0;
    *T = (uint64_t)floor(ldexp(q, 64));
}

/* Threshold of a sampling probability q: take all when q >= 1, else
 * T = floor(q 2^64) (a key is kept when its word is below T). */
void oracle_threshold_q(double q, uint64_t* T, int* take_all)
{
    if (q >= 1.0) { *take_all = 1; *T = 0; return; }
    *take_all = 0;
    *T = (uint64_t)floor(ldexp(q, 64));
}

/* The sampling probability of round j (1-based) of the k-round schedule of
 * Sec. 4.2.2 and Theorem 4.7: s_j = (2 ln p / eps)^(j/k) and every key of the
 * unresolved region is drawn with probability p s_j / N (rounds past k keep
 * s_k). */
double oracle_theory_q(uint32_t p, double eps, uint64_t N, uint32_t j, uint32_t k)
{
    const uint32_t jj = j < k ? j : k;
    const double sj = pow(2.0 * log((double)p) / eps, (double)jj / (double)k);
    return ((double)p * sj) / (double)N;
}

uint64_t oracle_tolerance(uint64_t N, uint32_t p, double eps)
{
    return (uint64_t)floor(((double)N * eps) / (2.0 * (double)p));
}

/* ------------------------------------------------------------------------- */
/* Tags and cuts                                                             */
/* ------------------------------------------------------------------------- */
enum { CUT_NEG_INF = 0, CUT_MEMBER = 1, CUT_NONMEMBER = 2, CUT_POS_INF = 3 };

typedef struct {
    int kind;
    uint64_t okey;    /* order-preserving key bits */
    int32_t seg;      /* -1 for a non-member cut */
    uint32_t spos;
    uint64_t rank;    /* #{elements strictly below} */
} ocut;

/* Three-way comparison of two cuts in tag order. */
static int cut_cmp(const ocut* a, const ocut* b)
{
    if (a->kind == CUT_NEG_INF || b->kind == CUT_NEG_INF) {
        if (a->kind == b->kind) return 0;
        return a->kind == CUT_NEG_INF ? -1 : 1;
    }
    if (a->kind == CUT_POS_INF || b->kind == CUT_POS_INF) {
        if (a->kind == b->kind) return 0;
        return a->kind == CUT_POS_INF ? 1 : -1;
    }
    if (a->okey != b->okey) return a->okey < b->okey ? -1 : 1;
    if (a->seg != b->seg) return a->seg < b->seg ? -1 : 1;
    if (a->spos != b->spos) return a->spos < b->spos ? -1 : 1;
    return 0;
}

/* Is the element (okey, seg, spos) strictly below cut c? */
static int elem_lt_cut(uint64_t okey, int32_t seg, uint32_t spos, const ocut* c)
{
    if (c->kind == CUT_NEG_INF) return 0;
    if (c->kind == CUT_POS_INF) return 1;
    if (okey != c->okey) return okey < c->okey;
    if (seg != c->seg) return seg < c->seg;
    return spos < c->spos;
}

typedef struct {
    uint64_t N;
    uint32_t p;
    const uint64_t* seg_start;  /* p+1 entries */
    const uint64_t* okeys;      /* segment-sorted, order-preserving keys */
} ostate;

/* lb_s(c): number of keys of sorted segment s strictly below cut c, by
 * binary search over the segment (its tags increase with position). */
static uint64_t seg_lower_bound(const ostate* st, uint32_t s, const ocut* c)
{
    uint64_t lo = 0, hi = st->seg_start[s + 1] - st->seg_start[s];
    const uint64_t* a = st->okeys + st->seg_start[s];
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (elem_lt_cut(a[mid], (int32_t)s, (uint32_t)mid, c)) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* The histogram of Sec. 4.2.2 step 2 for one probe: its global rank is the sum
 * over processors of the local counts below it. */
static uint64_t global_rank(const ostate* st, const ocut* c)
{
    uint64_t r = 0;
    for (uint32_t s = 0; s < st->p; ++s) r += seg_lower_bound(st, s, c);
    return r;
}

/* ------------------------------------------------------------------------- */
/* Local sort (stable, by order-preserving key)                              */
/* ------------------------------------------------------------------------- */
typedef struct { uint64_t okey; uint64_t idx; } kv;

static int kv_cmp(const void* a, const void* b)
{
    const kv* x = (const kv*)a; const kv* y = (const kv*)b;
    if (x->okey != y->okey) return x->okey < y->okey ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

static uint64_t to_okey(uint64_t k, int key_type) { return key_type == 1 ? (k ^ 0x8000000000000000ull) : k; }
static uint64_t from_okey(uint64_t k, int key_type) { return key_type == 1 ? (k ^ 0x8000000000000000ull) : k; }

static void segment_bounds(uint64_t N, uint32_t p, uint64_t* seg_start)
{
    for (uint32_t s = 0; s <= p; ++s)
        seg_start[s] = (uint64_t)(((unsigned __int128)s * N) / p);
}

/* Stable sort of every segment: (key, original index) order is exactly the
 * stable order.  Writes order-preserving keys and the permuted payload. */
static void local_sort(const uint64_t* keys, const uint32_t* payload, uint64_t N, int key_type,
                       uint32_t p, const uint64_t* seg_start, uint64_t* okeys, uint32_t* opay)
{
    for (uint32_t s = 0; s < p; ++s) {
        uint64_t b = seg_start[s], n = seg_start[s + 1] - b;
        if (n == 0) continue;
        kv* t = (kv*)malloc(sizeof(kv) * n);
        for (uint64_t i = 0; i < n; ++i) { t[i].okey = to_okey(keys[b + i], key_type); t[i].idx = b + i; }
        qsort(t, n, sizeof(kv), kv_cmp);
        for (uint64_t i = 0; i < n; ++i) {
            okeys[b + i] = t[i].okey;
            if (opay) opay[b + i] = payload ? payload[t[i].idx] : 0u;
        }
        free(t);
    }
}

void oracle_segment_sort(const uint64_t* keys, const uint32_t* payload, uint64_t N, int key_type, uint32_t p,
                         uint64_t* out_keys, uint32_t* out_payload)
{
    uint64_t* seg_start = (uint64_t*)malloc(sizeof(uint64_t) * (p + 1));
    segment_bounds(N, p, seg_start);
    local_sort(keys, payload, N, key_type, p, seg_start, out_keys, out_payload);
    for (uint64_t i = 0; i < N; ++i) out_keys[i] = from_okey(out_keys[i], key_type);
    free(seg_start);
}

/* ------------------------------------------------------------------------- */
/* HSS rounds                                                                */
/* ------------------------------------------------------------------------- */
#define ORACLE_MAX_ROUNDS 64

typedef struct {
    uint32_t rounds;
    int32_t status;                         /* 0 ok, -3 round limit */
    uint64_t tol;
    uint64_t sample_size[ORACLE_MAX_ROUNDS];  /* Z_j of round j+1 */
    uint64_t gamma[ORACLE_MAX_ROUNDS];        /* |gamma| sampled in round j+1 */
    uint64_t unresolved[ORACLE_MAX_ROUNDS + 1]; /* unresolved splitters before round j+1; last = after */
} oracle_stats;

/* Proposed cut supplied from outside (learned proposal): a non-member cut at
 * key k (it sorts before every key equal to k). */
typedef struct { uint64_t key; } oracle_proposal;

static int sample_cmp(const void* a, const void* b) { return cut_cmp((const ocut*)a, (const ocut*)b); }

/* Interval of splitter i is "the same" as that of splitter i' when both end
 * cuts coincide (Sec. 4.2.2: splitter intervals are identical or disjoint). */
static int same_interval(const ocut* L, const ocut* U, uint32_t a, uint32_t b)
{
    return cut_cmp(&L[a], &L[b]) == 0 && cut_cmp(&U[a], &U[b]) == 0;
}

static int is_resolved(const ocut* L, const ocut* U, uint64_t t, uint64_t tol)
{
    uint64_t dl = t - L->rank;           /* L->rank <= t */
    uint64_t du = U->rank - t;           /* U->rank >= t */
    return dl <= tol || du <= tol;
}

/* Trace byte: bit 0 resolved, bit 1 L is an input key, bit 2 U is an input key. */
static uint8_t trace_flags(const ocut* L, const ocut* U, uint8_t resolved)
{
    return (uint8_t)(resolved | ((L->kind == CUT_MEMBER) << 1) | ((U->kind == CUT_MEMBER) << 2));
}

/* Improve L/U of one splitter with a ranked cut c. */
static void offer(ocut* L, ocut* U, uint64_t t, const ocut* c)
{
    if (c->rank <= t) {
        if (c->rank > L->rank || (c->rank == L->rank && cut_cmp(c, L) < 0)) *L = *c;
    }
    if (c->rank >= t) {
        if (c->rank < U->rank || (c->rank == U->rank && cut_cmp(c, U) < 0)) *U = *c;
    }
}

/*
 * Full HSS run.  Outputs:
 *   spl_key/spl_seg/spl_spos[p-1]: final splitter tags (key in the caller's
 *       representation; seg = -1 for a non-member cut, -2 for -inf, -3 for +inf)
 *   offsets[p+1]: chi(0..p)
 *   out_keys/out_payload[N] (nullable): the globally sorted output, bucket b
 *       occupying [chi(b), chi(b+1)), each bucket a stable p-way merge.
 *   trace_lrank/trace_urank/trace_resolved (nullable): per round r = 0..rounds
 *       the (p-1) L/U ranks and resolved flags after round r (r = 0: initial).
 *   trace_samples (nullable, cap trace_cap): sorted probes of every round,
 *       as (key, seg, spos) triples, rounds concatenated.
 */
/* HSS over p processors into nb buckets (nb = p: the single-stage method;
 * nb < p: the partition step of a stage of multi-stage HSS, Sec. 5.3, whose
 * nb - 1 splitters target ranks i N / nb with tolerance N eps / (2 nb) and
 * draw s nb probes per round).  exchange_only: out_keys receives each
 * bucket as the concatenation of its runs in processor order (the data
 * exchange without the merge). */
int oracle_hss_groups(const uint64_t* keys, const uint32_t* payload, uint64_t N, int key_type,
                      uint32_t p, uint32_t nb, int exchange_only, double eps, uint64_t seed, float oversample,
                      uint32_t max_rounds, const uint64_t* proposal_keys, uint32_t nprop, int schedule,
                      uint32_t schedule_k, uint64_t* spl_key, int32_t* spl_seg, uint32_t* spl_spos, uint64_t* offsets,
                      uint64_t* out_keys, uint32_t* out_payload, oracle_stats* stats,
                      uint64_t* trace_lrank, uint64_t* trace_urank, uint8_t* trace_resolved,
                      uint64_t* trace_samples, uint64_t trace_cap)
{
    if (p == 0 || nb == 0 || nb > p || !(eps > 0.0) || max_rounds > ORACLE_MAX_ROUNDS) return -1;
    if (schedule < 0 || schedule > 2 || (schedule == 1 && schedule_k == 0)) return -1;
    memset(stats, 0, sizeof(*stats));

    /* Step 1: processors and targets. */
    uint64_t* seg_start = (uint64_t*)malloc(sizeof(uint64_t) * (p + 1));
    segment_bounds(N, p, seg_start);
    uint64_t tol = oracle_tolerance(N, nb, eps);
    stats->tol = tol;
    uint32_t S = nb - 1;  /* number of splitters */
    uint64_t* t = (uint64_t*)malloc(sizeof(uint64_t) * (S + 1));
    for (uint32_t i = 1; i <= S; ++i) t[i - 1] = (uint64_t)(((unsigned __int128)i * N) / nb);

    /* Step 2: local sort with implicit tagging. */
    uint64_t* okeys = (uint64_t*)malloc(sizeof(uint64_t) * (N ? N : 1));
    uint32_t* opay = (uint32_t*)malloc(sizeof(uint32_t) * (N ? N : 1));
    local_sort(keys, payload, N, key_type, p, seg_start, okeys, opay);
    ostate st = { N, p, seg_start, okeys };

    /* Step 3: splitter intervals start as (-inf, +inf). */
    ocut* L = (ocut*)calloc(S + 1, sizeof(ocut));
    ocut* U = (ocut*)calloc(S + 1, sizeof(ocut));
    uint8_t* res = (uint8_t*)calloc(S + 1, 1);
    for (uint32_t i = 0; i < S; ++i) {
        L[i].kind = CUT_NEG_INF; L[i].rank = 0;
        U[i].kind = CUT_POS_INF; U[i].rank = N;
    }

    /* Externally proposed cuts (learned proposal) are histogrammed before
     * round 1 exactly like probes. */
    for (uint32_t k = 0; k < nprop; ++k) {
        ocut c; memset(&c, 0, sizeof c);
        c.kind = CUT_NONMEMBER; c.okey = to_okey(proposal_keys[k], key_type); c.seg = -1; c.spos = 0;
        c.rank = global_rank(&st, &c);
        for (uint32_t i = 0; i < S; ++i) offer(&L[i], &U[i], t[i], &c);
    }

    uint32_t unresolved = 0;
    for (uint32_t i = 0; i < S; ++i) { res[i] = (uint8_t)is_resolved(&L[i], &U[i], t[i], tol); unresolved += !res[i]; }
    if (trace_lrank) for (uint32_t i = 0; i < S; ++i) { trace_lrank[i] = L[i].rank; trace_urank[i] = U[i].rank; trace_resolved[i] = trace_flags(&L[i], &U[i], res[i]); }
    stats->unresolved[0] = unresolved;

    uint64_t trace_used = 0;
    uint32_t j = 0;
    while (unresolved > 0 && j < max_rounds) {
        ++j;
        /* |gamma_{j-1}|: keys strictly inside the distinct unresolved intervals. */
        uint64_t gamma = 0;
        uint32_t nint = 0;                            /* distinct unresolved intervals */
        for (uint32_t i = 0; i < S; ++i) {
            if (res[i]) continue;
            int dup = 0;
            for (uint32_t i2 = i; i2-- > 0;) {       /* identical intervals are adjacent */
                if (!same_interval(L, U, i, i2)) break;
                if (!res[i2]) { dup = 1; break; }
            }
            if (dup) continue;
            gamma += U[i].rank - L[i].rank - (L[i].kind == CUT_MEMBER ? 1u : 0u);
            ++nint;
        }
        /* Sampling probability: proportional (Sec. 6: s p / |gamma| for every
         * key of the region), the k-round schedule of Theorem 4.7, or equal
         * per interval (HykSort, Sec. 4.2.2 remark): s p / nint expected
         * samples for each distinct unresolved interval. */
        uint64_t T; int take_all;
        if (schedule == 1) oracle_threshold_q(oracle_theory_q(nb, eps, N, j, schedule_k), &T, &take_all);
        else oracle_threshold((double)oversample, nb, gamma, &T, &take_all);
        const double per_int = nint ? ((double)oversample * (double)nb) / (double)nint : 0.0;

        /* Sampling phase: every key strictly inside an unresolved interval is
         * drawn independently. */
        uint64_t cap = 1024, Z = 0;
        ocut* smp = (ocut*)malloc(sizeof(ocut) * cap);
        for (uint32_t i = 0; i < S; ++i) {
            if (res[i]) continue;
            int dup = 0;
            for (uint32_t i2 = i; i2-- > 0;) {
                if (!same_interval(L, U, i, i2)) break;
                if (!res[i2]) { dup = 1; break; }
            }
            if (dup) continue;
            uint64_t Ti = T; int all_i = take_all;
            if (schedule == 2) {
                const uint64_t len = U[i].rank - L[i].rank - (L[i].kind == CUT_MEMBER ? 1u : 0u);
                oracle_threshold_q(len ? per_int / (double)len : 1.0, &Ti, &all_i);
            }
            for (uint32_t s = 0; s < p; ++s) {
                uint64_t a = seg_lower_bound(&st, s, &L[i]);
                if (L[i].kind == CUT_MEMBER && (uint32_t)L[i].seg == s) a += 1;   /* strictly above L */
                uint64_t b = seg_lower_bound(&st, s, &U[i]);                        /* strictly below U */
                for (uint64_t pos = a; pos < b; ++pos) {
                    uint64_t u = oracle_sample_draw(seed, s, (uint32_t)pos, j);
                    if (!(all_i || u < Ti)) continue;
                    if (Z == cap) { cap *= 2; smp = (ocut*)realloc(smp, sizeof(ocut) * cap); }
                    ocut* c = &smp[Z++];
                    c->kind = CUT_MEMBER; c->okey = okeys[seg_start[s] + pos]; c->seg = (int32_t)s; c->spos = (uint32_t)pos;
                    c->rank = 0;
                }
            }
        }
        /* Gather at the central processor and sort: the probes. */
        qsort(smp, Z, sizeof(ocut), sample_cmp);
        /* Histogramming: exact global rank of every probe. */
        for (uint64_t k = 0; k < Z; ++k) smp[k].rank = global_rank(&st, &smp[k]);
        if (trace_samples) {
            for (uint64_t k = 0; k < Z && trace_used < trace_cap; ++k, ++trace_used) {
                trace_samples[3 * trace_used + 0] = from_okey(smp[k].okey, key_type);
                trace_samples[3 * trace_used + 1] = (uint64_t)smp[k].seg;
                trace_samples[3 * trace_used + 2] = smp[k].spos;
            }
        }
        /* Update L_j(i), U_j(i) of every splitter.  The probe ranks increase
         * with tag order (distinct keys have distinct ranks), so the best
         * probe below / above t_i is found by binary search. */
        for (uint32_t i = 0; i < S; ++i) {
            uint64_t lo = 0, hi = Z;                 /* first probe with rank > t */
            while (lo < hi) { uint64_t m = lo + (hi - lo) / 2; if (smp[m].rank <= t[i]) lo = m + 1; else hi = m; }
            if (lo > 0) offer(&L[i], &U[i], t[i], &smp[lo - 1]);
            lo = 0; hi = Z;                          /* first probe with rank >= t */
            while (lo < hi) { uint64_t m = lo + (hi - lo) / 2; if (smp[m].rank < t[i]) lo = m + 1; else hi = m; }
            if (lo < Z) offer(&L[i], &U[i], t[i], &smp[lo]);
        }
        unresolved = 0;
        for (uint32_t i = 0; i < S; ++i) { res[i] = (uint8_t)is_resolved(&L[i], &U[i], t[i], tol); unresolved += !res[i]; }
        stats->sample_size[j - 1] = Z;
        stats->gamma[j - 1] = gamma;
        stats->unresolved[j] = unresolved;
        if (trace_lrank) {
            for (uint32_t i = 0; i < S; ++i) {
                trace_lrank[(uint64_t)j * S + i] = L[i].rank;
                trace_urank[(uint64_t)j * S + i] = U[i].rank;
                trace_resolved[(uint64_t)j * S + i] = trace_flags(&L[i], &U[i], res[i]);
            }
        }
        free(smp);
    }
    stats->rounds = j;
    stats->status = unresolved > 0 ? -3 : 0;

    /* Step 4: final splitters, the seen cut closest to t_i (tie -> L). */
    ocut* spl = (ocut*)malloc(sizeof(ocut) * (S + 2));
    memset(&spl[0], 0, sizeof(ocut)); spl[0].kind = CUT_NEG_INF; spl[0].rank = 0;
    for (uint32_t i = 0; i < S; ++i) {
        uint64_t dl = t[i] - L[i].rank, du = U[i].rank - t[i];
        spl[i + 1] = (dl <= du) ? L[i] : U[i];
    }
    memset(&spl[S + 1], 0, sizeof(ocut)); spl[S + 1].kind = CUT_POS_INF; spl[S + 1].rank = N;
    for (uint32_t b = 0; b <= nb; ++b) offsets[b] = spl[b].rank;
    for (uint32_t i = 0; i < S; ++i) {
        const ocut* c = &spl[i + 1];
        if (c->kind == CUT_MEMBER)          { spl_key[i] = from_okey(c->okey, key_type); spl_seg[i] = c->seg; spl_spos[i] = c->spos; }
        else if (c->kind == CUT_NONMEMBER)  { spl_key[i] = from_okey(c->okey, key_type); spl_seg[i] = -1; spl_spos[i] = 0; }
        else if (c->kind == CUT_NEG_INF)    { spl_key[i] = 0; spl_seg[i] = -2; spl_spos[i] = 0; }
        else                                { spl_key[i] = 0; spl_seg[i] = -3; spl_spos[i] = 0; }
    }

    /* Step 5: exchange and merge.  Bucket b takes, from every processor s in
     * order, the run of keys in [S(b), S(b+1)); the bucket is then merged by
     * (key, processor, index), i.e. a stable sort of the concatenated runs. */
    if (out_keys) {
        /* one bucket at a time: the buffer holds the largest bucket */
        uint64_t maxb = 1;
        for (uint32_t b = 0; b < nb; ++b) if (offsets[b + 1] - offsets[b] > maxb) maxb = offsets[b + 1] - offsets[b];
        kv* buf = (kv*)malloc(sizeof(kv) * maxb);
        for (uint32_t b = 0; b < nb; ++b) {
            uint64_t n = 0, base = offsets[b];
            for (uint32_t s = 0; s < p; ++s) {
                uint64_t a = seg_lower_bound(&st, s, &spl[b]);
                uint64_t e = seg_lower_bound(&st, s, &spl[b + 1]);
                for (uint64_t pos = a; pos < e; ++pos) {
                    buf[n].okey = okeys[seg_start[s] + pos];
                    buf[n].idx = seg_start[s] + pos;  /* increasing in (seg, spos) */
                    ++n;
                }
            }
            if (!exchange_only) qsort(buf, n, sizeof(kv), kv_cmp);
            for (uint64_t k = 0; k < n; ++k) {
                out_keys[base + k] = from_okey(buf[k].okey, key_type);
                if (out_payload) out_payload[base + k] = opay[buf[k].idx];
            }
        }
        free(buf);
    }

    free(spl); free(res); free(U); free(L); free(opay); free(okeys); free(t); free(seg_start);
    return stats->status;
}

/* The single-stage method: p processors, p buckets, exchange and merge. */
int oracle_hss(const uint64_t* keys, const uint32_t* payload, uint64_t N, int key_type,
               uint32_t p, double eps, uint64_t seed, float oversample, uint32_t max_rounds,
               const uint64_t* proposal_keys, uint32_t nprop, int schedule, uint32_t schedule_k,
               uint64_t* spl_key, int32_t* spl_seg, uint32_t* spl_spos, uint64_t* offsets,
               uint64_t* out_keys, uint32_t* out_payload, oracle_stats* stats,
               uint64_t* trace_lrank, uint64_t* trace_urank, uint8_t* trace_resolved,
               uint64_t* trace_samples, uint64_t trace_cap)
{
    return oracle_hss_groups(keys, payload, N, key_type, p, p, 0, eps, seed, oversample, max_rounds, proposal_keys,
                             nprop, schedule, schedule_k, spl_key, spl_seg, spl_spos, offsets, out_keys, out_payload,
                             stats, trace_lrank, trace_urank, trace_resolved, trace_samples, trace_cap);
}

/* Global rank of an arbitrary cut over the locally sorted segments of an input
 * (the histogram of one probe), for tests that pin the histogram against brute
 * force.  kind: 1 member (key, seg, spos), 2 non-member (key). */
uint64_t oracle_cut_rank(const uint64_t* keys, uint64_t N, int key_type, uint32_t p,
                         int kind, uint64_t key, int32_t seg, uint32_t spos)
{
    uint64_t* seg_start = (uint64_t*)malloc(sizeof(uint64_t) * (p + 1));
    segment_bounds(N, p, seg_start);
    uint64_t* okeys = (uint64_t*)malloc(sizeof(uint64_t) * (N ? N : 1));
    local_sort(keys, NULL, N, key_type, p, seg_start, okeys, NULL);
    ostate st = { N, p, seg_start, okeys };
    ocut c; memset(&c, 0, sizeof c);
    c.kind = kind; c.okey = to_okey(key, key_type); c.seg = kind == CUT_NONMEMBER ? -1 : seg; c.spos = spos;
    uint64_t r = global_rank(&st, &c);
    free(okeys); free(seg_start);
    return r;
}
