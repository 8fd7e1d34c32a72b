// cpu_baselines.cpp -- timed CPU baselines for the benchmark (TEST AND
// BENCHMARK INFRASTRUCTURE ONLY; the product library never links or calls it).
//
//  * cpu_hss_omp: Histogram Sort with Sampling (Harsh, Kale, Solomonik,
//    SPAA'19) on all host cores with OpenMP, keys alone.  It takes the same
//    steps and readings as the single-threaded oracle (hss_oracle.c) --
//    local sort of each processor's segment (Sec. 5), histogram rounds over
//    the unresolved splitter intervals with the per-key Philox4x32-10 draw
//    (Sec. 4.2.2 and 6), the closest seen key as splitter, exchange and
//    per-bucket merge (Sec. 3.1 step 3) -- but runs every loop over
//    processors, probes, splitters and buckets in parallel and sorts with
//    std::sort.  It produces the oracle's splitters, offsets, round
//    statistics and output (checked in tests/test_cpu_baselines.py), so its
//    time is a fair all-cores CPU reference for the same result.
//  * cpu_std_sort: std::sort of the whole input on one core, for context.
//
// It shares no code with the CUDA library (nor with the oracle: the two C
// sources are independent restatements of the same steps).
#include <stdint.h>
#include <string.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include <omp.h>

namespace {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, each
// multiplying two words by fixed 32-bit constants, mixing the high halves
// with the other words and the round key; the key advances by the Weyl
// constants between rounds.
inline void philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)M0 * c[0], p1 = (uint64_t)M1 * c[2];
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        c[0] = n0; c[1] = (uint32_t)p1; c[2] = n2; c[3] = (uint32_t)p0;
        k0 += W0; k1 += W1;
    }
}

// The 64-bit Bernoulli word of position spos of segment seg in round j:
// counter (spos >> 1, seg, j, 0), key (seed_lo, seed_hi); even positions take
// words (x1:x0), odd ones (x3:x2).
inline uint64_t draw(uint64_t seed, uint32_t seg, uint32_t spos, uint32_t j) {
    uint32_t c[4] = {spos >> 1, seg, j, 0u};
    philox(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    return (spos & 1u) ? (((uint64_t)c[3] << 32) | c[2]) : (((uint64_t)c[1] << 32) | c[0]);
}

enum { NEG = 0, MEM = 1, POS = 3 };

struct Cut {
    int kind;
    uint64_t key;  // order-preserving bits
    int32_t seg;
    uint32_t spos;
    uint64_t rank;
};

inline bool less_cut(const Cut& a, const Cut& b) {
    if (a.kind != b.kind && (a.kind == NEG || b.kind == NEG || a.kind == POS || b.kind == POS)) return a.kind < b.kind;
    if (a.kind == NEG || a.kind == POS) return false;
    if (a.key != b.key) return a.key < b.key;
    if (a.seg != b.seg) return a.seg < b.seg;
    return a.spos < b.spos;
}
inline bool same_cut(const Cut& a, const Cut& b) { return !less_cut(a, b) && !less_cut(b, a); }

struct State {
    uint64_t N;
    uint32_t p;
    std::vector<uint64_t> start;  // p + 1
    std::vector<uint64_t> k;      // locally sorted, order-preserving
};

// Keys of segment s strictly below cut c in tag order (key, seg, spos).
inline uint64_t below(const State& st, uint32_t s, const Cut& c) {
    if (c.kind == NEG) return 0;
    const uint64_t* a = st.k.data() + st.start[s];
    const uint64_t n = st.start[s + 1] - st.start[s];
    if (c.kind == POS) return n;
    const uint64_t lt = (uint64_t)(std::lower_bound(a, a + n, c.key) - a);
    if ((int32_t)s < c.seg) return (uint64_t)(std::upper_bound(a, a + n, c.key) - a);
    if ((int32_t)s > c.seg) return lt;
    return c.spos;  // the cut is the element at spos of this segment
}

inline uint64_t global_rank(const State& st, const Cut& c) {
    uint64_t r = 0;
    for (uint32_t s = 0; s < st.p; ++s) r += below(st, s, c);
    return r;
}

inline void offer(Cut& L, Cut& U, uint64_t t, const Cut& c) {
    if (c.rank <= t && (c.rank > L.rank || (c.rank == L.rank && less_cut(c, L)))) L = c;
    if (c.rank >= t && (c.rank < U.rank || (c.rank == U.rank && less_cut(c, U)))) U = c;
}

}  // namespace

extern "C" {

int cpu_baseline_threads(void) { return omp_get_max_threads(); }

// std::sort of the whole input (one core), keys as unsigned 64-bit.
void cpu_std_sort(uint64_t* keys, uint64_t N) { std::sort(keys, keys + N); }

// HSS on all cores, keys alone (unsigned 64-bit).  Outputs as the oracle:
// spl_key/spl_seg/spl_spos[p-1], offsets[p+1], out_keys[N] (nullable),
// rounds and per-round sample sizes (sample_size[max_rounds]).  Returns 0,
// -3 at the round limit, -1 for bad arguments.
int cpu_hss_omp(const uint64_t* keys, uint64_t N, uint32_t p, double eps, uint64_t seed, float oversample,
                uint32_t max_rounds, uint64_t* spl_key, int32_t* spl_seg, uint32_t* spl_spos, uint64_t* offsets,
                uint64_t* out_keys, uint32_t* rounds_out, uint64_t* sample_size) {
    if (p == 0 || !(eps > 0.0) || max_rounds > 64) return -1;
    State st;
    st.N = N;
    st.p = p;
    st.start.resize(p + 1);
    for (uint32_t s = 0; s <= p; ++s) st.start[s] = (uint64_t)(((unsigned __int128)s * N) / p);
    st.k.assign(keys, keys + N);
    // local sort (Sec. 5): every processor in parallel
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < (int64_t)p; ++s) std::sort(st.k.begin() + st.start[s], st.k.begin() + st.start[s + 1]);

    const uint32_t S = p - 1;
    const uint64_t tol = (uint64_t)floor(((double)N * eps) / (2.0 * (double)p));
    std::vector<uint64_t> t(S);
    for (uint32_t i = 0; i < S; ++i) t[i] = (uint64_t)(((unsigned __int128)(i + 1) * N) / p);
    std::vector<Cut> L(S), U(S);
    for (uint32_t i = 0; i < S; ++i) {
        L[i] = Cut{NEG, 0, -2, 0, 0};
        U[i] = Cut{POS, 0, -3, 0, N};
    }
    auto resolved = [&](uint32_t i) { return (t[i] - L[i].rank) <= tol || (U[i].rank - t[i]) <= tol; };
    uint32_t unresolved = 0;
    for (uint32_t i = 0; i < S; ++i) unresolved += !resolved(i);
    uint32_t j = 0;
    while (unresolved > 0 && j < max_rounds) {
        ++j;
        // distinct unresolved intervals (identical or disjoint, Sec. 4.2.2)
        std::vector<uint32_t> reps;
        uint64_t gamma = 0;
        for (uint32_t i = 0; i < S; ++i) {
            if (resolved(i)) continue;
            bool dup = false;
            for (uint32_t i2 = i; i2-- > 0;) {
                if (!(same_cut(L[i], L[i2]) && same_cut(U[i], U[i2]))) break;
                if (!resolved(i2)) { dup = true; break; }
            }
            if (dup) continue;
            reps.push_back(i);
            gamma += U[i].rank - L[i].rank - (L[i].kind == MEM ? 1u : 0u);
        }
        const double q = gamma == 0 ? 1.0 : ((double)oversample * (double)p) / (double)gamma;
        const bool all = q >= 1.0;
        const uint64_t T = all ? 0 : (uint64_t)floor(ldexp(q, 64));
        // sampling: processors in parallel
        std::vector<std::vector<Cut>> part(p);
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t s = 0; s < (int64_t)p; ++s) {
            for (uint32_t i : reps) {
                uint64_t a = below(st, (uint32_t)s, L[i]);
                if (L[i].kind == MEM && L[i].seg == (int32_t)s) a += 1;
                const uint64_t b = below(st, (uint32_t)s, U[i]);
                for (uint64_t pos = a; pos < b; ++pos) {
                    if (!all && draw(seed, (uint32_t)s, (uint32_t)pos, j) >= T) continue;
                    part[s].push_back(Cut{MEM, st.k[st.start[s] + pos], (int32_t)s, (uint32_t)pos, 0});
                }
            }
        }
        std::vector<Cut> probes;
        for (auto& v : part) probes.insert(probes.end(), v.begin(), v.end());
        std::sort(probes.begin(), probes.end(), less_cut);
        // histogram: probes in parallel
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t k = 0; k < (int64_t)probes.size(); ++k) probes[k].rank = global_rank(st, probes[k]);
        // L/U update: splitters in parallel
        const uint64_t Z = probes.size();
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < (int64_t)S; ++i) {
            const uint64_t ti = t[i];
            uint64_t lo = 0, hi = Z;
            while (lo < hi) { const uint64_t m = (lo + hi) / 2; if (probes[m].rank <= ti) lo = m + 1; else hi = m; }
            if (lo > 0) offer(L[i], U[i], ti, probes[lo - 1]);
            lo = 0; hi = Z;
            while (lo < hi) { const uint64_t m = (lo + hi) / 2; if (probes[m].rank < ti) lo = m + 1; else hi = m; }
            if (lo < Z) offer(L[i], U[i], ti, probes[lo]);
        }
        if (sample_size) sample_size[j - 1] = Z;
        unresolved = 0;
        for (uint32_t i = 0; i < S; ++i) unresolved += !resolved(i);
    }
    if (rounds_out) *rounds_out = j;
    // final splitters: the seen cut closest to t_i (tie -> L)
    std::vector<Cut> spl(S + 2);
    spl[0] = Cut{NEG, 0, -2, 0, 0};
    for (uint32_t i = 0; i < S; ++i) spl[i + 1] = (t[i] - L[i].rank <= U[i].rank - t[i]) ? L[i] : U[i];
    spl[S + 1] = Cut{POS, 0, -3, 0, N};
    for (uint32_t b = 0; b <= p; ++b) offsets[b] = spl[b].rank;
    for (uint32_t i = 0; i < S; ++i) {
        const Cut& c = spl[i + 1];
        spl_key[i] = c.kind == MEM ? c.key : 0;
        spl_seg[i] = c.kind == MEM ? c.seg : (c.kind == NEG ? -2 : -3);
        spl_spos[i] = c.kind == MEM ? c.spos : 0;
    }
    // exchange and merge: buckets in parallel
    if (out_keys) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t b = 0; b < (int64_t)p; ++b) {
            uint64_t o = offsets[b];
            for (uint32_t s = 0; s < p; ++s) {
                const uint64_t a = below(st, s, spl[b]), e = below(st, s, spl[b + 1]);
                memcpy(out_keys + o, st.k.data() + st.start[s] + a, (e - a) * 8);
                o += e - a;
            }
            std::sort(out_keys + offsets[b], out_keys + offsets[b + 1]);
        }
    }
    return unresolved > 0 ? -3 : 0;
}

}  // extern "C"
