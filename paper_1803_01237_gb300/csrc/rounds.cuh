// rounds.cuh -- the splitter-determination rounds of HSS on one device.
#pragma once

#include "hss_internal.cuh"
#include "segsort.cuh"

namespace hss {

// Device-resident state of the round loop (one per call).
struct RoundCtl {
    uint64_t gamma;        // |gamma| of the region the next round samples
    uint64_t T;            // threshold of the next round (u < T selects)
    uint32_t take_all;     // q >= 1: select every key of the region
    uint32_t nint;         // distinct unresolved intervals
    uint32_t unresolved;   // unresolved splitters
    uint32_t round;        // rounds started (device-driven loop)
    uint64_t Z;            // probes drawn by the last sampling pass
    uint64_t seg_off_z[2]; // {0, min(Z, cap)}: one "segment" for the probe sort
    // Device-driven loop: the decision kernel keeps the loop state and the
    // round statistics here, and reads the call's parameters from here (so one
    // captured graph serves every call on the same workspace).
    int32_t status;        // HSS_OK, HSS_ERR_ROUND_LIMIT or HSS_ERR_CAPACITY
    uint32_t staged;       // the next histogram takes the staged form
    uint64_t seed;         // Philox key of the sampling
    uint32_t max_rounds;
    uint32_t pad;
    uint64_t hist_Z[HSS_MAX_ROUNDS];
    uint64_t hist_gamma[HSS_MAX_ROUNDS];
    uint64_t hist_unres[HSS_MAX_ROUNDS + 1];
};

// Workspace of the rounds, carved from the caller's buffer.
struct RoundWs {
    RoundCtl* ctl;
    DCut* Lcut;          // [S]
    DCut* Ucut;          // [S]
    uint32_t* Lpos;      // [p][S]  keys of segment s below L_i
    uint32_t* Upos;      // [p][S]
    uint32_t* res;       // [S] resolved flags
    int32_t* chgL;       // [S]
    int32_t* chgU;       // [S]
    uint32_t* choose_u;  // [S]
    uint32_t* int_rep;   // [S] representative splitter of each distinct unresolved interval
    uint64_t* int_T;     // [S] per-interval threshold (equal-per-interval schedule)
    uint32_t* int_all;   // [S] per-interval take-all flag
    uint32_t* bitmap;    // [N/32 + 2]
    uint32_t* seg_cnt;   // [p]
    uint32_t* seg_cnt_off;  // [p + 1]
    uint64_t* skey;      // [cap] sampled keys (order-preserving bits) in (seg, spos) order
    uint32_t* sseg;      // [cap]
    uint32_t* sspos;     // [cap]
    uint32_t* siota;     // [cap]
    uint64_t* skey_sorted;  // [cap]
    uint32_t* sperm;     // [cap]
    uint64_t* stmp;      // [cap] sort scratch
    uint32_t* ptmp;      // [cap]
    uint64_t* pkey;      // [cap] probes
    int32_t* pseg;       // [cap]
    uint32_t* pspos;     // [cap]
    uint32_t* pint;      // [cap]
    uint64_t* prank;     // [cap]
    uint32_t* probe_pos; // [p][cap]
    uint64_t* fin_okey;  // [S] order-preserving key of each final splitter
    uint32_t* fin_kind;  // [S]
    uint64_t* bucket_lo;    // [p] lower key bound of each bucket (its first split digit is
    uint64_t* key_range;    // [2] smallest and largest key of the input
    uint64_t* bucket_mult;  // [p] mulhi(key - lo, mult), an interpolation of [lo, hi] onto 0..255)
    SegSortWs sws;       // scratch of the probe sort
    uint64_t cap;        // sample capacity
};

// nb (0: p) buckets: the per-splitter arrays hold nb - 1 entries, the
// per-(segment, splitter) arrays p x (nb - 1).
size_t rounds_ws_bytes(uint64_t N, uint64_t p, uint64_t cap, uint64_t nb = 0);
RoundWs rounds_ws_carve(void* base, uint64_t N, uint64_t p, uint64_t cap, uint32_t* err, uint64_t nb = 0);
uint64_t sample_capacity(uint64_t N, uint64_t p, float oversample);

struct RoundResult {
    uint32_t rounds = 0;
    int status = 0;
    uint64_t sample_size[HSS_MAX_ROUNDS] = {};
    uint64_t gamma[HSS_MAX_ROUNDS] = {};
    uint64_t unresolved[HSS_MAX_ROUNDS + 1] = {};
};

// Histogram form of the rounds: chosen per round, or forced (tests).
constexpr uint32_t kHistAuto = 0, kHistProbe = 1, kHistStaged = 2;

// Driver of the round loop: the host; the device graph from the second call
// of a shape on (a first call of a shape drives its rounds from the host);
// the device graph always.
constexpr uint32_t kLoopHost = 0, kLoopAdaptive = 1, kLoopDevice = 2;

// Run the histogram rounds over the p locally sorted segments skeys
// (order-preserving key bits) and write the splitters, offsets and the final
// per-segment positions of the splitters (into ws.Lpos).  nb (0: p) is the
// number of buckets: nb - 1 splitters at ranks i N / nb (a stage of
// multi-stage HSS partitions p processors' keys into nb < p groups).  d_prop[nprop]
// (nullable; keys in the caller's representation, nprop <= ws.cap) are
// proposed cuts ranked and offered to every splitter before round 1.
// With the device loop (loop_mode) the rounds run as one CUDA graph (a WHILE
// conditional node whose body is one round; a device kernel decides whether
// another round is needed), so the call does not wait for the GPU: out is
// then left for read_round_result() once the stream has passed the rounds.  The loop is
// taken only when the round's probe sort needs no host planning (sample
// capacity <= the on-chip capacity) and the schedule is computed on the device
// (not the k-round schedule); else the host drives the rounds as before.
int run_rounds(const uint64_t* skeys, const uint64_t* d_seg_off, uint64_t N, uint32_t p, double eps, uint64_t seed,
               float oversample, uint32_t max_rounds, int key_type, hss_cut* d_splitters, uint64_t* d_offsets,
               const RoundWs& ws, cudaStream_t st, RoundResult* out, const uint64_t* d_prop = nullptr,
               uint32_t nprop = 0, uint32_t schedule = HSS_SCHEDULE_PROPORTIONAL, uint32_t schedule_k = 0,
               uint32_t hist_mode = kHistAuto, uint32_t loop_mode = kLoopHost, bool* used_device_loop = nullptr,
               uint32_t nb = 0);

// Whether run_rounds can drive these rounds on the device.
bool device_loop_possible(uint64_t cap, uint32_t schedule);

// Fill out from the device record of a device-driven run (synchronises
// `st`).  Returns the status.
int read_round_result(const RoundWs& ws, RoundResult* out, cudaStream_t st);
// Kernels one round of the device-driven loop launches.
uint32_t device_round_kernels();

// Per-bucket split windows for the merge, from the final splitters: the key
// range of the p locally sorted segments, cut into nb (0: p) buckets.
cudaError_t bucket_hints(const RoundWs& ws, const uint64_t* skeys, const uint64_t* d_seg_off, uint32_t p,
                         cudaStream_t st, uint32_t nb = 0);

// Exchange: per-(segment, bucket) destinations, then the run copy.
cudaError_t exchange(const uint64_t* skeys, const uint32_t* spay, uint64_t N, uint32_t p, const uint64_t* d_seg_off,
                     const uint32_t* pos /*[p][nb-1]*/, const uint64_t* d_offsets, uint64_t* bkeys, uint32_t* bpay,
                     uint64_t* dst_scratch /*[p][nb]*/, uint32_t* err, cudaStream_t st, uint32_t nb = 0);

// Ranks of arbitrary cuts (keys in caller representation).
cudaError_t rank_cuts(const uint64_t* skeys, int key_type, uint64_t N, uint32_t p,
                      const hss_cut* cuts, uint32_t ncuts, uint64_t* ranks, uint32_t* seg_pos, cudaStream_t st);

cudaError_t sample_words_launch(uint64_t seed, uint32_t seg, uint32_t round, uint32_t spos0, uint32_t count,
                                uint64_t* out, cudaStream_t st);

}  // namespace hss
