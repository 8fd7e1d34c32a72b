// two_stage.cu -- two-stage HSS (hss_sort_two_stage).
//
// Multi-stage HSS (Sec. 5.3; Sec. 7.3 runs two stages with r = sqrt(p) groups
// and the same eps in each) first splits the p processors' keys into r groups
// of p / r processors and then sorts every group on its own:
//
//   stage 1   local sort of the p segments, histogram rounds for the r - 1
//             group splitters (targets i N / r, tolerance floor(N eps / 2r),
//             s r probes per round), exchange of every segment's runs to the
//             groups (group g: its runs in processor order);
//   stage 2   group g's keys, dealt by position to its p / r processors, are
//             sorted by single-stage HSS with seed + 1 + g: the r groups form
//             one batch (hss_sort_batch), whose local sort starts from the
//             group's key window (between its two group splitters) instead
//             of the top digit.
//
// The final buckets are the groups' buckets in group order.  On one device
// the second stage re-sorts the data once more than a single stage does; what
// it saves is the rounds' work, which grows with the number of (segment,
// splitter) pairs: p (r - 1) in stage 1 and p (p / r - 1) in stage 2 instead
// of p (p - 1), and every probe is ranked in p / r segments instead of p.
#include "hss_internal.cuh"
#include "segsort.cuh"
#include "rounds.cuh"
#include "batch.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace hss {
namespace {

inline size_t aup(size_t x) { return (x + 255) / 256 * 256; }

template <typename T>
T* at(void* base, size_t off) { return (T*)((char*)base + off); }

// Buffers of a two-stage call.  The first block lives through both stages;
// the stage-1 block is dead once the groups are exchanged and their windows
// computed, and the stage-2 batch workspace is laid over it.
struct TLayout {
    size_t keysG, payG, hint_lo, hint_mult, goff, joff, err;     // live
    size_t keysA, payA, seg_off, sws, rws, dst;                  // stage 1
    size_t shared, stage1, batch, total;
};

TLayout plan_two(uint64_t N, uint32_t p, uint32_t r, const hss_params* prm, bool pay) {
    TLayout L{};
    size_t o = 0;
    auto take = [&](size_t b) { size_t x = o; o += aup(std::max<size_t>(b, 1)); return x; };
    const uint64_t N1 = std::max<uint64_t>(N, 1);
    const uint32_t pg = p / r;
    L.keysG = take(N1 * 8);
    L.payG = pay ? take(N1 * 4) : 0;
    L.hint_lo = take((uint64_t)p * 8);
    L.hint_mult = take((uint64_t)p * 8);
    L.goff = take(((uint64_t)r + 1) * 8);
    L.joff = take((uint64_t)r * (pg + 1) * 8);
    L.err = take(256);
    L.shared = o;
    L.keysA = take(N1 * 8);
    L.payA = pay ? take(N1 * 4) : 0;
    L.seg_off = take(((uint64_t)p + 1) * 8);
    L.sws = take(segsort_ws_bytes(N1, p));
    const uint64_t cap = sample_capacity(N, r, prm->oversample);
    L.rws = take(rounds_ws_bytes(N1, p, cap, r));
    L.dst = take((uint64_t)p * r * 8);
    L.stage1 = o - L.shared;
    L.batch = batch_bytes_bound(N, r, pg, prm, pay);
    L.total = L.batch ? L.shared + std::max(L.stage1, L.batch) : 0;
    return L;
}

bool args_ok(uint64_t N, const hss_params* prm, uint32_t r) {
    if (!prm || !(prm->eps > 0.0) || !std::isfinite(prm->eps)) return false;
    if (!(prm->oversample > 0.0f) || !std::isfinite(prm->oversample)) return false;
    if (prm->max_rounds > HSS_MAX_ROUNDS || prm->schedule != HSS_SCHEDULE_PROPORTIONAL) return false;
    if ((prm->flags & HSS_FLAG_HIST_PROBE) && (prm->flags & HSS_FLAG_HIST_STAGED)) return false;
    if ((prm->flags & HSS_FLAG_HOST_ROUNDS) && (prm->flags & HSS_FLAG_DEVICE_ROUNDS)) return false;
    const uint32_t p = prm->p;
    if (r < 2 || p < r || p % r != 0 || p / r > (1u << 16) || p > (1u << 22)) return false;
    // every processor of every group holds a key when stage 1 balances
    if (N < 2ull * p || N >= (1ull << 40)) return false;
    // stage-1 segments and groups, and stage-2 segments, below 2^30 keys
    const double tol1 = std::floor(((double)N * prm->eps) / (2.0 * (double)r));
    return (double)(N / r) + 2.0 * tol1 + 2.0 < (double)kMaxSegKeys && (N + p - 1) / p < kMaxSegKeys;
}

// Window of every stage-2 segment: its group's window (segments of group g
// are g pg .. g pg + pg - 1 in the batch).
__global__ void k_group_hints(uint32_t p, uint32_t pg, const uint64_t* __restrict__ glo,
                              const uint64_t* __restrict__ gmult, uint64_t* __restrict__ lo,
                              uint64_t* __restrict__ mult) {
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= p) return;
    lo[s] = glo[s / pg];
    mult[s] = gmult[s / pg];
}

// Final offsets: bucket g pg + i starts at group g's start plus the start of
// bucket i inside the group.
__global__ void k_two_stage_offsets(uint32_t r, uint32_t pg, uint64_t N, const uint64_t* __restrict__ goff,
                                    const uint64_t* __restrict__ joff, uint64_t* __restrict__ off) {
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t p = (uint64_t)r * pg;
    if (b > p) return;
    if (b == p) { off[p] = N; return; }
    const uint64_t g = b / pg, i = b % pg;
    off[b] = goff[g] + joff[g * (pg + 1) + i];
}

#define HSS_TTRY(x) do { if ((x) != cudaSuccess) return HSS_ERR_CUDA; } while (0)

int run_two_stage(const void* d_keys, const uint32_t* d_payload, int key_type, uint64_t N, const hss_params* prm,
                  uint32_t r, void* d_keys_out, uint32_t* d_payload_out, hss_cut* d_group_splitters,
                  hss_cut* d_splitters, uint64_t* d_offsets, void* d_work, size_t work_bytes,
                  hss_two_stage_stats* h_stats, hss_job_stats* h_group_stats, cudaStream_t st) {
    const uint64_t mark = hss_kernel_launch_count();
    if (h_stats) std::memset(h_stats, 0, sizeof(*h_stats));
    if (!args_ok(N, prm, r) || (key_type != HSS_KEY_U64 && key_type != HSS_KEY_I64)) return HSS_ERR_INVALID;
    const uint32_t p = prm->p, pg = p / r;
    if (!d_keys || !d_keys_out || !d_offsets || !d_group_splitters || (pg > 1 && !d_splitters) || !d_work)
        return HSS_ERR_INVALID;
    if ((d_payload == nullptr) != (d_payload_out == nullptr)) return HSS_ERR_INVALID;
    const bool pay = d_payload != nullptr;
    const TLayout L = plan_two(N, p, r, prm, pay);
    if (L.total == 0) return HSS_ERR_INVALID;
    if (work_bytes < L.total) return HSS_ERR_WORKSPACE;
    const bool i64 = key_type == HSS_KEY_I64;
    const bool timing = (prm->flags & HSS_FLAG_TIMING) != 0;

    uint64_t* keysG = at<uint64_t>(d_work, L.keysG);
    uint32_t* payG = pay ? at<uint32_t>(d_work, L.payG) : nullptr;
    uint64_t* hint_lo = at<uint64_t>(d_work, L.hint_lo);
    uint64_t* hint_mult = at<uint64_t>(d_work, L.hint_mult);
    uint64_t* goff = at<uint64_t>(d_work, L.goff);
    uint64_t* joff = at<uint64_t>(d_work, L.joff);
    uint32_t* err = at<uint32_t>(d_work, L.err);
    uint64_t* keysA = at<uint64_t>(d_work, L.keysA);
    uint32_t* payA = pay ? at<uint32_t>(d_work, L.payA) : nullptr;
    uint64_t* seg_off = at<uint64_t>(d_work, L.seg_off);
    SegSortWs sws = segsort_ws_carve(at<void>(d_work, L.sws), std::max<uint64_t>(N, 1), p, err);
    const uint64_t cap = sample_capacity(N, r, prm->oversample);
    RoundWs rws = rounds_ws_carve(at<void>(d_work, L.rws), std::max<uint64_t>(N, 1), p, cap, err, r);
    uint64_t* dst = at<uint64_t>(d_work, L.dst);

    TimingEvents<4> tev;
    cudaEvent_t* ev = tev.ev;
    if (timing) {
        tev.create();
        cudaEventRecord(ev[0], st);
    }
    HSS_TTRY(cudaMemsetAsync(err, 0, 256, st));
    HSS_TTRY(fill_even_offsets(seg_off, N, p, st));

    // Stage 1: local sort (keysG serves as the sort's scratch), the group
    // splitters, the exchange into keysG, and the groups' key windows.
    HSS_TTRY(segsort((const uint64_t*)d_keys, keysA, keysG, d_payload, payA, payG, N, p, seg_off, i64, false, sws, st,
                     nullptr));
    if (timing) cudaEventRecord(ev[1], st);
    const uint32_t hist = (prm->flags & HSS_FLAG_HIST_PROBE) ? kHistProbe
                          : (prm->flags & HSS_FLAG_HIST_STAGED) ? kHistStaged : kHistAuto;
    const uint32_t loop = (prm->flags & HSS_FLAG_HOST_ROUNDS) ? kLoopHost
                          : (prm->flags & HSS_FLAG_DEVICE_ROUNDS) ? kLoopDevice : kLoopAdaptive;
    const uint32_t max_rounds = prm->max_rounds == 0 ? HSS_MAX_ROUNDS : prm->max_rounds;
    RoundResult rr;
    bool device_loop = false;
    int status1 = run_rounds(keysA, seg_off, N, p, prm->eps, prm->seed, prm->oversample, max_rounds, key_type,
                             d_group_splitters, goff, rws, st, &rr, nullptr, 0, HSS_SCHEDULE_PROPORTIONAL, 0, hist,
                             loop, &device_loop, r);
    if (status1 == HSS_ERR_CUDA || status1 == HSS_ERR_INVALID) return status1;
    if (timing) cudaEventRecord(ev[2], st);
    HSS_TTRY(exchange(keysA, payA, N, p, seg_off, rws.Lpos, goff, keysG, payG, dst, err, st, r));
    HSS_TTRY(bucket_hints(rws, keysA, seg_off, p, st, r));
    HSS_LAUNCH(k_group_hints, (unsigned)((p + 255) / 256), 256, 0, st, p, pg, rws.bucket_lo, rws.bucket_mult, hint_lo,
               hint_mult);
    if (timing) cudaEventRecord(ev[3], st);

    // The group sizes decide the batch's tables.
    std::vector<uint64_t> h_goff(r + 1);
    uint32_t h_err = 0;
    HSS_TTRY(read_small(h_goff.data(), goff, ((size_t)r + 1) * 8, st));
    HSS_TTRY(read_small(&h_err, err, 4, st));
    if (device_loop) {
        status1 = read_round_result(rws, &rr, st);
        add_launches(1 + (uint64_t)rr.rounds * device_round_kernels());
    }
    if (h_err & kDevErrTimeout) return HSS_ERR_TIMEOUT;
    if (h_err & kDevErrSize) return HSS_ERR_INVALID;
    if (h_err & kDevErrBounds) return HSS_ERR_CUDA;
    std::vector<uint64_t> sizes(r);
    std::vector<uint32_t> ps(r, pg);
    for (uint32_t g = 0; g < r; ++g) {
        sizes[g] = h_goff[g + 1] - h_goff[g];
        if (sizes[g] < pg) return HSS_ERR_INVALID;  // a processor of the group would hold no key
    }

    // Stage 2: the groups as one batch, seed + 1 + g for group g.
    hss_params prm2 = *prm;
    prm2.seed = prm->seed + 1;
    prm2.p = pg;
    BatchExtra ex;
    ex.keys_ordered = true;
    ex.hint_lo = hint_lo;
    ex.hint_mult = hint_mult;
    hss_batch_stats bst;
    const int status2 = run_batch(keysG, payG, key_type, sizes.data(), ps.data(), r, &prm2, d_keys_out, d_payload_out,
                                  d_splitters, joff, at<void>(d_work, L.shared), work_bytes - L.shared, &bst,
                                  h_group_stats, st, true, ex);
    if (status2 == HSS_ERR_CUDA || status2 == HSS_ERR_INVALID || status2 == HSS_ERR_WORKSPACE) return status2;
    HSS_LAUNCH(k_two_stage_offsets, (unsigned)(((uint64_t)p + 1 + 255) / 256), 256, 0, st, r, pg, N, goff, joff,
               d_offsets);
    HSS_TTRY(cudaGetLastError());
    HSS_TTRY(cudaStreamSynchronize(st));
    const int status = status1 != HSS_OK ? status1 : status2;

    if (h_stats) {
        hss_stats& s1 = h_stats->stage1;
        s1.rounds = rr.rounds;
        s1.status = status1;
        s1.tol = (uint64_t)std::floor(((double)N * prm->eps) / (2.0 * (double)r));
        for (uint32_t j = 0; j < rr.rounds && j < HSS_MAX_ROUNDS; ++j) {
            s1.sample_size[j] = rr.sample_size[j];
            s1.gamma[j] = rr.gamma[j];
        }
        for (uint32_t j = 0; j <= rr.rounds && j <= HSS_MAX_ROUNDS; ++j) s1.unresolved[j] = rr.unresolved[j];
        h_stats->stage2 = bst;
        h_stats->groups = r;
        h_stats->status = status;
        if (timing) {
            cudaEventElapsedTime(&s1.ms_phase[HSS_PHASE_LOCAL_SORT], ev[0], ev[1]);
            cudaEventElapsedTime(&s1.ms_phase[HSS_PHASE_ROUNDS], ev[1], ev[2]);
            cudaEventElapsedTime(&s1.ms_phase[HSS_PHASE_EXCHANGE], ev[2], ev[3]);
        }
        h_stats->kernel_launches = (uint32_t)(hss_kernel_launch_count() - mark);
    }
    return status;
}

}  // namespace
}  // namespace hss

using namespace hss;

extern "C" {

size_t hss_two_stage_workspace_bytes(uint64_t N, const hss_params* prm, uint32_t groups, int key_type,
                                     int has_payload) {
    (void)key_type;
    if (!args_ok(N, prm, groups)) return 0;
    return plan_two(N, prm->p, groups, prm, has_payload != 0).total;
}

int hss_sort_two_stage(const void* d_keys, const uint32_t* d_payload, int key_type, uint64_t N, const hss_params* prm,
                       uint32_t groups, void* d_keys_out, uint32_t* d_payload_out, hss_cut* d_group_splitters,
                       hss_cut* d_splitters, uint64_t* d_offsets, void* d_work, size_t work_bytes,
                       hss_two_stage_stats* h_stats, hss_job_stats* h_group_stats, void* stream) {
    return run_two_stage(d_keys, d_payload, key_type, N, prm, groups, d_keys_out, d_payload_out, d_group_splitters,
                         d_splitters, d_offsets, d_work, work_bytes, h_stats, h_group_stats, (cudaStream_t)stream);
}

}  // extern "C"
