// hss_api.cu -- the C ABI of libhss.so (declared in include/hss.h).
//
// Orchestrates the hot path of Histogram Sort with Sampling on one device:
// local sort (segmented radix sort over the p processor segments), the
// splitter rounds, the exchange of runs to buckets and the per-bucket merge.
// All scratch comes from the caller's workspace; the library never allocates.
#include "hss_internal.cuh"
#include "segsort.cuh"
#include "rounds.cuh"

#include <atomic>
#include <cmath>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <map>
#include <set>
#include <utility>

namespace hss {

static std::atomic<uint64_t> g_launches{0};
static thread_local int t_capture_depth = 0;
static thread_local uint64_t t_captured = 0;
void note_launch() {
    if (t_capture_depth > 0) ++t_captured;
    else g_launches.fetch_add(1, std::memory_order_relaxed);
}
void add_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
LaunchCountPause::LaunchCountPause() { ++t_capture_depth; }
LaunchCountPause::~LaunchCountPause() { --t_capture_depth; }
uint64_t LaunchCountPause::captured() const { return t_captured; }

// Per-device bookkeeping of kernel attributes and SM counts: a kernel's
// shared-memory limit set on one device does not carry over to another, and
// server threads call in concurrently.
static std::mutex g_attr_mu;
static std::set<std::pair<int, const void*>> g_attr_done;
constexpr int kMaxDevices = 256;
static std::atomic<int> g_sm_count[kMaxDevices];

cudaError_t ensure_func_attrs(const void* func, int max_dyn_smem, int carveout) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_attr_mu);
    if (g_attr_done.count({dev, func})) return cudaSuccess;
    if ((e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn_smem)) != cudaSuccess)
        return e;
    if (carveout >= 0 &&
        (e = cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout, carveout)) != cudaSuccess)
        return e;
    g_attr_done.insert({dev, func});
    return cudaSuccess;
}

int resident_ctas(const void* func, int threads, size_t dyn_smem) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> lock(mu);
    const auto it = cache.find({dev, func});
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, func, threads, dyn_smem) != cudaSuccess || n < 1) n = 1;
    cache[{dev, func}] = n;
    return n;
}

__global__ void k_copy_words(const uint32_t* __restrict__ src, volatile uint32_t* dst, uint32_t n) {
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

static constexpr size_t kSmallRead = 8192;
struct SmallReadBuf {
    volatile uint32_t* host = nullptr;
    uint32_t* dev = nullptr;
    bool tried = false;
};
static thread_local SmallReadBuf t_small;

cudaError_t read_small(void* h_dst, const void* d_src, size_t bytes, cudaStream_t st) {
    if (!t_small.tried) {
        t_small.tried = true;
        void* p = nullptr;
        if (cudaHostAlloc(&p, kSmallRead, cudaHostAllocMapped | cudaHostAllocPortable) == cudaSuccess) {
            void* dp = nullptr;
            if (cudaHostGetDevicePointer(&dp, p, 0) == cudaSuccess) {
                t_small.host = (volatile uint32_t*)p;
                t_small.dev = (uint32_t*)dp;
            } else {
                (void)cudaGetLastError();
                cudaFreeHost(p);
            }
        } else {
            (void)cudaGetLastError();
        }
    }
    cudaError_t e;
    if (!t_small.host || bytes > kSmallRead || bytes % 4 != 0 || ((uintptr_t)d_src & 3u) != 0) {
        if ((e = cudaMemcpyAsync(h_dst, d_src, bytes, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
        return cudaStreamSynchronize(st);
    }
    const uint32_t n = (uint32_t)(bytes / 4);
    HSS_LAUNCH(k_copy_words, 1, 256, 0, st, (const uint32_t*)d_src, t_small.dev, n);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    uint32_t* out = (uint32_t*)h_dst;
    for (uint32_t i = 0; i < n; ++i) out[i] = t_small.host[i];
    return cudaSuccess;
}

int device_sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 148;
    int n = g_sm_count[dev].load(std::memory_order_relaxed);
    if (n <= 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
        g_sm_count[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

static inline size_t aup(size_t x) { return (x + 255) / 256 * 256; }

struct Layout {
    size_t keysA = 0, keysB = 0, payA = 0, payB = 0, seg_off = 0, err = 0, sws = 0, rws = 0, dst = 0;
    size_t io_keys = 0, io_pay = 0, io_spl = 0, io_off = 0;
    size_t total = 0;
    bool has_pay = false;
};

static const uint64_t kMaxN = 1ull << 40;
static const uint32_t kMaxP = 1u << 22;
// A segment or bucket holds fewer than 2^30 keys: the look-back words of the
// split pack a digit's count into 30 bits and in-segment positions are u32.
static const uint64_t kMaxSeg = 1ull << 30;

// Every processor segment of N keys over p processors is below the limit.
static bool segments_fit(uint64_t N, uint32_t p) { return p > 0 && (N + p - 1) / p < kMaxSeg; }
// ... and so is every bucket of an eps-balanced partition: at most
// ceil(N/p) + 2 floor(N eps/(2p)) keys.
static bool buckets_fit(uint64_t N, uint32_t p, double eps) {
    if (!segments_fit(N, p)) return false;
    const double extra = std::floor(((double)N * eps) / (2.0 * (double)p)) * 2.0;
    return (double)((N + p - 1) / p) + extra + 1.0 < (double)kMaxSeg;
}

static Layout plan(int op, uint64_t N, uint32_t p, float oversample, bool pay) {
    Layout L;
    L.has_pay = pay;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t r = off; off += aup(bytes); return r; };
    const uint64_t N1 = std::max<uint64_t>(N, 1);
    switch (op) {
    case HSS_OP_LOCAL_SORT:
    case HSS_OP_MERGE:
        L.keysB = take(N1 * 8);
        if (pay) L.payB = take(N1 * 4);
        L.seg_off = take((uint64_t)(p + 1) * 8);
        L.err = take(256);
        L.sws = take(segsort_ws_bytes(N1, p));
        break;
    case HSS_OP_EXCHANGE:
        L.seg_off = take((uint64_t)(p + 1) * 8);
        L.err = take(256);
        L.dst = take((uint64_t)p * p * 8);
        break;
    case HSS_OP_PARTITION:
    case HSS_OP_SORT:
    case HSS_OP_SORT_HOST: {
        L.keysA = take(N1 * 8);
        L.keysB = take(N1 * 8);
        if (pay && op != HSS_OP_PARTITION) { L.payA = take(N1 * 4); L.payB = take(N1 * 4); }
        L.seg_off = take((uint64_t)(p + 1) * 8);
        L.err = take(256);
        L.sws = take(segsort_ws_bytes(N1, p));
        const uint64_t cap = sample_capacity(N, p, oversample);
        L.rws = take(rounds_ws_bytes(N1, p, cap));
        if (op != HSS_OP_PARTITION) L.dst = take((uint64_t)p * p * 8);
        if (op == HSS_OP_SORT_HOST) {
            L.io_keys = take(N1 * 8);
            if (pay) L.io_pay = take(N1 * 4);
            L.io_spl = take((uint64_t)std::max<uint32_t>(p - 1, 1) * sizeof(hss_cut));
            L.io_off = take((uint64_t)(p + 1) * 8);
        }
        break;
    }
    default:
        return L;
    }
    L.total = off;
    return L;
}

template <typename T>
static T* at(void* base, size_t off) { return (T*)((char*)base + off); }

static bool params_ok(const hss_params* prm) {
    if (!prm) return false;
    if (!(prm->eps > 0.0) || !std::isfinite(prm->eps)) return false;
    if (prm->p == 0 || prm->p > kMaxP) return false;
    if (!(prm->oversample > 0.0f) || !std::isfinite(prm->oversample)) return false;
    if (prm->max_rounds > HSS_MAX_ROUNDS) return false;
    if (prm->schedule > HSS_SCHEDULE_EQUAL || (prm->schedule == HSS_SCHEDULE_THEORY && prm->schedule_k == 0)) return false;
    if ((prm->flags & HSS_FLAG_HIST_PROBE) && (prm->flags & HSS_FLAG_HIST_STAGED)) return false;
    if ((prm->flags & HSS_FLAG_HOST_ROUNDS) && (prm->flags & HSS_FLAG_DEVICE_ROUNDS)) return false;
    return true;
}
static uint32_t hist_mode(const hss_params* prm) {
    if (prm->flags & HSS_FLAG_HIST_PROBE) return kHistProbe;
    if (prm->flags & HSS_FLAG_HIST_STAGED) return kHistStaged;
    return kHistAuto;
}

static uint32_t loop_mode(const hss_params* prm) {
    if (prm->flags & HSS_FLAG_HOST_ROUNDS) return kLoopHost;
    if (prm->flags & HSS_FLAG_DEVICE_ROUNDS) return kLoopDevice;
    return kLoopAdaptive;
}

// Oversampling that sizes the round sample buffers: s, or under the k-round
// schedule 5 (2 ln p / eps)^(1/k), the bound of Lemma 4.6 on a round's probes
// per processor (round 1 draws p (2 ln p / eps)^(1/k) of the whole input).
static float eff_oversample(const hss_params* prm) {
    if (!prm) return 5.0f;
    if (prm->schedule == HSS_SCHEDULE_THEORY && prm->schedule_k > 0 && prm->p > 1) {
        const double r = std::pow(2.0 * std::log((double)prm->p) / prm->eps, 1.0 / (double)prm->schedule_k);
        return (float)std::max<double>(prm->oversample, 5.0 * r);
    }
    return prm->oversample;
}
static uint32_t eff_rounds(const hss_params* prm) { return prm->max_rounds == 0 ? HSS_MAX_ROUNDS : prm->max_rounds; }

struct PhaseTimer {
    bool on = false;
    cudaStream_t st = nullptr;
    cudaEvent_t ev[HSS_NUM_PHASES + 1] = {};
    void start(bool enable, cudaStream_t s) {
        on = enable; st = s;
        if (!on) return;
        for (auto& e : ev) cudaEventCreate(&e);
        cudaEventRecord(ev[0], st);
    }
    void mark(int phase_end) { if (on) cudaEventRecord(ev[phase_end + 1], st); }
    void finish(hss_stats* out, int last_phase) {
        if (!on) return;
        cudaEventSynchronize(ev[last_phase + 1]);
        if (out) {
            for (int i = 0; i <= last_phase; ++i) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
                out->ms_phase[i] = ms;
            }
        }
        for (auto& e : ev) cudaEventDestroy(e);
        on = false;
    }
    ~PhaseTimer() {  // a call that returned early
        if (on)
            for (auto& e : ev)
                if (e) cudaEventDestroy(e);
    }
};

static int read_dev_err(uint32_t* d_err, cudaStream_t st) {
    uint32_t h = 0;
    if (read_small(&h, d_err, sizeof(h), st) != cudaSuccess) return HSS_ERR_CUDA;
    if (h & kDevErrTimeout) return HSS_ERR_TIMEOUT;
    if (h & kDevErrSize) return HSS_ERR_INVALID;
    if (h & kDevErrBounds) return HSS_ERR_CUDA;
    return HSS_OK;
}

// Host buffers of hss_sort_host: the copies run on a second stream in
// chunks, overlapping the local sort (input, a group of processors at a time)
// and the merge (output, a group of buckets at a time).
struct HostIO {
    const void* h_keys;
    const uint32_t* h_payload;
    void* h_keys_out;
    uint32_t* h_payload_out;
    uint64_t* h_offsets;  // filled before the merge (the output copies need them)
    cudaStream_t cs;      // copy stream
    cudaEvent_t ev[2 * 64];
    uint32_t groups;      // chunks each way
};

static std::mutex g_io_mu;
static std::mutex g_io_call_mu[256];  // one hss_sort_host at a time per device (they share the copy stream)
static cudaStream_t g_io_stream[256] = {};
static cudaEvent_t g_io_events[256][2 * 64] = {};

// Copy stream and events of the current device (created once).
static int io_resources(cudaStream_t* cs, cudaEvent_t** ev, int* dev_out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return HSS_ERR_CUDA;
    *dev_out = dev;
    std::lock_guard<std::mutex> lock(g_io_mu);
    if (!g_io_stream[dev]) {
        if (cudaStreamCreateWithFlags(&g_io_stream[dev], cudaStreamNonBlocking) != cudaSuccess) return HSS_ERR_CUDA;
        for (auto& e : g_io_events[dev])
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return HSS_ERR_CUDA;
    }
    *cs = g_io_stream[dev];
    *ev = g_io_events[dev];
    return HSS_OK;
}

// Core of hss_partition / hss_sort.
static int run_path(const void* d_keys, const uint32_t* d_payload, int key_type, uint64_t N, const hss_params* prm,
                    void* d_keys_out, uint32_t* d_payload_out, hss_cut* d_splitters, uint64_t* d_offsets,
                    void* d_work, size_t work_bytes, hss_stats* h_stats, cudaStream_t st, bool sort,
                    const void* d_prop = nullptr, uint32_t nprop = 0, HostIO* hio = nullptr) {
    const uint64_t mark = g_launches.load();
    if (h_stats) std::memset(h_stats, 0, sizeof(*h_stats));
    if (!params_ok(prm) || (key_type != HSS_KEY_U64 && key_type != HSS_KEY_I64) || N >= kMaxN) return HSS_ERR_INVALID;
    if (!(sort ? buckets_fit(N, prm->p, prm->eps) : segments_fit(N, prm->p))) return HSS_ERR_INVALID;
    if ((N > 0 && !d_keys) || !d_offsets || (prm->p > 1 && !d_splitters) || !d_work) return HSS_ERR_INVALID;
    if (sort && N > 0 && !d_keys_out) return HSS_ERR_INVALID;
    const bool pay = sort && d_payload != nullptr;
    if (sort && ((d_payload == nullptr) != (d_payload_out == nullptr))) return HSS_ERR_INVALID;
    const uint32_t p = prm->p;
    const float s = prm->oversample;
    const float s_cap = eff_oversample(prm);
    const Layout L = plan(sort ? HSS_OP_SORT : HSS_OP_PARTITION, N, p, s_cap, pay);
    if (work_bytes < L.total) return HSS_ERR_WORKSPACE;

    uint64_t* keysA = at<uint64_t>(d_work, L.keysA);
    uint64_t* keysB = at<uint64_t>(d_work, L.keysB);
    uint32_t* payA = pay ? at<uint32_t>(d_work, L.payA) : nullptr;
    uint32_t* payB = pay ? at<uint32_t>(d_work, L.payB) : nullptr;
    uint64_t* seg_off = at<uint64_t>(d_work, L.seg_off);
    uint32_t* err = at<uint32_t>(d_work, L.err);
    const uint64_t cap = sample_capacity(N, p, s_cap);
    SegSortWs sws = segsort_ws_carve(at<void>(d_work, L.sws), std::max<uint64_t>(N, 1), p, err);
    RoundWs rws = rounds_ws_carve(at<void>(d_work, L.rws), std::max<uint64_t>(N, 1), p, cap, err);
    const bool i64 = key_type == HSS_KEY_I64;
    const bool timing = (prm->flags & HSS_FLAG_TIMING) != 0;

    if (cudaMemsetAsync(err, 0, 256, st) != cudaSuccess) return HSS_ERR_CUDA;
    if (fill_even_offsets(seg_off, N, p, st) != cudaSuccess) return HSS_ERR_CUDA;

    PhaseTimer tm;
    tm.start(timing, st);
    SegSortTiming stime;
    stime.enabled = timing;

    // Local sort (Sec. 5): order-preserving bits into keysA.  With a single
    // processor the locally sorted segment is already the output.
    const bool single = sort && p == 1;
    if (hio) {
        // Input in chunks of whole processors: every chunk's copy is queued
        // on the copy stream first (the copy engine then runs without a gap
        // while the host plans the sorts), and the processors of chunk g are
        // sorted as soon as it has landed.
        const uint32_t G = hio->groups;
        for (uint32_t g = 0; g < G; ++g) {
            const uint64_t s0 = (uint64_t)g * p / G, s1 = (uint64_t)(g + 1) * p / G;
            const uint64_t a = (uint64_t)(((unsigned __int128)s0 * N) / p), b = (uint64_t)(((unsigned __int128)s1 * N) / p);
            if (b > a && cudaMemcpyAsync((uint64_t*)d_keys + a, (const uint64_t*)hio->h_keys + a, (b - a) * 8,
                                         cudaMemcpyHostToDevice, hio->cs) != cudaSuccess)
                return HSS_ERR_CUDA;
            if (pay && b > a && cudaMemcpyAsync((uint32_t*)d_payload + a, hio->h_payload + a, (b - a) * 4,
                                                cudaMemcpyHostToDevice, hio->cs) != cudaSuccess)
                return HSS_ERR_CUDA;
            if (cudaEventRecord(hio->ev[g], hio->cs) != cudaSuccess) return HSS_ERR_CUDA;
        }
        for (uint32_t g = 0; g < G; ++g) {
            const uint64_t s0 = (uint64_t)g * p / G, s1 = (uint64_t)(g + 1) * p / G;
            const uint64_t a = (uint64_t)(((unsigned __int128)s0 * N) / p), b = (uint64_t)(((unsigned __int128)s1 * N) / p);
            if (cudaStreamWaitEvent(st, hio->ev[g], 0) != cudaSuccess) return HSS_ERR_CUDA;
            if (s1 > s0 && segsort((const uint64_t*)d_keys, single ? (uint64_t*)d_keys_out : keysA, keysB, d_payload,
                                   single ? d_payload_out : payA, payB, b - a, s1 - s0, seg_off + s0, i64, single && i64,
                                   sws, st, &stime) != cudaSuccess)
                return HSS_ERR_CUDA;
        }
    } else if (segsort((const uint64_t*)d_keys, single ? (uint64_t*)d_keys_out : keysA, keysB, d_payload,
                       single ? d_payload_out : payA, payB, N, p, seg_off, i64, single && i64, sws, st, &stime) !=
               cudaSuccess) {
        return HSS_ERR_CUDA;
    }
    tm.mark(HSS_PHASE_LOCAL_SORT);

    // Splitter rounds (Sec. 4.2.2).
    RoundResult rr;
    bool device_loop = false;
    int status = run_rounds(keysA, seg_off, N, p, prm->eps, prm->seed, s, eff_rounds(prm), key_type, d_splitters,
                            d_offsets, rws, st, &rr, (const uint64_t*)d_prop, nprop, prm->schedule, prm->schedule_k,
                            hist_mode(prm), loop_mode(prm), &device_loop);
    tm.mark(HSS_PHASE_ROUNDS);
    if (status == HSS_ERR_CUDA || status == HSS_ERR_INVALID) return status;

    if (sort) {
        if (single) {
            tm.mark(HSS_PHASE_EXCHANGE);
            tm.mark(HSS_PHASE_MERGE);
        } else {
            uint64_t* dst = at<uint64_t>(d_work, L.dst);
            // Exchange (Sec. 3.1 step 3): runs to buckets, keysA -> keysB.
            if (exchange(keysA, payA, N, p, seg_off, rws.Lpos, d_offsets, keysB, payB, dst, err, st) != cudaSuccess)
                return HSS_ERR_CUDA;
            tm.mark(HSS_PHASE_EXCHANGE);
            // Merge (Sec. 6 local merging): stable sort of each bucket's runs.
            // The keys of bucket b lie between splitters b and b+1, so the first
            // split of each bucket spreads that key range over 256 sub-buckets.
            if (bucket_hints(rws, keysA, seg_off, p, st) != cudaSuccess) return HSS_ERR_CUDA;
            if (hio) {
                // Output in chunks of whole buckets: chunk g goes back on the
                // copy stream while the next chunk merges.  The bucket bounds
                // come first (the host needs them to cut the chunks).
                if (cudaMemcpyAsync(hio->h_offsets, d_offsets, (uint64_t)(p + 1) * 8, cudaMemcpyDeviceToHost, st) !=
                        cudaSuccess ||
                    cudaStreamSynchronize(st) != cudaSuccess)
                    return HSS_ERR_CUDA;
                const uint32_t G = hio->groups;
                for (uint32_t g = 0; g < G; ++g) {
                    const uint64_t b0 = (uint64_t)g * p / G, b1 = (uint64_t)(g + 1) * p / G;
                    const uint64_t a = hio->h_offsets[b0], b = hio->h_offsets[b1];
                    if (b1 > b0 && b > a &&
                        segsort(keysB, (uint64_t*)d_keys_out, keysA, payB, d_payload_out, payA, b - a, b1 - b0,
                                d_offsets + b0, false, i64, sws, st, &stime, rws.bucket_lo + b0,
                                rws.bucket_mult + b0) != cudaSuccess)
                        return HSS_ERR_CUDA;
                    if (cudaEventRecord(hio->ev[64 + g], st) != cudaSuccess) return HSS_ERR_CUDA;
                    if (cudaStreamWaitEvent(hio->cs, hio->ev[64 + g], 0) != cudaSuccess) return HSS_ERR_CUDA;
                    if (b > a && cudaMemcpyAsync((uint64_t*)hio->h_keys_out + a, (uint64_t*)d_keys_out + a, (b - a) * 8,
                                                 cudaMemcpyDeviceToHost, hio->cs) != cudaSuccess)
                        return HSS_ERR_CUDA;
                    if (pay && b > a && cudaMemcpyAsync(hio->h_payload_out + a, d_payload_out + a, (b - a) * 4,
                                                        cudaMemcpyDeviceToHost, hio->cs) != cudaSuccess)
                        return HSS_ERR_CUDA;
                }
            } else if (segsort(keysB, (uint64_t*)d_keys_out, keysA, payB, d_payload_out, payA, N, p, d_offsets, false, i64,
                               sws, st, &stime, rws.bucket_lo, rws.bucket_mult) != cudaSuccess) {
                return HSS_ERR_CUDA;
            }
            tm.mark(HSS_PHASE_MERGE);
        }
    }
    tm.finish(h_stats, sort ? HSS_PHASE_MERGE : HSS_PHASE_ROUNDS);

    // With the device-driven rounds nothing above waited for the GPU (a
    // partition returns at once; a sort waits only where the merge plans its
    // levels): the statistics and the device status are read here when asked
    // for, else later through hss_call_stats.
    const bool sync = (prm->flags & (HSS_FLAG_SYNC | HSS_FLAG_TIMING)) != 0 || h_stats != nullptr;
    if (device_loop && sync) {
        status = read_round_result(rws, &rr, st);
        add_launches(1 + (uint64_t)rr.rounds * device_round_kernels());
    }
    if (sync || (!device_loop && status == HSS_OK)) {
        const int e = read_dev_err(err, st);
        if (e != HSS_OK && status == HSS_OK) status = e;
    }
    if (h_stats) {
        h_stats->rounds = rr.rounds;
        h_stats->status = status;
        h_stats->tol = (uint64_t)std::floor(((double)N * prm->eps) / (2.0 * (double)p));
        for (uint32_t j = 0; j < rr.rounds && j < HSS_MAX_ROUNDS; ++j) {
            h_stats->sample_size[j] = rr.sample_size[j];
            h_stats->gamma[j] = rr.gamma[j];
        }
        for (uint32_t j = 0; j <= rr.rounds && j <= HSS_MAX_ROUNDS; ++j) h_stats->unresolved[j] = rr.unresolved[j];
        stime.collect(&h_stats->ms_radix_pass_total, &h_stats->radix_pass_launches, &h_stats->radix_pass_keys);
        h_stats->kernel_launches = (uint32_t)(g_launches.load() - mark);
    }
    if (stime.n) stime.collect(nullptr, nullptr, nullptr);
    return status;
}

}  // namespace hss

using namespace hss;

extern "C" {

size_t hss_workspace_bytes(int op, uint64_t N, const hss_params* prm, uint32_t p_if_no_params, int key_type,
                           int has_payload) {
    (void)key_type;
    const uint32_t p = prm ? prm->p : p_if_no_params;
    if (p == 0) return 0;
    const Layout L = plan(op, N, p, eff_oversample(prm), has_payload != 0);
    return L.total;
}

int hss_local_sort(const void* d_keys, const uint32_t* d_payload, int key_type, uint64_t N, uint32_t p,
                   void* d_keys_out, uint32_t* d_payload_out, void* d_work, size_t work_bytes, void* stream) {
    if ((key_type != HSS_KEY_U64 && key_type != HSS_KEY_I64) || p == 0 || p > kMaxP || N >= kMaxN) return HSS_ERR_INVALID;
    if (!segments_fit(N, p)) return HSS_ERR_INVALID;
    if (N > 0 && (!d_keys || !d_keys_out)) return HSS_ERR_INVALID;
    if ((d_payload == nullptr) != (d_payload_out == nullptr) || !d_work) return HSS_ERR_INVALID;
    const bool pay = d_payload != nullptr;
    const Layout L = plan(HSS_OP_LOCAL_SORT, N, p, 5.0f, pay);
    if (work_bytes < L.total) return HSS_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t* err = at<uint32_t>(d_work, L.err);
    uint64_t* seg_off = at<uint64_t>(d_work, L.seg_off);
    SegSortWs sws = segsort_ws_carve(at<void>(d_work, L.sws), std::max<uint64_t>(N, 1), p, err);
    if (cudaMemsetAsync(err, 0, 256, st) != cudaSuccess) return HSS_ERR_CUDA;
    if (fill_even_offsets(seg_off, N, p, st) != cudaSuccess) return HSS_ERR_CUDA;
    const bool i64 = key_type == HSS_KEY_I64;
    if (segsort((const uint64_t*)d_keys, (uint64_t*)d_keys_out, at<uint64_t>(d_work, L.keysB), d_payload, d_payload_out,
                pay ? at<uint32_t>(d_work, L.payB) : nullptr, N, p, seg_off, i64, i64, sws, st, nullptr) != cudaSuccess)
        return HSS_ERR_CUDA;
    return read_dev_err(err, st);
}

int hss_rank_cuts(const void* d_sorted_keys, int key_type, uint64_t N, uint32_t p, const hss_cut* d_cuts, uint32_t ncuts,
                  uint64_t* d_ranks, uint32_t* d_seg_pos, void* stream) {
    if ((key_type != HSS_KEY_U64 && key_type != HSS_KEY_I64) || p == 0 || p > kMaxP || N >= kMaxN) return HSS_ERR_INVALID;
    if (!segments_fit(N, p)) return HSS_ERR_INVALID;
    if (ncuts > 0 && (!d_cuts || !d_ranks || (N > 0 && !d_sorted_keys))) return HSS_ERR_INVALID;
    if (rank_cuts((const uint64_t*)d_sorted_keys, key_type, N, p, d_cuts, ncuts, d_ranks, d_seg_pos,
                  (cudaStream_t)stream) != cudaSuccess)
        return HSS_ERR_CUDA;
    return HSS_OK;
}

int hss_partition(const void* d_keys, int key_type, uint64_t N, const hss_params* prm, hss_cut* d_splitters,
                  uint64_t* d_offsets, void* d_work, size_t work_bytes, hss_stats* h_stats, void* stream) {
    return run_path(d_keys, nullptr, key_type, N, prm, nullptr, nullptr, d_splitters, d_offsets, d_work, work_bytes, h_stats,
                    (cudaStream_t)stream, false);
}

int hss_partition_with_proposal(const void* d_keys, int key_type, uint64_t N, const hss_params* prm,
                                const void* d_proposal, uint32_t nprop, hss_cut* d_splitters, uint64_t* d_offsets,
                                void* d_work, size_t work_bytes, hss_stats* h_stats, void* stream) {
    if (nprop > 0 && !d_proposal) return HSS_ERR_INVALID;
    return run_path(d_keys, nullptr, key_type, N, prm, nullptr, nullptr, d_splitters, d_offsets, d_work, work_bytes, h_stats,
                    (cudaStream_t)stream, false, d_proposal, nprop);
}

int hss_sort_with_proposal(const void* d_keys, const uint32_t* d_payload, int key_type, uint64_t N, const hss_params* prm,
                           const void* d_proposal, uint32_t nprop, void* d_keys_out, uint32_t* d_payload_out,
                           hss_cut* d_splitters, uint64_t* d_offsets, void* d_work, size_t work_bytes, hss_stats* h_stats,
                           void* stream) {
    if (nprop > 0 && !d_proposal) return HSS_ERR_INVALID;
    return run_path(d_keys, d_payload, key_type, N, prm, d_keys_out, d_payload_out, d_splitters, d_offsets, d_work,
                    work_bytes, h_stats, (cudaStream_t)stream, true, d_proposal, nprop);
}

int hss_exchange(const void* d_sorted_keys, const uint32_t* d_sorted_payload, uint64_t N, uint32_t p,
                 const uint32_t* d_seg_pos, const uint64_t* d_offsets, void* d_bucket_keys, uint32_t* d_bucket_payload,
                 void* d_work, size_t work_bytes, void* stream) {
    if (p == 0 || p > kMaxP || N >= kMaxN || !segments_fit(N, p) || !d_offsets || !d_work) return HSS_ERR_INVALID;
    if (N > 0 && (!d_sorted_keys || !d_bucket_keys || (p > 1 && !d_seg_pos))) return HSS_ERR_INVALID;
    if ((d_sorted_payload == nullptr) != (d_bucket_payload == nullptr)) return HSS_ERR_INVALID;
    const Layout L = plan(HSS_OP_EXCHANGE, N, p, 5.0f, d_sorted_payload != nullptr);
    if (work_bytes < L.total) return HSS_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t* err = at<uint32_t>(d_work, L.err);
    uint64_t* seg_off = at<uint64_t>(d_work, L.seg_off);
    if (cudaMemsetAsync(err, 0, 256, st) != cudaSuccess) return HSS_ERR_CUDA;
    if (fill_even_offsets(seg_off, N, p, st) != cudaSuccess) return HSS_ERR_CUDA;
    if (p == 1) {
        if (N > 0 && cudaMemcpyAsync(d_bucket_keys, d_sorted_keys, N * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return HSS_ERR_CUDA;
        if (N > 0 && d_sorted_payload &&
            cudaMemcpyAsync(d_bucket_payload, d_sorted_payload, N * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return HSS_ERR_CUDA;
        return HSS_OK;
    }
    if (exchange((const uint64_t*)d_sorted_keys, d_sorted_payload, N, p, seg_off, d_seg_pos, d_offsets,
                 (uint64_t*)d_bucket_keys, d_bucket_payload, at<uint64_t>(d_work, L.dst), err, st) != cudaSuccess)
        return HSS_ERR_CUDA;
    return read_dev_err(err, st);
}

int hss_merge(const void* d_bucket_keys, const uint32_t* d_bucket_payload, int key_type, uint64_t N, uint32_t p,
              const uint64_t* d_offsets, void* d_keys_out, uint32_t* d_payload_out, void* d_work, size_t work_bytes,
              void* stream) {
    if ((key_type != HSS_KEY_U64 && key_type != HSS_KEY_I64) || p == 0 || p > kMaxP || N >= kMaxN) return HSS_ERR_INVALID;
    if (!d_offsets || !d_work || (N > 0 && (!d_bucket_keys || !d_keys_out))) return HSS_ERR_INVALID;
    if ((d_bucket_payload == nullptr) != (d_payload_out == nullptr)) return HSS_ERR_INVALID;
    const bool pay = d_bucket_payload != nullptr;
    const Layout L = plan(HSS_OP_MERGE, N, p, 5.0f, pay);
    if (work_bytes < L.total) return HSS_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t* err = at<uint32_t>(d_work, L.err);
    SegSortWs sws = segsort_ws_carve(at<void>(d_work, L.sws), std::max<uint64_t>(N, 1), p, err);
    if (cudaMemsetAsync(err, 0, 256, st) != cudaSuccess) return HSS_ERR_CUDA;
    const bool i64 = key_type == HSS_KEY_I64;
    if (segsort((const uint64_t*)d_bucket_keys, (uint64_t*)d_keys_out, at<uint64_t>(d_work, L.keysB), d_bucket_payload,
                d_payload_out, pay ? at<uint32_t>(d_work, L.payB) : nullptr, N, p, d_offsets, i64, i64, sws, st,
                nullptr) != cudaSuccess)
        return HSS_ERR_CUDA;
    return read_dev_err(err, st);
}

int hss_sort(const void* d_keys, const uint32_t* d_payload, int key_type, uint64_t N, const hss_params* prm,
             void* d_keys_out, uint32_t* d_payload_out, hss_cut* d_splitters, uint64_t* d_offsets, void* d_work,
             size_t work_bytes, hss_stats* h_stats, void* stream) {
    return run_path(d_keys, d_payload, key_type, N, prm, d_keys_out, d_payload_out, d_splitters, d_offsets, d_work,
                    work_bytes, h_stats, (cudaStream_t)stream, true);
}

int hss_sort_host(const void* h_keys, const uint32_t* h_payload, int key_type, uint64_t N, const hss_params* prm,
                  void* h_keys_out, uint32_t* h_payload_out, hss_cut* h_splitters, uint64_t* h_offsets, void* d_work,
                  size_t work_bytes, hss_stats* h_stats, void* stream) {
    if (!params_ok(prm) || !d_work || !h_offsets || (N > 0 && (!h_keys || !h_keys_out))) return HSS_ERR_INVALID;
    if ((h_payload == nullptr) != (h_payload_out == nullptr)) return HSS_ERR_INVALID;
    const uint32_t p = prm->p;
    const bool pay = h_payload != nullptr;
    const Layout L = plan(HSS_OP_SORT_HOST, N, p, eff_oversample(prm), pay);
    if (work_bytes < L.total) return HSS_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    uint64_t* io = at<uint64_t>(d_work, L.io_keys);
    uint32_t* iop = pay ? at<uint32_t>(d_work, L.io_pay) : nullptr;
    hss_cut* spl = at<hss_cut>(d_work, L.io_spl);
    uint64_t* off = at<uint64_t>(d_work, L.io_off);
    HostIO hio{};
    cudaEvent_t* ev = nullptr;
    int dev = 0;
    if (io_resources(&hio.cs, &ev, &dev) != HSS_OK) return HSS_ERR_CUDA;
    std::lock_guard<std::mutex> call_lock(g_io_call_mu[dev]);
    for (int i = 0; i < 2 * 64; ++i) hio.ev[i] = ev[i];
    hio.h_keys = h_keys;
    hio.h_payload = h_payload;
    hio.h_keys_out = h_keys_out;
    hio.h_payload_out = h_payload_out;
    hio.h_offsets = h_offsets;
    // chunks of at least 16 Mi keys, at most 32 and one per processor
    hio.groups = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>({32, (uint64_t)p, N >> 24}));
    // the copy stream starts after the work already on the caller's stream
    if (cudaEventRecord(hio.ev[127], st) != cudaSuccess || cudaStreamWaitEvent(hio.cs, hio.ev[127], 0) != cudaSuccess)
        return HSS_ERR_CUDA;
    // run with the SORT layout inside the same workspace (it is a prefix of SORT_HOST's)
    int rc = run_path(io, iop, key_type, N, prm, io, iop, spl, off, d_work, work_bytes, h_stats, st, true, nullptr, 0,
                      &hio);
    if (rc == HSS_ERR_CUDA || rc == HSS_ERR_INVALID || rc == HSS_ERR_WORKSPACE) {
        cudaStreamSynchronize(hio.cs);
        return rc;
    }
    if (p == 1) {  // no merge: the locally sorted keys are the output
        if (N > 0 && cudaMemcpyAsync(h_keys_out, io, N * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) return HSS_ERR_CUDA;
        if (pay && N > 0 && cudaMemcpyAsync(h_payload_out, iop, N * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return HSS_ERR_CUDA;
        if (cudaMemcpyAsync(h_offsets, off, (uint64_t)(p + 1) * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return HSS_ERR_CUDA;
    }
    if (p > 1 && h_splitters &&
        cudaMemcpyAsync(h_splitters, spl, (uint64_t)(p - 1) * sizeof(hss_cut), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return HSS_ERR_CUDA;
    if (cudaStreamSynchronize(hio.cs) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return HSS_ERR_CUDA;
    return rc;
}

int hss_call_stats(int op, uint64_t N, const hss_params* prm, int key_type, int has_payload, const void* d_work,
                   size_t work_bytes, hss_stats* h_stats, void* stream) {
    if (!params_ok(prm) || !d_work || !h_stats || (op != HSS_OP_SORT && op != HSS_OP_PARTITION)) return HSS_ERR_INVALID;
    (void)key_type;
    const uint32_t p = prm->p;
    const Layout L = plan(op, N, p, eff_oversample(prm), op == HSS_OP_SORT && has_payload != 0);
    if (work_bytes < L.total) return HSS_ERR_WORKSPACE;
    std::memset(h_stats, 0, sizeof(*h_stats));
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t* err = at<uint32_t>((void*)d_work, L.err);
    const uint64_t cap = sample_capacity(N, p, eff_oversample(prm));
    RoundWs rws = rounds_ws_carve(at<void>((void*)d_work, L.rws), std::max<uint64_t>(N, 1), p, cap, err);
    RoundResult rr;
    int status = p > 1 ? read_round_result(rws, &rr, st) : HSS_OK;
    const int e = read_dev_err(err, st);
    if (e != HSS_OK && status == HSS_OK) status = e;
    h_stats->rounds = rr.rounds;
    h_stats->status = status;
    h_stats->tol = (uint64_t)std::floor(((double)N * prm->eps) / (2.0 * (double)p));
    for (uint32_t j = 0; j < rr.rounds && j < HSS_MAX_ROUNDS; ++j) {
        h_stats->sample_size[j] = rr.sample_size[j];
        h_stats->gamma[j] = rr.gamma[j];
    }
    for (uint32_t j = 0; j <= rr.rounds && j <= HSS_MAX_ROUNDS; ++j) h_stats->unresolved[j] = rr.unresolved[j];
    return status;
}

int hss_sample_words(uint64_t seed, uint32_t seg, uint32_t round, uint32_t spos0, uint32_t count, uint64_t* d_out,
                     void* stream) {
    if (count > 0 && !d_out) return HSS_ERR_INVALID;
    if ((uint64_t)spos0 + count > (1ull << 32)) return HSS_ERR_INVALID;
    if (sample_words_launch(seed, seg, round, spos0, count, d_out, (cudaStream_t)stream) != cudaSuccess) return HSS_ERR_CUDA;
    return HSS_OK;
}

int hss_set_tuning(const hss_tuning* t) { return set_tuning(t); }

int hss_get_tuning(hss_tuning* t) {
    if (!t) return HSS_ERR_INVALID;
    get_tuning(t);
    return HSS_OK;
}

uint64_t hss_kernel_launch_count(void) { return g_launches.load(); }

const char* hss_strerror(int code) {
    switch (code) {
    case HSS_OK: return "ok";
    case HSS_ERR_INVALID: return "invalid argument";
    case HSS_ERR_WORKSPACE: return "workspace too small";
    case HSS_ERR_ROUND_LIMIT: return "round limit reached with unresolved splitters";
    case HSS_ERR_TIMEOUT: return "a bounded device-side wait timed out";
    case HSS_ERR_CUDA: return "CUDA runtime error";
    case HSS_ERR_CAPACITY: return "a round drew more probes than the sample buffer holds";
    case HSS_ERR_NOALLOC_LIMIT: return "input exceeds the fixed scratch of hss_local_sort_noalloc (N <= 524288, 16 MiB)";
    default: return "unknown error";
    }
}

}  // extern "C"
