// hss_internal.cuh -- device helpers shared by the kernels of libhss.so.
#pragma once

#include <cstdint>
#include <cstddef>
#include <cuda_runtime.h>
#include <cuda/atomic>

#include "hss.h"

namespace hss {

typedef unsigned long long ull;

constexpr uint64_t kSignBit = 0x8000000000000000ull;

// Device error bits (OR-ed into a status word in the workspace).
constexpr uint32_t kDevErrTimeout = 1u;
constexpr uint32_t kDevErrBounds = 2u;
constexpr uint32_t kDevErrSize = 4u;  // a segment of 2^30 keys or more (reported as HSS_ERR_INVALID)
constexpr uint64_t kMaxSegKeys = 1ull << 30;

// No kernel of the library waits on another CTA or kernel (the split pass
// takes its tile offsets from a scan, not a look-back), so kDevErrTimeout is
// set by none today; the status it maps to stays part of the ABI.

// Cut kinds, ordered so that comparison by (kind class, key, seg, spos) is the
// tag order of Sec. 6.1.
constexpr int kNegInf = 0;
constexpr int kMember = 1;
constexpr int kNonMember = 2;
constexpr int kPosInf = 3;

// A cut kept on the device during the rounds: order-preserving key bits,
// processor, position, kind, rank.
struct DCut {
    uint64_t okey;
    int32_t seg;   // -1 for a non-member cut
    uint32_t spos;
    uint64_t rank;
    int32_t kind;
    int32_t pad;
};

// Tag comparison a < b (Sec. 6.1 implicit tagging, extended by sentinels and
// non-member cuts).  Non-member cuts carry seg = -1 so they sort first among
// equal keys.
__host__ __device__ inline bool cut_less(const DCut& a, const DCut& b) {
    if (a.kind == kNegInf) return b.kind != kNegInf;
    if (b.kind == kNegInf) return false;
    if (b.kind == kPosInf) return a.kind != kPosInf;
    if (a.kind == kPosInf) return false;
    if (a.okey != b.okey) return a.okey < b.okey;
    if (a.seg != b.seg) return a.seg < b.seg;
    return a.spos < b.spos;
}

__host__ __device__ inline bool cut_equal(const DCut& a, const DCut& b) {
    return !cut_less(a, b) && !cut_less(b, a);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplies whose high halves are mixed into the other two words with the
// round key; the key advances by the golden-ratio Weyl increments.
// ---------------------------------------------------------------------------
struct Philox4 {
    uint32_t v[4];
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                  uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = M0 * c0, hi0 = __umulhi(M0, c0);
        const uint32_t lo1 = M1 * c2, hi1 = __umulhi(M1, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += W0; k1 += W1;
    }
    Philox4 o;
    o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
    return o;
}

// The two 64-bit sampling words of the position pair (2m, 2m+1) of segment
// `seg` in round `round`: counter (m, seg, round, 0), key = seed halves.
__device__ __forceinline__ void sample_words(uint64_t seed, uint32_t seg, uint32_t round, uint32_t m,
                                             uint64_t& even, uint64_t& odd) {
    const Philox4 x = philox4x32_10(m, seg, round, 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
    even = ((uint64_t)x.v[1] << 32) | x.v[0];
    odd = ((uint64_t)x.v[3] << 32) | x.v[2];
}

// ---------------------------------------------------------------------------
// Relaxed device-scope atomics for the decoupled look-back status words.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_relaxed(uint32_t* p) {
    cuda::atomic_ref<uint32_t, cuda::thread_scope_device> r(*p);
    return r.load(cuda::memory_order_relaxed);
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    cuda::atomic_ref<uint32_t, cuda::thread_scope_device> r(*p);
    r.store(v, cuda::memory_order_relaxed);
}

// Launch accounting: every kernel launch of the library goes through this.
void note_launch();
uint32_t launches_since(uint64_t mark);
// Kernels that ran inside a graph (counted when their number is known).
void add_launches(uint64_t n);
// While one is alive, launches on this thread are being captured into a
// graph: they are counted apart (captured()), not as launches.
struct LaunchCountPause {
    LaunchCountPause();
    ~LaunchCountPause();
    uint64_t captured() const;
};

// Kernel attributes are per device: set the dynamic shared-memory limit (and,
// when carveout >= 0, the preferred shared-memory carveout) of `func` once per
// device, thread-safely.  Returns the first failing CUDA error.
cudaError_t ensure_func_attrs(const void* func, int max_dyn_smem, int carveout = -1);
// Streaming multiprocessors of the current device (cached per device).
int device_sm_count();
// CTAs of `func` resident per SM at this block size and dynamic shared
// memory (the occupancy calculator, cached per device; at least 1).  Call
// after ensure_func_attrs so that the shared-memory settings count.
int resident_ctas(const void* func, int threads, size_t dyn_smem);
// Timing events of a call (HSS_FLAG_TIMING), destroyed on every way out of it.
template <int K>
struct TimingEvents {
    cudaEvent_t ev[K] = {};
    bool on = false;
    void create() {
        on = true;
        for (auto& e : ev) cudaEventCreate(&e);
    }
    ~TimingEvents() {
        if (on)
            for (auto& e : ev)
                if (e) cudaEventDestroy(e);
    }
};

// Read `bytes` (a multiple of 4, d_src 4-byte aligned) of device memory that
// the host needs for a decision (round state, status words), after the work
// queued on `st`; synchronises `st`.  Up to 8 KiB go through this thread's
// mapped pinned buffer, written by a copy kernel: no copy engine is involved,
// so the read never waits behind bulk copies queued on other streams.  Larger
// reads (or no pinned buffer) take cudaMemcpyAsync.
cudaError_t read_small(void* h_dst, const void* d_src, size_t bytes, cudaStream_t st);

}  // namespace hss

#define HSS_LAUNCH(kernel, grid, block, smem, stream, ...)                 \
    do {                                                                   \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);        \
        ::hss::note_launch();                                              \
    } while (0)
