// segsort.cuh -- stable segmented LSD radix sort of 64-bit keys (+ u32 payload).
//
// Segments are given by a device array seg_off[nseg+1] of u64 offsets.  A
// segment that fits in shared memory (<= kSmallCap keys) is sorted by one CTA
// entirely on chip; larger segments go through eight 8-bit digit passes of a
// one-sweep radix sort whose tiles chain their digit prefixes per segment by
// decoupled look-back.
#pragma once

#include "hss_internal.cuh"

namespace hss {

constexpr int kRadixBits = 8;
constexpr int kRadix = 256;
constexpr int kPasses = 8;

constexpr int kOsThreads = 256;
constexpr int kOsWarps = kOsThreads / 32;
constexpr int kOsItems = 16;
constexpr int kOsTile = kOsThreads * kOsItems;  // 4096 keys per tile

constexpr int kSmThreads = 512;
constexpr int kSmWarps = kSmThreads / 32;
constexpr int kSmItems = 32;
constexpr int kSmallCap = kSmThreads * kSmItems;  // 16384 keys per on-chip segment

struct SegSortWs {
    uint32_t* digit_off;   // [nseg][8][256] digit counts, then exclusive offsets
    uint32_t* tile_start;  // [nseg + 1] first tile of each large segment
    uint32_t* status;      // [2][max_tiles][256] look-back words
    uint32_t* counters;    // [kPasses] dynamic tile counters
    uint32_t* err;         // device error word (kDevErr*)
    uint64_t max_tiles;
};

// Bytes of scratch a segmented sort of N keys in nseg segments needs.
size_t segsort_ws_bytes(uint64_t N, uint64_t nseg);
// Carve the scratch out of `base`.
SegSortWs segsort_ws_carve(void* base, uint64_t N, uint64_t nseg, uint32_t* err);

struct SegSortTiming {
    bool enabled = false;
    int n = 0;                      // recorded (start, end) pairs around digit-pass groups
    cudaEvent_t ev[8][2] = {};
    uint32_t launches[8] = {};
    // Sum the recorded pass times (call after the stream has passed the last
    // recorded event) and release the events.
    void collect(float* ms_total, uint32_t* n_launches) {
        float tot = 0.f;
        uint32_t nl = 0;
        for (int i = 0; i < n; ++i) {
            float ms = 0.f;
            cudaEventSynchronize(ev[i][1]);
            cudaEventElapsedTime(&ms, ev[i][0], ev[i][1]);
            tot += ms;
            nl += launches[i];
            cudaEventDestroy(ev[i][0]);
            cudaEventDestroy(ev[i][1]);
        }
        n = 0;
        if (ms_total) *ms_total = tot;
        if (n_launches) *n_launches = nl;
    }
};

// Stable sort of every segment [seg_off[s], seg_off[s+1]) of src into dst.
// tmp (and ptmp) must not alias src/dst; dst may alias src.  flip_in XORs the
// sign bit into keys as they are read (signed keys), flip_out as they are
// written.  psrc/pdst/ptmp are all null or all non-null.
cudaError_t segsort(const uint64_t* src, uint64_t* dst, uint64_t* tmp,
                    const uint32_t* psrc, uint32_t* pdst, uint32_t* ptmp,
                    uint64_t N, uint64_t nseg, const uint64_t* d_seg_off,
                    bool flip_in, bool flip_out, const SegSortWs& ws, cudaStream_t st,
                    SegSortTiming* timing);

// seg_off[s] = floor(s * N / p) for s = 0..p.
cudaError_t fill_even_offsets(uint64_t* d_seg_off, uint64_t N, uint64_t p, cudaStream_t st);

}  // namespace hss
