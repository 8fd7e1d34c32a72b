// segsort.cuh -- stable segmented radix sort of 64-bit keys (+ u32 payload).
//
// Segments are given by a device array seg_off[nseg+1] of u64 offsets.  A
// segment of at most kSmallCap keys is sorted by one CTA entirely on chip.  A
// larger segment is split by one most-significant-digit pass (per-tile digit
// counts, a scan into per-tile offsets, then a scatter of every tile) on its top
// varying 8-bit window into 256 sub-buckets, which are sorted the same way,
// recursively; a segment whose keys are all equal is copied straight to the
// output.
#pragma once

#include "hss_internal.cuh"

namespace hss {

constexpr int kRadixBits = 8;
constexpr int kRadix = 256;
// Levels of the split recursion: byte splits need at most 8 (one per byte of
// the key) and one more to copy single-valued sub-buckets; interpolated splits
// of sub-buckets choose their width to finish within the limit.
constexpr int kMaxDepth = 16;

constexpr int kOsThreads = 256;
constexpr int kOsWarps = kOsThreads / 32;
constexpr int kOsItems = 16;
constexpr int kOsTile = kOsThreads * kOsItems;  // 4096 keys per split tile

// On-chip sort: three CTA shapes by segment size (threads x items per thread).
constexpr int kC0Threads = 128, kC0Items = 12;  // up to 1536 keys
constexpr int kC1Threads = 256, kC1Items = 16;  // up to 4096 keys
constexpr int kC2Threads = 512, kC2Items = 28;  // up to 14336 keys
constexpr int kC0Cap = kC0Threads * kC0Items;
constexpr int kC1Cap = kC1Threads * kC1Items;
constexpr int kSmallCap = kC2Threads * kC2Items;
constexpr int kTinyGroup = 64;  // on chip: rank inside the groups of one MSD pass when none is larger

struct SegSortWs {
    uint64_t max_large;    // bound on segments larger than kSmallCap at any depth
    uint64_t max_list;     // bound on the length of any segment list
    uint64_t max_tiles;
    uint32_t* tile_start;  // [max_list + 1]
    uint32_t* tile_seg;    // [max_tiles] segment of every tile of this level's large segments
    uint32_t* large_id;    // [max_list]
    uint32_t* large_seg;   // [max_large]
    uint16_t* tile_hist;   // [max_tiles][2][256] digit counts of every tile: the speculative window, then a recount
    uint8_t* tile_skew;    // [max_tiles] one digit holds more than an eighth of the tile
    uint64_t max_spl;      // segments of the first level that can take sampled splitters
    uint64_t* spl_tab;     // [max_spl][256] sampled splitters of each first-level segment split
    uint8_t* spl_mode;     // [max_spl] 1: that segment's first split uses them
    unsigned long long* vor;   // [max_large] OR of the keys
    unsigned long long* vand;  // [max_large] AND of the keys
    uint32_t* msd_shift[2];  // [max_large] split window (bits) of each large segment, by level parity
    uint32_t* spec;        // [max_large] byte counted speculatively by the statistics pass
    uint64_t* msd_base;    // [max_large] digit = ((key >> shift) - base) & 255, or
    uint64_t* msd_mult;    // [max_large] when mult != 0: digit = mulhi(key - base, mult)
    uint32_t* direct;      // [max_large] all keys equal: copy to the output
    uint64_t* sub_lo[2];   // [max_large * 256] sub-bucket bounds, double-buffered by depth
    uint64_t* sub_hi[2];
    // Sub-buckets that will be split again: their smallest and largest key
    // (gathered by the split pass) and the interpolating digit of their own
    // split, double-buffered by depth like the bounds.
    uint64_t* cmin[2];     // [max_large * 256]
    uint64_t* cmax[2];
    uint64_t* cmult[2];
    uint32_t* large_mask;  // [max_large * 8] sub-buckets above the on-chip limit, one bit per digit
    uint32_t* any_large;   // [max_large]
    uint32_t* tile_off;    // [max_tiles][256] destination of each tile's digit-d keys, relative to its segment
    uint32_t* counters;    // [64]
    uint32_t* list[3];     // [max_list] segments of each on-chip size class
    uint32_t* fb_list;     // [max_list] segments left to the stable LSD kernel (count in counters[24])
    uint32_t* slow_list;   // [max_list] segments the register kernel leaves to the shared-memory kernel (counters[25])
    uint32_t* slow_keys[3];  // [max_list] per size class: segments the keys-only kernel leaves (counters[26..28])
    uint32_t* blk;         // [8 * (max_list / 1024 + 2)] per-chunk counts of the planning scan
    uint32_t* err;         // device error word (kDevErr*)
    // false: the planning counts come back by a copy into pageable host
    // memory (nothing allocated: hss_local_sort_noalloc); true: a kernel
    // writes them into this thread's mapped pinned buffer, which needs no copy
    // engine (a count read then never waits behind the caller's bulk copies).
    bool mapped_counts = true;
};

// Bytes of scratch a segmented sort of N keys in nseg segments needs.
size_t segsort_ws_bytes(uint64_t N, uint64_t nseg);
// Carve the scratch out of `base`.
SegSortWs segsort_ws_carve(void* base, uint64_t N, uint64_t nseg, uint32_t* err);

struct SegSortTiming {
    bool enabled = false;
    int n = 0;                      // recorded (start, end) pairs around MSD passes
    cudaEvent_t ev[16][2] = {};
    uint64_t keys[16] = {};         // keys moved by each recorded pass
    // Sum the recorded pass times (call after the stream has passed the last
    // recorded event) and release the events.
    void collect(float* ms_total, uint32_t* n_launches, uint64_t* n_keys) {
        float tot = 0.f;
        uint64_t nk = 0;
        for (int i = 0; i < n; ++i) {
            float ms = 0.f;
            cudaEventSynchronize(ev[i][1]);
            cudaEventElapsedTime(&ms, ev[i][0], ev[i][1]);
            tot += ms;
            nk += keys[i];
            cudaEventDestroy(ev[i][0]);
            cudaEventDestroy(ev[i][1]);
        }
        if (ms_total) *ms_total = tot;
        if (n_launches) *n_launches = (uint32_t)n;
        if (n_keys) *n_keys = nk;
        n = 0;
    }
};

// Stable sort of every segment [seg_off[s], seg_off[s+1]) of src into dst.
// tmp (and ptmp) must not alias src/dst; dst may alias src.  flip_in XORs the
// sign bit into keys as they are read (signed keys), flip_out as they are
// written.  psrc/pdst/ptmp are all null or all non-null.  hint_lo and
// hint_mult (both null or both per segment) promise that every key k of
// segment s satisfies hint_lo[s] <= k and mulhi(k - hint_lo[s], hint_mult[s])
// <= 255; the first split of s then uses that value, which is monotone in k,
// as its digit (an interpolation of the key range over 256 sub-buckets).
cudaError_t segsort(const uint64_t* src, uint64_t* dst, uint64_t* tmp,
                    const uint32_t* psrc, uint32_t* pdst, uint32_t* ptmp,
                    uint64_t N, uint64_t nseg, const uint64_t* d_seg_off,
                    bool flip_in, bool flip_out, const SegSortWs& ws, cudaStream_t st,
                    SegSortTiming* timing, const uint64_t* hint_lo = nullptr,
                    const uint64_t* hint_mult = nullptr);

// Process-wide tuning of the sort (hss_set_tuning / hss_get_tuning).
int set_tuning(const hss_tuning* t);
void get_tuning(hss_tuning* t);

// seg_off[s] = floor(s * N / p) for s = 0..p.
cudaError_t fill_even_offsets(uint64_t* d_seg_off, uint64_t N, uint64_t p, cudaStream_t st);

}  // namespace hss
