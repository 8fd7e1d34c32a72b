// noalloc.cu -- the local sort for callers that cannot allocate device memory.
//
// hss_local_sort_noalloc runs the same segmented radix sort as hss_local_sort,
// but takes its scratch (the ping-pong key/payload buffers, the segment
// offsets, the digit offsets and the look-back words) from one fixed array
// that lives in the library's device image instead of from a caller
// workspace.  The array is kNoAllocScratchBytes per device and stays resident
// on every device that loads the library until the process exits.
#include "hss_internal.cuh"
#include "segsort.cuh"

#include <algorithm>

namespace hss {

constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;  // 16 MiB per device
constexpr uint64_t kNoAllocMaxKeys = (uint64_t)1 << 19;     // 524288 keys per call

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

// Device address of the scratch array on the current device.  The host-side
// symbol is only a stand-in: kernels must be given the address looked up here.
// It is looked up on every call (cheap next to the sort): a cached address
// would go stale if the caller reset the device and the library image were
// loaded again.
int scratch_on_current_device(void** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return HSS_ERR_CUDA;
    *out = p;
    return HSS_OK;
}

size_t aup256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace
}  // namespace hss

using namespace hss;

extern "C" int hss_local_sort_noalloc(const void* d_keys, const uint32_t* d_payload, int key_type, uint64_t N,
                                      uint32_t p, void* d_keys_out, uint32_t* d_payload_out, void* stream) {
    if ((key_type != HSS_KEY_U64 && key_type != HSS_KEY_I64) || p == 0) return HSS_ERR_INVALID;
    if (N > 0 && (!d_keys || !d_keys_out)) return HSS_ERR_INVALID;
    if ((d_payload == nullptr) != (d_payload_out == nullptr)) return HSS_ERR_INVALID;
    if (N > kNoAllocMaxKeys) return HSS_ERR_NOALLOC_LIMIT;
    cudaStream_t st = (cudaStream_t)stream;
    // The call ends with a stream synchronisation to read the kernels' status
    // word; on a stream that is capturing work that would end the caller's
    // capture, so such a stream is refused before anything is enqueued.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return HSS_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return HSS_ERR_INVALID;
    const bool pay = d_payload != nullptr;
    const uint64_t N1 = std::max<uint64_t>(N, 1);
    // Layout inside the fixed array: tmp keys, tmp payload, segment offsets,
    // error word, sort scratch.
    size_t off = 0;
    const size_t o_keys = off; off += aup256(N1 * 8);
    const size_t o_pay = off; off += pay ? aup256(N1 * 4) : 0;
    const size_t o_seg = off; off += aup256(((size_t)p + 1) * 8);
    const size_t o_err = off; off += 256;
    const size_t o_ws = off; off += segsort_ws_bytes(N1, p);
    if (off > kNoAllocScratchBytes) return HSS_ERR_NOALLOC_LIMIT;
    void* base = nullptr;
    const int rc = scratch_on_current_device(&base);
    if (rc != HSS_OK) return rc;
    char* b = (char*)base;
    uint32_t* err = (uint32_t*)(b + o_err);
    uint64_t* seg_off = (uint64_t*)(b + o_seg);
    // The array keeps the previous call's contents: zero the error word here;
    // the sort zeroes its own counters and look-back words before use.
    if (cudaMemsetAsync(err, 0, 256, st) != cudaSuccess) return HSS_ERR_CUDA;
    if (fill_even_offsets(seg_off, N, p, st) != cudaSuccess) return HSS_ERR_CUDA;
    SegSortWs ws = segsort_ws_carve(b + o_ws, N1, p, err);
    ws.mapped_counts = false;  // allocate nothing, not even the pinned count buffer
    const bool i64 = key_type == HSS_KEY_I64;
    if (segsort((const uint64_t*)d_keys, (uint64_t*)d_keys_out, (uint64_t*)(b + o_keys), d_payload, d_payload_out,
                pay ? (uint32_t*)(b + o_pay) : nullptr, N, p, seg_off, i64, i64, ws, st, nullptr) != cudaSuccess)
        return HSS_ERR_CUDA;
    uint32_t h = 0;
    if (cudaMemcpyAsync(&h, err, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return HSS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return HSS_ERR_CUDA;
    if (h & kDevErrTimeout) return HSS_ERR_TIMEOUT;
    if (h & kDevErrSize) return HSS_ERR_INVALID;
    if (h & kDevErrBounds) return HSS_ERR_CUDA;
    return HSS_OK;
}
