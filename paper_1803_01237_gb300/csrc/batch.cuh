// batch.cuh -- the batched sort as a building block of other entry points.
#pragma once

#include "hss_internal.cuh"

namespace hss {

// Options of a batched call made from inside the library.
struct BatchExtra {
    // The keys are already order-preserving bits (a signed key type then
    // only decides how splitters and output are written back).
    bool keys_ordered = false;
    // Per segment of the batch (all jobs' segments in order; both null or
    // both set): the interpolation window of the local sort's first split,
    // as for segsort().
    const uint64_t* hint_lo = nullptr;
    const uint64_t* hint_mult = nullptr;
    // Host array of each job's Philox key (null: prm->seed + j).
    const uint64_t* seeds = nullptr;
};

// hss_sort_batch (sort) / hss_partition_batch (!sort) with options.
int run_batch(const void* d_keys, const uint32_t* d_payload, int key_type, const uint64_t* h_sizes, const uint32_t* h_p,
              uint32_t njobs, const hss_params* prm, void* d_keys_out, uint32_t* d_payload_out, hss_cut* d_splitters,
              uint64_t* d_offsets, void* d_work, size_t work_bytes, hss_batch_stats* h_stats,
              hss_job_stats* h_job_stats, cudaStream_t st, bool sort, const BatchExtra& ex);

// Workspace bytes of a batched sort of njobs jobs of p_j = pj processors
// each, N keys in all, whatever the split of N among the jobs (0 when some
// split would be refused: a job below pj keys aside, the per-job limits).
size_t batch_bytes_bound(uint64_t N, uint32_t njobs, uint32_t pj, const hss_params* prm, bool pay);

}  // namespace hss
