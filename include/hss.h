/*
 * hss.h -- C ABI of the GB300 Histogram Sort with Sampling library (libhss.so).
 *
 * The method is Histogram Sort with Sampling (HSS) of Harsh, Kale and
 * Solomonik (SPAA'19).  Its p "processors" are p contiguous segments of one
 * device array: processor s owns input positions [floor(sN/p), floor((s+1)N/p)).
 *
 * Conventions shared by every entry point
 *   - Every buffer belongs to the caller.  Pointers named d_* are device
 *     pointers on the current device, h_* are host pointers.  The library
 *     never allocates device memory: scratch comes from the caller's
 *     workspace (d_work, work_bytes), sized with hss_workspace_bytes().  The
 *     small reads the host needs (a level's counts, a round's state, status
 *     words) go through two mapped pinned host buffers per calling thread,
 *     allocated at its first call (so they never wait behind bulk copies on
 *     the copy engine); hss_local_sort_noalloc uses neither.
 *   - Work is enqueued on `stream` (a cudaStream_t passed as void*, NULL =
 *     the legacy default stream).  The splitter rounds of a repeated shape
 *     run on the device (a CUDA graph loop, see HSS_FLAG_DEVICE_ROUNDS), so
 *     hss_partition returns without waiting for the GPU unless statistics
 *     are asked for (h_stats non-NULL) or HSS_FLAG_SYNC / HSS_FLAG_TIMING is
 *     set; hss_call_stats reads them later.  The local sort and the merge
 *     wait where they plan a level of their radix recursion (one small read
 *     per level).  Rounds driven from the host (a shape's first call, large
 *     samples, the k-round schedule, HSS_FLAG_HOST_ROUNDS) read one small
 *     record per round.
 *   - Keys are 64-bit, unsigned (HSS_KEY_U64) or signed (HSS_KEY_I64).  An
 *     optional 32-bit payload travels with its key.
 *   - Ties between equal keys are broken by (processor, position), which is
 *     the (key, processor, index) implicit tagging of the paper's Sec. 6.1;
 *     every sort here is therefore stable with respect to input order.
 *   - Return value: HSS_OK (0) or a negative HSS_ERR_* code.  Device-side
 *     failures (an index check that failed, a segment too large) travel
 *     through a status word and are reported as an error code; nothing traps
 *     the GPU.  No kernel waits on another, so HSS_ERR_TIMEOUT is reserved.
 *   - Limits: N < 2^40; 1 <= p <= 2^22 and p*(samples per round) positions
 *     must fit the workspace; a segment or bucket holds fewer than 2^30 keys.
 *     Calls whose even segments (ceil(N/p)), or for the sorting calls whose
 *     eps-balanced buckets (ceil(N/p) + 2 floor(N eps/(2p))), could reach
 *     2^30 keys return HSS_ERR_INVALID before any device work; a caller's
 *     bucket of 2^30 keys or more given to hss_merge is reported as
 *     HSS_ERR_INVALID after the call's device work.
 */
#ifndef HSS_H
#define HSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HSS_OK 0
#define HSS_ERR_INVALID (-1)      /* bad argument: null pointer, p = 0, eps <= 0, sizes out of range */
#define HSS_ERR_WORKSPACE (-2)    /* work_bytes smaller than hss_workspace_bytes() */
#define HSS_ERR_ROUND_LIMIT (-3)  /* max_rounds reached with splitters unresolved */
#define HSS_ERR_TIMEOUT (-4)      /* reserved: a bounded device-side wait gave up (no kernel waits today) */
#define HSS_ERR_CUDA (-5)         /* a CUDA runtime call failed, or a device index check did */
#define HSS_ERR_CAPACITY (-6)     /* a round drew more probes than the sample buffer holds */
#define HSS_ERR_NOALLOC_LIMIT (-7) /* input larger than the fixed scratch of hss_local_sort_noalloc */

#define HSS_KEY_U64 0
#define HSS_KEY_I64 1

#define HSS_MAX_ROUNDS 64

/* params.flags */
#define HSS_FLAG_SYNC 1u     /* synchronize `stream` before returning */
#define HSS_FLAG_TIMING 2u   /* record per-phase device times into hss_stats (implies SYNC) */
/* Histogram form of the splitter rounds (Sec. 3.3 step 2; the result is the
 * same either way).  By default each round chooses: when all its probes
 * share one interval (round 1) and searching every segment for every probe
 * (Z p log2(N/p) dependent loads) would cost more than eight reads of the
 * keys, a staged form ranks blocks of sorted probes against the keys between
 * the block's first and last probe, staged in shared memory; else every
 * probe is searched in every segment.  These flags force one form (at most
 * one may be set, else HSS_ERR_INVALID). */
#define HSS_FLAG_HIST_PROBE 4u
#define HSS_FLAG_HIST_STAGED 8u
/* Drivers of the splitter rounds.  A call whose round sample fits one
 * on-chip sort (sample capacity min(N, ceil(2 s p) + 4096) <= 14336) and
 * whose schedule is not the k-round one can run its rounds as one CUDA
 * graph: a WHILE conditional node whose body is one round (sample, sort,
 * histogram, L/U update, intervals, next sample) and whose condition a device
 * kernel sets after each round (all resolved, round limit, sample capacity);
 * the graph is built once per shape (workspace, stream, N, p, eps, s, ...)
 * and cached.  By default a shape's first call drives its rounds from the
 * host (one small device-to-host read per round decides the next launch:
 * cheaper than building a graph used once) and later calls of the same
 * shape run the graph.  HSS_FLAG_HOST_ROUNDS always drives from the host,
 * HSS_FLAG_DEVICE_ROUNDS always runs the graph (built at the first call);
 * both together are HSS_ERR_INVALID.  The results are identical in every
 * case. */
#define HSS_FLAG_HOST_ROUNDS 16u
#define HSS_FLAG_DEVICE_ROUNDS 32u

/* Workspace queries (op argument of hss_workspace_bytes). */
#define HSS_OP_SORT 0
#define HSS_OP_PARTITION 1
#define HSS_OP_LOCAL_SORT 2
#define HSS_OP_MERGE 3
#define HSS_OP_EXCHANGE 4
#define HSS_OP_SORT_HOST 5

/* A cut in the tag order of Sec. 6.1: the key itself (caller's
 * representation), the processor it lies on and its position in that
 * processor's locally sorted keys.  Special values of seg:
 *   -1  a non-member cut: sorts before every key equal to `key`;
 *   -2  minus infinity;  -3  plus infinity. */
typedef struct {
    uint64_t key;
    int32_t seg;
    uint32_t spos;
} hss_cut;

typedef struct {
    double eps;          /* balance: bucket i's start rank lies within floor(N eps/(2p)) of floor(iN/p) (Sec. 2) */
    uint64_t seed;       /* Philox key of the Bernoulli sampling */
    uint32_t p;          /* number of processors = buckets */
    float oversample;    /* s: expected probes per processor per round (default 5, Sec. 7.2) */
    uint32_t max_rounds; /* <= HSS_MAX_ROUNDS (0 means HSS_MAX_ROUNDS) */
    uint32_t flags;      /* HSS_FLAG_* */
    uint32_t schedule;   /* HSS_SCHEDULE_*: how a round's sampling probability is chosen */
    uint32_t schedule_k; /* HSS_SCHEDULE_THEORY: the number of rounds k (>= 1) */
} hss_params;

/* Sampling schedules (single calls; the batch entry points take only the
 * proportional one):
 *   PROPORTIONAL  every key of the unresolved region with probability
 *                 min(1, s p / |gamma|) (Sec. 6: s p probes per round);
 *   THEORY        round j draws every key of the region with probability
 *                 min(1, p s_j / N), s_j = (2 ln p / eps)^(min(j,k)/k)
 *                 (Sec. 4.2.2, Theorem 4.7), computed on the host in IEEE
 *                 double with the C library's log and pow;
 *   EQUAL         every distinct unresolved interval gets s p / nint expected
 *                 probes (probability min(1, (s p / nint) / its length)), the
 *                 HykSort sampling the paper contrasts with (Sec. 4.2.2). */
#define HSS_SCHEDULE_PROPORTIONAL 0
#define HSS_SCHEDULE_THEORY 1
#define HSS_SCHEDULE_EQUAL 2

#define HSS_PHASE_LOCAL_SORT 0
#define HSS_PHASE_ROUNDS 1
#define HSS_PHASE_EXCHANGE 2
#define HSS_PHASE_MERGE 3
#define HSS_NUM_PHASES 4

typedef struct {
    uint32_t rounds;                         /* histogram rounds run */
    int32_t status;                          /* same code as the return value */
    uint64_t tol;                            /* floor(N eps / (2p)) */
    uint64_t sample_size[HSS_MAX_ROUNDS];    /* Z_j: probes drawn in round j+1 */
    uint64_t gamma[HSS_MAX_ROUNDS];          /* |gamma|: keys inside unresolved intervals sampled in round j+1 */
    uint64_t unresolved[HSS_MAX_ROUNDS + 1]; /* unresolved splitters before round 1 .. after the last round */
    float ms_phase[HSS_NUM_PHASES];          /* device time per phase (HSS_FLAG_TIMING) */
    float ms_radix_pass_total;               /* summed device time of the radix digit-pass kernels (HSS_FLAG_TIMING) */
    uint32_t radix_pass_launches;            /* number of those launches */
    uint64_t radix_pass_keys;                /* keys moved by those launches, summed */
    uint32_t kernel_launches;                /* kernels this call launched */
} hss_stats;

/* Bytes of device workspace needed by operation `op` (HSS_OP_*) for N keys.
 * prm may be NULL for HSS_OP_LOCAL_SORT, HSS_OP_MERGE and HSS_OP_EXCHANGE
 * except that p is then taken from `p_if_no_params`. */
size_t hss_workspace_bytes(int op, uint64_t N, const hss_params* prm, uint32_t p_if_no_params,
                           int key_type, int has_payload);

/* Local sort (paper Sec. 5 "local sorting", Sec. 6 phase 1): stably sort each
 * of the p contiguous segments of d_keys by key.  d_keys_out may equal d_keys.
 * d_payload / d_payload_out are both NULL or both non-NULL. */
int hss_local_sort(const void* d_keys, const uint32_t* d_payload, int key_type, uint64_t N, uint32_t p,
                   void* d_keys_out, uint32_t* d_payload_out, void* d_work, size_t work_bytes, void* stream);

/* Histogram of Sec. 3.3 step 2 / Sec. 4.2.2 step 2: for each of ncuts cuts,
 * its exact global rank (#keys strictly below it in tag order) over the p
 * locally sorted segments of d_sorted_keys (as produced by hss_local_sort).
 * Optionally also the per-segment counts, d_seg_pos[s * ncuts + k] (u32).
 * d_ranks: ncuts u64. */
int hss_rank_cuts(const void* d_sorted_keys, int key_type, uint64_t N, uint32_t p,
                  const hss_cut* d_cuts, uint32_t ncuts, uint64_t* d_ranks, uint32_t* d_seg_pos, void* stream);

/* Splitter determination (Sec. 4.2.2, with the Sec. 6 sampling of
 * probability s*p/|gamma|): local sort, then histogram rounds until every
 * splitter i has a probe whose rank is within floor(N eps/(2p)) of
 * floor(iN/p), then the closest probe becomes the splitter.
 * Outputs: d_splitters[p-1], d_offsets[p+1] (chi(0)=0 .. chi(p)=N; bucket b
 * holds ranks [chi(b), chi(b+1))).  The locally sorted keys stay at the start
 * of d_work.  h_stats (nullable) receives the round statistics. */
int hss_partition(const void* d_keys, int key_type, uint64_t N, const hss_params* prm,
                  hss_cut* d_splitters, uint64_t* d_offsets,
                  void* d_work, size_t work_bytes, hss_stats* h_stats, void* stream);

/* hss_partition with externally proposed splitters (a learned model of the
 * key distribution, or the splitters of an earlier call on similar data).
 * Each of the nprop keys of d_proposal (device, the caller's key type) is a
 * non-member cut: it sorts before every input key equal to it, and its rank
 * is the number of input keys strictly below it.  Before the first round the
 * cuts are histogrammed like probes (Sec. 4.2.2 step 2) and offered to every
 * splitter's L/U (step 3; equal ranks keep the smaller cut), so good proposals
 * resolve splitters without sampling while the rounds still decide balance:
 * the contract on d_offsets is that of hss_partition whatever the proposal.
 * A splitter may end on a proposed cut (seg = -1 in d_splitters).  The paper
 * proposes no such step; it is the hook of the learned proposal.  nprop may be
 * 0; it must not exceed the round sample capacity, min(N, ceil(2 s p) + 4096),
 * else HSS_ERR_INVALID.  Workspace as hss_partition. */
int hss_partition_with_proposal(const void* d_keys, int key_type, uint64_t N, const hss_params* prm,
                                const void* d_proposal, uint32_t nprop, hss_cut* d_splitters, uint64_t* d_offsets,
                                void* d_work, size_t work_bytes, hss_stats* h_stats, void* stream);

/* Data exchange (Sec. 3.1 step 3, Sec. 6 "data exchange"): move every run of
 * locally sorted keys to its bucket.  d_seg_pos[s*(p-1)+i] is the number of
 * keys of segment s below splitter i (hss_rank_cuts output for the p-1
 * splitters); d_offsets[p+1] as above.  Bucket b of d_bucket_keys holds the
 * runs of segments 0..p-1 in order. */
int hss_exchange(const void* d_sorted_keys, const uint32_t* d_sorted_payload, uint64_t N, uint32_t p,
                 const uint32_t* d_seg_pos, const uint64_t* d_offsets,
                 void* d_bucket_keys, uint32_t* d_bucket_payload, void* d_work, size_t work_bytes, void* stream);

/* Local merge (Sec. 5 "merges them", Sec. 6 "local merging"): stably merge the
 * sorted runs inside each bucket [d_offsets[b], d_offsets[b+1]) by key,
 * giving the globally sorted output. */
int hss_merge(const void* d_bucket_keys, const uint32_t* d_bucket_payload, int key_type, uint64_t N, uint32_t p,
              const uint64_t* d_offsets, void* d_keys_out, uint32_t* d_payload_out,
              void* d_work, size_t work_bytes, void* stream);

/* The whole method: local sort, splitter rounds, exchange, merge.  Writes the
 * globally sorted keys (and payload) with processor i owning
 * [d_offsets[i], d_offsets[i+1]).  d_keys_out may equal d_keys. */
int hss_sort(const void* d_keys, const uint32_t* d_payload, int key_type, uint64_t N, const hss_params* prm,
             void* d_keys_out, uint32_t* d_payload_out, hss_cut* d_splitters, uint64_t* d_offsets,
             void* d_work, size_t work_bytes, hss_stats* h_stats, void* stream);

/* hss_sort with proposed splitters: the rounds start from d_proposal[nprop]
 * exactly as in hss_partition_with_proposal; the rest as hss_sort.  Workspace
 * as hss_sort. */
int hss_sort_with_proposal(const void* d_keys, const uint32_t* d_payload, int key_type, uint64_t N,
                           const hss_params* prm, const void* d_proposal, uint32_t nprop, void* d_keys_out,
                           uint32_t* d_payload_out, hss_cut* d_splitters, uint64_t* d_offsets, void* d_work,
                           size_t work_bytes, hss_stats* h_stats, void* stream);

/* hss_sort from host buffers: copies the keys (and payload) to the
 * workspace, sorts, and copies the sorted keys, payload, splitters and
 * offsets back to host memory.  The copies run on a library stream in chunks
 * of whole processors (in) and whole buckets (out) so that they overlap the
 * local sort and the merge; pinned host memory gives full copy speed.
 * Synchronous; calls on one device are serialised (they share that stream).
 * Workspace: hss_workspace_bytes(HSS_OP_SORT_HOST, ...). */
int hss_sort_host(const void* h_keys, const uint32_t* h_payload, int key_type, uint64_t N, const hss_params* prm,
                  void* h_keys_out, uint32_t* h_payload_out, hss_cut* h_splitters, uint64_t* h_offsets,
                  void* d_work, size_t work_bytes, hss_stats* h_stats, void* stream);

/* Statistics and status of the last hss_partition / hss_sort (or their
 * _with_proposal forms; op = HSS_OP_PARTITION or HSS_OP_SORT) made on the
 * workspace d_work with these arguments: a call that returned without waiting
 * for the GPU leaves its round statistics and device-side status in the
 * workspace until the next call on it.  Synchronises `stream`; the return
 * value is that call's status (HSS_OK, HSS_ERR_ROUND_LIMIT, HSS_ERR_CAPACITY,
 * HSS_ERR_TIMEOUT, ...).  h_stats's device times are not filled. */
int hss_call_stats(int op, uint64_t N, const hss_params* prm, int key_type, int has_payload, const void* d_work,
                   size_t work_bytes, hss_stats* h_stats, void* stream);

/* The 64-bit Bernoulli words of the sampling phase (Sec. 4.2.1): for
 * positions spos0 .. spos0+count-1 of sorted segment `seg` in round `round`,
 * the Philox4x32-10 word each key is compared against.  d_out: count u64. */
int hss_sample_words(uint64_t seed, uint32_t seg, uint32_t round, uint32_t spos0, uint32_t count,
                     uint64_t* d_out, void* stream);

/* hss_local_sort for callers that may not allocate device memory at all:
 * code running inside a host framework that owns every device allocation
 * (a database or stream engine calling a user function, a plugin of a
 * serving runtime with a fixed memory budget), or a thread that must not
 * take the allocator's locks or synchronise the device the way cudaMalloc
 * and cudaFree can.  The paper has no counterpart; this is a library
 * service, not a step of the method.
 *
 * Same arguments and result as hss_local_sort without d_work/work_bytes: the
 * scratch is a fixed 16 MiB array inside the library's device image, resident
 * on every device that loads the library until the process exits.  Limits:
 * N <= 524288 keys, and the scratch the sort needs for (N, p) must fit those
 * 16 MiB (the call computes it); otherwise it returns HSS_ERR_NOALLOC_LIMIT
 * before any device work.  Every call looks up the array's device address
 * (cudaGetSymbolAddress) on the current device.  Every call, from any thread
 * or stream, uses the same array and leaves its contents behind, so calls
 * that can overlap on the GPU race with each other: serialise them.  The
 * call synchronises `stream` to read the kernels' status word; on a stream
 * that is capturing work it returns HSS_ERR_INVALID before enqueuing
 * anything.  It allocates nothing, neither through CUDA nor through any
 * other library. */
int hss_local_sort_noalloc(const void* d_keys, const uint32_t* d_payload, int key_type, uint64_t N, uint32_t p,
                           void* d_keys_out, uint32_t* d_payload_out, void* stream);

/* ---------------------------------------------------------------------------
 * Batches of independent jobs.
 *
 * Job j is the n_j = h_sizes[j] keys following job j-1 in d_keys (job 0
 * starts at 0), split over p_j = h_p[j] processors (1 <= p_j <= max(n_j, 1),
 * p_j <= 65536).  Each job gets exactly what hss_sort (hss_partition) would
 * compute for it alone with params prm and seed prm->seed + j; the jobs run
 * together: one segmented local sort over the segments of all jobs, rounds in
 * lock step (a job stops sampling once its splitters are resolved or it
 * fails), one exchange and one merge over all buckets.  A round costs one
 * 16-byte device-to-host read for the whole batch.
 *
 * Outputs, job-major: d_splitters[sum (p_j - 1)], d_offsets[sum (p_j + 1)]
 * (relative to the job's first key, chi(0) = 0 .. chi(p_j) = n_j), and for
 * hss_sort_batch the sorted keys (payload) of every job in its own range.
 * h_job_stats (host, nullable, njobs entries) receives each job's round
 * statistics.  The return value is the first failing job's code (or a
 * device error), HSS_OK when every job succeeded.  Synchronous.
 * ------------------------------------------------------------------------- */
typedef struct {
    uint32_t rounds;                          /* histogram rounds of this job */
    int32_t status;                           /* HSS_OK or the job's error */
    uint64_t tol;                             /* floor(n eps / (2p)) */
    uint64_t sample_size[HSS_MAX_ROUNDS];
    uint64_t gamma[HSS_MAX_ROUNDS];
    uint64_t unresolved[HSS_MAX_ROUNDS + 1];
} hss_job_stats;

typedef struct {
    uint32_t njobs;
    uint32_t max_rounds;       /* most rounds any job took */
    uint32_t lockstep_rounds;  /* rounds the batch ran */
    int32_t status;
    uint64_t total_samples;    /* probes drawn over all jobs and rounds */
    uint64_t total_keys;
    uint32_t total_segments;
    uint32_t kernel_launches;
    float ms_phase[HSS_NUM_PHASES];  /* with HSS_FLAG_TIMING */
} hss_batch_stats;

/* Workspace bytes of hss_sort_batch (sort = 1) or hss_partition_batch
 * (sort = 0); 0 for invalid job lists. */
size_t hss_batch_workspace_bytes(const uint64_t* h_sizes, const uint32_t* h_p, uint32_t njobs, const hss_params* prm,
                                 int key_type, int has_payload, int sort);

int hss_sort_batch(const void* d_keys, const uint32_t* d_payload, int key_type, const uint64_t* h_sizes,
                   const uint32_t* h_p, uint32_t njobs, const hss_params* prm, void* d_keys_out, uint32_t* d_payload_out,
                   hss_cut* d_splitters, uint64_t* d_offsets, void* d_work, size_t work_bytes, hss_batch_stats* h_stats,
                   hss_job_stats* h_job_stats, void* stream);

int hss_partition_batch(const void* d_keys, int key_type, const uint64_t* h_sizes, const uint32_t* h_p, uint32_t njobs,
                        const hss_params* prm, hss_cut* d_splitters, uint64_t* d_offsets, void* d_work,
                        size_t work_bytes, hss_batch_stats* h_stats, hss_job_stats* h_job_stats, void* stream);

/* The same calls with a seed per job: job j uses h_seeds[j] (host array of
 * njobs entries) instead of prm->seed + j, so each job equals hss_sort
 * (hss_partition) alone with its own seed -- a server batching independent
 * requests keeps every request's result.  h_seeds = NULL is the plain form.
 * Workspace: hss_batch_workspace_bytes (seeds do not change it). */
int hss_sort_batch_seeded(const void* d_keys, const uint32_t* d_payload, int key_type, const uint64_t* h_sizes,
                          const uint32_t* h_p, const uint64_t* h_seeds, uint32_t njobs, const hss_params* prm,
                          void* d_keys_out, uint32_t* d_payload_out, hss_cut* d_splitters, uint64_t* d_offsets,
                          void* d_work, size_t work_bytes, hss_batch_stats* h_stats, hss_job_stats* h_job_stats,
                          void* stream);
int hss_partition_batch_seeded(const void* d_keys, int key_type, const uint64_t* h_sizes, const uint32_t* h_p,
                               const uint64_t* h_seeds, uint32_t njobs, const hss_params* prm, hss_cut* d_splitters,
                               uint64_t* d_offsets, void* d_work, size_t work_bytes, hss_batch_stats* h_stats,
                               hss_job_stats* h_job_stats, void* stream);

/* ---------------------------------------------------------------------------
 * Two-stage HSS (Sec. 5.3, multi-stage with two stages; Sec. 7.3 uses
 * r = sqrt(p) groups and the same eps in both stages).
 *
 * Stage 1 splits the N keys of p = prm->p processors (segments as for
 * hss_sort) into `groups` = r groups: the same local sort, then histogram
 * rounds for r - 1 group splitters whose target ranks are i N / r with
 * tolerance floor(N eps / (2r)) and s r expected probes per round, then the
 * exchange (group g holds its runs in processor order).  Stage 2 deals group
 * g's keys by position to its p / r processors and sorts them with
 * single-stage HSS, seed prm->seed + 1 + g (as hss_sort_batch does with
 * seed prm->seed + 1).  The final p buckets are the groups' buckets in group
 * order; the output is the stable sort of the input (payload in tow).
 *
 * Requirements (else HSS_ERR_INVALID before any device work): 2 <= r <= p,
 * r divides p, p / r <= 65536, N >= 2p, the proportional schedule, u64 or
 * i64 keys; and every group stays below 2^30 keys at its balance bound
 * (N / r + 2 floor(N eps / (2r)) + 2 < 2^30) as every stage-1 segment
 * (ceil(N / p) < 2^30).  If stage 1 leaves a group with fewer than p / r keys
 * (only when it did not balance) the call returns HSS_ERR_INVALID after
 * stage 1.  d_work holds at least hss_two_stage_workspace_bytes(...) bytes
 * of the same arguments (else HSS_ERR_WORKSPACE); its contents are undefined
 * afterwards.
 *
 * Outputs (device): d_keys_out[N] (d_payload_out[N] when d_payload is set),
 * d_group_splitters[r - 1] (stage-1 cuts: seg / spos name an input processor
 * and a position in its locally sorted keys), d_splitters[r (p/r - 1)]
 * (stage-2 cuts, group-major; seg / spos name a processor of the group and
 * a position in its sorted share; may be NULL when p = r), d_offsets[p + 1]
 * (absolute: bucket g (p/r) + i of group g).  h_stats and h_group_stats[r]
 * (host, nullable) receive each stage's round statistics.  The return value
 * is stage 1's status if it failed, else the first failing group's.
 * Synchronous (stage 2's tables depend on the group sizes).
 * ------------------------------------------------------------------------- */
typedef struct {
    uint32_t groups;
    int32_t status;
    uint32_t kernel_launches;    /* kernels both stages launched */
    uint32_t pad;
    hss_stats stage1;            /* the group split: rounds, sample sizes, |gamma|; ms_phase 0..2 with HSS_FLAG_TIMING */
    hss_batch_stats stage2;      /* the r group sorts */
} hss_two_stage_stats;

/* Workspace bytes of hss_sort_two_stage; 0 when the arguments are refused. */
size_t hss_two_stage_workspace_bytes(uint64_t N, const hss_params* prm, uint32_t groups, int key_type,
                                     int has_payload);

int hss_sort_two_stage(const void* d_keys, const uint32_t* d_payload, int key_type, uint64_t N, const hss_params* prm,
                       uint32_t groups, void* d_keys_out, uint32_t* d_payload_out, hss_cut* d_group_splitters,
                       hss_cut* d_splitters, uint64_t* d_offsets, void* d_work, size_t work_bytes,
                       hss_two_stage_stats* h_stats, hss_job_stats* h_group_stats, void* stream);

/* ---------------------------------------------------------------------------
 * Learned splitter proposal: a 1-32-32-1 CDF network of the keys.
 *
 * The paper proposes no model; its rounds (Sec. 4.2.2) take any candidate
 * cuts, and hss_partition_with_proposal feeds them the cuts a model of the
 * key distribution predicts.  The network maps a key to its estimated
 * empirical CDF value:
 *   u   = the key's order-preserving bits (int64: sign bit flipped)
 *   x   = clip((raw(u) - lo) / (hi - lo), 0, 1), raw(u) = u (HSS_CDF_LINEAR)
 *         or log2(1 + u) (HSS_CDF_LOG), in double precision
 *   y   = w3 . relu(W2 relu(w1 x + b1) + b2) + b3, float32
 * trained on (key, rank) pairs of earlier jobs (for instance the splitters
 * and offsets an HSS call returns: exact ranks of sampled keys) to minimise
 * (1/n) sum (y - rank/N)^2 with Adam (beta1 0.9, beta2 0.999, eps 1e-8).
 * The model is one caller-owned device struct; its parameters can be read
 * and written directly.  All calls are asynchronous on `stream`.
 * ------------------------------------------------------------------------- */
#define HSS_CDF_HIDDEN 32
#define HSS_CDF_NPARAM 1153  /* 32 + 32 + 32*32 + 32 + 32 + 1 */
#define HSS_CDF_LINEAR 0
#define HSS_CDF_LOG 1
#define HSS_CDF_W_FP32 0
#define HSS_CDF_W_BF16 1

typedef struct {
    float theta[HSS_CDF_NPARAM];  /* w1[32], b1[32], W2[32*32] (row i = hidden-2 unit), b2[32], w3[32], b3 */
    float m[HSS_CDF_NPARAM];      /* Adam first moments */
    float v[HSS_CDF_NPARAM];      /* Adam second moments */
    uint32_t step;                /* Adam steps taken */
    int32_t feature;              /* HSS_CDF_LINEAR or HSS_CDF_LOG */
    int32_t key_type;             /* HSS_KEY_U64 or HSS_KEY_I64 */
    int32_t weights;              /* HSS_CDF_W_FP32, or HSS_CDF_W_BF16: every network evaluation (eval,
                                     propose, the forward and backward pass of training) uses theta
                                     rounded to bfloat16 (round to nearest, ties to even); theta and the
                                     Adam moments stay float32 (the master copy the updates go to) */
    double lo, hi;                /* raw feature bounds of x = 0 and x = 1 */
} hss_cdf_model;

/* Initialise d_model: feature map from the key bounds lo_key < hi_key (the
 * caller's key type), Adam state zero, parameters from Philox4x32-10 words of
 * `seed` (counter (k, 0, 0, 0x43444621) for parameter k, u = (x0 >> 8) 2^-24):
 * hidden-1 units alternate in sign with |w1| = 4 (1 + u) and knots -b1/w1 at
 * (i + 0.5)/32; W2 and w3 uniform in +-sqrt(6/32); b2 = 0.1; b3 = 0.5.
 * HSS_ERR_INVALID for a bad mode or key type, or bounds not increasing. */
int hss_cdf_init(hss_cdf_model* d_model, uint64_t seed, int feature, int key_type, uint64_t lo_key, uint64_t hi_key,
                 void* stream);

/* The weight precision of every later evaluation of d_model (weights =
 * HSS_CDF_W_FP32 or HSS_CDF_W_BF16; hss_cdf_init sets FP32).  HSS_ERR_INVALID
 * for another value. */
int hss_cdf_set_weights(hss_cdf_model* d_model, int weights, void* stream);

/* sizeof(hss_cdf_model), for callers without this header's struct. */
size_t hss_cdf_model_bytes(void);

/* Device scratch (bytes) of hss_cdf_grad / hss_cdf_train for n points. */
size_t hss_cdf_work_bytes(uint32_t n);

/* Gradient of the loss at the current parameters over n points (d_keys[n]
 * in the model's key type, d_ranks[n] their ranks among N keys): d_grad[1153]
 * (float, nullable) and the loss d_loss[1] (nullable).  No update. */
int hss_cdf_grad(const hss_cdf_model* d_model, const void* d_keys, const uint64_t* d_ranks, uint32_t n, uint64_t N,
                 float* d_grad, float* d_loss, void* d_work, size_t work_bytes, void* stream);

/* `steps` full-batch Adam steps of learning rate lr on the n points; the loss
 * before the last step into d_loss (nullable).  Two kernels per step. */
int hss_cdf_train(hss_cdf_model* d_model, const void* d_keys, const uint64_t* d_ranks, uint32_t n, uint64_t N,
                  uint32_t steps, float lr, float* d_loss, void* d_work, size_t work_bytes, void* stream);

/* Network output y for n keys: d_y[n] float. */
int hss_cdf_eval(const hss_cdf_model* d_model, const void* d_keys, uint32_t n, float* d_y, void* stream);

/* Proposed cuts: for each splitter i = 1..p-1 and k = 0..per_splitter-1 the
 * CDF target tau = i/p + delta (2k/(per_splitter-1) - 1), clipped to [0, 1]
 * (just i/p when per_splitter = 1); bisection (40 halvings, float32) for the
 * smallest x in [0, 1] with y(x) >= tau, mapped back through the inverse
 * feature map to a key (clamped to the key range).  Several cuts per splitter
 * spread over the model's error band (delta about a few times its RMS error)
 * bracket the target rank from both sides, so the histogram of the cuts
 * narrows both L_i and U_i.  d_out_keys[(p-1) per_splitter], splitter-major,
 * in the model's key type, ready for hss_partition_with_proposal. */
int hss_cdf_propose(const hss_cdf_model* d_model, uint32_t p, uint32_t per_splitter, double delta, void* d_out_keys,
                    void* stream);

/* ---------------------------------------------------------------------------
 * Tuning of the segmented sort (the local sort and the merge), process-wide.
 * The project's autotuner (paper_1803_01237_gb300/autotune.py) measures the
 * choices per workload shape and sets them here; the sorted output,
 * splitters and offsets do not depend on them.
 * ------------------------------------------------------------------------- */
typedef struct {
    /* The largest segment sorted on chip; a larger one is split again.  4096
     * (the default) or 14336 (the largest on-chip class). */
    uint32_t chip_max_keys;
    /* 1: a sub-bucket that is split again interpolates its own key range
     * (gathered by the split that made it) with a digit width giving about
     * child_bucket_keys keys per sub-bucket; 0 (default): its top varying
     * byte. */
    uint32_t child_interp;
    uint32_t child_bucket_keys;  /* 128 .. 4096 (0 = 384) */
    /* Packing of small sub-buckets: after a split, runs of consecutive
     * sub-buckets that are sorted on chip are merged into one on-chip sort of
     * up to pack_keys keys (their keys are already in order between them, so
     * sorting the run sorts each).  1 .. 4096; 0 = 1024; 1 packs nothing. */
    uint32_t pack_keys;
    /* First split of each segment of a local sort: 0 (default) on its top
     * varying byte; 1 samples the segment first and, when the sample's top
     * varying byte crowds its keys into few values (Gaussian clusters, heavy
     * duplicates, spatially clustered Morton codes), splits on 255 splitters
     * taken from the sorted sample (a binary search per key) and packs those
     * sub-buckets by at most 256 keys.  Faster on the clustered Morton
     * payload workload, slower on the Gaussian mixture and Zipf keys: off by
     * default, left to the autotuner. */
    uint32_t first_split;
    /* How the split pass writes a tile: 0 stages the tile in shared memory in
     * digit order and writes each digit's run with consecutive stores; 1
     * writes every key straight to its slot in its digit's run (no staging,
     * no second pass over shared memory; the L2 cache assembles the runs),
     * except in tiles whose sub-buckets' key ranges are gathered for the next
     * level, which stay staged. */
    uint32_t split_scatter;
    uint32_t reserved[2];        /* zero */
} hss_tuning;

/* Set the tuning (NULL restores the defaults); HSS_ERR_INVALID for a value
 * out of range.  Calls already enqueued keep the tuning they started with. */
int hss_set_tuning(const hss_tuning* t);
int hss_get_tuning(hss_tuning* t);

/* Kernels launched by this library in this process so far. */
uint64_t hss_kernel_launch_count(void);

/* Static description of an error code. */
const char* hss_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* HSS_H */
