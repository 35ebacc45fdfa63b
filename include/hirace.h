/*
 * hirace.h - C-ABI of the GB300 race checker (HiRace, arXiv 2401.04701).
 *
 * The checker folds the access history of every monitored word into a
 * constant-size shadow value with a parallel finite-state machine (Sec. III;
 * Algorithm 1 "UpdateShadow"; 8 bytes per word by default, 4 with the compact
 * packing, 24 in every-epoch report mode; Sec. IV-B) and reports the words on
 * which two accesses race (Sec. II-A:
 * different threads, at least one write, not ordered by happens-before;
 * Sec. II-B: __syncthreads orders a block, __syncwarp a warp, nothing orders
 * two blocks of one kernel, kernel end orders everything).
 *
 * Every entry point is extern "C", takes plain pointers and sizes, returns an
 * hr_status and never throws.  Device pointers are CUDA global-memory
 * addresses of the current device; streams are cudaStream_t values (NULL is
 * the legacy default stream).  All work is issued asynchronously on the given
 * stream unless a call says otherwise.
 */
#ifndef HIRACE_H
#define HIRACE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* hr_stream_t; /* same type as cudaStream_t */
typedef struct hr_ctx hr_ctx;            /* opaque checker context */

typedef enum hr_status {
    HR_OK = 0,
    HR_ERR_INVALID = 1,        /* bad argument or region descriptor */
    HR_ERR_OOM = 2,            /* device or host allocation failed */
    HR_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    HR_ERR_ORDER = 4,          /* trace not sorted by (kernel, bc, wc), or older than the region's last record */
    HR_ERR_RANGE = 5,          /* word index >= n_words */
    HR_ERR_CLOCK_OVERFLOW = 6, /* a clock or thread id does not fit the shadow packing (Sec. III-A footnote) */
    HR_ERR_CONTENTION = 7,     /* the CAS retry cap was reached on some word */
    HR_ERR_TIMEOUT = 8,        /* a bounded device-side wait expired */
    HR_ERR_UNSUPPORTED = 9,    /* partial-mask __syncwarp or an unknown op code */
    HR_ERR_CAPACITY = 10,      /* more waves in one call than the wave table holds */
    HR_ERR_NOT_READY = 11      /* the region has work in flight on another stream */
} hr_status;

/* report modes of a region (hr_region_desc.report_mode) */
#define HR_REPORT_FIRST 0u       /* the first racy epoch of each word per kernel (RACE absorbing) */
#define HR_REPORT_EVERY_EPOCH 1u /* every racy (word, kernel, epoch) */

/* hr_report flag bits */
#define HR_FLAG_TRUNCATED 1u /* more races than the report ring holds; n_total stays exact */

/* memory space of a region (informational: the shadow always lives in HBM) */
#define HR_SPACE_GLOBAL 0u
#define HR_SPACE_SHARED 1u

/* hr_sync scopes */
#define HR_SYNC_KERNEL 0u

/* access operations (Algorithm 1 input `access`: read / write / atomic) and
 * barrier records (Sec. II-B) */
typedef enum hr_op {
    HR_R = 0,
    HR_W = 1,
    HR_A = 2,
    HR_SYNCTHREADS = 3,
    HR_SYNCWARP = 4
} hr_op;

#define HR_RECFLAG_ATOMIC_LOAD 1u  /* informational */
#define HR_RECFLAG_PARTIAL_MASK 2u /* __syncwarp with a partial mask: unsupported (Sec. VI future work) */

/*
 * One trace record, 16 bytes, little endian.  `tid` is the global thread id
 * blockIdx*blockDim+threadIdx (Algorithm 1 input "Global thread ID"); `bc`
 * and `wc` are the thread-private block-scope and warp-scope scalar clocks
 * (Algorithm 1 inputs `bc`, `wc`; Sec. III-A Scenario 2): bc counts the
 * __syncthreads the thread has executed in this kernel, wc the full-warp
 * __syncwarp since its last __syncthreads.  A barrier record carries the
 * clocks the thread holds after the barrier.  Bytes 8..13 read as a
 * little-endian u64 masked to 48 bits form the wave key (kernel, bc, wc).
 */
typedef struct hr_record {
    uint32_t word;   /* word index inside the region (ignored for barrier records) */
    uint32_t tid;
    uint16_t wc;
    uint16_t bc;
    uint16_t kernel; /* launch ordinal of the traced kernel */
    uint8_t op;      /* hr_op */
    uint8_t flags;   /* HR_RECFLAG_* */
} hr_record;

/*
 * One race report, 16 bytes: the first racy pair on `word` inside `kernel`
 * was completed by an access of thread `tid` doing `op` in block epoch
 * `epoch` (its bc).  `prior` is the FSM state the word held just before
 * (hr_fsm_state_name).  Races are reported once per (word, kernel): the
 * paper reports races per distinct address (Sec. V-B).  In every-epoch mode
 * a report is made once per (word, kernel, epoch) and `prior` is the scope
 * level (1 thread .. 4 grid) of the accesses the reporting one conflicts with.
 */
typedef struct hr_race {
    uint32_t word;
    uint32_t tid;
    uint16_t kernel;
    uint16_t epoch;
    uint16_t region;
    uint8_t op;
    uint8_t prior;
} hr_race;

/* Geometry of one monitored region: its words and the traced launch shape. */
typedef struct hr_region_desc {
    uint64_t n_words;         /* monitored words, >= 1 */
    uint32_t block_dim;       /* threads per block of the traced kernels, >= 1 */
    uint32_t warp_size;       /* 32 on NVIDIA GPUs; 1..32 for small test universes */
    uint32_t space;           /* HR_SPACE_GLOBAL or HR_SPACE_SHARED (informational) */
    uint8_t shadow_bytes;     /* bytes per shadow word: 8 (0 = default) or 4 (compact packing) */
    uint8_t tid_bits;         /* compact packing only: tid field width, 4..22 (0 = 16); bc and wc
                                 share the other 24 - tid_bits bits (hirace_device.cuh) */
    uint8_t report_mode;      /* HR_REPORT_FIRST (0): one report per racy word and kernel, the
                                 first racy epoch (RACE absorbing); HR_REPORT_EVERY_EPOCH (1): one
                                 per racy (word, kernel, epoch), 24 shadow bytes per word, 8-byte
                                 packing only */
    uint8_t reserved;         /* must be 0 */
    uint64_t report_capacity; /* race records kept for this region; 0 = the hr_init default */
} hr_region_desc;

/*
 * hr_init - create a checker context with one shadow store per region
 * (Sec. III-A: one shadow entry per monitored array element; 8 bytes per
 * word, Sec. IV-B).  Every shadow word starts in INIT.
 *   out              receives the context (host pointer; NULL on failure)
 *   regions          n_regions host descriptors
 *   report_capacity  default race records per region (>= 1)
 *   stream           stream for the initial clears
 * The context owns all device memory it allocates (shadow: shadow_bytes *
 * n_words bytes per region; report ring: 16*report_capacity bytes per region;
 * a wave table and control block).  Errors: HR_ERR_INVALID (also for a
 * compact region whose block_dim exceeds 2^tid_bits), HR_ERR_OOM, HR_ERR_CUDA.
 */
hr_status hr_init(hr_ctx** out, const hr_region_desc* regions, uint32_t n_regions,
                  uint64_t report_capacity, hr_stream_t stream);

/*
 * hr_init_with_buffers - hr_init over shadow stores (and optionally report
 * rings) the caller already owns, e.g. tensors from a framework's allocator.
 *   shadows  n_regions device pointers, each to shadow_bytes * n_words bytes,
 *            16-byte aligned; every word is set to INIT (zero) on `stream`
 *   rings    NULL, or n_regions device pointers (NULL entries: allocated by
 *            the context) to 16 * capacity bytes, 16-byte aligned
 * The caller keeps ownership: the buffers must outlive the context and are
 * not freed by hr_destroy; nothing else may write them while it lives.  The
 * context still allocates its own scratch.  Errors: those of hr_init, and
 * HR_ERR_INVALID for a NULL or misaligned buffer.
 */
hr_status hr_init_with_buffers(hr_ctx** out, const hr_region_desc* regions, uint32_t n_regions,
                               uint64_t report_capacity, void* const* shadows, hr_race* const* rings,
                               hr_stream_t stream);

/*
 * hr_check_trace - apply a device-resident trace to one region (Algorithm 1
 * for every access record, in an order consistent with happens-before).
 *   d_trace  n records in device memory, caller-owned, alive until `stream`
 *            passes this call; sorted by wave key (kernel, bc, wc), each
 *            thread's records in program order, kernels not older than the
 *            region's last processed record
 * d_trace must be 16-byte aligned.  Asynchronous.  Violations found on the
 * device set the region's sticky
 * error (HR_ERR_ORDER, HR_ERR_RANGE, HR_ERR_CLOCK_OVERFLOW,
 * HR_ERR_CONTENTION, HR_ERR_UNSUPPORTED, HR_ERR_CAPACITY, HR_ERR_TIMEOUT);
 * checking of that region stops after the races found so far are reported
 * (Sec. III-A footnote), and hr_report returns the error.  Returns
 * HR_ERR_INVALID for a bad region or NULL trace with n > 0.
 */
hr_status hr_check_trace(hr_ctx* ctx, uint32_t region, const hr_record* d_trace, uint64_t n,
                         hr_stream_t stream);

/*
 * hr_check_trace_host - hr_check_trace over a trace in HOST memory: the trace
 * is copied in chunks of chunk_records records (0: 2^24, i.e. 256 MB) through
 * two device staging buffers owned by the context, each chunk's copy (on a
 * copy stream of the context) overlapping the check of the chunk before it on
 * `stream`.  Chunks may cut waves (the shadow stays resident between them).
 * Asynchronous: h_trace must stay valid, and unchanged, until `stream` has
 * passed this call; page-locked memory lets the copies overlap the checks.
 * Growing the staging buffers synchronises the device once.  Not for use
 * inside stream capture.  Errors: those of hr_check_trace, HR_ERR_OOM.
 */
hr_status hr_check_trace_host(hr_ctx* ctx, uint32_t region, const hr_record* h_trace, uint64_t n,
                              uint64_t chunk_records, hr_stream_t stream);

/*
 * hr_check_trace_kbase - hr_check_trace with `kernel_base` (0..65535) added to
 * every record's kernel ordinal: one recorded trace can be checked again as a
 * later launch without clearing the region (kernel end orders everything,
 * Sec. II-B, so shadow values of older launches read as INIT).  The rebased
 * ordinals must fit in 16 bits.  Same ownership and errors as hr_check_trace.
 */
hr_status hr_check_trace_kbase(hr_ctx* ctx, uint32_t region, const hr_record* d_trace, uint64_t n,
                               uint32_t kernel_base, hr_stream_t stream);

/*
 * hr_check_trace_plain - the same check without warp aggregation: every lane
 * applies its own record with its own CAS loop.  Same arguments, ownership
 * and errors as hr_check_trace; kept as the one-record-per-update baseline.
 */
hr_status hr_check_trace_plain(hr_ctx* ctx, uint32_t region, const hr_record* d_trace, uint64_t n,
                               hr_stream_t stream);

/* One job of a batched check: a trace for one region of the context. */
typedef struct hr_job {
    uint32_t region;
    uint32_t reserved;       /* must be 0 */
    const hr_record* trace;  /* device pointer, 16-byte aligned, same rules as hr_check_trace */
    uint64_t n;
} hr_job;

/*
 * hr_check_batch - check many traces, each on its own region, in one
 * persistent launch (the per-job result equals hr_check_trace on that job
 * alone).  jobs is a host array of n_jobs <= 512 entries naming distinct
 * regions (HR_ERR_INVALID otherwise).  The jobs' stages are interleaved
 * wave-major (every job's first wave, then every job's second wave, ...) and
 * each stage waits only for the previous stage of its own job, so independent
 * traces fill each other's wave boundaries.  Asynchronous.  The first call
 * allocates the batch scratch (call hr_batch_reserve first to keep later calls
 * allocation-free, e.g. inside CUDA-graph capture).
 */
hr_status hr_check_batch(hr_ctx* ctx, const hr_job* jobs, uint32_t n_jobs, hr_stream_t stream);

/* Calls queued inside a stream capture (CUDA graphs) record no completion
 * event: synchronise the replay stream before hr_report on those regions
 * (hr_report then waits for the whole device). */

/* Size the batch scratch for up to max_jobs jobs and max_waves waves per call
 * (synchronises the device).  Errors: HR_ERR_INVALID, HR_ERR_OOM. */
hr_status hr_batch_reserve(hr_ctx* ctx, uint32_t max_jobs, uint64_t max_waves);

/*
 * hr_batch_job_times - completion time of each job of the last hr_check_batch,
 * in nanoseconds after the batch's first kernel started (device clock): the
 * moment the tile that finished the job's last wave was done.  ns_out[i] is
 * for jobs[i] of that call (0 for an empty trace or a job that failed before
 * running).  Synchronises the device.  HR_ERR_INVALID if n exceeds that call's
 * job count.
 */
hr_status hr_batch_job_times(hr_ctx* ctx, uint64_t* ns_out, uint32_t n);

/*
 * hr_sync - kernel end for a region (Sec. II-B: the end of a kernel orders
 * every access of that kernel before every access of the next one).  Only
 * HR_SYNC_KERNEL exists: block and warp barriers arrive as trace records or
 * through the device header.  Later trace records must carry a larger kernel
 * ordinal; the next device view uses the next kernel ordinal.  Asynchronous.
 */
hr_status hr_sync(hr_ctx* ctx, uint32_t region, uint32_t scope, hr_stream_t stream);

/*
 * hr_report - wait for the region's outstanding work, then copy its race
 * records to host memory.
 *   host_out  host array of cap records (may be NULL when cap == 0)
 *   n_total   receives the number of races found (may exceed cap)
 *   flags     receives HR_FLAG_* bits (may be NULL)
 * Records are in the order the device appended them (sort them for a set
 * comparison).  Returns the region's sticky error, HR_OK if none.
 */
hr_status hr_report(hr_ctx* ctx, uint32_t region, hr_race* host_out, uint64_t cap, uint64_t* n_total,
                    uint32_t* flags);

/* Counters of one region since init/reset: accesses applied, CAS attempts,
 * CAS retries, and accesses applied without a shadow access of their own
 * (lanes folded by warp aggregation, exact repeats, and accesses to a word
 * the per-wave checker has cached in a state that absorbs them).
 * Synchronises like hr_report. */
hr_status hr_counters(hr_ctx* ctx, uint32_t region, uint64_t out[4]);

/* hr_reset - every shadow word of the region back to INIT, reports, counters
 * and error cleared, kernel ordinal back to 0.  Asynchronous. */
hr_status hr_reset(hr_ctx* ctx, uint32_t region, hr_stream_t stream);

/*
 * hr_region_reconfigure - give a region new geometry (n_words up to the
 * n_words it was created with, block_dim, warp_size) and reset it like
 * hr_reset, without allocating: lets a server reuse pre-allocated region
 * slots for jobs of different shapes.  Stream-ordered.  HR_ERR_INVALID if
 * n_words exceeds the region's allocation.
 */
hr_status hr_region_reconfigure(hr_ctx* ctx, uint32_t region, uint64_t n_words, uint32_t block_dim,
                                uint32_t warp_size, hr_stream_t stream);

/*
 * Selective monitoring (Sec. IV-A: instrumentation can be switched on or off
 * per thread and per address, and symmetric work groups can be represented by
 * a few threads to save work and memory).  Accesses outside the filter are not
 * checked and raise no error; the races reported are exactly those among the
 * monitored accesses.
 */
typedef struct hr_filter {
    uint64_t word_lo;   /* word window [word_lo, word_hi): shadow word i holds word word_lo + i, */
    uint64_t word_hi;   /*   so the region needs only word_hi - word_lo words; word_hi 0 = no window */
    uint32_t block_lo;  /* monitored blocks [block_lo, block_hi); block_hi 0 = every block */
    uint32_t block_hi;
    uint32_t lane_mask; /* monitored lanes of each warp (bit l: lane l = tid mod block_dim mod
                           warp_size); 0xFFFFFFFF = every lane, 0 is invalid */
    uint32_t reserved;  /* must be 0 */
    /* Symmetric work group (Sec. IV-A: only representative threads of a
     * user-declared symmetric group are tracked).  Blocks [sym_lo, sym_hi)
     * are declared to run the same program, block sym_lo + m on the words of
     * block sym_lo shifted up by m * sym_stride.  An access of thread tid of
     * block sym_lo + m to word w is applied as the access of thread
     * tid - m * block_dim (the same thread of block sym_lo) to word
     * w - m * sym_stride (not monitored if w < m * sym_stride); the block
     * range, lane mask and word window then apply to that representative
     * access, and a race on it is reported with the representative's tid and
     * word.  With a word window over the representative's data the shadow
     * shrinks by the group size.  sym_hi 0 = no group. */
    uint32_t sym_lo;
    uint32_t sym_hi;
    uint64_t sym_stride;
} hr_filter;

/*
 * hr_set_filter - monitor only the accesses `filter` selects, on later checks
 * and device views of `region` (NULL: monitor everything again).  Race
 * records keep absolute word indices.  Stream-ordered; the filter stays set
 * across hr_reset and is cleared by hr_region_reconfigure.  HR_ERR_INVALID if
 * the window is empty or wider than the region, block_hi < block_lo (with
 * block_hi != 0), sym_hi <= sym_lo (with sym_hi != 0), lane_mask is 0 or
 * reserved is not 0.  A symmetric group finds the races inside each member
 * block, exactly when the members are symmetric; it misses races between two
 * members and races of other blocks on a member's (non-representative)
 * words, and if the members are not symmetric it may report races that only
 * the folded program has.
 */
hr_status hr_set_filter(hr_ctx* ctx, uint32_t region, const hr_filter* filter, hr_stream_t stream);

/* hr_destroy - synchronise and free everything the context owns. */
hr_status hr_destroy(hr_ctx* ctx);

/*
 * Kernel variants and the autotuner (no paper counterpart; the tile schedule
 * of the checker).  Ids 0..5 are shapes of the per-wave checker: a variant
 * fixes the consumer warps per CTA, the records each consumer lane takes per
 * tile and whether lanes on the same word are aggregated; even ids aggregate
 * and the odd id after each is the same shape without aggregation.  Id 6 is the
 * binned checker, which hr_variant_desc reports with zero records per lane and
 * zero consumer warps: the accesses are moved into (4096-word shadow segment,
 * wave) buckets and persistent thread groups apply each segment's buckets to a
 * shared-memory copy of the segment, wave by wave.  It takes single-trace checks of regions of at
 * most 2^26 words with at most 256 waves per call; batches, and calls it cannot
 * take, run the per-wave checker of id 3.  So does a check of at least 2^22
 * accesses whose fullest segment holds more than 1/256 of them (one thread
 * group applies a segment, so a few hot words would serialise the check); that
 * decision is taken on the device after the count and scan passes.  Its first check on a region
 * allocates the region's bucket tables (4 bytes per segment for each of 256
 * waves plus about one count slice per SM) and an access buffer of 8 bytes per
 * record, so make that check before capturing calls into a CUDA graph.  Its shared-memory CAS loops are bounded by the same cap.  hr_autotune checks the given trace on `region` with
 * every variant (reset before each run, a warm-up then a timed run on
 * `stream`, synchronous), keeps the fastest for this context's later checks,
 * writes it to *best and the per-variant milliseconds to ms[0..ms_cap), and
 * leaves the region reset.  A variant whose run ends with HR_ERR_CONTENTION or
 * HR_ERR_TIMEOUT (a bound of that variant ran out) is skipped and gets -1 ms;
 * any other error is the trace's, and hr_autotune returns it.
 * Regions in HR_REPORT_EVERY_EPOCH mode always use a checker of their own
 * (variant 3's shape): the variant setting does not apply to them, and
 * hr_autotune on such a region returns HR_ERR_INVALID.
 */
uint32_t hr_variant_count(void);
hr_status hr_variant_desc(uint32_t id, uint32_t* aggregate, uint32_t* records_per_lane, uint32_t* consumer_warps);
hr_status hr_set_variant(hr_ctx* ctx, uint32_t id);
hr_status hr_get_variant(hr_ctx* ctx, uint32_t* id);
hr_status hr_autotune(hr_ctx* ctx, uint32_t region, const hr_record* d_trace, uint64_t n, hr_stream_t stream,
                      uint32_t* best, float* ms, uint32_t ms_cap);

/*
 * hr_set_limits - bounds of the device-side waits and retries of this
 * context's later checks (Sec. III-A: checking stops with a report rather than
 * running on).  wait_ns (> 0, default 4e9) bounds every wait of a CTA on the
 * previous stage or on its copy pipeline; when it runs out the launch winds
 * down and the region reports HR_ERR_TIMEOUT.  cas_retry_cap (default 4096)
 * bounds the CAS retries of one update; beyond it the region reports
 * HR_ERR_CONTENTION.  test_flags is a test hook: HR_TEST_HOLD_STAGE makes the
 * second stage of a single-trace check wait for a completion that never comes,
 * so the bounded wait runs out; leave it 0 otherwise.
 */
#define HR_TEST_HOLD_STAGE 1u
hr_status hr_set_limits(hr_ctx* ctx, uint64_t wait_ns, uint32_t cas_retry_cap, uint32_t test_flags);

/*
 * Profiling (no paper counterpart; measurement support).  With profiling on,
 * every check call records CUDA events on its stream around the wave
 * pre-pass and around the FSM kernel.  hr_profile_read waits for those
 * events and returns the summed milliseconds, the number of profiled calls
 * and of library kernel launches since the previous read.  Host pointers may
 * be NULL.
 */
hr_status hr_profile_enable(hr_ctx* ctx, int on);
hr_status hr_profile_read(hr_ctx* ctx, double* check_ms, double* prepass_ms, uint64_t* calls, uint64_t* launches);

/*
 * hr_check_trace_noalloc - the aggregated trace check for callers that cannot
 * allocate device memory.  The paper has no counterpart: it is a deployment
 * variant of hr_check_trace.  Callers that cannot call cudaMalloc include
 * code running while another component owns the device memory budget (a
 * framework's caching allocator or a fixed pool that already holds the free
 * memory) and latency-critical paths where cudaMalloc/cudaFree would stall
 * on an implicit device synchronisation.  No context is needed and nothing is
 * allocated: no cudaMalloc, cudaFree or allocating library routine is called.
 *   d_trace   n records, device memory, same rules as hr_check_trace
 *   d_shadow  n_words 8-byte shadow values, caller-owned device memory.  Each
 *             call checks one complete trace as a fresh region: before the
 *             trace's first wave the call clears d_shadow (every word INIT),
 *             so what an earlier call or the caller left there does not
 *             matter, and kernel ordinals are not ordered against an earlier
 *             call's.  On return it holds the state after the trace.  A trace
 *             cut into several calls is not continued: use hr_check_trace on a
 *             context for that.
 *   d_races   race_cap race records (device), written from slot 0
 *   d_result  device hr_result, overwritten: races found by this call (may
 *             exceed race_cap), its sticky error, HR_FLAG_* flags
 * The wave pre-pass scratch is a file-scope device array of
 * HR_NOALLOC_SCRATCH_BYTES (611 KiB) inside the library; every GPU that loads
 * the library holds it until the process exits.  Its limit: at most
 * HR_NOALLOC_MAX_WAVES waves (distinct (kernel, bc, wc) keys) per call; a
 * longer trace is rejected on the device with d_result->error ==
 * HR_ERR_CAPACITY and nothing is checked.  The first call on each device
 * looks up the array's device address and copies the FSM table into it with
 * a synchronous cudaMemcpy, so make that first call before any stream
 * capture.  The address is cached per device for the life of the process, so
 * a cudaDeviceReset on a device invalidates this entry point there until the
 * library is reloaded.  All calls share the array and it keeps the last call's contents
 * (each call re-initialises what must start at zero); calls whose work
 * overlaps on the GPU race on it, so serialise them.  Asynchronous on
 * `stream` after the first call.  Returns HR_ERR_INVALID for bad arguments,
 * HR_ERR_CUDA if a launch or the set-up fails; device-side errors go to
 * d_result->error.
 */
#define HR_NOALLOC_MAX_WAVES 4096u
#define HR_NOALLOC_SCRATCH_BYTES 625664u

typedef struct hr_result {
    uint64_t n_races;
    uint32_t error;
    uint32_t flags;
} hr_result;

hr_status hr_check_trace_noalloc(const hr_record* d_trace, uint64_t n, uint64_t* d_shadow, uint64_t n_words,
                                 uint32_t block_dim, uint32_t warp_size, hr_race* d_races, uint64_t race_cap,
                                 hr_result* d_result, hr_stream_t stream);

/*
 * Word-range sharding (no paper counterpart; the paper checks on one GPU).
 * Ranks that each own a contiguous word range [bounds[r], bounds[r+1]) of a
 * region check one trace together: an access touches only its own word's
 * shadow value (Algorithm 1), so each rank checks the accesses to its words
 * on its own region, in wave order.
 *
 * hr_shard_partition - split the n records of d_trace (device, wave-sorted,
 * 16-byte aligned) by owner rank.  d_bounds: world + 1 device uint64 word
 * bounds, ascending, bounds[0] = 0 (world <= HR_SHARD_MAX_WORLD).  Each access
 * whose word w lies in [bounds[r], bounds[r+1]) is written, with word
 * w - bounds[r], to destination r's block of d_out (device, n records, 16-byte
 * aligned); blocks follow one another in rank order and keep trace order
 * inside (a stable partition, so each stays wave-sorted).  Barrier records
 * and words at or past bounds[world] are not routed.  d_counts (device,
 * world uint64) gets each block's record count.  d_scratch: device memory of
 * hr_shard_partition_scratch_bytes(n, world) bytes, 8-byte aligned.
 * Asynchronous on `stream`.  HR_ERR_INVALID for bad arguments, HR_ERR_CUDA if
 * a launch fails.
 */
#define HR_SHARD_MAX_WORLD 64u
uint64_t hr_shard_partition_scratch_bytes(uint64_t n, uint32_t world);
hr_status hr_shard_partition(const hr_record* d_trace, uint64_t n, const uint64_t* d_bounds, uint32_t world,
                             hr_record* d_out, uint64_t* d_counts, void* d_scratch, uint64_t scratch_bytes,
                             hr_stream_t stream);

/*
 * hr_shard_merge - merge n_chunks wave-sorted blocks of d_in (device; block c
 * is records [d_starts[c], d_starts[c+1]), d_starts: n_chunks + 1 device
 * uint64, d_starts[n_chunks] = n) into one wave-sorted trace in d_out (device,
 * n records): runs of equal wave key in key order, equal keys in block order.
 * Inside a wave any order is a valid execution order (Sec. II-B), so the
 * result checks like the blocks' union.  d_scratch: device memory of
 * hr_shard_merge_scratch_bytes(max_runs) bytes, 256-byte aligned, for up to
 * max_runs runs (a run: one block's records of one wave).  *d_status (device
 * uint32) gets 0, HR_ERR_ORDER when a block is not wave-sorted, or
 * HR_ERR_CAPACITY when the blocks hold more than max_runs runs (the output
 * is then incomplete).  Asynchronous on `stream`.  HR_ERR_INVALID for bad
 * arguments, HR_ERR_CUDA if a launch fails.
 */
uint64_t hr_shard_merge_scratch_bytes(uint64_t max_runs);
hr_status hr_shard_merge(const hr_record* d_in, const uint64_t* d_starts, uint32_t n_chunks, uint64_t n,
                         hr_record* d_out, void* d_scratch, uint64_t scratch_bytes, uint64_t max_runs,
                         uint32_t* d_status, hr_stream_t stream);

/* Static text for a status code. */
const char* hr_status_str(hr_status s);

/*
 * The FSM as a flat table (Sec. IV-B stores it as one array whose index
 * joins the old state and the transition label bits): entry
 * (oState << 6) | (access << 4) | (tRel << 2) | sRel gives the next state in
 * bits 0..4 and its scope level in bits 5..7 (0xFF marks unused labels).
 * access: 0 R, 1 W, 2 A.  tRel: 0 same thread, 1 same warp, 2 same block,
 * 3 other block.  sRel: 0 unsynchronised, 1 warp barrier between, 2 block
 * barrier between.  Copies 2048 bytes to out; *n_states gets the number of
 * reachable states.  Host only; needs no GPU.
 */
hr_status hr_fsm_table(uint8_t* out, uint32_t* n_states);

/* Name of an FSM state id (e.g. "INIT", "RACE", "T[R|R|R]"); "?" if unused. */
const char* hr_fsm_state_name(uint32_t state);

/* Library version string. */
const char* hr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HIRACE_H */
