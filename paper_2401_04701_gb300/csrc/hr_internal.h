// hr_internal.h - device-side data structures shared by the kernels and the API.
#pragma once

#include <cstdint>

#include "../../include/hirace.h"
#include "../../include/hirace_device.cuh"

// Geometry with exact reciprocals and, when both sizes are powers of two,
// shifts; plus the shadow packing (8 bytes, or 4 with a tid_bits-wide tid).
inline hr_geom hr_make_geom(uint32_t block_dim, uint32_t warp_size, uint32_t shadow_bytes = 8, uint32_t tid_bits = 0,
                            uint32_t report_mode = HR_REPORT_FIRST)
{
    auto magic = [](uint32_t d) { return d <= 1 ? 0ull : (~0ull) / d + 1ull; };
    auto log2_exact = [](uint32_t d) -> uint32_t {
        if (d == 0 || (d & (d - 1))) return ~0u;
        uint32_t s = 0;
        while ((1u << s) < d) ++s;
        return s;
    };
    hr_geom g{};
    g.block_dim = block_dim;
    g.warp_size = warp_size;
    g.bd_magic = magic(block_dim);
    g.ws_magic = magic(warp_size);
    const uint32_t bs = log2_exact(block_dim), ws = log2_exact(warp_size);
    g.bd_shift = (bs != ~0u && ws != ~0u) ? bs : ~0u;
    g.ws_shift = (bs != ~0u && ws != ~0u) ? ws : ~0u;
    g.report_mode = report_mode;
    g.shadow_bytes = report_mode == HR_REPORT_EVERY_EPOCH ? 24u : (shadow_bytes == 4 ? 4u : 8u);
    g.tid_bits = g.shadow_bytes == 4 ? (tid_bits ? tid_bits : 16u) : 0u;
    return g;
}

// Bytes per shadow word and tid width of a region descriptor (defaults applied):
// 8, 4 for the compact packing, 24 (three 8-byte arrays) in every-epoch mode.
inline uint32_t hr_desc_shadow_bytes(const hr_region_desc& d)
{
    return d.report_mode == HR_REPORT_EVERY_EPOCH ? 24u : (d.shadow_bytes == 4 ? 4u : 8u);
}
inline uint32_t hr_desc_tid_bits(const hr_region_desc& d)
{
    return d.shadow_bytes == 4 ? (d.tid_bits ? d.tid_bits : 16u) : 0u;
}
inline hr_geom hr_desc_geom(const hr_region_desc& d)
{
    return hr_make_geom(d.block_dim, d.warp_size, d.shadow_bytes == 4 ? 4u : 8u, hr_desc_tid_bits(d), d.report_mode);
}

// Per-region state in device memory.
struct hr_region_dev {
    unsigned long long* shadow;   // n_words shadow values
    hr_race* ring;                // ring_cap race records
    unsigned long long n_words;
    unsigned long long ring_cap;
    unsigned long long n_races;   // races found (may exceed ring_cap)
    unsigned int error;           // sticky first error (hr_status)
    unsigned int flags;           // HR_FLAG_* bits
    unsigned long long last_key;  // wave key after the region's last processed record
    unsigned int used;            // 1: a record was processed since init/reset; 2: the shadow's
                                  // contents are unknown (cleared before the first wave)
    unsigned int region;
    unsigned long long counters[4];  // accesses, CAS attempts, CAS retries, accesses without a shadow access
    hr_geom geom;
    hr_filter filter;             // monitored words, blocks, lanes (hr_set_filter)
};

// the filter that monitors every access
__host__ __device__ inline hr_filter hr_filter_all()
{
    hr_filter f{};
    f.lane_mask = 0xFFFFFFFFu;
    return f;
}

// One job = one trace checked on one region.  A single-trace check is a batch
// of one job; a batch interleaves the jobs' stages wave-major.
struct hr_jobd {
    const hr_record* trace;
    unsigned long long n;         // records
    unsigned long long kb;        // kernel base added to every record's kernel, shifted left by 32
    unsigned region;
    unsigned G;                   // records per pre-pass interval
    unsigned int_begin;           // first global pre-pass interval of this job
    unsigned n_int;
    unsigned wave_begin;          // first global wave index (written on the device)
    unsigned n_waves;             // waves of this job (written on the device)
    unsigned long long done_ns;   // device clock when the job's last stage completed (0: no stages)
};

// Work stages: per wave an optional shadow clear (when the kernel-tag group
// changes) followed by the wave's record tiles.  A stage waits for `dep`, the
// previous stage of the same job, to reach `dep_need` per-warp completions.
enum { HR_STAGE_RECORDS = 0, HR_STAGE_CLEAR = 1 };
constexpr unsigned HR_NO_DEP = 0xFFFFFFFFu;

struct hr_stage {
    unsigned item_begin;  // first global work-item index of the stage
    unsigned wave;        // global wave index
    unsigned type;
    unsigned done;        // per-warp completions of this stage's items
    unsigned dep;
    unsigned dep_need;
    unsigned job;
    unsigned last;        // 1: the job's last stage (its completion time is recorded)
};

constexpr unsigned HR_BIN_SKEW = 256;           // a segment with more than 1/this of the accesses ...
constexpr unsigned HR_BIN_SKEW_MIN = 1u << 22;  // ... of a check this large goes to the per-wave checker

struct hr_ctl {
    unsigned ticket;       // next work item
    unsigned abort;        // set when a bounded wait expired
    unsigned n_waves;
    unsigned n_stages;
    unsigned total_items;
    unsigned n_jobs;
    unsigned n_intervals;
    unsigned binned;       // 1: the binned checker took this check (the per-wave checker then has no items)
    unsigned long long t0_ns;  // device clock when the check's first kernel started
    unsigned bin_parts;    // binned checker: (slice, wave) parts of the trace
    unsigned bin_total;    // binned checker: accesses moved into buckets
    unsigned fresh;        // 1: every shadow value reads as INIT for this check's first wave (the region
                           // is new or reset, or its last record came from an older kernel and no device
                           // view writes it), so a shadow segment need not be read
    unsigned bin_max_tid;  // binned checker: largest thread id of an applied access
    unsigned bin_pack4;    // binned checker: bucketed accesses are 4 bytes (tid < 2^(30 - HR_BIN_SEG_SHIFT))
    unsigned bin_tbits;    // binned checker: 0, or the tid width of a 4-byte working shadow in shared memory
                           // (fresh checks whose tids and clocks fit it)
    unsigned seg_ticket;   // binned checker: next segment a thread group of the segment pass takes
    unsigned bin_max_seg;  // binned checker: accesses of the fullest segment
    unsigned bin_count;    // binned checker: accesses counted into buckets
};

// Whether the binned checker applies this check (the flag, and the skew guard:
// one thread group applies a segment's accesses, so a large check whose fullest
// segment holds more than 1/HR_BIN_SKEW of them - the hub words of a power-law
// graph - goes to the per-wave checker instead, which is launched after the
// binned kernels).  Read by the kernels after the count and scan passes.
__host__ __device__ inline bool hr_bin_taken(const hr_ctl* c)
{
    return c->binned && !(c->bin_count >= HR_BIN_SKEW_MIN && (unsigned long long)c->bin_max_seg * HR_BIN_SKEW > c->bin_count);
}

// Scratch of the binned checker (hr_binned.cu), one per region.  The region's
// shadow is cut into segments of HR_BIN_SEG words.  The trace is cut into one
// contiguous slice per streaming CTA, and a slice into parts, one per wave it
// meets; parts are numbered in trace order, so their waves ascend.  The table
// holds, for segment s and part p at s * n_parts + p, first the part's number
// of accesses to the segment, then (after an exclusive scan in that order) where
// they go in the bucketed access array: segment-major, waves ascending.
#ifndef HR_BIN_SEG_SHIFT_BITS
#define HR_BIN_SEG_SHIFT_BITS 12
#endif
constexpr unsigned HR_BIN_SEG_SHIFT = HR_BIN_SEG_SHIFT_BITS;
constexpr unsigned HR_BIN_SEG = 1u << HR_BIN_SEG_SHIFT;  // shadow words per segment (4 or 8 B each in shared memory)
static_assert(HR_BIN_SEG_SHIFT >= 10 && HR_BIN_SEG_SHIFT <= 13, "the packed access keeps 16 bits for the word");
constexpr unsigned HR_BIN_MAX_SEGS = 16384;              // larger regions take the per-wave checker
constexpr unsigned HR_BIN_MAX_WAVES = 256;               // checks with more waves take the per-wave checker
constexpr unsigned HR_BIN_SCAN = 4096;                   // table entries per scan block
constexpr unsigned HR_BIN_CLUSTER = 8;                   // CTAs sharing bucket cursors in the scatter
constexpr unsigned HR_BIN_MAX_SUB = 16;                  // count slices per cluster slice, at most
struct hr_bin {
    unsigned* table;         // [seg_cap * part_cap] counts, then offsets
    unsigned* sums;          // [seg_cap * part_cap / HR_BIN_SCAN + 1] per scan block
    unsigned* part_wave;     // [part_cap] wave of each part (ascending)
    unsigned char* clear;    // [HR_BIN_MAX_WAVES] 1: the shadow is cleared before this wave
    uint2* out;              // [out_cap] bucketed accesses {tid, op << 16 | word within the segment}, or
                             // when ctl->bin_pack4 as unsigned tid << (SEG_SHIFT + 2) | op << SEG_SHIFT | word
    unsigned long long out_cap;
    unsigned n_seg;          // segments of this check's region
    unsigned seg_cap;        // segments the table holds
    unsigned part_cap;       // parts the table holds: HR_BIN_MAX_WAVES + slices - 1
    unsigned clusters;       // scatter clusters (hr_bin_shape())
    unsigned sub;            // count slices per cluster slice
    unsigned slices;         // count slices (CTAs of the count pass): clusters * sub
    unsigned pow2;           // 1: block size and warp size are powers of two (bit-operation FSM step)
};

// Scratch of one check (device memory): job table, pre-pass counts, wave
// table, stage list and control block.
struct hr_work {
    hr_jobd* jobs;                   // [max_jobs]
    unsigned* counts;                // [max_intervals] boundaries per interval, then their offsets
    unsigned long long* wave_start;  // [max_waves] first record (index into the job's trace)
    unsigned long long* wave_end;    // [max_waves] one past the last record
    unsigned long long* wave_key;    // [max_waves] rebased wave key
    hr_stage* stages;                // [2 * max_waves + 1]
    hr_ctl* ctl;
    unsigned max_waves;
    unsigned max_intervals;
    unsigned max_jobs;
    unsigned tile;                   // records per work item (set per kernel variant)
    unsigned consumers;              // per-warp completions per work item
    unsigned cas_cap;                // CAS retries before HR_ERR_CONTENTION
    unsigned long long wait_ns;      // bound of every device-side wait
    unsigned test_flags;             // HR_TEST_* hooks (tests only)
    unsigned views;                  // 1: a device view of the checked region exists (inline writes may
                                     // carry kernel ordinals the region's last key does not know)
    hr_bin bin;                      // binned checker scratch (variant HR_BIN_VARIANT only)
};

constexpr unsigned long long HR_DEFAULT_WAIT_NS = 4000000000ull;  // 4 s
constexpr unsigned HR_DEFAULT_CAS_CAP = 4096;

// bytes of an hr_work scratch block for the given capacities (256-B aligned parts)
inline size_t hr_work_bytes(unsigned max_jobs, unsigned max_intervals, unsigned max_waves)
{
    auto a = [](size_t x) { return (x + 255) & ~size_t(255); };
    return a(sizeof(hr_ctl)) + a((size_t)max_jobs * sizeof(hr_jobd)) + a((size_t)max_intervals * 4) +
           3 * a((size_t)max_waves * 8) + a((size_t)(2 * max_waves + 1) * sizeof(hr_stage));
}

// carve an hr_work out of `mem` (hr_work_bytes(...) bytes, 256-B aligned)
inline hr_work hr_work_at(void* mem, unsigned max_jobs, unsigned max_intervals, unsigned max_waves)
{
    auto a = [](size_t x) { return (x + 255) & ~size_t(255); };
    char* p = (char*)mem;
    hr_work w{};
    w.ctl = (hr_ctl*)p;
    p += a(sizeof(hr_ctl));
    w.jobs = (hr_jobd*)p;
    p += a((size_t)max_jobs * sizeof(hr_jobd));
    w.counts = (unsigned*)p;
    p += a((size_t)max_intervals * 4);
    w.wave_start = (unsigned long long*)p;
    p += a((size_t)max_waves * 8);
    w.wave_end = (unsigned long long*)p;
    p += a((size_t)max_waves * 8);
    w.wave_key = (unsigned long long*)p;
    p += a((size_t)max_waves * 8);
    w.stages = (hr_stage*)p;
    w.max_waves = max_waves;
    w.max_intervals = max_intervals;
    w.max_jobs = max_jobs;
    w.cas_cap = HR_DEFAULT_CAS_CAP;
    w.wait_ns = HR_DEFAULT_WAIT_NS;
    w.test_flags = 0;
    return w;
}

constexpr unsigned HR_MAX_BATCH = 512;  // jobs per batched launch

// Kernel variants (chosen by hr_set_variant / hr_autotune): consumer warps per
// CTA, records per consumer lane, warp aggregation.  Even ids aggregate; the
// odd id after each is the same shape without aggregation.
struct hr_variant {
    int aggregate;
    int rpl;         // records per consumer lane per tile
    int consumers;   // consumer warps per CTA (plus one producer warp)
};
constexpr hr_variant HR_VARIANTS[] = {{1, 4, 8}, {0, 4, 8}, {1, 2, 8}, {0, 2, 8}, {1, 1, 8}, {0, 1, 8}};
constexpr unsigned HR_N_SHAPES = sizeof(HR_VARIANTS) / sizeof(HR_VARIANTS[0]);
// The binned checker (hr_binned.cu): single-trace checks of first-race regions
// only; batches, and checks it cannot take, run the per-wave checker of shape 3.
constexpr unsigned HR_BIN_VARIANT = HR_N_SHAPES;
constexpr unsigned HR_BIN_FALLBACK = 3;
constexpr unsigned HR_N_VARIANTS = HR_N_SHAPES + 1;  // ids a caller may choose
// Internal id of the checker that also carries the every-epoch path (shape of
// variant 3); checks on regions in that report mode use it.
constexpr unsigned HR_EVERY_EPOCH_VARIANT = HR_N_VARIANTS;
constexpr unsigned hr_variant_consumers(unsigned v)
{
    return v == HR_EVERY_EPOCH_VARIANT ? 8u
                                       : (unsigned)HR_VARIANTS[v == HR_BIN_VARIANT ? HR_BIN_FALLBACK : v].consumers;
}
constexpr unsigned hr_variant_tile(unsigned v)
{
    return v == HR_EVERY_EPOCH_VARIANT ? 8u * 32u * 2u
           : v == HR_BIN_VARIANT       ? hr_variant_tile(HR_BIN_FALLBACK)
                                       : HR_VARIANTS[v].consumers * 32u * HR_VARIANTS[v].rpl;
}
#ifndef HR_RING_DEPTH
#define HR_RING_DEPTH 2
#endif
#ifndef HR_BATCH
#define HR_BATCH 1
#endif
#ifndef HR_WAIT_SLEEP_MAX_NS
#define HR_WAIT_SLEEP_MAX_NS 1024  // longest back-off between polls of a stage counter
#endif
#ifndef HR_MIN_CTAS
#define HR_MIN_CTAS 3
#endif
constexpr int HR_RING = HR_RING_DEPTH;                   // tiles in flight in shared memory
constexpr unsigned HR_TICKET_BATCH = HR_BATCH;           // tiles a producer claims per ticket
constexpr unsigned HR_CLEAR_WORDS = 1u << 16;  // shadow words per clear item
constexpr unsigned HR_MAX_INTERVALS = 1u << 16;      // pre-pass intervals of a single-trace check
constexpr unsigned HR_BATCH_INTERVALS = 1u << 18;    // pre-pass intervals of a batch
constexpr unsigned long long HR_KEY_MASK = 0xFFFFFFFFFFFFull;

// kernel launch helpers (hr_kernels.cu)
// Check n_jobs jobs (1..HR_MAX_BATCH) on the regions of d_regions with the
// scratch w.  Jobs must name distinct regions and hold n > 0 records.
// *launches (if not NULL) receives the kernels launched: 2 for a small single
// trace (one-CTA pre-pass), 5 otherwise.
cudaError_t hr_launch_jobs(hr_region_dev* d_regions, const hr_work& w, const hr_jobd* jobs, unsigned n_jobs,
                           const unsigned char* d_table, unsigned variant, cudaStream_t stream,
                           cudaEvent_t before_check, unsigned* launches = nullptr);
// interval size and count for a job of n records when it may use up to budget intervals
void hr_plan_intervals(unsigned long long n, unsigned budget, unsigned* G, unsigned* n_int);
int hr_check_grid_size(unsigned variant);
constexpr unsigned HR_SMALL_INTERVALS = 4096;  // pre-pass intervals of a single trace (the one-CTA pre-pass)
// The binned checker's five launches (hr_binned.cu), queued after the pre-pass
// of a single-job check; the per-wave checker queued after them finds no items
// when they took the check.
cudaError_t hr_launch_binned(hr_region_dev* d_regions, const hr_work& w, const unsigned char* d_table,
                             cudaStream_t stream);
// The binned checker's streaming shape: as many scatter clusters as fit at once,
// and count slices per cluster slice so that the count pass fills the SMs.
void hr_bin_shape(unsigned* clusters, unsigned* sub);
// bytes of a region's binned-checker tables (without the access buffer)
inline size_t hr_bin_table_bytes(unsigned seg_cap, unsigned part_cap)
{
    auto a = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t e = (size_t)seg_cap * part_cap;
    return a(e * 4) + a((e / HR_BIN_SCAN + 1) * 4) + a((size_t)part_cap * 4) + a(HR_BIN_MAX_WAVES);
}
cudaError_t hr_launch_sync_kernel(hr_region_dev* d_region, cudaStream_t stream);
cudaError_t hr_launch_reset(hr_region_dev* d_region, unsigned long long* shadow, unsigned long long shadow_bytes,
                            cudaStream_t stream);
cudaError_t hr_launch_reconfigure(hr_region_dev* d_region, unsigned long long n_words, hr_geom geom,
                                  cudaStream_t stream);
cudaError_t hr_launch_set_filter(hr_region_dev* d_region, hr_filter filter, cudaStream_t stream);
