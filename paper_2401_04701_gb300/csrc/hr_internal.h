// hr_internal.h - device-side data structures shared by the kernels and the API.
#pragma once

#include <cstdint>

#include "../../include/hirace.h"
#include "../../include/hirace_device.cuh"

// Geometry with exact reciprocals and, when both sizes are powers of two, shifts.
inline hr_geom hr_make_geom(uint32_t block_dim, uint32_t warp_size)
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
    return g;
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
    unsigned int used;            // any record processed since init/reset
    unsigned int region;
    unsigned long long counters[4];  // accesses, CAS attempts, CAS retries, merged lanes
    hr_geom geom;
};

// Work stages of one check: per wave an optional shadow clear (when the kernel
// tag group changes) followed by the wave's record tiles.
enum { HR_STAGE_RECORDS = 0, HR_STAGE_CLEAR = 1 };

struct hr_stage {
    unsigned int item_begin;  // first global work-item index of the stage
    unsigned int wave;
    unsigned int type;
    unsigned int done;        // items of this stage finished
};

struct hr_ctl {
    unsigned int ticket;      // next work item
    unsigned int abort;       // set when a bounded wait expired
    unsigned int n_waves;
    unsigned int n_stages;
    unsigned int total_items;
    unsigned int n_intervals;
    unsigned int interval;    // records per pre-pass interval
    unsigned int pad;
};

// Scratch of one region's trace check (device memory).
struct hr_work {
    unsigned int* counts;          // [max_intervals] boundaries per interval, then their offsets
    unsigned long long* wave_start;  // [max_waves + 1]
    unsigned long long* wave_key;    // [max_waves]
    hr_stage* stages;                // [2 * max_waves + 1]
    hr_ctl* ctl;
    unsigned int max_waves;
    unsigned int max_intervals;
};

constexpr int HR_CONSUMERS = 8;                          // consumer warps per CTA
constexpr int HR_THREADS = (HR_CONSUMERS + 1) * 32;      // + one producer warp
constexpr int HR_RPL = 4;                                // records per consumer lane per tile
constexpr int HR_TILE = HR_CONSUMERS * 32 * HR_RPL;      // records per tile (one wave per tile)
#ifndef HR_RING_DEPTH
#define HR_RING_DEPTH 2
#endif
#ifndef HR_BATCH
#define HR_BATCH 1
#endif
#ifndef HR_MIN_CTAS
#define HR_MIN_CTAS 3
#endif
constexpr int HR_RING = HR_RING_DEPTH;                   // tiles in flight in shared memory
constexpr unsigned HR_TICKET_BATCH = HR_BATCH;           // tiles a producer claims per ticket
constexpr unsigned HR_CLEAR_WORDS = 1u << 16;  // shadow words per clear item
constexpr unsigned HR_MAX_INTERVALS = 1u << 16;
constexpr unsigned long long HR_KEY_MASK = 0xFFFFFFFFFFFFull;

// kernel launch helpers (hr_kernels.cu)
cudaError_t hr_launch_check(hr_region_dev* d_region, const hr_work& w, const hr_record* trace,
                            unsigned long long n, unsigned kernel_base, const unsigned char* d_table,
                            bool aggregate, int grid, cudaStream_t stream, cudaEvent_t before_check);
constexpr unsigned HR_LAUNCHES_PER_CHECK = 5;  // pre-pass (4) + checker (1)
int hr_check_grid_size(bool aggregate);
cudaError_t hr_launch_sync_kernel(hr_region_dev* d_region, cudaStream_t stream);
cudaError_t hr_launch_reset(hr_region_dev* d_region, unsigned long long* shadow, unsigned long long n_words,
                            cudaStream_t stream);
