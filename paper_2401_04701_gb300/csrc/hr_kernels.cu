// hr_kernels.cu - the trace checker's device code (sm_103a).
//
// A check covers one or more jobs (a job = one trace on one region).  It runs
// five launches on the caller's stream:
//   1. hr_scan_intervals : per pre-pass interval of a job's trace, count the
//                          wave boundaries (a wave is a run of equal
//                          (kernel, bc, wc) keys); an interval is read only
//                          when its two end keys differ
//   2. hr_scan_counts    : exclusive scan of the counts (one CTA): global wave
//                          numbers, each job's first wave and wave count
//   3. hr_write_waves    : wave start offsets and keys
//   4. hr_build_stages   : work stages per wave, an optional shadow clear
//                          (kernel-tag group change) then the record tiles;
//                          several jobs are interleaved wave-major
//   5. hr_check_kernel   : persistent CTAs take work items in ticket order; a
//                          stage waits (bounded) for the previous stage of the
//                          same job, so every region sees its waves in wave
//                          order: an order consistent with happens-before
//                          (Sec. II-B: every ordered pair differs in kernel,
//                          bc or wc)
// Inside a wave every cross-thread pair is unordered, so any order of its
// records is a valid execution order; each record is applied with the FSM step
// of Algorithm 1 (hr_fsm_step) and a 64-bit atomicCAS on its shadow word.
#include <cuda_runtime.h>

#include "hr_internal.h"

namespace {


template <unsigned CAP>
struct JobParams {
    unsigned n;
    hr_jobd job[CAP];
};

// wave key (kernel, bc, wc) of record i; kb is the caller's kernel base, already shifted by 32
__device__ __forceinline__ unsigned long long key_at(const hr_record* t, unsigned long long i,
                                                     unsigned long long kb)
{
    const unsigned long long* p = reinterpret_cast<const unsigned long long*>(t + i) + 1;
    return (__ldg(p) & HR_KEY_MASK) + kb;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// job holding global pre-pass interval i (jobs sorted by int_begin)
template <unsigned CAP>
__device__ __forceinline__ unsigned job_of_interval(const JobParams<CAP>& P, unsigned i)
{
    unsigned lo = 0, hi = P.n;
    while (hi - lo > 1) {
        const unsigned mid = (lo + hi) >> 1;
        if (P.job[mid].int_begin <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------------ wave discovery

template <unsigned CAP>
__global__ void hr_scan_intervals(const JobParams<CAP> P, unsigned total_int, hr_work w,
                                  hr_region_dev* __restrict__ regions)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned n_warps = (gridDim.x * blockDim.x) >> 5;
    if (blockIdx.x == 0) {
        for (unsigned j = threadIdx.x; j < P.n; j += blockDim.x) {
            hr_jobd jb = P.job[j];
            jb.done_ns = 0;
            w.jobs[j] = jb;
        }
        if (threadIdx.x == 0) {
            w.ctl->n_jobs = P.n;
            w.ctl->t0_ns = globaltimer();
        }
    }
    for (unsigned i = warp; i < total_int; i += n_warps) {
        const unsigned j = job_of_interval(P, i);
        const hr_jobd& jb = P.job[j];
        const hr_record* trace = jb.trace;
        const unsigned long long n = jb.n, kb = jb.kb;
        const unsigned local = i - jb.int_begin;
        const unsigned long long beg = (unsigned long long)local * jb.G;
        const unsigned long long end = min(n, beg + jb.G);
        int need = 0;
        if (lane == 0) need = (local == 0) || key_at(trace, beg - 1, kb) != key_at(trace, end - 1, kb);
        need = __shfl_sync(0xffffffffu, need, 0);
        unsigned cnt = 0;
        if (need) {
            bool bad = false;
#pragma unroll 8
            for (unsigned long long c = beg; c < end; c += 32) {
                const unsigned long long p = c + lane;
                if (p < end) {
                    const unsigned long long k = key_at(trace, p, kb);
                    if (p == 0) {
                        cnt++;
                    } else {
                        const unsigned long long kp = key_at(trace, p - 1, kb);
                        cnt += k != kp;
                        bad |= k < kp;
                    }
                }
            }
            if (bad) hr_set_error(&regions[jb.region].error, HR_ERR_ORDER);
            for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        }
        if (lane == 0) w.counts[i] = cnt;
    }
}

// block-wide exclusive scan of one value per thread (blockDim.x == 1024)
__device__ unsigned long long block_exclusive_scan(unsigned long long v, unsigned long long* total)
{
    __shared__ unsigned long long s_warp[32];
    const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long s = s_warp[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= (unsigned)o) s += y;
        }
        s_warp[lane] = s;
    }
    __syncthreads();
    const unsigned long long before = (wid ? s_warp[wid - 1] : 0ull) + x - v;
    *total = s_warp[31];
    __syncthreads();
    return before;
}

// Exclusive scan of the interval counts into wave offsets, each job's wave range,
// the control block's reset (one CTA of 1024 threads).
__device__ void scan_counts_body(hr_work& w, unsigned total_int, hr_region_dev* regions)
{
    const unsigned per = (total_int + 1023) / 1024;
    const unsigned b = threadIdx.x * per, e = min(total_int, b + per);
    unsigned local = 0;
#pragma unroll 8
    for (unsigned i = b; i < e; ++i) local += w.counts[i];
    unsigned long long total;
    unsigned run = (unsigned)block_exclusive_scan(local, &total);
#pragma unroll 8
    for (unsigned i = b; i < e; ++i) {
        const unsigned c = w.counts[i];
        w.counts[i] = run;
        run += c;
    }
    __syncthreads();
    const unsigned n_jobs = w.ctl->n_jobs;
    const bool over = total > w.max_waves;
    for (unsigned j = threadIdx.x; j < n_jobs; j += blockDim.x) {
        hr_jobd& jb = w.jobs[j];
        const unsigned first = w.counts[jb.int_begin];
        const unsigned next = jb.int_begin + jb.n_int < total_int ? w.counts[jb.int_begin + jb.n_int] : (unsigned)total;
        jb.wave_begin = over ? 0u : first;
        jb.n_waves = over ? 0u : next - first;
        if (over) hr_set_error(&regions[jb.region].error, HR_ERR_CAPACITY);
    }
    if (threadIdx.x == 0) {
        w.ctl->ticket = 0;
        w.ctl->abort = 0;
        w.ctl->total_items = 0;
        w.ctl->n_stages = 0;
        w.ctl->binned = 0;
        w.ctl->fresh = 0;
        w.ctl->bin_max_tid = 0;
        w.ctl->bin_max_seg = 0;
        w.ctl->bin_count = 0;
        w.ctl->n_waves = over ? 0u : (unsigned)total;
    }
}

__global__ void __launch_bounds__(1024) hr_scan_counts(hr_work w, unsigned total_int, hr_region_dev* regions)
{
    scan_counts_body(w, total_int, regions);
}

template <unsigned CAP>
__global__ void hr_write_waves(const JobParams<CAP> P, unsigned total_int, hr_work w)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned n_warps = (gridDim.x * blockDim.x) >> 5;
    const unsigned n_waves = w.ctl->n_waves;
    if (n_waves == 0) return;
    for (unsigned i = warp; i < total_int; i += n_warps) {
        const unsigned j = job_of_interval(P, i);
        const hr_jobd& jb = P.job[j];
        const unsigned long long kb = jb.kb;
        const unsigned local = i - jb.int_begin;
        const unsigned long long beg = (unsigned long long)local * jb.G;
        const unsigned long long end = min(jb.n, beg + jb.G);
        const unsigned next = (i + 1 < total_int) ? w.counts[i + 1] : n_waves;
        unsigned off = w.counts[i];
        if (off == next) continue;  // no boundary in this interval
#pragma unroll 8
        for (unsigned long long c = beg; c < end; c += 32) {
            const unsigned long long p = c + lane;
            bool is_b = false;
            unsigned long long k = 0;
            if (p < end) {
                k = key_at(jb.trace, p, kb);
                is_b = (p == 0) || k != key_at(jb.trace, p - 1, kb);
            }
            const unsigned mask = __ballot_sync(0xffffffffu, is_b);
            if (is_b) {
                const unsigned slot = off + __popc(mask & ((1u << lane) - 1u));
                if (slot < n_waves) {
                    w.wave_start[slot] = p;
                    w.wave_key[slot] = k;
                }
            }
            off += __popc(mask);
        }
    }
}

// stage and item counts of wave L of a job, and whether it starts with a clear
__device__ __forceinline__ void wave_plan(const hr_work& w, const hr_jobd& jb, const hr_region_dev& rg, unsigned L,
                                          bool* clear, unsigned* rec_items, unsigned* clr_items)
{
    const unsigned g = jb.wave_begin + L;
    const unsigned long long kern = w.wave_key[g] >> 32;
    const unsigned long long prev = L ? (w.wave_key[g - 1] >> 32) : (rg.last_key >> 32);
    // used == 2: the region's shadow holds unknown contents (a caller-owned
    // shadow handed to a one-shot check), so the first wave starts from a clear
    *clear = (L > 0 || rg.used) && ((kern >> 3) != (prev >> 3) || (L == 0 && rg.used == 2));
    const unsigned long long end = L + 1 < jb.n_waves ? w.wave_start[g + 1] : jb.n;
    w.wave_end[g] = end;
    *rec_items = (unsigned)((end - w.wave_start[g] + w.tile - 1) / w.tile);
    *clr_items = *clear ? (unsigned)((rg.n_words + HR_CLEAR_WORDS - 1) / HR_CLEAR_WORDS) : 0u;
}

// One job: stages follow its waves; threads take waves in parallel.
__device__ void stages_one_job(hr_work& w, hr_region_dev* regions)
{
    const hr_jobd jb = w.jobs[0];
    hr_region_dev& rg = regions[jb.region];
    const unsigned nw = jb.n_waves;
    const bool failed = rg.error != 0 || (nw > 0 && w.wave_key[jb.wave_begin] < rg.last_key);
    const unsigned per = (nw + 1023) / 1024;
    const unsigned b = threadIdx.x * per, e = min(nw, b + per);
    unsigned long long mine = 0;  // (stages << 32) | items
    for (unsigned L = b; L < e; ++L) {
        bool clear;
        unsigned ri, ci;
        wave_plan(w, jb, rg, L, &clear, &ri, &ci);
        mine += ((unsigned long long)(1 + clear) << 32) + ri + ci;
    }
    unsigned long long tot;
    const unsigned long long pre = block_exclusive_scan(mine, &tot);
    unsigned s = (unsigned)(pre >> 32), it = (unsigned)pre;
    for (unsigned L = b; L < e; ++L) {
        bool clear;
        unsigned ri, ci;
        wave_plan(w, jb, rg, L, &clear, &ri, &ci);
        const unsigned g = jb.wave_begin + L;
        if (clear) {
            w.stages[s] = hr_stage{it, g, HR_STAGE_CLEAR, 0u, s ? s - 1 : HR_NO_DEP, 0u, 0u, 0u};
            s++;
            it += ci;
        }
        w.stages[s] = hr_stage{it, g, HR_STAGE_RECORDS, 0u, s ? s - 1 : HR_NO_DEP, 0u, 0u, 0u};
        s++;
        it += ri;
    }
    __syncthreads();
    // dependency need = items of the previous stage (one completion per item)
    const unsigned n_st = (unsigned)(tot >> 32);
    for (unsigned i = threadIdx.x; i < n_st; i += blockDim.x)
        if (i > 0) w.stages[i].dep_need = w.stages[i].item_begin - w.stages[i - 1].item_begin;
    __syncthreads();
    // test hook: stage 1 waits for one completion more than stage 0 can give,
    // so its bounded wait must run out and report HR_ERR_TIMEOUT
    if (threadIdx.x == 0 && (w.test_flags & HR_TEST_HOLD_STAGE) && n_st > 1) w.stages[1].dep_need += 1;
    if (threadIdx.x == 0) {
        if (n_st > 0) w.stages[n_st - 1].last = 1u;
        w.stages[n_st] = hr_stage{(unsigned)tot, 0u, HR_STAGE_RECORDS, 0u, HR_NO_DEP, 0u, 0u, 0u};
        if (nw > 0 && w.wave_key[jb.wave_begin] < rg.last_key) hr_set_error(&rg.error, HR_ERR_ORDER);
        w.ctl->n_stages = n_st;
        w.ctl->total_items = failed ? 0u : (unsigned)tot;
        // a zero shadow (new or reset region), one cleared before the first wave
        // (used == 2), or one last written by an older kernel: nothing in it is live
        w.ctl->fresh = !failed && nw > 0 && !w.views &&
                       (rg.used != 1 || (w.wave_key[jb.wave_begin] >> 32) > (rg.last_key >> 32));
        if (!failed && nw > 0) {
            rg.last_key = w.wave_key[jb.wave_begin + nw - 1];
            rg.used = 1;
        }
    }
}

// Several jobs: stages interleaved wave-major (every job's wave 0, then every
// job's wave 1, ...), so jobs fill each other's wave-boundary bubbles.  Thread j
// owns job j.
__device__ void stages_many_jobs(hr_work& w, hr_region_dev* regions)
{
    const unsigned n_jobs = w.ctl->n_jobs;
    const unsigned j = threadIdx.x;
    hr_jobd jb{};
    bool failed = true;
    unsigned nw = 0;
    hr_region_dev* rg = nullptr;
    if (j < n_jobs) {
        jb = w.jobs[j];
        rg = &regions[jb.region];
        nw = jb.n_waves;
        failed = rg->error != 0 || (nw > 0 && w.wave_key[jb.wave_begin] < rg->last_key);
        if (nw > 0 && w.wave_key[jb.wave_begin] < rg->last_key) hr_set_error(&rg->error, HR_ERR_ORDER);
    }
    __shared__ unsigned s_max;
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    if (j < n_jobs && !failed) atomicMax(&s_max, nw);
    __syncthreads();
    const unsigned max_w = s_max;
    unsigned base_s = 0, base_i = 0, last = HR_NO_DEP, last_items = 0;
    for (unsigned L = 0; L < max_w; ++L) {
        const bool has = j < n_jobs && !failed && L < nw;
        bool clear = false;
        unsigned ri = 0, ci = 0;
        if (has) wave_plan(w, jb, *rg, L, &clear, &ri, &ci);
        const unsigned long long mine = has ? (((unsigned long long)(1 + clear) << 32) + ri + ci) : 0ull;
        unsigned long long tot;
        const unsigned long long pre = block_exclusive_scan(mine, &tot);
        if (has) {
            unsigned s = base_s + (unsigned)(pre >> 32), it = base_i + (unsigned)pre;
            const unsigned g = jb.wave_begin + L;
            if (clear) {
                w.stages[s] = hr_stage{it, g, HR_STAGE_CLEAR, 0u, last, last_items, j, 0u};
                last = s;
                last_items = ci;
                s++;
                it += ci;
            }
            w.stages[s] = hr_stage{it, g, HR_STAGE_RECORDS, 0u, last, last_items, j, 0u};
            last = s;
            last_items = ri;
        }
        base_s += (unsigned)(tot >> 32);
        base_i += (unsigned)tot;
    }
    if (j < n_jobs && !failed && nw > 0) {
        rg->last_key = w.wave_key[jb.wave_begin + nw - 1];
        rg->used = 1;
    }
    if (j < n_jobs && last != HR_NO_DEP) w.stages[last].last = 1u;
    if (threadIdx.x == 0) {
        w.stages[base_s] = hr_stage{base_i, 0u, HR_STAGE_RECORDS, 0u, HR_NO_DEP, 0u, 0u, 0u};
        w.ctl->n_stages = base_s;
        w.ctl->total_items = base_i;
    }
}

__global__ void __launch_bounds__(1024) hr_build_stages(hr_work w, hr_region_dev* regions)
{
    if (w.ctl->n_jobs == 1)
        stages_one_job(w, regions);
    else
        stages_many_jobs(w, regions);
}

// The wave boundaries of records [beg, end) of a trace (a boundary is a
// position p whose key differs from the key at p - 1; p = 0 is one), found by
// one warp without reading every record: from the key k at the current
// position, a 32-way search (each lane probes one position per round, the
// range shrinks 32-fold) finds the first later position whose key differs, so
// a boundary costs about log32(end - beg) rounds of one load per lane.  emit(p,
// key) is called by every lane for each boundary, in ascending order.  Returns
// false if a boundary's key is below the key before it (the trace is not wave
// sorted there); records that differ from their wave's key without forming a
// boundary are caught by the checkers, which compare every record with its
// wave's key.
template <class Emit>
__device__ __forceinline__ bool interval_boundaries(const hr_record* t, unsigned long long kb, unsigned long long beg,
                                                    unsigned long long end, Emit emit)
{
    const unsigned lane = threadIdx.x & 31;
    if (beg >= end) return true;
    bool ordered = true;
    unsigned long long lo = beg, k;
    if (beg == 0) {
        k = key_at(t, 0, kb);
        emit(0ull, k);
        lo = 1;
    } else {
        k = key_at(t, beg - 1, kb);
    }
    const unsigned long long k_end = key_at(t, end - 1, kb);
    while (lo < end && k_end != k) {
        // the first position in [lo, end) whose key differs from k: the key at h - 1 differs
        unsigned long long l = lo, h = end;
        while (h - l > 1) {
            const unsigned long long step = (h - l + 31) / 32;
            const unsigned long long x = min(l + (lane + 1) * step, h) - 1;
            const bool differs = key_at(t, x, kb) != k;
            const unsigned j = __ffs(__ballot_sync(0xffffffffu, differs)) - 1;  // some lane differs: x(31) = h - 1
            h = min(l + (j + 1) * step, h);
            l = l + j * step;
        }
        const unsigned long long kq = key_at(t, l, kb);
        ordered = ordered && kq > k;
        emit(l, kq);
        k = kq;
        lo = l + 1;
    }
    return ordered;
}

// The whole pre-pass of one small trace (at most HR_SMALL_INTERVALS intervals)
// in one CTA: the four kernels above as phases separated by block barriers, so
// a small check costs two launches instead of five.  Phase (a) finds the
// intervals holding a wave boundary (one lane per interval, two keys each),
// (b) counts each one's boundaries (a warp per interval), (c) scans the counts,
// (d) writes the wave table, (e) builds the stages.
__global__ void __launch_bounds__(1024) hr_prepass_small(const JobParams<1> P, unsigned total_int, hr_work w,
                                                         hr_region_dev* regions)
{
    __shared__ unsigned s_list[HR_SMALL_INTERVALS];  // intervals holding a boundary
    __shared__ unsigned s_n;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const hr_jobd& jb = P.job[0];
    const unsigned long long n = jb.n, kb = jb.kb, G = jb.G;
    if (threadIdx.x == 0) {
        hr_jobd j0 = jb;
        j0.done_ns = 0;
        w.jobs[0] = j0;
        w.ctl->n_jobs = 1;
        w.ctl->t0_ns = globaltimer();
        s_n = 0;
    }
    __syncthreads();
    // (a)
    for (unsigned i = threadIdx.x; i < total_int; i += blockDim.x) {
        const unsigned long long beg = (unsigned long long)i * G, end = min(n, beg + G);
        if (i == 0 || key_at(jb.trace, beg - 1, kb) != key_at(jb.trace, end - 1, kb))
            s_list[atomicAdd(&s_n, 1u)] = i;
        else
            w.counts[i] = 0;
    }
    __syncthreads();
    const unsigned n_need = s_n;
    // (b)
    for (unsigned q = warp; q < n_need; q += blockDim.x >> 5) {
        const unsigned i = s_list[q];
        const unsigned long long beg = (unsigned long long)i * G, end = min(n, beg + G);
        unsigned cnt = 0;
        const bool ordered = interval_boundaries(jb.trace, kb, beg, end, [&](unsigned long long, unsigned long long) {
            ++cnt;
        });
        if (!ordered && lane == 0) hr_set_error(&regions[jb.region].error, HR_ERR_ORDER);
        if (lane == 0) w.counts[i] = cnt;
    }
    __syncthreads();
    // (c)
    scan_counts_body(w, total_int, regions);
    __syncthreads();
    // (d)
    const unsigned n_waves = w.ctl->n_waves;
    for (unsigned q = warp; q < n_need && n_waves; q += blockDim.x >> 5) {
        const unsigned i = s_list[q];
        const unsigned long long beg = (unsigned long long)i * G, end = min(n, beg + G);
        unsigned off = w.counts[i];
        interval_boundaries(jb.trace, kb, beg, end, [&](unsigned long long p, unsigned long long k) {
            if (lane == 0 && off < n_waves) {
                w.wave_start[off] = p;
                w.wave_key[off] = k;
            }
            ++off;
        });
    }
    __syncthreads();
    // (e)
    stages_one_job(w, regions);
}

// ------------------------------------------------------------ the FSM checker
//
// Warp-specialised persistent CTAs.  One producer warp (lane 0) takes work
// items in ticket order and streams each tile of records into a shared-memory
// ring with a bulk asynchronous copy (cp.async.bulk, completion on an mbarrier,
// L2 evict-first so the stream does not push shadow lines out of L2).  Eight
// consumer warps take the tiles from the ring, release the slot as soon as
// their records sit in registers, and apply them to the shadow.  A tile of
// wave w may only touch the shadow once every tile of the previous stage is
// done (per-warp completion counts with release/acquire); while it waits, the
// warp touches its shadow words so they sit in L2.

struct TileInfo {
    unsigned long long rb, re, key;  // record range (in the job's trace) and wave key of the tile
    unsigned long long kb;           // the job's kernel base (shifted), to rebase record keys
    unsigned stage, type, item, valid;
    unsigned skip, dep, dep_need, region;
    unsigned ready;                   // the producer saw the dependency complete
    unsigned last;                    // the stage is its job's last (its completion is timed)
    unsigned pad[2];
};

struct Acc {
    unsigned tid;
    unsigned op;
};

template <int RPL, int CONS>
struct Shape {
    static constexpr int TILE = CONS * 32 * RPL;
    static constexpr int THREADS = (CONS + 1) * 32;
    static constexpr int SLOTS = CONS * RPL * 32;  // records a tile gives its consumer lanes
    static constexpr size_t REC = (size_t)HR_RING * TILE * sizeof(uint4);
    // records ring, FSM table, per-slot decoded access (tid, op), word and
    // (group mask, race), tile infos, full/empty mbarriers, tile-finish
    // counters, per-warp geometry and filter
    static constexpr size_t BYTES = REC + 2048 + (size_t)SLOTS * (sizeof(Acc) + 4 + 8) + HR_RING * sizeof(TileInfo) +
                                    2 * HR_RING * 8 + 2 * HR_RING * 4 + CONS * sizeof(hr_geom) +
                                    CONS * sizeof(hr_filter);
    static constexpr int MIN_CTAS = CONS >= 8 ? HR_MIN_CTAS : 4;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

__device__ __forceinline__ unsigned smem_add_acq_rel(unsigned* p, unsigned v)
{
    unsigned old;
    asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(smem_u32(p)), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned atom_add_release(unsigned* p, unsigned v)
{
    unsigned old;
    asm volatile("atom.release.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded mbarrier wait: gives up (and raises the abort flag) after wait_ns
// or when another CTA aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned* abort_flag, unsigned* err,
                                          unsigned long long wait_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (unsigned n = 0;; ++n) {
        if (mbar_try_wait(bar, parity)) return true;
        // The abort flag and the clock are looked at every 32 tries only: reading
        // the flag is a round trip to L2, and a phase that completes meanwhile
        // would be noticed only after it.  Each try is itself bounded, so the
        // wait stays bounded.
        if ((n & 31u) == 31u) {
            if (*(volatile unsigned*)abort_flag) return false;
            if (globaltimer() - t0 > wait_ns) {
                atomicExch(abort_flag, 1u);
                hr_set_error(err, HR_ERR_TIMEOUT);
                return false;
            }
        }
    }
}

// Bounded wait until a stage's completion count reaches `need`.
__device__ __forceinline__ bool stage_wait(const unsigned* done, unsigned need, unsigned* abort_flag, unsigned* err,
                                           unsigned long long wait_ns)
{
    const unsigned long long t0 = globaltimer();
    unsigned ns = 64;
    while (ld_acquire_u32(done) < need) {
        if (*(volatile unsigned*)abort_flag) return false;
        if (globaltimer() - t0 > wait_ns) {
            atomicExch(abort_flag, 1u);
            hr_set_error(err, HR_ERR_TIMEOUT);
            return false;
        }
        __nanosleep(ns);
        if (ns < HR_WAIT_SLEEP_MAX_NS) ns <<= 1;
    }
    return true;
}

// Result of folding accesses into a shadow value: the new value, 1 + the
// prior state when the fold entered RACE (else 0), and the lane whose access
// did it.  Returned by value so the callers' state stays in registers.
struct Fold {
    unsigned long long n;
    unsigned raced, who;
};

// Fold the accesses of one lane group (lanes in `grp`, in lane order) into o.
__device__ __forceinline__ Fold fold_group(unsigned long long o, unsigned grp, const Acc* acc, unsigned bc, unsigned wc,
                                        unsigned ktag, const hr_geom& g, const unsigned char* table)
{
    Fold f{o, 0u, threadIdx.x & 31};
    unsigned last_tid = ~0u, last_op = ~0u;
    while (grp) {
        const unsigned l = __ffs(grp) - 1;
        grp &= grp - 1;
        // the summary depends on the set of accesses: a repeat of the access
        // just applied (same thread, same op, same wave) changes nothing
        if (acc[l].tid == last_tid && acc[l].op == last_op) continue;
        last_tid = acc[l].tid;
        last_op = acc[l].op;
        unsigned r = 0;
        f.n = hr_fsm_step(f.n, acc[l].tid, acc[l].op, bc, wc, ktag, g, table, &r);
        if (r && !f.raced) {
            f.raced = r;
            f.who = l;
        }
    }
    return f;
}

// Outcome of the cold CAS path.
struct Retry {
    unsigned raced, who;
    unsigned attempts;  // extra CAS attempts
    unsigned ok;        // a CAS stuck (or the access needed none)
};

// Cold path: the first CAS lost a race (or validated a stale speculative
// load).  Re-fold from the value it returned until a CAS sticks or the retry
// cap is reached.
__device__ __forceinline__ Retry retry_cas(unsigned long long* shadow, unsigned word, unsigned long long seen,
                                        unsigned tid, unsigned op, unsigned grp, const Acc* acc, unsigned bc,
                                        unsigned wc, unsigned ktag, const hr_geom& g, const unsigned char* table,
                                        unsigned cap)
{
    const unsigned lane = threadIdx.x & 31;
    Retry r{0u, lane, 0u, 0u};
    for (unsigned tries = 0; tries < cap; ++tries) {
        const unsigned long long o = seen;
        Fold f{o, 0u, lane};
        if (grp == (1u << lane))
            f.n = hr_fsm_step(o, tid, op, bc, wc, ktag, g, table, &f.raced);
        else
            f = fold_group(o, grp, acc, bc, wc, ktag, g, table);
        r.raced = f.raced;
        r.who = f.who;
        if (f.n == o) {
            r.ok = 1;
            return r;
        }
        r.attempts++;
        seen = hr_shadow_cas(shadow, word, o, f.n, g);
        if (seen == o) {
            r.ok = 1;
            return r;
        }
    }
    return r;
}

// Every-epoch mode for a lane's RPL accesses at once (bit k of `act`: slot k
// holds one): the steps of hr_ep_apply, each over every slot before the next,
// so each step costs one round trip for all of them and one fence serves them
// all.  Per access: fold it into the summaries of the conflict kinds it holds
// (CAS loops), then a sequentially consistent fence, then read the summaries
// of the kinds it conflicts with; a conflicting holder is reported once per
// (word, kernel, epoch) through a CAS on the stamp word.  Of two concurrent
// conflicting accesses at least one therefore sees the other.  Returns 0 or
// HR_ERR_CONTENTION when a CAS loop reached `cap` tries.
template <int RPL>
__device__ __forceinline__ unsigned every_epoch_slots(unsigned long long* shadow, unsigned long long n_words,
                                                      unsigned act, const unsigned* idx, const unsigned* report_word,
                                                      const unsigned* tid, const unsigned* op, unsigned bc,
                                                      unsigned wc, unsigned kernel, const hr_geom& g,
                                                      hr_region_dev* region, unsigned cap)
{
    const unsigned ktag = kernel & 7u;
    unsigned err = 0;
    auto holds = [&](int k) { return op[k] == HR_R ? 1u : (op[k] == HR_A ? 2u : 3u); };
    auto against = [&](int k) { return op[k] == HR_R ? 2u : (op[k] == HR_A ? 1u : 3u); };
    // 1. the held kinds' summaries, all loaded at once, then every first CAS
    unsigned long long o[RPL][2], seen[RPL][2];
    unsigned casm = 0;  // bit 2k+b: a CAS went out on summary b of slot k
#pragma unroll
    for (int k = 0; k < RPL; ++k)
#pragma unroll
        for (int b = 0; b < 2; ++b)
            if (((act >> k) & 1u) && ((holds(k) >> b) & 1u)) o[k][b] = hr_ld_relaxed(shadow + b * n_words + idx[k]);
#pragma unroll
    for (int k = 0; k < RPL; ++k)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            if (!((act >> k) & 1u) || !((holds(k) >> b) & 1u)) continue;
            const unsigned long long n = hr_ep_update(o[k][b], tid[k], bc, wc, ktag, g);
            if (n == o[k][b]) continue;
            seen[k][b] = atomicCAS(shadow + b * n_words + idx[k], o[k][b], n);
            casm |= 1u << (2 * k + b);
        }
    // a CAS that lost: fold again into what it saw
#pragma unroll
    for (int k = 0; k < RPL; ++k)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            if (!((casm >> (2 * k + b)) & 1u) || seen[k][b] == o[k][b]) continue;
            unsigned long long* p = shadow + b * n_words + idx[k];
            unsigned long long cur = seen[k][b];
            bool ok = false;
            for (unsigned tries = 1; tries < cap; ++tries) {
                const unsigned long long n = hr_ep_update(cur, tid[k], bc, wc, ktag, g);
                if (n == cur) { ok = true; break; }
                const unsigned long long sv = atomicCAS(p, cur, n);
                if (sv == cur) { ok = true; break; }
                cur = sv;
            }
            if (!ok) {
                err = HR_ERR_CONTENTION;
                act &= ~(1u << k);  // this access is not applied: it reports nothing
            }
        }
    if (!act) return err;
    asm volatile("fence.sc.gpu;" ::: "memory");
    // 2. the conflicting kinds' summaries, all loaded at once
    unsigned long long sv[RPL][2];
#pragma unroll
    for (int k = 0; k < RPL; ++k)
#pragma unroll
        for (int b = 0; b < 2; ++b)
            if (((act >> k) & 1u) && ((against(k) >> b) & 1u)) sv[k][b] = hr_ld_relaxed(shadow + b * n_words + idx[k]);
    // 3. a conflicting holder: claim the (kernel, epoch) of the report
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
        if (!((act >> k) & 1u)) continue;
        unsigned prior = 0;
#pragma unroll
        for (int b = 0; b < 2; ++b)
            if (!prior && ((against(k) >> b) & 1u) && hr_ep_pred(sv[k][b], tid[k], bc, wc, ktag, g))
                prior = hr_ep_level(sv[k][b], ktag);
        if (!prior) continue;
        unsigned long long* st = shadow + 2 * n_words + idx[k];
        const unsigned long long mine = ((((unsigned long long)kernel) << 16) | bc) + 1ull;
        unsigned long long cur = hr_ld_relaxed(st);
        bool claimed = false;
        for (unsigned tries = 0; cur < mine && tries < cap; ++tries) {
            const unsigned long long x = atomicCAS(st, cur, mine);
            if (x == cur) { claimed = true; break; }
            cur = x;
        }
        if (claimed)
            hr_append_race(region->ring, region->ring_cap, &region->n_races, &region->flags, report_word[k], tid[k],
                           kernel, bc, region->region, op[k], prior);
        else if (cur < mine)
            err = HR_ERR_CONTENTION;
    }
    return err;
}

template <int TILE>
__device__ void producer_loop(hr_work& w, hr_region_dev* regions, uint4* s_rec, TileInfo* s_info, uint64_t* s_full,
                              uint64_t* s_empty)
{
    const uint64_t pol = policy_evict_first();
    const unsigned total = hr_bin_taken(w.ctl) ? 0u : w.ctl->total_items;  // binned: the work is done already
    unsigned s = 0, s_begin = 0, s_end = 0, type = 0, dep = HR_NO_DEP, dep_need = 0, region = 0, last = 0;
    unsigned long long w_start = 0, w_end = 0, key = 0, kb = 0;
    const hr_record* trace = nullptr;
    bool have = false, skip = false;
    unsigned pend = 0, pend_end = 0, polls = 0;
    unsigned known = HR_NO_DEP;  // last dependency seen complete
    // Tickets are claimed one batch ahead, so the claim's round trip to L2
    // overlaps the wait for a free slot instead of delaying every tile.  A
    // claimed tile only waits on stages of lower tickets, so holding one
    // blocks nobody.
    unsigned next = atomicAdd(&w.ctl->ticket, HR_TICKET_BATCH);
    for (unsigned it = 0;; ++it) {
        const unsigned b = it % HR_RING;
        if (it >= HR_RING &&
            !mbar_wait(&s_empty[b], ((it / HR_RING) - 1) & 1u, &w.ctl->abort, &regions[region].error, w.wait_ns)) {
            s_info[b].valid = 0;
            mbar_arrive(&s_full[b]);
            return;
        }
        if (pend == pend_end) {  // take the batch claimed ahead, claim the one after it
            pend = next;
            pend_end = min(pend + HR_TICKET_BATCH, total);
            if (pend < total) next = atomicAdd(&w.ctl->ticket, HR_TICKET_BATCH);
            ++polls;
        }
        const unsigned t = pend++;
        if (t >= total || (polls % 8 == 0 && *(volatile unsigned*)&w.ctl->abort)) {
            s_info[b].valid = 0;
            mbar_arrive(&s_full[b]);
            return;
        }
        if (!have || t >= s_end) {  // move to the stage holding ticket t
            while (w.stages[s + 1].item_begin <= t) ++s;
            const hr_stage st = w.stages[s];
            s_begin = st.item_begin;
            s_end = w.stages[s + 1].item_begin;
            type = st.type;
            dep = st.dep;
            dep_need = st.dep_need;
            last = st.last;
            const hr_jobd jb = w.jobs[st.job];
            region = jb.region;
            trace = jb.trace;
            kb = jb.kb;
            w_start = w.wave_start[st.wave];
            w_end = w.wave_end[st.wave];
            key = w.wave_key[st.wave];  // already rebased by the pre-pass
            skip = *(volatile unsigned*)&regions[region].error != 0;
            have = true;
        } else if (polls % 8 == 0) {
            skip = *(volatile unsigned*)&regions[region].error != 0;
        }
        TileInfo info;
        info.valid = 1;
        info.stage = s;
        info.type = type;
        info.item = t - s_begin;
        info.dep = dep;
        info.dep_need = dep_need;
        info.last = last;
        // one look at the dependency here spares every consumer warp its own poll
        info.ready = dep == HR_NO_DEP || dep == known;
        if (!info.ready && ld_acquire_u32(&w.stages[dep].done) >= dep_need) {
            info.ready = 1;
            known = dep;
        }
        info.region = region;
        info.skip = skip;
        info.key = key;
        info.kb = kb;
        info.rb = w_start + (unsigned long long)info.item * TILE;
        info.re = min(info.rb + TILE, w_end);
        s_info[b] = info;
        if (type == HR_STAGE_RECORDS && !info.skip) {
            const uint32_t bytes = (uint32_t)(info.re - info.rb) * (uint32_t)sizeof(hr_record);
            mbar_arrive_tx(&s_full[b], bytes);
            bulk_g2s(s_rec + (size_t)b * TILE, trace + info.rb, bytes, &s_full[b], pol);
        } else {
            mbar_arrive(&s_full[b]);
        }
    }
}

template <bool AGG, int HR_RPL, int HR_CONSUMERS, bool EVERY>
__global__ void __launch_bounds__(Shape<HR_RPL, HR_CONSUMERS>::THREADS, Shape<HR_RPL, HR_CONSUMERS>::MIN_CTAS)
    hr_check_kernel(hr_region_dev* __restrict__ regions, hr_work w, const unsigned char* __restrict__ gtable)
{
    using S = Shape<HR_RPL, HR_CONSUMERS>;
    constexpr int HR_TILE = S::TILE;
    constexpr int HR_THREADS = S::THREADS;
    extern __shared__ __align__(128) unsigned char smem[];
    uint4* s_rec = reinterpret_cast<uint4*>(smem);                                  // [HR_RING][HR_TILE]
    unsigned char* s_table = smem + S::REC;                                         // [2048]
    Acc* s_acc = reinterpret_cast<Acc*>(s_table + 2048);                            // [SLOTS]: (tid, op)
    unsigned* s_word = reinterpret_cast<unsigned*>(s_acc + S::SLOTS);               // [SLOTS]: shadow index
    uint2* s_aux = reinterpret_cast<uint2*>(s_word + S::SLOTS);                     // [SLOTS]: (group, race)
    TileInfo* s_info = reinterpret_cast<TileInfo*>(s_aux + S::SLOTS);               // [HR_RING]
    uint64_t* s_full = reinterpret_cast<uint64_t*>(s_info + HR_RING);
    uint64_t* s_empty = s_full + HR_RING;
    unsigned* s_fin = reinterpret_cast<unsigned*>(s_empty + HR_RING);               // [2 * HR_RING]
    hr_geom* s_geom = reinterpret_cast<hr_geom*>(s_fin + 2 * HR_RING);              // [HR_CONSUMERS]
    hr_filter* s_filt = reinterpret_cast<hr_filter*>(s_geom + HR_CONSUMERS);        // [HR_CONSUMERS]

    const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (unsigned i = threadIdx.x; i < 256; i += HR_THREADS)
        reinterpret_cast<uint2*>(s_table)[i] = reinterpret_cast<const uint2*>(gtable)[i];
    if (threadIdx.x == 0) {
        for (int b = 0; b < HR_RING; ++b) {
            mbar_init(&s_full[b], 1);
            mbar_init(&s_empty[b], HR_CONSUMERS);
        }
        for (int b = 0; b < 2 * HR_RING; ++b) s_fin[b] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (wid == HR_CONSUMERS) {
        if (lane == 0) producer_loop<HR_TILE>(w, regions, s_rec, s_info, s_full, s_empty);
        return;
    }

    // ---- consumer warp
    unsigned cur = ~0u;  // region of the previous tile
    hr_region_dev* region = nullptr;
    // the region's geometry lives in this warp's shared slot (read per use, not held in registers)
    const hr_geom& g = s_geom[wid];
    const hr_filter& filt = s_filt[wid];
    bool filtering = false;  // the region's filter selects only part of the accesses
    unsigned long long* shadow = nullptr;
    unsigned long long n_words = 0;
    unsigned tid_hi = 0;     // tid bits the region's shadow packing cannot hold
    // this warp's slots: lane + 32 k holds the lane's k-th record of the tile
    Acc* my_acc = s_acc + (size_t)wid * HR_RPL * 32;
    unsigned* my_word = s_word + (size_t)wid * HR_RPL * 32;
    uint2* my_aux = s_aux + (size_t)wid * HR_RPL * 32;
    unsigned known = HR_NO_DEP;  // last dependency this warp has seen complete
    // diagnostics: this lane's counts since the warp last added them to the region
    unsigned lc_acc = 0, lc_cas = 0, lc_retry = 0, lc_merged = 0;
    auto flush = [&]() {
        unsigned long long v[4] = {lc_acc, lc_cas, lc_retry, lc_merged};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            for (int o2 = 16; o2 > 0; o2 >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o2);
            if (lane == 0 && region && v[i]) atomicAdd(&region->counters[i], v[i]);
        }
        lc_acc = lc_cas = lc_retry = lc_merged = 0;
    };
    // The warp's part of tile `tn` (stage `stage`, bit 31: the job's last) is
    // done: the CTA's last warp to finish the tile publishes one completion for
    // the stage.  Counters indexed by tile number mod 2*ring never mix two
    // tiles: a warp cannot finish tile tn+2*ring before every warp has
    // finished tile tn.
    auto publish = [&](unsigned tn, unsigned stage) {
        __syncwarp();
        if (lane == 0) {
            const unsigned old = smem_add_acq_rel(&s_fin[tn % (2 * HR_RING)], 1u);
            if ((old + 1u) % HR_CONSUMERS == 0) {
                hr_stage* st = &w.stages[stage & 0x7FFFFFFFu];
                if (stage >> 31) {
                    // the job's last stage: the tile that completes it stamps the job's end
                    const unsigned prev = atom_add_release(&st->done, 1u);
                    if (prev + 1u == st[1].item_begin - st->item_begin) w.jobs[st->job].done_ns = globaltimer();
                } else {
                    red_release_add(&st->done, 1u);
                }
            }
        }
    };
    // Bounded wait for the tile's dependency; false when the check is aborting.
    auto wait_dep = [&](unsigned dep, unsigned need) {
        bool ok = true;
        if (lane == 0) ok = stage_wait(&w.stages[dep].done, need, &w.ctl->abort, &region->error, w.wait_ns);
        ok = __shfl_sync(0xffffffffu, ok, 0) != 0;
        __syncwarp();
        if (ok) known = dep;
        return ok;
    };

    for (unsigned it = 0;; ++it) {
        const unsigned b = it % HR_RING;
        if (!mbar_wait(&s_full[b], (it / HR_RING) & 1u, &w.ctl->abort, region ? &region->error : &regions[0].error,
                       w.wait_ns))
            break;
        const TileInfo& ti = s_info[b];
        if (!ti.valid) break;
        const unsigned t_type = ti.type, t_skip = ti.skip, t_dep = ti.dep;
        const unsigned t_stage = ti.stage | (ti.last << 31);  // bit 31: the job's last stage
        const unsigned t_need = ti.dep_need, t_item = ti.item, t_region = ti.region, t_ready = ti.ready;
        const unsigned t_n = (unsigned)(ti.re - ti.rb);  // records in this tile (<= HR_TILE)
        const unsigned kern = (unsigned)(ti.key >> 32);  // wave key: kernel (rebased), bc, wc
        const unsigned bcwc = (unsigned)ti.key;
        const unsigned kb = (unsigned)(ti.kb >> 32);     // the job's kernel base
        const bool records = t_type == HR_STAGE_RECORDS && !t_skip;
        if (!records) {  // nothing to read from the slot
            __syncwarp();
            if (lane == 0) mbar_arrive(&s_empty[b]);
        }
        if (t_region != cur) {
            flush();
            cur = t_region;
            region = regions + cur;
            if (lane == 0) {
                s_geom[wid] = region->geom;
                s_filt[wid] = region->filter;
            }
            __syncwarp();
            filtering = hr_filter_active(filt);
            shadow = region->shadow;
            n_words = region->n_words;
            tid_hi = (g.shadow_bytes == 4 && g.tid_bits < 32) ? ~((1u << g.tid_bits) - 1u) : 0u;
        }

        bool ready = t_dep == HR_NO_DEP || t_dep == known || t_ready;
        if (!ready) {
            unsigned r = 0;
            if (lane == 0) r = ld_acquire_u32(&w.stages[t_dep].done) >= t_need;
            ready = __shfl_sync(0xffffffffu, r, 0) != 0;
            __syncwarp();
        }
        if (ready && t_dep != HR_NO_DEP) known = t_dep;

        if (t_type == HR_STAGE_CLEAR && !t_skip) {
            if (!ready && !wait_dep(t_dep, t_need)) break;
            // bytes [bb, be) of the shadow: 16-byte stores, a 4-byte tail
            const unsigned long long sb = g.shadow_bytes;
            const unsigned long long span = (unsigned long long)(HR_CLEAR_WORDS / HR_CONSUMERS) * sb;
            const unsigned long long bb = (unsigned long long)t_item * HR_CLEAR_WORDS * sb + wid * span;
            const unsigned long long be = min(n_words * sb, bb + span);
            unsigned char* base8 = reinterpret_cast<unsigned char*>(shadow);
            for (unsigned long long i = bb + 16ull * lane; i < be; i += 512ull) {
                if (i + 16 <= be)
                    *reinterpret_cast<ulonglong2*>(base8 + i) = make_ulonglong2(0ull, 0ull);
                else
                    for (unsigned long long j = i; j < be; j += 4) *reinterpret_cast<unsigned*>(base8 + j) = 0u;
            }
        } else if (records) {
            const unsigned bc = bcwc >> 16;
            const unsigned wc = bcwc & 0xFFFFu;
            const unsigned ktag = kern & 7u;
            // non-absorbing reports: only the EVERY instantiation carries that path
            const bool every = EVERY && g.report_mode == HR_REPORT_EVERY_EPOCH;
            // the wave's clocks fit the region's shadow packing (else every access overflows it)
            const bool clk_fit = g.shadow_bytes != 4 ? (bc <= HR_BC_MAX && wc <= HR_WC_MAX)
                                                     : ((wc >> hr_wc_bits(g)) == 0 && (bc >> hr_bc_bits(g)) == 0);
            // Phase 1: decode the lane's records, drop or group repeats (warp
            // aggregation), note each access in the warp's slots and issue every
            // shadow load of the tile at once.  When the previous stage is still
            // running the loads go out before waiting for it (they overlap the
            // wait) and may be stale: every CAS then goes out, so a stale value
            // fails and is refolded from the value the CAS returns.
            const uint4* trec = s_rec + (size_t)b * HR_TILE;
            const unsigned base = wid * 32 * HR_RPL + lane;
            unsigned err = 0;
            unsigned actm = 0;  // bit k: slot k applies an access (a group's leader applies the group)
            unsigned grpm = 0;  // bit k: slot k leads a group of distinct accesses to one word
            unsigned long long o[HR_RPL];
#pragma unroll
            for (int k = 0; k < HR_RPL; ++k) {
                const unsigned idx = base + k * 32;
                const bool in = idx < t_n;
                const uint4 v = in ? trec[idx] : make_uint4(0, 0, 0, 0xFFFFFFFFu);
                const unsigned op = (v.w >> 16) & 0xFFu;
                const unsigned flags = v.w >> 24;
                // record key (kernel + kernel base, bc, wc) against the wave's
                const bool same_wave = v.z == bcwc && (v.w & 0xFFFFu) + kb == kern;
                bool a = in && op <= HR_A;
                // selective monitoring: unmonitored accesses are skipped, a word window
                // maps words to shadow indices
                // (a symmetric group folds the access onto its representative: tidf, widx)
                unsigned widx = v.x, tidf = v.y;
                bool mon = true;
                if (filtering && a && same_wave) {
                    unsigned long long ix = v.x;
                    mon = hr_monitored(filt, g, &tidf, v.x, &ix);
                    widx = (unsigned)ix;
                }
                if (in) {
                    if (!same_wave) err = HR_ERR_ORDER;
                    else if (op > HR_SYNCWARP || (op == HR_SYNCWARP && (flags & HR_RECFLAG_PARTIAL_MASK)))
                        err = HR_ERR_UNSUPPORTED;
                    else if (a && mon && widx >= n_words)
                        err = HR_ERR_RANGE;
                }
                a = a && same_wave && mon && widx < n_words;
                if (a && (!clk_fit || (tidf & tid_hi))) {
                    err = HR_ERR_CLOCK_OVERFLOW;  // tid, bc or wc wider than the shadow packing
                    a = false;
                }
                lc_acc += a;
                if (AGG && !every) {
                    // lanes of this slot applying the same word
                    const unsigned am = __ballot_sync(0xffffffffu, a);
                    const unsigned mw = __match_any_sync(0xffffffffu, a ? widx : 0xFFFFFFFFu) & am;
                    if (__any_sync(0xffffffffu, a && mw != (1u << lane))) {
                        // an exact repeat (same word, thread, op, wave) of a lower lane's
                        // access adds nothing to the summary: drop it
                        const unsigned me =
                            __match_any_sync(0xffffffffu, ((unsigned long long)tidf << 32) | op) & mw;
                        if (a && (unsigned)(__ffs(me) - 1) != lane) {
                            a = false;
                            lc_merged++;
                        }
                        // distinct accesses to one word: the lowest lane folds them
                        const unsigned m = mw & __ballot_sync(0xffffffffu, a);
                        if (a && m != (1u << lane)) {
                            if ((unsigned)(__ffs(m) - 1) != lane) {
                                a = false;  // folded by the group leader
                                lc_merged++;
                            } else {
                                grpm |= 1u << k;
                                my_aux[k * 32 + lane].x = m;
                            }
                        }
                    }
                }
                my_acc[k * 32 + lane] = Acc{tidf, op};
                my_word[k * 32 + lane] = widx;
                if (a && !every) o[k] = hr_shadow_load(shadow, widx, g);
                actm |= (unsigned)a << k;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&s_empty[b]);  // decoded: the slot may be refilled
            if (err) hr_set_error(&region->error, err);

            if (every) {
                if (!ready && !wait_dep(t_dep, t_need)) break;
                unsigned ix[HR_RPL], rw[HR_RPL], tv[HR_RPL], ov[HR_RPL];
#pragma unroll
                for (int k = 0; k < HR_RPL; ++k) {
                    const Acc me = my_acc[k * 32 + lane];
                    ix[k] = my_word[k * 32 + lane];
                    rw[k] = ix[k] + (filtering ? (unsigned)filt.word_lo : 0u);
                    tv[k] = me.tid;
                    ov[k] = me.op;
                }
                const unsigned st = every_epoch_slots<HR_RPL>(shadow, n_words, actm, ix, rw, tv, ov, bc, wc, kern, g,
                                                              region, w.cas_cap);
                if (st) hr_set_error(&region->error, st);
            } else {
                const bool spec = !ready;
                if (!ready && !wait_dep(t_dep, t_need)) break;
                // Phase 2: fold each access into its loaded value and send out every
                // CAS of the tile before reading any of their results.
                unsigned long long seen[HR_RPL];
                unsigned casm = 0;  // bit k: a CAS went out for slot k
                unsigned racem = 0; // bit k: slot k's fold moves the word into RACE (details in my_aux.y)
#pragma unroll
                for (int k = 0; k < HR_RPL; ++k) {
                    if (!((actm >> k) & 1u)) continue;
                    unsigned r = 0, who = lane;
                    unsigned long long nv;
                    if (AGG && ((grpm >> k) & 1u)) {
                        const Fold f = fold_group(o[k], my_aux[k * 32 + lane].x, my_acc + k * 32, bc, wc, ktag, g,
                                                  s_table);
                        nv = f.n;
                        r = f.raced;
                        who = f.who;
                    } else {
                        const Acc me = my_acc[k * 32 + lane];
                        nv = hr_fsm_step(o[k], me.tid, me.op, bc, wc, ktag, g, s_table, &r);
                    }
                    if (spec || nv != o[k]) {
                        seen[k] = hr_shadow_cas(shadow, my_word[k * 32 + lane], o[k], nv, g);
                        casm |= 1u << k;
                        if (r) {
                            racem |= 1u << k;
                            my_aux[k * 32 + lane].y = r | (who << 8);
                        }
                    }
                }
                // Phase 3: a CAS that returned the value it expected stuck.  One that
                // lost mostly lost to an equal transition (another lane or CTA applied
                // the same access pattern first): the value seen then already absorbs
                // this access, which one inline look settles; otherwise refold and retry.
#pragma unroll
                for (int k = 0; k < HR_RPL; ++k) {
                    if (!((casm >> k) & 1u)) continue;
                    lc_cas++;
                    unsigned raced = 0, who = lane;
                    if ((racem >> k) & 1u) {
                        const unsigned y = my_aux[k * 32 + lane].y;
                        raced = y & 0xFFu;
                        who = y >> 8;
                    }
                    bool done = seen[k] == o[k];
                    if (!done) {
                        lc_retry++;
                        const Acc me = my_acc[k * 32 + lane];
                        const unsigned m = (AGG && ((grpm >> k) & 1u)) ? my_aux[k * 32 + lane].x : (1u << lane);
                        if (m == (1u << lane)) {
                            unsigned r2 = 0;
                            if (hr_fsm_step(seen[k], me.tid, me.op, bc, wc, ktag, g, s_table, &r2) == seen[k]) {
                                done = true;
                                raced = 0;  // no change: this access moved nothing into RACE
                                who = lane;
                            }
                        }
                        if (!done) {
                            const Retry rr = retry_cas(shadow, my_word[k * 32 + lane], seen[k], me.tid, me.op, m,
                                                       my_acc + k * 32, bc, wc, ktag, g, s_table, w.cas_cap);
                            lc_cas += rr.attempts;
                            raced = rr.raced;
                            who = rr.who;
                            done = rr.ok != 0;
                            if (!done) hr_set_error(&region->error, HR_ERR_CONTENTION);
                        }
                    }
                    if (done && raced) {
                        const Acc ra = my_acc[k * 32 + who];
                        const unsigned abs_word = my_word[k * 32 + lane] + (filtering ? (unsigned)filt.word_lo : 0u);
                        hr_append_race(region->ring, region->ring_cap, &region->n_races, &region->flags, abs_word,
                                       ra.tid, kern, bc, region->region, ra.op, raced - 1u);
                    }
                }
            }  // first-race mode
        }
        publish(it, t_stage);
    }
    flush();
}

__global__ void hr_sync_kernel(hr_region_dev* region)
{
    // kernel end: the next record must come from a later kernel ordinal
    const unsigned long long k = region->last_key >> 32;
    region->last_key = (k + 1) << 32;
    region->used = 1;
}

__global__ void hr_reset_state(hr_region_dev* region)
{
    region->n_races = 0;
    region->error = 0;
    region->flags = 0;
    region->last_key = 0;
    region->used = 0;
    for (int i = 0; i < 4; ++i) region->counters[i] = 0;
}

__global__ void hr_reconfigure_state(hr_region_dev* region, unsigned long long n_words, hr_geom geom)
{
    region->n_words = n_words;
    region->geom = geom;
    region->filter = hr_filter_all();
}

__global__ void hr_set_filter_state(hr_region_dev* region, hr_filter filter) { region->filter = filter; }

int g_grid[HR_N_VARIANTS + 1] = {};

template <bool AGG, int RPL, int CONS, bool EVERY = false>
int grid_for()
{
    using S = Shape<RPL, CONS>;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(hr_check_kernel<AGG, RPL, CONS, EVERY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)S::BYTES);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hr_check_kernel<AGG, RPL, CONS, EVERY>, S::THREADS,
                                                  S::BYTES);
    if (per_sm < 1) per_sm = 1;
    return sms * per_sm;
}

template <bool AGG, int RPL, int CONS, bool EVERY = false>
void launch_variant(int grid, hr_region_dev* d_regions, const hr_work& w, const unsigned char* d_table,
                    cudaStream_t stream)
{
    using S = Shape<RPL, CONS>;
    hr_check_kernel<AGG, RPL, CONS, EVERY><<<grid, S::THREADS, S::BYTES, stream>>>(d_regions, w, d_table);
}

}  // namespace

int hr_check_grid_size(unsigned variant)
{
    if (variant > HR_EVERY_EPOCH_VARIANT) variant = 0;
    if (variant == HR_BIN_VARIANT) variant = HR_BIN_FALLBACK;
    int& cached = g_grid[variant];
    if (cached) return cached;
    switch (variant) {
    case 0: cached = grid_for<true, 4, 8>(); break;
    case 1: cached = grid_for<false, 4, 8>(); break;
    case 2: cached = grid_for<true, 2, 8>(); break;
    case 3: cached = grid_for<false, 2, 8>(); break;
    case 4: cached = grid_for<true, 1, 8>(); break;
    case 5: cached = grid_for<false, 1, 8>(); break;
    default: cached = grid_for<false, 2, 8, true>(); break;
    }
    return cached;
}

void hr_plan_intervals(unsigned long long n, unsigned budget, unsigned* G, unsigned* n_int)
{
    unsigned g = 1024;
    if (budget < 1) budget = 1;
    while ((n + g - 1) / g > budget && g < (1u << 30)) g <<= 1;
    *G = g;
    *n_int = (unsigned)((n + g - 1) / g);
}

template <unsigned CAP>
static void launch_prepass(const JobParams<CAP>& P, unsigned total_int, hr_region_dev* d_regions, const hr_work& w,
                           cudaStream_t stream)
{
    const unsigned blocks = (total_int + 7) / 8 < 4096 ? (total_int + 7) / 8 : 4096;
    hr_scan_intervals<CAP><<<blocks, 256, 0, stream>>>(P, total_int, w, d_regions);
    hr_scan_counts<<<1, 1024, 0, stream>>>(w, total_int, d_regions);
    hr_write_waves<CAP><<<blocks, 256, 0, stream>>>(P, total_int, w);
    hr_build_stages<<<1, 1024, 0, stream>>>(w, d_regions);
}

cudaError_t hr_launch_jobs(hr_region_dev* d_regions, const hr_work& w_in, const hr_jobd* jobs, unsigned n_jobs,
                           const unsigned char* d_table, unsigned variant, cudaStream_t stream,
                           cudaEvent_t before_check, unsigned* launches)
{
    if (variant > HR_EVERY_EPOCH_VARIANT) return cudaErrorInvalidValue;
    const bool binned = variant == HR_BIN_VARIANT;
    if (binned && (n_jobs != 1 || !w_in.bin.table)) return cudaErrorInvalidValue;
    if (binned) variant = HR_BIN_FALLBACK;  // the per-wave checker runs after it (and finds no work when binned)
    hr_work w = w_in;
    w.tile = hr_variant_tile(variant);
    w.consumers = hr_variant_consumers(variant);
    const int grid = hr_check_grid_size(variant);
    if (n_jobs == 0 || n_jobs > HR_MAX_BATCH || n_jobs > w.max_jobs) return cudaErrorInvalidValue;
    const unsigned total_int = jobs[n_jobs - 1].int_begin + jobs[n_jobs - 1].n_int;
    if (total_int > w.max_intervals) return cudaErrorInvalidValue;
    unsigned prepass_launches = 4;
    if (n_jobs == 1) {
        JobParams<1> P;
        P.n = 1;
        P.job[0] = jobs[0];
        if (total_int <= HR_SMALL_INTERVALS) {  // the whole pre-pass in one CTA
            hr_prepass_small<<<1, 1024, 0, stream>>>(P, total_int, w, d_regions);
            prepass_launches = 1;
        } else {
            launch_prepass(P, total_int, d_regions, w, stream);
        }
    } else {
        static thread_local JobParams<HR_MAX_BATCH> P;  // 24 KB: off the stack; copied into the launch
        P.n = n_jobs;
        for (unsigned j = 0; j < n_jobs; ++j) P.job[j] = jobs[j];
        launch_prepass(P, total_int, d_regions, w, stream);
    }
    if (before_check) cudaEventRecord(before_check, stream);
    if (launches) *launches = prepass_launches + 1 + (binned ? 5 : 0);
    if (binned) {
        const cudaError_t e = hr_launch_binned(d_regions, w, d_table, stream);
        if (e != cudaSuccess) return e;
    }
    switch (variant) {
    case 0: launch_variant<true, 4, 8>(grid, d_regions, w, d_table, stream); break;
    case 1: launch_variant<false, 4, 8>(grid, d_regions, w, d_table, stream); break;
    case 2: launch_variant<true, 2, 8>(grid, d_regions, w, d_table, stream); break;
    case 3: launch_variant<false, 2, 8>(grid, d_regions, w, d_table, stream); break;
    case 4: launch_variant<true, 1, 8>(grid, d_regions, w, d_table, stream); break;
    case 5: launch_variant<false, 1, 8>(grid, d_regions, w, d_table, stream); break;
    default: launch_variant<false, 2, 8, true>(grid, d_regions, w, d_table, stream); break;
    }
    return cudaGetLastError();
}

cudaError_t hr_launch_reconfigure(hr_region_dev* d_region, unsigned long long n_words, hr_geom geom,
                                  cudaStream_t stream)
{
    hr_reconfigure_state<<<1, 1, 0, stream>>>(d_region, n_words, geom);
    return cudaGetLastError();
}

cudaError_t hr_launch_set_filter(hr_region_dev* d_region, hr_filter filter, cudaStream_t stream)
{
    hr_set_filter_state<<<1, 1, 0, stream>>>(d_region, filter);
    return cudaGetLastError();
}

cudaError_t hr_launch_sync_kernel(hr_region_dev* d_region, cudaStream_t stream)
{
    hr_sync_kernel<<<1, 1, 0, stream>>>(d_region);
    return cudaGetLastError();
}

cudaError_t hr_launch_reset(hr_region_dev* d_region, unsigned long long* shadow, unsigned long long shadow_bytes,
                            cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(shadow, 0, shadow_bytes, stream);
    if (e != cudaSuccess) return e;
    hr_reset_state<<<1, 1, 0, stream>>>(d_region);
    return cudaGetLastError();
}
