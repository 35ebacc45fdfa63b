// hr_kernels.cu - the trace checker's device code (sm_103a).
//
// One hr_check_trace call runs five launches on the caller's stream:
//   1. hr_scan_intervals   : per interval of G records, count wave boundaries
//                            (a wave is a run of equal (kernel, bc, wc) keys);
//                            only intervals whose two end keys differ are read
//   2. hr_scan_counts      : exclusive scan of the counts (one CTA)
//   3. hr_write_waves      : wave start offsets and keys
//   4. hr_build_stages     : work stages: per wave an optional shadow clear
//                            (kernel-tag group change) then its record tiles
//   5. hr_check_kernel     : persistent CTAs take work items in ticket order;
//                            an item waits (bounded) until the previous stage
//                            is complete, so waves are applied in wave order —
//                            an order consistent with happens-before (Sec. II-B:
//                            every ordered pair differs in kernel, bc or wc)
// Inside a wave every cross-thread pair is unordered, so any order of its
// records is a valid execution order; each record is applied with the FSM step
// of Algorithm 1 (hr_fsm_step) and a 64-bit atomicCAS on its shadow word.
#include <cuda_runtime.h>

#include "hr_internal.h"

namespace {

constexpr unsigned long long HR_WAIT_NS = 4000000000ull;  // bounded wait: 4 s

// wave key (kernel, bc, wc) of record i; kb is the caller's kernel base, already shifted by 32
__device__ __forceinline__ unsigned long long key_at(const hr_record* t, unsigned long long i,
                                                     unsigned long long kb)
{
    const unsigned long long* p = reinterpret_cast<const unsigned long long*>(t + i) + 1;
    return (__ldg(p) & HR_KEY_MASK) + kb;
}

__device__ __forceinline__ uint4 ld_stream(const hr_record* p)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
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

// ------------------------------------------------------------ wave discovery

__global__ void hr_scan_intervals(const hr_record* __restrict__ trace, unsigned long long n, unsigned G,
                                  unsigned n_int, unsigned* __restrict__ counts, hr_region_dev* region,
                                  unsigned long long kb)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned n_warps = (gridDim.x * blockDim.x) >> 5;
    for (unsigned i = warp; i < n_int; i += n_warps) {
        const unsigned long long beg = (unsigned long long)i * G;
        const unsigned long long end = min(n, beg + G);
        int need = 0;
        if (lane == 0) need = (i == 0) || key_at(trace, beg - 1, kb) != key_at(trace, end - 1, kb);
        need = __shfl_sync(0xffffffffu, need, 0);
        unsigned cnt = 0;
        if (need) {
            bool bad = false;
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
            if (bad) hr_set_error(&region->error, HR_ERR_ORDER);
            for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        }
        if (lane == 0) counts[i] = cnt;
    }
}

// block-wide exclusive scan of one value per thread (blockDim.x == 1024)
__device__ unsigned block_exclusive_scan(unsigned v, unsigned* total)
{
    __shared__ unsigned s_warp[32];
    const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned s = s_warp[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= (unsigned)o) s += y;
        }
        s_warp[lane] = s;
    }
    __syncthreads();
    const unsigned before = (wid ? s_warp[wid - 1] : 0u) + x - v;
    *total = s_warp[31];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(1024) hr_scan_counts(unsigned* counts, unsigned n_int, hr_work w,
                                                       hr_region_dev* region)
{
    const unsigned per = (n_int + 1023) / 1024;
    const unsigned b = threadIdx.x * per, e = min(n_int, b + per);
    unsigned local = 0;
    for (unsigned i = b; i < e; ++i) local += counts[i];
    unsigned total;
    unsigned run = block_exclusive_scan(local, &total);
    for (unsigned i = b; i < e; ++i) {
        const unsigned c = counts[i];
        counts[i] = run;
        run += c;
    }
    if (threadIdx.x == 0) {
        w.ctl->ticket = 0;
        w.ctl->abort = 0;
        w.ctl->total_items = 0;
        w.ctl->n_stages = 0;
        if (total > w.max_waves) {
            hr_set_error(&region->error, HR_ERR_CAPACITY);
            total = 0;
        }
        w.ctl->n_waves = total;
    }
}

__global__ void hr_write_waves(const hr_record* __restrict__ trace, unsigned long long n, unsigned G,
                               unsigned n_int, hr_work w, unsigned long long kb)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned n_warps = (gridDim.x * blockDim.x) >> 5;
    const unsigned n_waves = w.ctl->n_waves;
    if (warp == 0 && lane == 0) w.wave_start[n_waves] = n;
    if (n_waves == 0) return;
    for (unsigned i = warp; i < n_int; i += n_warps) {
        const unsigned long long beg = (unsigned long long)i * G;
        const unsigned long long end = min(n, beg + G);
        const unsigned next = (i + 1 < n_int) ? w.counts[i + 1] : n_waves;
        unsigned off = w.counts[i];
        if (off == next) continue;  // no boundary in this interval
        for (unsigned long long c = beg; c < end; c += 32) {
            const unsigned long long p = c + lane;
            bool is_b = false;
            unsigned long long k = 0;
            if (p < end) {
                k = key_at(trace, p, kb);
                is_b = (p == 0) || k != key_at(trace, p - 1, kb);
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

__global__ void __launch_bounds__(1024) hr_build_stages(hr_work w, hr_region_dev* region)
{
    const unsigned n_waves = w.ctl->n_waves;
    const unsigned per = (n_waves + 1023) / 1024;
    const unsigned b = threadIdx.x * per, e = min(n_waves, b + per);
    const unsigned long long n_words = region->n_words;
    const unsigned clear_items = (unsigned)((n_words + HR_CLEAR_WORDS - 1) / HR_CLEAR_WORDS);
    const bool used = region->used != 0;
    const unsigned long long last_key = region->last_key;
    const bool failed = region->error != 0 || (n_waves > 0 && w.wave_key[0] < last_key);
    // pass 1: stages and items per thread chunk
    unsigned my_stages = 0, my_items = 0;
    for (unsigned i = b; i < e; ++i) {
        const unsigned long long kern = w.wave_key[i] >> 32;
        const unsigned long long prev = i ? (w.wave_key[i - 1] >> 32) : (last_key >> 32);
        const bool clear = (i > 0 || used) && (kern >> 3) != (prev >> 3);
        const unsigned long long len = w.wave_start[i + 1] - w.wave_start[i];
        my_stages += 1 + clear;
        my_items += (unsigned)((len + HR_TILE - 1) / HR_TILE) + (clear ? clear_items : 0);
    }
    unsigned tot_stages, tot_items;
    unsigned s = block_exclusive_scan(my_stages, &tot_stages);
    unsigned it = block_exclusive_scan(my_items, &tot_items);
    for (unsigned i = b; i < e; ++i) {
        const unsigned long long kern = w.wave_key[i] >> 32;
        const unsigned long long prev = i ? (w.wave_key[i - 1] >> 32) : (last_key >> 32);
        const bool clear = (i > 0 || used) && (kern >> 3) != (prev >> 3);
        const unsigned long long len = w.wave_start[i + 1] - w.wave_start[i];
        if (clear) {
            w.stages[s] = hr_stage{it, i, HR_STAGE_CLEAR, 0u};
            s++;
            it += clear_items;
        }
        w.stages[s] = hr_stage{it, i, HR_STAGE_RECORDS, 0u};
        s++;
        it += (unsigned)((len + HR_TILE - 1) / HR_TILE);
    }
    if (threadIdx.x == 0) {
        w.stages[tot_stages] = hr_stage{tot_items, n_waves, HR_STAGE_RECORDS, 0u};
        if (n_waves > 0 && w.wave_key[0] < last_key) hr_set_error(&region->error, HR_ERR_ORDER);
        w.ctl->n_stages = tot_stages;
        w.ctl->total_items = failed ? 0u : tot_items;
        if (!failed && n_waves > 0) {
            region->last_key = w.wave_key[n_waves - 1];
            region->used = 1;
        }
    }
}

// ------------------------------------------------------------ the FSM checker

struct Acc {
    unsigned tid;
    unsigned op;
};

// Fold the accesses of one lane group (lanes in `grp`, in lane order) into o.
__device__ __forceinline__ unsigned long long fold_group(unsigned long long o, unsigned grp, const Acc* acc,
                                                         unsigned bc, unsigned wc, unsigned ktag,
                                                         const hr_geom& g, const unsigned char* table,
                                                         unsigned* raced, unsigned* who)
{
    while (grp) {
        const unsigned l = __ffs(grp) - 1;
        grp &= grp - 1;
        unsigned r = 0;
        o = hr_fsm_step(o, acc[l].tid, acc[l].op, bc, wc, ktag, g, table, &r);
        if (r && !*raced) {
            *raced = r;
            *who = l;
        }
    }
    return o;
}

template <bool AGG>
__global__ void __launch_bounds__(HR_THREADS, 2) hr_check_kernel(hr_region_dev* __restrict__ region, hr_work w,
                                                              const hr_record* __restrict__ trace,
                                                              const unsigned char* __restrict__ gtable,
                                                              unsigned long long kb)
{
    __shared__ unsigned char s_table[2048];
    __shared__ Acc s_acc[HR_THREADS / 32][HR_RPT][32];
    __shared__ unsigned s_item, s_stage, s_skip;
    __shared__ unsigned long long s_cnt[4];

    reinterpret_cast<uint2*>(s_table)[threadIdx.x] = reinterpret_cast<const uint2*>(gtable)[threadIdx.x];
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0;
    const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const hr_geom g = region->geom;
    unsigned long long* __restrict__ shadow = region->shadow;
    const unsigned long long n_words = region->n_words;
    const unsigned total = w.ctl->total_items;
    unsigned hint = 0;
    unsigned long long c_acc = 0, c_cas = 0, c_retry = 0, c_merged = 0;
    __syncthreads();

    while (true) {
        if (threadIdx.x == 0) {
            const unsigned t = atomicAdd(&w.ctl->ticket, 1u);
            s_item = t;
            if (t < total) {
                unsigned s = hint;
                while (w.stages[s + 1].item_begin <= t) ++s;
                s_stage = s;
            }
        }
        __syncthreads();
        const unsigned t = s_item;
        if (t >= total) break;
        const unsigned s = s_stage;
        hint = s;
        const hr_stage st = w.stages[s];
        const unsigned item = t - st.item_begin;

        // stage the tile's records in registers before waiting on the previous stage
        uint4 rec[HR_RPT];
        unsigned long long rb = 0, re = 0, wkey = 0;
        if (st.type == HR_STAGE_RECORDS) {
            rb = w.wave_start[st.wave] + (unsigned long long)item * HR_TILE;
            re = min(rb + HR_TILE, w.wave_start[st.wave + 1]);
            wkey = w.wave_key[st.wave];
#pragma unroll
            for (int k = 0; k < HR_RPT; ++k) {
                const unsigned long long r = rb + (unsigned long long)k * HR_THREADS + threadIdx.x;
                rec[k] = r < re ? ld_stream(trace + r) : make_uint4(0, 0, 0, 0xFFFFFFFFu);
            }
        }

        if (threadIdx.x == 0) {
            bool ok = true;
            if (s > 0) {
                const unsigned need = st.item_begin - w.stages[s - 1].item_begin;
                const unsigned long long t0 = globaltimer();
                unsigned ns = 32;
                while (ld_acquire_u32(&w.stages[s - 1].done) < need) {
                    if (*(volatile unsigned*)&w.ctl->abort) { ok = false; break; }
                    if (globaltimer() - t0 > HR_WAIT_NS) {
                        atomicExch(&w.ctl->abort, 1u);
                        hr_set_error(&region->error, HR_ERR_TIMEOUT);
                        ok = false;
                        break;
                    }
                    __nanosleep(ns);
                    if (ns < 2048) ns <<= 1;
                }
            }
            s_skip = ok ? (*(volatile unsigned*)&region->error != 0 ? 1u : 0u) : 2u;
        }
        __syncthreads();
        const unsigned skip = s_skip;
        if (skip == 2) break;  // aborted: a bounded wait expired somewhere

        if (!skip && st.type == HR_STAGE_CLEAR) {
            const unsigned long long wb = (unsigned long long)item * HR_CLEAR_WORDS;
            const unsigned long long we = min(n_words, wb + HR_CLEAR_WORDS);
            for (unsigned long long i = wb + 2ull * threadIdx.x; i < we; i += 2ull * HR_THREADS) {
                if (i + 1 < we)
                    *reinterpret_cast<ulonglong2*>(shadow + i) = make_ulonglong2(0ull, 0ull);
                else
                    shadow[i] = 0ull;
            }
        } else if (!skip) {
            const unsigned bc = (unsigned)(wkey >> 16) & 0xFFFFu;
            const unsigned wc = (unsigned)wkey & 0xFFFFu;
            const unsigned kern = (unsigned)(wkey >> 32);
            const unsigned ktag = kern & 7u;
            unsigned err = 0;
            if (wc > HR_WC_MAX) err = HR_ERR_CLOCK_OVERFLOW;
            unsigned word[HR_RPT], grp[HR_RPT];
            bool act[HR_RPT];
#pragma unroll
            for (int k = 0; k < HR_RPT; ++k) {
                const uint4 v = rec[k];
                const unsigned op = (v.w >> 16) & 0xFFu;
                const unsigned flags = v.w >> 24;
                const bool in = rb + (unsigned long long)k * HR_THREADS + threadIdx.x < re;
                const unsigned long long key = (((unsigned long long)(v.w & 0xFFFFu) << 32) |
                                                ((unsigned long long)(v.z >> 16) << 16) | (v.z & 0xFFFFu)) + kb;
                bool a = in && op <= HR_A;
                if (in) {
                    if (key != wkey) err = HR_ERR_ORDER;
                    else if (op > HR_SYNCWARP || (op == HR_SYNCWARP && (flags & HR_RECFLAG_PARTIAL_MASK)))
                        err = HR_ERR_UNSUPPORTED;
                    else if (a && v.x >= n_words)
                        err = HR_ERR_RANGE;
                }
                a = a && key == wkey && v.x < n_words && wc <= HR_WC_MAX;
                act[k] = a;
                word[k] = v.x;
                s_acc[wid][k][lane] = Acc{v.y, op};
                if (AGG) {
                    const unsigned long long mk = a ? (unsigned long long)v.x : (0xFFFFFFFF00000000ull | lane);
                    grp[k] = __match_any_sync(0xffffffffu, mk);
                    if (a && (__ffs(grp[k]) - 1) != lane) {
                        act[k] = false;  // folded by the group leader
                        c_merged++;
                    }
                } else {
                    grp[k] = 1u << lane;
                }
            }
            if (err) hr_set_error(&region->error, err);
            __syncwarp();

            unsigned long long o[HR_RPT], nv[HR_RPT], prev[HR_RPT];
            unsigned raced[HR_RPT], who[HR_RPT];
#pragma unroll
            for (int k = 0; k < HR_RPT; ++k)
                if (act[k]) o[k] = hr_ld_relaxed(shadow + word[k]);
#pragma unroll
            for (int k = 0; k < HR_RPT; ++k) {
                raced[k] = 0;
                who[k] = lane;
                if (act[k]) {
                    c_acc += __popc(grp[k]);
                    nv[k] = fold_group(o[k], grp[k], s_acc[wid][k], bc, wc, ktag, g, s_table, &raced[k], &who[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < HR_RPT; ++k)
                if (act[k] && nv[k] != o[k]) prev[k] = atomicCAS(shadow + word[k], o[k], nv[k]);
#pragma unroll
            for (int k = 0; k < HR_RPT; ++k) {
                if (!act[k]) continue;
                bool done = nv[k] == o[k];
                if (!done) {
                    c_cas++;
                    done = prev[k] == o[k];
                    int tries = 0;
                    while (!done && tries < HR_CAS_RETRY_CAP) {
                        ++tries;
                        c_retry++;
                        o[k] = prev[k];
                        raced[k] = 0;
                        nv[k] = fold_group(o[k], grp[k], s_acc[wid][k], bc, wc, ktag, g, s_table, &raced[k],
                                           &who[k]);
                        if (nv[k] == o[k]) {
                            done = true;
                            break;
                        }
                        c_cas++;
                        prev[k] = atomicCAS(shadow + word[k], o[k], nv[k]);
                        done = prev[k] == o[k];
                    }
                    if (!done) hr_set_error(&region->error, HR_ERR_CONTENTION);
                    if (done && raced[k]) {
                        const Acc a = s_acc[wid][k][who[k]];
                        hr_append_race(region->ring, region->ring_cap, &region->n_races, &region->flags, word[k],
                                       a.tid, kern, bc, region->region, a.op, raced[k] - 1u);
                    }
                }
            }
            __syncwarp();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&w.stages[s].done, 1u);
        }
    }
    // counters: one atomic per CTA
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
        c_acc += __shfl_xor_sync(0xffffffffu, c_acc, o2);
        c_cas += __shfl_xor_sync(0xffffffffu, c_cas, o2);
        c_retry += __shfl_xor_sync(0xffffffffu, c_retry, o2);
        c_merged += __shfl_xor_sync(0xffffffffu, c_merged, o2);
    }
    if (lane == 0) {
        atomicAdd(&s_cnt[0], c_acc);
        atomicAdd(&s_cnt[1], c_cas);
        atomicAdd(&s_cnt[2], c_retry);
        atomicAdd(&s_cnt[3], c_merged);
    }
    __syncthreads();
    if (threadIdx.x < 4 && s_cnt[threadIdx.x]) atomicAdd(&region->counters[threadIdx.x], s_cnt[threadIdx.x]);
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

int g_grid[2] = {0, 0};

}  // namespace

int hr_check_grid_size(bool aggregate)
{
    int& cached = g_grid[aggregate ? 1 : 0];
    if (cached) return cached;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (aggregate)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hr_check_kernel<true>, HR_THREADS, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hr_check_kernel<false>, HR_THREADS, 0);
    if (per_sm < 1) per_sm = 1;
    cached = sms * per_sm;
    return cached;
}

cudaError_t hr_launch_check(hr_region_dev* d_region, const hr_work& w, const hr_record* trace,
                            unsigned long long n, unsigned kernel_base, const unsigned char* d_table,
                            bool aggregate, int grid, cudaStream_t stream, cudaEvent_t before_check)
{
    const unsigned long long kb = (unsigned long long)kernel_base << 32;
    unsigned G = 1024;
    while ((n + G - 1) / G > HR_MAX_INTERVALS) G <<= 1;
    const unsigned n_int = (unsigned)((n + G - 1) / G);
    const unsigned scan_blocks = (n_int + 7) / 8 < 4096 ? (n_int + 7) / 8 : 4096;
    hr_scan_intervals<<<scan_blocks, 256, 0, stream>>>(trace, n, G, n_int, w.counts, d_region, kb);
    hr_scan_counts<<<1, 1024, 0, stream>>>(w.counts, n_int, w, d_region);
    hr_write_waves<<<scan_blocks, 256, 0, stream>>>(trace, n, G, n_int, w, kb);
    hr_build_stages<<<1, 1024, 0, stream>>>(w, d_region);
    if (before_check) cudaEventRecord(before_check, stream);
    if (aggregate)
        hr_check_kernel<true><<<grid, HR_THREADS, 0, stream>>>(d_region, w, trace, d_table, kb);
    else
        hr_check_kernel<false><<<grid, HR_THREADS, 0, stream>>>(d_region, w, trace, d_table, kb);
    return cudaGetLastError();
}

cudaError_t hr_launch_sync_kernel(hr_region_dev* d_region, cudaStream_t stream)
{
    hr_sync_kernel<<<1, 1, 0, stream>>>(d_region);
    return cudaGetLastError();
}

cudaError_t hr_launch_reset(hr_region_dev* d_region, unsigned long long* shadow, unsigned long long n_words,
                            cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(shadow, 0, n_words * sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
    hr_reset_state<<<1, 1, 0, stream>>>(d_region);
    return cudaGetLastError();
}
