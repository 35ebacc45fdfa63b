// hr_binned.cu - the binned trace checker (variant HR_BIN_VARIANT, sm_103a).
//
// The per-wave checker (hr_kernels.cu) applies each wave's accesses to the
// shadow in HBM and orders the waves across the whole GPU with stage counters;
// every access then costs a random read-modify-write of an 8-byte shadow value
// and every wave boundary drains the GPU.  This checker organises the same
// work around the shadow instead.  The region's shadow is cut into segments of
// HR_BIN_SEG words, each access of the trace is moved into the bucket of its
// (segment, wave), and a thread group holds one segment's shadow in shared
// memory and applies its buckets in wave order, with a barrier of the group
// between waves.
//
// Why this is the same computation: Algorithm 1 folds the accesses of a word
// into its shadow value one at a time, and Sec. II-B orders two accesses only
// through a barrier or a kernel end, so every pair inside one wave (records of
// equal (kernel, bc, wc)) is unordered and any order of a wave's accesses is a
// valid execution order; processing the waves in order keeps every ordered
// pair in order.  A word's accesses all land in one segment, and the segment's
// group applies its buckets in wave order, so each word sees exactly what the
// per-wave checker would show it.  Buckets need no stable order, so accesses
// are appended with atomics.
//
// Launches after the shared pre-pass (wave table and stage list):
//   1. hr_bin_count     : one CTA per SM takes a contiguous slice of the trace;
//                         for each part (the slice's records of one wave) it
//                         validates the records (the per-wave checker's checks
//                         and errors) and counts the accesses per segment in a
//                         shared-memory histogram, then writes the histogram
//                         into the table column of that part
//   2. hr_bin_scan_sums : the sum of each block of the table; the per-wave
//                         shadow-clear flags; the "binned" flag; the accesses
//                         of the check and of its fullest segment, for the
//                         skew guard (hr_bin_taken)
//   3. hr_bin_scan      : exclusive scan of the table (segment-major, parts in
//                         trace order) into bucket offsets
//   4. hr_bin_scatter   : clusters of CTAs walk the same slices wave by wave;
//                         each access, packed to 4 or 8 bytes (tid, op, word
//                         within the segment), goes to its bucket's next slot
//                         (cursors in distributed shared memory: no global atomics)
//   5. hr_bin_groups    : persistent thread groups, one segment at a time: its
//                         shadow in shared memory (or zeros when nothing in it
//                         is live), its accesses in wave order with a
//                         shared-memory CAS per access, races appended to the
//                         region's ring, the segment written back
// A check with more than HR_BIN_MAX_WAVES waves is not binned: the flag stays
// clear and the per-wave checker launched after these kernels does the work.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <type_traits>

#include "hr_internal.h"

namespace cg = cooperative_groups;

namespace {

constexpr unsigned STREAM_THREADS = 1024;      // threads of the two streaming passes (one CTA per SM)
constexpr unsigned STREAM_R = 4;               // records each streaming thread loads per step
constexpr unsigned STREAM_STEP = STREAM_THREADS * STREAM_R;
constexpr unsigned SCAN_THREADS = 1024;
// 4-byte bucketed access: tid << (SEG_SHIFT + 2) | op << SEG_SHIFT | word within the segment
constexpr unsigned PACK4_TID_SHIFT = HR_BIN_SEG_SHIFT + 2;
constexpr unsigned PACK4_TID_LIMIT = 1u << (32 - PACK4_TID_SHIFT);

// whether this check is one the binned checker takes (read from the pre-pass
// results; every kernel below decides the same way)
__device__ __forceinline__ bool bin_fits(const hr_ctl* c)
{
    return c->n_jobs == 1 && c->total_items > 0 && c->n_waves >= 1 && c->n_waves <= HR_BIN_MAX_WAVES;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async8(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// wait until at most N of this thread's copy groups are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait_group()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Records of a streaming step: thread tx owns slots j * STREAM_THREADS + tx of
// a step (the same slots it processes), so a thread's copies are visible to it
// after its own wait and no block barrier is needed; two steps are in flight.
__device__ __forceinline__ void stream_issue(uint4* tile, const hr_record* trace, unsigned long long base,
                                             unsigned long long end)
{
#pragma unroll
    for (unsigned j = 0; j < STREAM_R; ++j) {
        const unsigned long long i = base + j * STREAM_THREADS + threadIdx.x;
        if (i < end) cp_async16(&tile[j * STREAM_THREADS + threadIdx.x], trace + i);
    }
    cp_async_commit();
}

// One record classified for the binned checker: the checks of the per-wave
// checker (wave key, op, filter, range, packing), its segment and packed form.
struct BinAcc {
    unsigned seg;
    uint2 rec;
    unsigned err;
    bool act;
};

// clocks_fit: the wave's bc and wc fit the region's packing (hr_fits without the tid)
__device__ __forceinline__ BinAcc bin_decode(const uint4 v, bool in, unsigned long long key, unsigned kb,
                                             const hr_geom& g, const hr_filter& f, bool filtering,
                                             unsigned long long n_words, bool clocks_fit)
{
    BinAcc r{0u, make_uint2(0u, 0u), 0u, false};
    const unsigned kern = (unsigned)(key >> 32), bcwc = (unsigned)key;
    const unsigned op = (v.w >> 16) & 0xFFu;
    const unsigned flags = v.w >> 24;
    const bool same_wave = v.z == bcwc && (v.w & 0xFFFFu) + kb == kern;
    bool a = in && op <= HR_A;
    // (a symmetric group folds the access onto its representative: tid, widx)
    unsigned widx = v.x, tid = v.y;
    bool mon = true;
    if (filtering && a && same_wave) {
        unsigned long long ix = v.x;
        mon = hr_monitored(f, g, &tid, v.x, &ix);
        widx = (unsigned)ix;
    }
    if (in) {
        if (!same_wave) r.err = HR_ERR_ORDER;
        else if (op > HR_SYNCWARP || (op == HR_SYNCWARP && (flags & HR_RECFLAG_PARTIAL_MASK)))
            r.err = HR_ERR_UNSUPPORTED;
        else if (a && mon && widx >= n_words)
            r.err = HR_ERR_RANGE;
    }
    a = a && same_wave && mon && widx < n_words;
    if (a && !(clocks_fit && (g.shadow_bytes != 4 || (tid >> g.tid_bits) == 0))) {
        r.err = HR_ERR_CLOCK_OVERFLOW;
        a = false;
    }
    r.act = a;
    r.seg = widx >> HR_BIN_SEG_SHIFT;
    r.rec = make_uint2(tid, (op << 16) | (widx & (HR_BIN_SEG - 1u)));
    return r;
}

__device__ __forceinline__ unsigned block_sum(unsigned v, unsigned* s_warp)
{
    const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if (lane == 0) s_warp[wid] = v;
    __syncthreads();
    unsigned t = 0;
    for (unsigned i = 0; i < (blockDim.x >> 5); ++i) t += s_warp[i];
    __syncthreads();
    return t;
}

// exclusive scan of one value per thread over the block (a multiple of 32 threads)
__device__ __forceinline__ unsigned block_exclusive(unsigned v, unsigned* s_warp)
{
    const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned s = lane < nw ? s_warp[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xFFFFFFFFu, s, o);
            if (lane >= (unsigned)o) s += y;
        }
        s_warp[lane] = s;
    }
    __syncthreads();
    const unsigned before = (wid ? s_warp[wid - 1] : 0u) + x - v;
    __syncthreads();
    return before;
}

// Shared-memory state of the two streaming passes: the job's wave table, this
// CTA's slice and its first part, and a per-segment array (histogram or cursors).
struct StreamSmem {
    unsigned long long start[HR_BIN_MAX_WAVES + 1];  // first record of each wave; start[W] = n
    unsigned long long key[HR_BIN_MAX_WAVES];        // rebased wave keys
    unsigned s_warp[32];
    unsigned p0, np, w0, n_parts;
    unsigned long long a, b;                         // this CTA's records [a, b)
    unsigned seg[HR_BIN_MAX_SEGS];
    uint4 tile[2][STREAM_STEP];                      // two steps of records in flight
};
constexpr size_t STREAM_SMEM = sizeof(StreamSmem);

// first wave holding record i (binary search)
__device__ __forceinline__ unsigned wave_find(const StreamSmem& S, unsigned W, unsigned long long i)
{
    unsigned lo = 0, hi = W;
    while (hi - lo > 1) {
        const unsigned mid = (lo + hi) >> 1;
        if (S.start[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// Count slice c: the trace is cut into one slice per scatter cluster, and each
// of those into `sub` count slices, so a cluster's records are the union of
// consecutive count slices.
__device__ __forceinline__ void count_slice(unsigned long long n, const hr_bin& bin, unsigned c,
                                            unsigned long long* a, unsigned long long* b)
{
    const unsigned long long per_cl = (n + bin.clusters - 1) / bin.clusters;
    const unsigned long long per_sub = (per_cl + bin.sub - 1) / bin.sub;
    const unsigned cl = c / bin.sub, j = c % bin.sub;
    const unsigned long long A = min(n, cl * per_cl), B = min(n, A + per_cl);
    *a = min(B, A + j * per_sub);
    *b = min(B, *a + per_sub);
}

// The wave table, then the slices of all count CTAs (thread c < slices
// measures slice c), their parts and this CTA's first part.
__device__ void stream_prologue(const hr_work& w, const hr_jobd& jb, unsigned W, StreamSmem& S)
{
    for (unsigned i = threadIdx.x; i < W; i += blockDim.x) {
        S.start[i] = w.wave_start[jb.wave_begin + i];
        S.key[i] = w.wave_key[jb.wave_begin + i];
    }
    if (threadIdx.x == 0) S.start[W] = jb.n;
    __syncthreads();
    const unsigned c = threadIdx.x;
    unsigned np = 0, w0 = 0;
    unsigned long long a = 0, b = 0;
    if (c < w.bin.slices) {
        count_slice(jb.n, w.bin, c, &a, &b);
        if (a < b) {
            w0 = wave_find(S, W, a);
            np = wave_find(S, W, b - 1) - w0 + 1;
        }
    }
    const unsigned before = block_exclusive(np, S.s_warp);
    if (c == blockIdx.x) {
        S.p0 = before;
        S.np = np;
        S.w0 = w0;
        S.a = a;
        S.b = b;
    }
    if (c == w.bin.slices - 1) S.n_parts = before + np;
    __syncthreads();
}

// ------------------------------------------------------------ 1. counts

__global__ void __launch_bounds__(STREAM_THREADS) hr_bin_count(hr_region_dev* __restrict__ regions, hr_work w)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StreamSmem& S = *reinterpret_cast<StreamSmem*>(smem_raw);
    if (!bin_fits(w.ctl)) return;
    const unsigned W = w.ctl->n_waves;
    const hr_jobd jb = w.jobs[0];
    hr_region_dev* rg = regions + jb.region;
    const hr_geom g = rg->geom;
    const hr_filter f = rg->filter;
    const bool filtering = hr_filter_active(f);
    const unsigned long long n_words = rg->n_words;
    const unsigned kb = (unsigned)(jb.kb >> 32);
    const unsigned n_seg = w.bin.n_seg;
    stream_prologue(w, jb, W, S);
    const unsigned P = S.n_parts, tx = threadIdx.x, lane = tx & 31;
    if (blockIdx.x == 0 && tx == 0) w.ctl->bin_parts = P;
    unsigned err = 0, max_tid = 0;
    for (unsigned k = 0; k < S.np; ++k) {
        const unsigned gw = S.w0 + k, part = S.p0 + k;
        const unsigned long long pa = max(S.a, S.start[gw]), pb = min(S.b, S.start[gw + 1]);
        const unsigned long long key = S.key[gw];
        const bool fit = hr_fits(0u, ((unsigned)key) >> 16, (unsigned)key & 0xFFFFu, g);
        for (unsigned i = tx; i < n_seg; i += STREAM_THREADS) S.seg[i] = 0u;
        if (tx == 0) w.bin.part_wave[part] = gw;
        __syncthreads();
        if (pa < pb) stream_issue(S.tile[0], jb.trace, pa, pb);
        unsigned buf = 0;
        for (unsigned long long base = pa; base < pb; base += STREAM_STEP, buf ^= 1u) {
            if (base + STREAM_STEP < pb) {
                stream_issue(S.tile[buf ^ 1u], jb.trace, base + STREAM_STEP, pb);
                cp_async_wait_group<1>();
            } else {
                cp_async_wait_group<0>();
            }
#pragma unroll
            for (unsigned j = 0; j < STREAM_R; ++j) {
                const bool in = base + j * STREAM_THREADS + tx < pb;
                const uint4 v = in ? S.tile[buf][j * STREAM_THREADS + tx] : make_uint4(0u, 0u, 0u, 0u);
                const BinAcc r = bin_decode(v, in, key, kb, g, f, filtering, n_words, fit);
                if (r.err) err = r.err;
                if (r.act) {
                    atomicAdd(&S.seg[r.seg], 1u);
                    max_tid = max(max_tid, r.rec.x);
                }
            }
        }
        __syncthreads();
        // the part's column of the table (every entry: the table is dense)
        for (unsigned i = tx; i < n_seg; i += STREAM_THREADS) w.bin.table[(size_t)i * P + part] = S.seg[i];
        __syncthreads();
    }
    if (err) hr_set_error(&rg->error, err);
    // the largest thread id decides the packing of the bucketed accesses
    for (int o = 16; o > 0; o >>= 1) max_tid = max(max_tid, __shfl_xor_sync(0xFFFFFFFFu, max_tid, o));
    if (lane == 0 && max_tid) atomicMax(&w.ctl->bin_max_tid, max_tid);
}

// ------------------------------------------------------------ 2-3. scan

__global__ void __launch_bounds__(SCAN_THREADS) hr_bin_scan_sums(hr_work w)
{
    __shared__ unsigned s_warp[32];
    if (!bin_fits(w.ctl)) return;
    if (blockIdx.x == 0) {
        // a wave's shadow clear is the stage right before its record stage
        const unsigned n_st = w.ctl->n_stages, wb = w.jobs[0].wave_begin;
        for (unsigned s = threadIdx.x; s < n_st; s += blockDim.x) {
            const hr_stage st = w.stages[s];
            if (st.type == HR_STAGE_RECORDS)
                w.bin.clear[st.wave - wb] = s > 0 && w.stages[s - 1].type == HR_STAGE_CLEAR;
        }
        // the largest bc and wc of the check's waves, for the working-shadow packing
        __shared__ unsigned s_max_bc, s_max_wc;
        if (threadIdx.x == 0) s_max_bc = s_max_wc = 0;
        __syncthreads();
        const unsigned W = w.ctl->n_waves, wb0 = w.jobs[0].wave_begin;
        for (unsigned i = threadIdx.x; i < W; i += blockDim.x) {
            const unsigned k = (unsigned)w.wave_key[wb0 + i];
            atomicMax(&s_max_bc, k >> 16);
            atomicMax(&s_max_wc, k & 0xFFFFu);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            w.ctl->binned = 1;
            const unsigned mt = w.ctl->bin_max_tid;
            w.ctl->bin_pack4 = mt < PACK4_TID_LIMIT;
            w.ctl->seg_ticket = 0;
            // a 4-byte working shadow (tid in tb bits, wc and bc in the rest of 24) when
            // nothing in the region is live and the check's tids and clocks fit it
            unsigned tb = 1;
            while (tb < 24 && (mt >> tb)) ++tb;
            const unsigned wcb = (24 - tb) / 2, bcb = 24 - tb - wcb;
            const bool fits = tb <= 22 && s_max_wc < (1u << wcb) && s_max_bc < (1u << bcb);
            w.ctl->bin_tbits = (w.ctl->fresh && fits) ? tb : 0u;
        }
    }
    const unsigned P = w.ctl->bin_parts, n_seg = w.bin.n_seg;
    const unsigned long long E = (unsigned long long)n_seg * P;
    const unsigned long long b0 = (unsigned long long)blockIdx.x * HR_BIN_SCAN;
    if (b0 >= E) return;
    unsigned v = 0;
    for (unsigned long long i = b0 + threadIdx.x; i < min(E, b0 + HR_BIN_SCAN); i += blockDim.x) v += w.bin.table[i];
    v = block_sum(v, s_warp);
    // the skew guard's inputs: the segments whose first entry lies in this block,
    // each summed whole by one warp (its row may run into the next block)
    const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned long long s_lo = (b0 + P - 1) / P;
    const unsigned long long s_hi = min((unsigned long long)n_seg, (min(E, b0 + HR_BIN_SCAN) + P - 1) / P);
    unsigned m = 0;
    for (unsigned long long sg = s_lo + wid; sg < s_hi; sg += blockDim.x >> 5) {
        unsigned t = 0;
        for (unsigned i = lane; i < P; i += 32) t += w.bin.table[sg * P + i];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
        m = max(m, t);
    }
    __shared__ unsigned s_max;
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    if (lane == 0 && m) atomicMax(&s_max, m);
    __syncthreads();
    if (threadIdx.x == 0) {  // one global atomic of each kind per block
        w.bin.sums[blockIdx.x] = v;
        if (v) atomicAdd(&w.ctl->bin_count, v);
        if (s_max) atomicMax(&w.ctl->bin_max_seg, s_max);
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) hr_bin_scan(hr_work w)
{
    __shared__ unsigned s_warp[32];
    if (!hr_bin_taken(w.ctl)) return;
    const unsigned long long E = (unsigned long long)w.bin.n_seg * w.ctl->bin_parts;
    const unsigned long long b0 = (unsigned long long)blockIdx.x * HR_BIN_SCAN;
    if (b0 >= E) return;
    unsigned part = 0;
    for (unsigned i = threadIdx.x; i < blockIdx.x; i += blockDim.x) part += w.bin.sums[i];
    const unsigned base = block_sum(part, s_warp);
    constexpr unsigned PER = HR_BIN_SCAN / SCAN_THREADS;
    const unsigned long long i0 = b0 + (unsigned long long)threadIdx.x * PER;
    unsigned c[PER], local = 0;
#pragma unroll
    for (unsigned k = 0; k < PER; ++k) {
        c[k] = i0 + k < E ? w.bin.table[i0 + k] : 0u;
        local += c[k];
    }
    const unsigned pre = block_exclusive(local, s_warp);
    unsigned run = base + pre;
#pragma unroll
    for (unsigned k = 0; k < PER; ++k) {
        if (i0 + k < E) {
            w.bin.table[i0 + k] = run;
            run += c[k];
        }
    }
    if (i0 < E && i0 + PER >= E) w.ctl->bin_total = run;  // the thread holding the last entry
}

// ------------------------------------------------------------ 4. scatter
//
// Clusters of HR_BIN_CLUSTER CTAs; a cluster's slice is the slices of its CTAs
// in the count pass, so a (cluster, wave) covers consecutive parts of the
// table and owns one contiguous range per segment, starting at the table entry
// of its first part.  The cluster walks its waves in order; for each, the
// segment cursors are spread over the cluster's shared memory (segment s on
// rank s % HR_BIN_CLUSTER) and every CTA appends its share of the wave's
// records with atomics on those cursors (distributed shared memory).  One
// bucket range per cluster is being filled at a time, so L2 holds one partly
// written sector per (cluster, segment) and merges the 4- or 8-byte stores.

constexpr unsigned CL = HR_BIN_CLUSTER;
constexpr unsigned SCATTER_R = 4;  // records per thread per step: their atomics are in flight together

struct ScatterSmem {
    unsigned long long start[HR_BIN_MAX_WAVES + 1];
    unsigned long long key[HR_BIN_MAX_WAVES];
    unsigned s_warp[32];
    unsigned p0[HR_BIN_MAX_SUB], w0[HR_BIN_MAX_SUB], np[HR_BIN_MAX_SUB];  // the cluster's count slices
    unsigned cur[HR_BIN_MAX_SEGS / CL];
};
constexpr size_t SCATTER_SMEM = sizeof(ScatterSmem);

__global__ void __cluster_dims__(HR_BIN_CLUSTER, 1, 1) __launch_bounds__(STREAM_THREADS)
    hr_bin_scatter(hr_region_dev* __restrict__ regions, hr_work w)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ScatterSmem& S = *reinterpret_cast<ScatterSmem*>(smem_raw);
    cg::cluster_group cluster = cg::this_cluster();
    if (!hr_bin_taken(w.ctl)) return;  // the same for every CTA: no remote access happens
    const unsigned W = w.ctl->n_waves, P = w.ctl->bin_parts;
    const hr_jobd jb = w.jobs[0];
    hr_region_dev* rg = regions + jb.region;
    if (*(volatile unsigned*)&rg->error) return;  // no writer runs now: the same for every CTA
    const hr_geom g = rg->geom;
    const hr_filter f = rg->filter;
    const bool filtering = hr_filter_active(f);
    const unsigned long long n_words = rg->n_words;
    const unsigned kb = (unsigned)(jb.kb >> 32);
    const unsigned n_seg = w.bin.n_seg, tx = threadIdx.x, lane = tx & 31;
    const unsigned rank = cluster.block_rank(), cl = blockIdx.x / CL, sub = w.bin.sub;
    for (unsigned i = tx; i < W; i += STREAM_THREADS) {
        S.start[i] = w.wave_start[jb.wave_begin + i];
        S.key[i] = w.wave_key[jb.wave_begin + i];
    }
    if (tx == 0) S.start[W] = jb.n;
    __syncthreads();
    // the count pass's slices and their parts
    {
        const unsigned c = tx;
        unsigned np = 0, w0 = 0;
        if (c < w.bin.slices) {
            unsigned long long a, b;
            count_slice(jb.n, w.bin, c, &a, &b);
            if (a < b) {
                unsigned lo = 0, hi = W;
                while (hi - lo > 1) { const unsigned mid = (lo + hi) >> 1; if (S.start[mid] <= a) lo = mid; else hi = mid; }
                w0 = lo;
                hi = W;
                while (hi - lo > 1) { const unsigned mid = (lo + hi) >> 1; if (S.start[mid] <= b - 1) lo = mid; else hi = mid; }
                np = lo - w0 + 1;
            }
        }
        const unsigned before = block_exclusive(np, S.s_warp);
        if (c >= cl * sub && c < (cl + 1) * sub) {
            S.p0[c - cl * sub] = before;
            S.w0[c - cl * sub] = w0;
            S.np[c - cl * sub] = np;
        }
        __syncthreads();
    }
    const unsigned long long per_cl = (jb.n + w.bin.clusters - 1) / w.bin.clusters;
    const unsigned long long A = min(jb.n, cl * per_cl), B = min(jb.n, A + per_cl);
    unsigned w_lo = W, w_hi = 0;  // waves of the cluster's slice
    for (unsigned r = 0; r < sub; ++r)
        if (S.np[r]) {
            w_lo = min(w_lo, S.w0[r]);
            w_hi = max(w_hi, S.w0[r] + S.np[r]);
        }
    const unsigned my_segs = (n_seg + CL - 1 - rank) / CL;  // segments s with s % CL == rank
    const bool pack4 = w.ctl->bin_pack4 != 0;
    unsigned* out4 = reinterpret_cast<unsigned*>(w.bin.out);
    for (unsigned gw = w_lo; gw < w_hi; ++gw) {
        // the cluster's first part of this wave: the first of its CTAs that met it
        unsigned fp = 0;
        for (unsigned r = sub; r-- > 0;)
            if (S.np[r] && S.w0[r] <= gw && gw < S.w0[r] + S.np[r]) fp = S.p0[r] + (gw - S.w0[r]);
        for (unsigned i = tx; i < my_segs; i += STREAM_THREADS) S.cur[i] = w.bin.table[(size_t)(i * CL + rank) * P + fp];
        cluster.sync();  // every cursor is loaded before any CTA adds to it
        const unsigned long long wa = max(A, S.start[gw]), wb = min(B, S.start[gw + 1]);
        const unsigned long long span = (wb - wa + CL - 1) / CL;
        const unsigned long long a = min(wb, wa + rank * span), b = min(wb, a + span);
        const unsigned long long key = S.key[gw];
        const bool fit = hr_fits(0u, ((unsigned)key) >> 16, (unsigned)key & 0xFFFFu, g);
        for (unsigned long long base = a; base < b; base += STREAM_STEP) {
            uint4 v[SCATTER_R];  // every record of the step in flight at once
#pragma unroll
            for (unsigned j = 0; j < SCATTER_R; ++j) {
                const unsigned long long i = base + j * STREAM_THREADS + tx;
                v[j] = i < b ? __ldcs(reinterpret_cast<const uint4*>(jb.trace + i)) : make_uint4(0u, 0u, 0u, 0u);
            }
            uint2 rec[SCATTER_R];
            unsigned pos[SCATTER_R], grp[SCATTER_R];
            bool act[SCATTER_R];
#pragma unroll
            for (unsigned j = 0; j < SCATTER_R; ++j) {
                const bool in = base + j * STREAM_THREADS + tx < b;
                const BinAcc r = bin_decode(v[j], in, key, kb, g, f, filtering, n_words, fit);
                const unsigned m = __match_any_sync(0xFFFFFFFFu, r.act ? r.seg : 0xFFFFFFFFu);
                pos[j] = 0;
                if (r.act && lane == (unsigned)(__ffs(m) - 1)) {
                    unsigned* c = cluster.map_shared_rank(&S.cur[r.seg / CL], r.seg % CL);
                    pos[j] = atomicAdd(c, (unsigned)__popc(m));
                }
                rec[j] = r.rec;
                grp[j] = m;
                act[j] = r.act;
            }
#pragma unroll
            for (unsigned j = 0; j < SCATTER_R; ++j) {
                const unsigned p = __shfl_sync(0xFFFFFFFFu, pos[j], __ffs(grp[j]) - 1);
                const unsigned slot = p + __popc(grp[j] & ((1u << lane) - 1u));
                if (act[j]) {
                    if (pack4) out4[slot] = (rec[j].x << PACK4_TID_SHIFT) | ((rec[j].y >> 16) << HR_BIN_SEG_SHIFT) |
                                            (rec[j].y & (HR_BIN_SEG - 1u));
                    else w.bin.out[slot] = rec[j];
                }
            }
        }
        cluster.sync();  // every add is done before the cursors are reloaded (or the CTAs exit)
    }
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

// ------------------------------------------------------------ 5. segments, persistent groups
//
// One CTA of 1024 threads per SM, cut into independent thread groups; a group
// takes a segment (atomic ticket, so uneven segments balance), loads (or,
// when nothing in the shadow is live, zeroes) its working shadow, applies the
// segment's buckets wave by wave with a shared-memory CAS per access, writes
// the segment back and takes the next.  A group synchronises with a named
// barrier of its own, never the whole CTA.  Two layouts:
//   compact (ctl->bin_tbits != 0): 8 groups of 128 threads, the segment's
//     working shadow 4 bytes per word (tid in tbits bits, wc and bc in the rest
//     of 24, state and kernel tag on top: the compact storage form of the 8-byte
//     value, which the checker expands for every FSM step).  Taken only when
//     nothing in the shadow is live and every tid and clock of the check fits,
//     so each value the FSM stores fits too.  About one thread per access of a
//     wave of the benchmark trace.
//   full: 4 groups of 256 threads, 8-byte working shadow.

constexpr unsigned PG_THREADS = 1024;
constexpr unsigned PG_RACES = 64;           // races a group buffers per segment
constexpr unsigned PG_STAGE_BYTES_C = 8192; // staged accesses per group, compact layout
constexpr unsigned PG_STAGE_BYTES_F = 16384;

struct alignas(16) PGroupC {
    unsigned sh[HR_BIN_SEG];
    unsigned char stage[PG_STAGE_BYTES_C];
    unsigned wend[HR_BIN_MAX_WAVES];
    hr_race races[PG_RACES];
    unsigned seg, n_races;
    unsigned long long race_base;
};
struct alignas(16) PGroupF {
    unsigned long long sh[HR_BIN_SEG];
    unsigned char stage[PG_STAGE_BYTES_F];
    unsigned wend[HR_BIN_MAX_WAVES];
    hr_race races[PG_RACES];
    unsigned seg, n_races;
    unsigned long long race_base;
};
struct alignas(16) PCommon {
    unsigned char tab[2048];
    unsigned wave_y[HR_BIN_MAX_WAVES];  // bc << 16 | clear << 15 | ktag << 8 | wc
    unsigned kern[HR_BIN_MAX_WAVES];
    unsigned lastp[HR_BIN_MAX_WAVES];   // the last part of each wave (parts are in trace order)
    unsigned red[3][PG_THREADS / 32];
    int any_clear;
};
constexpr size_t PG_GROUPS_BYTES = sizeof(PGroupC) * 8 > sizeof(PGroupF) * 4 ? sizeof(PGroupC) * 8 : sizeof(PGroupF) * 4;
constexpr size_t PG_SMEM = sizeof(PCommon) + PG_GROUPS_BYTES;
static_assert(PG_SMEM <= 227 * 1024, "the persistent segment CTA fits in shared memory");
// every group (and its 8-byte fields, its 16-byte cp.async destinations) starts 16-byte aligned
static_assert(sizeof(PCommon) % 16 == 0 && sizeof(PGroupC) % 16 == 0 && sizeof(PGroupF) % 16 == 0,
              "16-byte aligned group layouts");
static_assert(offsetof(PGroupF, stage) % 16 == 0 && offsetof(PGroupC, stage) % 16 == 0 &&
                  offsetof(PGroupF, race_base) % 8 == 0 && offsetof(PGroupC, race_base) % 8 == 0,
              "aligned group fields");
static_assert(PG_STAGE_BYTES_C >= HR_BIN_SEG * 4 / 2, "staging sizes");

__device__ __forceinline__ void group_sync(unsigned id, unsigned n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// working value (4 bytes) <-> 8-byte layout, tid in tb bits
__device__ __forceinline__ unsigned long long pg_expand(unsigned x, const hr_geom& gw) { return hr_expand32(x, gw); }
__device__ __forceinline__ unsigned pg_compress(unsigned long long v, const hr_geom& gw) { return hr_compress64(v, gw); }

// The FSM step of Algorithm 1 on the 4-byte working form (the compact storage
// form with tid width tb, hr_expand32): the same transition as
// hr_fsm_step_pow2 on the expanded value, with 32-bit operations only.  wbits
// is the wave's kernel tag, bc and wc placed where the form keeps them; mbc and
// mwc mask the bc and wc fields; keep_w and keep_b keep the tid bits of a
// warp's and of a block's first thread (~(warp_size - 1), ~(block_dim - 1)).
__device__ __forceinline__ unsigned compact_step(unsigned x, unsigned tid, unsigned op, unsigned wbits, unsigned mbc,
                                                 unsigned mwc, unsigned tidmask, unsigned bd_shift,
                                                 unsigned ws_shift, unsigned keep_w, unsigned keep_b,
                                                 const unsigned char* tab, unsigned* raced)
{
    const unsigned d = x ^ wbits;
    unsigned os = x >> 27;
    if (d & 0x07000000u) os = HR_STATE_INIT;  // another kernel's value (or INIT already)
    const unsigned xt = (x & tidmask) ^ tid;
    const unsigned trel = xt == 0u ? HR_TREL_SAME : (xt >> bd_shift) ? HR_TREL_GRID
                        : (xt >> ws_shift) ? HR_TREL_BLOCK : HR_TREL_WARP;
    const unsigned srel = (d & mbc) ? HR_SREL_BLOCK : ((d & mwc) ? HR_SREL_WARP : HR_SREL_UNSYNC);
    const unsigned e = tab[(os << 6) | (op << 4) | (trel << 2) | srel];
    const unsigned ns = e & 31u, lvl = e >> 5;
    unsigned nx = (ns << 27) | (wbits & 0x07000000u);
    if (lvl >= HR_LVL_THREAD && lvl <= HR_LVL_BLOCK)
        nx |= (tid & (lvl == HR_LVL_THREAD ? ~0u : (lvl == HR_LVL_WARP ? keep_w : keep_b))) |
              (wbits & (lvl == HR_LVL_BLOCK ? mbc : (mbc | mwc)));
    if (ns == HR_STATE_RACE && os != HR_STATE_RACE) *raced = 1u + os;
    return nx;
}

template <bool COMPACT, typename T>
__device__ __forceinline__ unsigned long long as64_store(T v, const hr_geom& gw)
{
    if constexpr (COMPACT) return hr_expand32((unsigned)v, gw);
    else return (unsigned long long)v;
}

template <bool POW2, bool COMPACT, bool PACK4>
__device__ __forceinline__ void pg_run(unsigned char* gbase, PCommon& C, const hr_work& w, hr_region_dev* rg,
                                       const hr_geom& g, unsigned W, unsigned P, unsigned gid, unsigned* cnt)
{
    using Grp = typename std::conditional<COMPACT, PGroupC, PGroupF>::type;
    constexpr unsigned GT = COMPACT ? 128u : 256u;
    constexpr unsigned STAGE = COMPACT ? PG_STAGE_BYTES_C : PG_STAGE_BYTES_F;
    constexpr unsigned CH = STAGE / (PACK4 ? 4u : 8u);  // accesses staged at a time
    Grp& G = reinterpret_cast<Grp*>(gbase)[gid];
    const unsigned bar = gid + 1, t = threadIdx.x - gid * GT;
    hr_geom gw = g;  // the working form's packing (compact layout)
    gw.tid_bits = w.ctl->bin_tbits;
    const unsigned tb = gw.tid_bits, wcb = (24u - tb) >> 1;
    const unsigned tidmask = tb ? (1u << tb) - 1u : 0u;
    const unsigned mwc = ((1u << wcb) - 1u) << tb, mbc = 0x00FFFFFFu & ~((1u << (tb + wcb)) - 1u);
    const unsigned keep_w = POW2 ? ~((1u << min(g.ws_shift, g.bd_shift)) - 1u) : 0u;
    const unsigned keep_b = POW2 ? ~((1u << g.bd_shift) - 1u) : 0u;
    const bool fresh = w.ctl->fresh != 0;
    const bool store4 = g.shadow_bytes == 4;
    const unsigned cap = w.cas_cap;
    const unsigned ring_region = rg->region;
    const unsigned long long word_lo = hr_filter_active(rg->filter) ? rg->filter.word_lo : 0ull;
    unsigned long long* shadow = rg->shadow;
    const unsigned n_seg = w.bin.n_seg;
    unsigned n_acc = 0, n_cas = 0, n_retry = 0, err = 0;
    if (t == 0) G.n_races = 0;
    for (;;) {
        if (t == 0) G.seg = atomicAdd(&w.ctl->seg_ticket, 1u);
        group_sync(bar, GT);
        const unsigned seg = G.seg;
        if (seg >= n_seg) break;
        // the segment's wave ends: a wave's accesses end where its last part's do
        const unsigned* row = w.bin.table + (size_t)seg * P;
        for (unsigned wv = t; wv < W; wv += GT) {
            const unsigned lp = C.lastp[wv];
            G.wend[wv] = lp + 1 < P ? row[lp + 1] : (seg + 1 < n_seg ? row[P] : w.ctl->bin_total);
        }
        const unsigned r0 = row[0];
        group_sync(bar, GT);
        const unsigned r1 = G.wend[W - 1];
        const unsigned long long w0 = (unsigned long long)seg * HR_BIN_SEG;
        const unsigned nws = (unsigned)min((unsigned long long)HR_BIN_SEG, rg->n_words - w0);
        if (r0 == r1) {
            if (C.any_clear) {  // only clears: the segment ends cleared
                for (unsigned i = t; i < nws; i += GT) {
                    if (store4) reinterpret_cast<unsigned*>(shadow)[w0 + i] = 0u;
                    else shadow[w0 + i] = 0ull;
                }
            }
            group_sync(bar, GT);  // G.seg and G.wend are reused
            continue;
        }
        // the working shadow: zeros when nothing is live, else the stored values
        if (COMPACT || fresh) {
            for (unsigned i = t; i < HR_BIN_SEG; i += GT) G.sh[i] = 0;
        } else if constexpr (!COMPACT) {
            if (!store4) {
                for (unsigned i = t; i < nws / 2; i += GT) cp_async16(&G.sh[2 * i], shadow + w0 + 2 * i);
                if ((nws & 1u) && t == 0) G.sh[nws - 1] = shadow[w0 + nws - 1];
            } else {
                const unsigned* src = reinterpret_cast<const unsigned*>(shadow) + w0;
                for (unsigned i = t; i < nws; i += GT) G.sh[i] = hr_expand32(src[i], g);
            }
        }
        unsigned c0 = r0, c1 = min(r0 + CH, r1);
        if (PACK4) {
            unsigned* dst = reinterpret_cast<unsigned*>(G.stage);
            const unsigned* src = reinterpret_cast<const unsigned*>(w.bin.out);
            for (unsigned i = c0 + t; i < c1; i += GT) cp_async4(&dst[i - c0], &src[i]);
        } else {
            uint2* dst = reinterpret_cast<uint2*>(G.stage);
            for (unsigned i = c0 + t; i < c1; i += GT) cp_async8(&dst[i - c0], &w.bin.out[i]);
        }
        cp_async_wait_all();
        group_sync(bar, GT);
        n_acc += t == 0 ? r1 - r0 : 0u;
        unsigned b0 = r0;
        for (unsigned gwv = 0; gwv < W; ++gwv) {
            const unsigned wy = C.wave_y[gwv];
            if (wy & 0x8000u) {  // kernel-tag group change before this wave: the shadow starts over
                for (unsigned i = t; i < HR_BIN_SEG; i += GT) G.sh[i] = 0;
                group_sync(bar, GT);
            }
            const unsigned b1 = G.wend[gwv];
            const unsigned bc = wy >> 16, wc = wy & 0xFFu, ktag = (wy >> 8) & 7u;
            const unsigned wbits = (ktag << 24) | (bc << (tb + wcb)) | (wc << tb);  // compact layout only
            while (b0 < b1) {
                if (b0 >= c1) {  // the next accesses (every thread is done with the staged ones)
                    c0 = b0;
                    c1 = min(c0 + CH, r1);
                    if (PACK4) {
                        unsigned* dst = reinterpret_cast<unsigned*>(G.stage);
                        const unsigned* src = reinterpret_cast<const unsigned*>(w.bin.out);
                        for (unsigned i = c0 + t; i < c1; i += GT) cp_async4(&dst[i - c0], &src[i]);
                    } else {
                        uint2* dst = reinterpret_cast<uint2*>(G.stage);
                        for (unsigned i = c0 + t; i < c1; i += GT) cp_async8(&dst[i - c0], &w.bin.out[i]);
                    }
                    cp_async_wait_all();
                    group_sync(bar, GT);
                }
                const unsigned e = min(b1, c1);
                for (unsigned i = b0 + t; i < e; i += GT) {
                    unsigned wis, op, tid;
                    if (PACK4) {
                        const unsigned x = reinterpret_cast<const unsigned*>(G.stage)[i - c0];
                        wis = x & (HR_BIN_SEG - 1u);
                        op = (x >> HR_BIN_SEG_SHIFT) & 3u;
                        tid = x >> PACK4_TID_SHIFT;
                    } else {
                        const uint2 r = reinterpret_cast<const uint2*>(G.stage)[i - c0];
                        wis = r.y & (HR_BIN_SEG - 1u);
                        op = (r.y >> 16) & 0xFFu;
                        tid = r.x;
                    }
                    auto as64 = [&](auto v) -> unsigned long long {
                        if constexpr (COMPACT) return pg_expand((unsigned)v, gw);
                        else return (unsigned long long)v;
                    };
                    // one FSM step from a stored value to the value to store
                    auto step = [&](auto stored, unsigned* raced) -> decltype(stored) {
                        if constexpr (COMPACT && POW2) {
                            return compact_step(stored, tid, op, wbits, mbc, mwc, tidmask, g.bd_shift, g.ws_shift,
                                                keep_w, keep_b, C.tab, raced);
                        } else {
                            const unsigned long long o = as64(stored);
                            const unsigned long long nv =
                                POW2 ? hr_fsm_step_pow2(o, tid, op, bc, wc, ktag, g.bd_shift, g.ws_shift, C.tab, raced)
                                     : hr_fsm_step(o, tid, op, bc, wc, ktag, g, C.tab, raced);
                            if constexpr (COMPACT) return pg_compress(nv, gw);
                            else return nv;
                        }
                    };
                    auto stored = G.sh[wis];
                    unsigned raced = 0;
                    auto nst = step(stored, &raced);
                    bool done = true;
                    if (nst != stored) {
                        ++n_cas;
                        auto seen = atomicCAS(&G.sh[wis], stored, nst);
                        if (seen != stored) {
                            // another access of this wave changed the word first: fold into
                            // what it left, at most cap more times
                            ++n_retry;
                            done = false;
                            for (unsigned tries = 0; tries < cap; ++tries) {
                                stored = seen;
                                raced = 0;
                                nst = step(stored, &raced);
                                if (nst == stored) {
                                    done = true;
                                    break;
                                }
                                ++n_cas;
                                seen = atomicCAS(&G.sh[wis], stored, nst);
                                if (seen == stored) {
                                    done = true;
                                    break;
                                }
                            }
                        }
                    }
                    if (!done) {
                        err = HR_ERR_CONTENTION;
                    } else if (raced) {
                        const unsigned k = atomicAdd(&G.n_races, 1u);
                        const unsigned word = (unsigned)(word_lo + w0 + wis);
                        if (k < PG_RACES) {
                            hr_race& x = G.races[k];
                            x.word = word;
                            x.tid = tid;
                            x.kernel = (uint16_t)C.kern[gwv];
                            x.epoch = (uint16_t)bc;
                            x.region = (uint16_t)ring_region;
                            x.op = (uint8_t)op;
                            x.prior = (uint8_t)(raced - 1u);
                        } else {
                            hr_append_race(rg->ring, rg->ring_cap, &rg->n_races, &rg->flags, word, tid, C.kern[gwv],
                                           bc, ring_region, op, raced - 1u);
                        }
                    }
                }
                group_sync(bar, GT);
                b0 = e;
            }
        }
        // write the segment back in the region's storage form
        for (unsigned i = t; i < nws; i += GT) {
            const unsigned long long v = as64_store<COMPACT>(G.sh[i], gw);
            if (store4) reinterpret_cast<unsigned*>(shadow)[w0 + i] = hr_compress64(v, g);
            else shadow[w0 + i] = v;
        }
        // the buffered races: one reservation on the region's counter
        const unsigned nr = min(G.n_races, PG_RACES);
        if (nr) {
            if (t == 0) G.race_base = atomicAdd(&rg->n_races, (unsigned long long)nr);
            group_sync(bar, GT);
            for (unsigned i = t; i < nr; i += GT) {
                const unsigned long long slot = G.race_base + i;
                if (slot < rg->ring_cap) rg->ring[slot] = G.races[i];
                else atomicOr(&rg->flags, HR_FLAG_TRUNCATED);
            }
        }
        group_sync(bar, GT);  // every thread is done with G before it is reused
        if (t == 0) G.n_races = 0;
    }
    if (err) hr_set_error(&rg->error, err);
    cnt[0] = n_acc;
    cnt[1] = n_cas;
    cnt[2] = n_retry;
}

template <bool POW2>
__global__ void __launch_bounds__(PG_THREADS, 1)
    hr_bin_groups(hr_region_dev* __restrict__ regions, hr_work w, const unsigned char* __restrict__ gtable)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PCommon& C = *reinterpret_cast<PCommon*>(smem_raw);
    unsigned char* gbase = smem_raw + sizeof(PCommon);
    if (!hr_bin_taken(w.ctl)) return;
    const hr_jobd jb = w.jobs[0];
    hr_region_dev* rg = regions + jb.region;
    if (*(volatile unsigned*)&rg->error) return;
    const unsigned W = w.ctl->n_waves, P = w.ctl->bin_parts, tx = threadIdx.x;
    for (unsigned i = tx; i < W; i += PG_THREADS) {
        const unsigned long long key = w.wave_key[jb.wave_begin + i];
        const unsigned kern = (unsigned)(key >> 32);
        C.wave_y[i] = ((unsigned)key & 0xFFFF0000u) | (w.bin.clear[i] ? 0x8000u : 0u) | ((kern & 7u) << 8) |
                      ((unsigned)key & 0xFFu);
        C.kern[i] = kern;
    }
    for (unsigned i = tx; i < 2048 / 4; i += PG_THREADS)
        reinterpret_cast<unsigned*>(C.tab)[i] = reinterpret_cast<const unsigned*>(gtable)[i];
    for (unsigned p = tx; p < P; p += PG_THREADS) {
        const unsigned wv = w.bin.part_wave[p];
        if (p + 1 == P || w.bin.part_wave[p + 1] != wv) C.lastp[wv] = p;
    }
    const int any_clear = __syncthreads_or(tx < W && w.bin.clear[tx]);
    if (tx == 0) C.any_clear = any_clear;
    __syncthreads();
    const hr_geom g = rg->geom;
    const bool compact = w.ctl->bin_tbits != 0, pack4 = w.ctl->bin_pack4 != 0;
    unsigned cnt[3] = {0, 0, 0};
    if (compact) {
        if (pack4) pg_run<POW2, true, true>(gbase, C, w, rg, g, W, P, tx >> 7, cnt);
        else pg_run<POW2, true, false>(gbase, C, w, rg, g, W, P, tx >> 7, cnt);
    } else {
        if (pack4) pg_run<POW2, false, true>(gbase, C, w, rg, g, W, P, tx >> 8, cnt);
        else pg_run<POW2, false, false>(gbase, C, w, rg, g, W, P, tx >> 8, cnt);
    }
    // diagnostics: accesses, CAS attempts, retries
    const unsigned lane = tx & 31, wid = tx >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        for (int o = 16; o > 0; o >>= 1) cnt[k] += __shfl_xor_sync(0xFFFFFFFFu, cnt[k], o);
        if (lane == 0) C.red[k][wid] = cnt[k];
    }
    __syncthreads();
    if (tx < 3) {
        unsigned long long t = 0;
        for (unsigned i = 0; i < PG_THREADS / 32; ++i) t += C.red[tx][i];
        if (t) atomicAdd(&rg->counters[tx], t);
    }
}

bool g_attrs = false;

}  // namespace

cudaError_t hr_launch_binned(hr_region_dev* d_regions, const hr_work& w, const unsigned char* d_table,
                             cudaStream_t stream)
{
    if (!g_attrs) {
        // the shared-memory carveout at its maximum (the groups kernel takes nearly all of it)
        for (const void* k : {(const void*)hr_bin_count, (const void*)hr_bin_groups<true>,
                              (const void*)hr_bin_groups<false>})
            cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaFuncSetAttribute(hr_bin_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)STREAM_SMEM);
        cudaFuncSetAttribute(hr_bin_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SCATTER_SMEM);
        cudaFuncSetAttribute(hr_bin_groups<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PG_SMEM);
        cudaFuncSetAttribute(hr_bin_groups<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PG_SMEM);
        g_attrs = true;
    }
    const hr_bin& b = w.bin;
    if (b.n_seg == 0 || b.n_seg > b.seg_cap || b.n_seg > HR_BIN_MAX_SEGS || b.clusters == 0 || b.sub == 0 ||
        b.sub > HR_BIN_MAX_SUB || b.slices != b.clusters * b.sub || b.slices > STREAM_THREADS ||
        b.part_cap < HR_BIN_MAX_WAVES + b.slices - 1)
        return cudaErrorInvalidValue;
    const unsigned scan_blocks = (unsigned)(((unsigned long long)b.n_seg * b.part_cap + HR_BIN_SCAN - 1) / HR_BIN_SCAN);
    hr_bin_count<<<b.slices, STREAM_THREADS, STREAM_SMEM, stream>>>(d_regions, w);
    hr_bin_scan_sums<<<scan_blocks, SCAN_THREADS, 0, stream>>>(w);
    hr_bin_scan<<<scan_blocks, SCAN_THREADS, 0, stream>>>(w);
    hr_bin_scatter<<<b.clusters * CL, STREAM_THREADS, SCATTER_SMEM, stream>>>(d_regions, w);
    static int sms = 0;  // one persistent segment CTA per SM
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    if (b.pow2) hr_bin_groups<true><<<sms, PG_THREADS, PG_SMEM, stream>>>(d_regions, w, d_table);
    else hr_bin_groups<false><<<sms, PG_THREADS, PG_SMEM, stream>>>(d_regions, w, d_table);
    return cudaGetLastError();
}

// The binned checker's streaming shape: scatter clusters of HR_BIN_CLUSTER CTAs,
// as many as can be resident at once (one CTA per SM), and count slices per
// cluster slice so that the count pass (one CTA per SM) fills the SMs.
void hr_bin_shape(unsigned* clusters_out, unsigned* sub_out)
{
    static unsigned c_cached = 0, s_cached = 0;
    if (!c_cached) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < (int)CL) sms = CL;
        cudaFuncSetAttribute(hr_bin_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SCATTER_SMEM);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(sms / CL * CL));
        cfg.blockDim = dim3(STREAM_THREADS);
        cfg.dynamicSmemBytes = SCATTER_SMEM;
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = CL;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, (void*)hr_bin_scatter, &cfg) != cudaSuccess || clusters < 1) {
            (void)cudaGetLastError();
            clusters = sms / (int)CL;
        }
        unsigned sub = (unsigned)sms / (unsigned)clusters;
        if (sub < 1) sub = 1;
        if (sub > HR_BIN_MAX_SUB) sub = HR_BIN_MAX_SUB;
        while ((unsigned)clusters * sub > STREAM_THREADS) --sub;
        c_cached = (unsigned)clusters;
        s_cached = sub;
    }
    *clusters_out = c_cached;
    *sub_out = s_cached;
}
