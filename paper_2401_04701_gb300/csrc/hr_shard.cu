// hr_shard.cu - word-range sharding of a trace check over several ranks.
//
// The check of one trace can be spread over ranks that each own a contiguous
// range of the region's words (and that range's shadow).  An access only
// touches its own word's shadow value (Algorithm 1), so rank r can check the
// accesses to its words on its own, provided it sees them in wave order.  The
// data path has one real exchange step:
//   1. hr_shard_partition: every rank splits its part of the trace by owner
//      rank (a stable partition: each destination's records keep trace order,
//      so they stay wave-sorted), rebasing each word to the owner's range;
//      barrier records carry no word and are not routed (the checker reads
//      the clocks of every access record itself);
//   2. an all-to-all of those blocks (the caller's collective);
//   3. hr_shard_merge: a rank merges the wave-sorted blocks it received (one
//      per source) into one wave-sorted trace: runs of equal wave key are
//      placed in key order, equal keys in source order;
//   4. hr_check_trace on the rank's own region; race reports are gathered and
//      their words shifted back by the range start.
// Inside one wave every pair is unordered (Sec. II-B), so interleaving the
// sources' records of a wave in any order is a valid execution order.
#include <cuda_runtime.h>

#include "hr_internal.h"

namespace {

constexpr unsigned PT_WARPS = 8;
constexpr unsigned PT_THREADS = PT_WARPS * 32;
constexpr unsigned PT_ROUNDS = 8;                          // 32-record rounds per warp
constexpr unsigned PT_TILE = PT_THREADS * PT_ROUNDS;       // records per partition tile
constexpr unsigned MERGE_THREADS = 256;

__device__ __forceinline__ unsigned owner_of(unsigned word, const unsigned long long* bounds, unsigned world)
{
    // bounds[0] = 0 <= ... <= bounds[world] = n_words: the last r with bounds[r] <= word
    unsigned lo = 0, hi = world;
    while (hi - lo > 1) {
        const unsigned mid = (lo + hi) >> 1;
        if (bounds[mid] <= word) lo = mid; else hi = mid;
    }
    return lo;
}

// destination of record v (world when it is not routed: a barrier record or a
// word at or beyond the last bound)
__device__ __forceinline__ unsigned dest_of(const uint4 v, const unsigned long long* b, unsigned world)
{
    const unsigned op = (v.w >> 16) & 0xFFu;
    if (op > HR_A || v.x >= b[world]) return world;
    return owner_of(v.x, b, world);
}

// Per tile, the routed records per destination, destination-major:
// cnt[d * n_tiles + tile].
__global__ void __launch_bounds__(PT_THREADS) shard_count(const hr_record* __restrict__ t, unsigned long long n,
                                                          const unsigned long long* __restrict__ bounds,
                                                          unsigned world, unsigned n_tiles,
                                                          unsigned long long* __restrict__ cnt)
{
    __shared__ unsigned s_cnt[HR_SHARD_MAX_WORLD];
    __shared__ unsigned long long s_b[HR_SHARD_MAX_WORLD + 1];
    for (unsigned i = threadIdx.x; i <= world; i += PT_THREADS) s_b[i] = bounds[i];
    for (unsigned i = threadIdx.x; i < world; i += PT_THREADS) s_cnt[i] = 0;
    __syncthreads();
    const unsigned long long b0 = (unsigned long long)blockIdx.x * PT_TILE;
    for (unsigned j = threadIdx.x; j < PT_TILE; j += PT_THREADS) {
        const unsigned long long i = b0 + j;
        if (i >= n) break;
        const unsigned d = dest_of(__ldg(reinterpret_cast<const uint4*>(t + i)), s_b, world);
        if (d < world) atomicAdd(&s_cnt[d], 1u);
    }
    __syncthreads();
    for (unsigned d = threadIdx.x; d < world; d += PT_THREADS) cnt[(size_t)d * n_tiles + blockIdx.x] = s_cnt[d];
}

// Exclusive scan of cnt in place (destination-major, one CTA): every
// destination's block starts where the previous one ends.  counts[d] gets the
// records routed to destination d.
__global__ void __launch_bounds__(1024) shard_scan(unsigned long long* __restrict__ cnt, unsigned world,
                                                   unsigned n_tiles, unsigned long long* __restrict__ counts)
{
    __shared__ unsigned long long s_warp[32];
    const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned long long total = (unsigned long long)world * n_tiles;
    const unsigned long long per = (total + 1023) / 1024;
    const unsigned long long b = min(total, threadIdx.x * per), e = min(total, b + per);
    unsigned long long local = 0;
    for (unsigned long long i = b; i < e; ++i) local += cnt[i];
    unsigned long long x = local;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long v = s_warp[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= (unsigned)o) v += y;
        }
        s_warp[lane] = v;
    }
    __syncthreads();
    unsigned long long run = (wid ? s_warp[wid - 1] : 0ull) + x - local;
    for (unsigned long long i = b; i < e; ++i) {
        const unsigned long long c = cnt[i];
        cnt[i] = run;
        run += c;
    }
    __syncthreads();
    for (unsigned d = threadIdx.x; d < world; d += blockDim.x) {
        const unsigned long long s0 = cnt[(size_t)d * n_tiles];
        const unsigned long long s1 = d + 1 < world ? cnt[(size_t)(d + 1) * n_tiles] : s_warp[31];
        counts[d] = s1 - s0;
    }
}

// Stable placement: warp w of a tile owns records [w * 256, w * 256 + 256) of
// it, in 32-record rounds; a record's slot is its destination's offset for the
// tile, plus the records of lower warps, plus those of earlier rounds and
// lower lanes of its own warp with the same destination.
__global__ void __launch_bounds__(PT_THREADS) shard_place(const hr_record* __restrict__ t, unsigned long long n,
                                                          const unsigned long long* __restrict__ bounds,
                                                          unsigned world, unsigned n_tiles,
                                                          const unsigned long long* __restrict__ off,
                                                          hr_record* __restrict__ out)
{
    __shared__ unsigned long long s_b[HR_SHARD_MAX_WORLD + 1];
    __shared__ unsigned s_wc[PT_WARPS][HR_SHARD_MAX_WORLD];
    __shared__ unsigned long long s_base[PT_WARPS][HR_SHARD_MAX_WORLD];
    const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (unsigned i = threadIdx.x; i <= world; i += PT_THREADS) s_b[i] = bounds[i];
    for (unsigned i = threadIdx.x; i < PT_WARPS * HR_SHARD_MAX_WORLD; i += PT_THREADS) (&s_wc[0][0])[i] = 0;
    __syncthreads();
    const unsigned long long w0 = (unsigned long long)blockIdx.x * PT_TILE + wid * (PT_ROUNDS * 32);
    unsigned dest[PT_ROUNDS];
#pragma unroll
    for (unsigned r = 0; r < PT_ROUNDS; ++r) {
        const unsigned long long i = w0 + r * 32 + lane;
        dest[r] = i < n ? dest_of(__ldg(reinterpret_cast<const uint4*>(t + i)), s_b, world) : world;
        const unsigned m = __match_any_sync(0xffffffffu, dest[r]);
        if (dest[r] < world && lane == (unsigned)(__ffs(m) - 1)) s_wc[wid][dest[r]] += __popc(m);
        __syncwarp();
    }
    __syncthreads();
    for (unsigned k = threadIdx.x; k < PT_WARPS * world; k += PT_THREADS) {
        const unsigned w = k / world, d = k % world;
        unsigned long long b = off[(size_t)d * n_tiles + blockIdx.x];
        for (unsigned v = 0; v < w; ++v) b += s_wc[v][d];
        s_base[w][d] = b;
    }
    __syncthreads();
#pragma unroll
    for (unsigned r = 0; r < PT_ROUNDS; ++r) {
        const unsigned long long i = w0 + r * 32 + lane;
        const unsigned d = dest[r];
        const unsigned m = __match_any_sync(0xffffffffu, d);
        if (d < world) {
            uint4 v = *reinterpret_cast<const uint4*>(t + i);
            v.x -= (unsigned)s_b[d];  // the word within the owner's range
            const unsigned long long slot = s_base[wid][d] + __popc(m & ((1u << lane) - 1u));
            *reinterpret_cast<uint4*>(out + slot) = v;
        }
        __syncwarp();
        if (d < world && lane == (unsigned)(__ffs(m) - 1)) s_base[wid][d] += __popc(m);
        __syncwarp();
    }
}

__device__ __forceinline__ unsigned long long mkey(const hr_record* t, unsigned long long i)
{
    return __ldg(reinterpret_cast<const unsigned long long*>(t + i) + 1) & HR_KEY_MASK;
}

// first position in [lo, hi) whose key is > k (strict) or >= k, by a warp
// 32-way search over a wave-sorted range
template <bool STRICT>
__device__ __forceinline__ unsigned long long warp_bound(const hr_record* t, unsigned long long lo,
                                                         unsigned long long hi, unsigned long long k)
{
    const unsigned lane = threadIdx.x & 31;
    // invariant: every position < lo is below the bound, every position >= hi is not
    while (hi > lo) {
        const unsigned long long step = (hi - lo + 31) / 32;
        const unsigned long long x = lo + lane * step;
        bool beyond = true;  // position x is at or past the bound
        if (x < hi) {
            const unsigned long long kx = mkey(t, x);
            beyond = STRICT ? kx > k : kx >= k;
        }
        const unsigned m = __ballot_sync(0xffffffffu, beyond);
        if (m == 0) {  // every probe below the bound: it lies past the last one
            lo = lo + 31 * step + 1;
            continue;
        }
        const unsigned j = __ffs(m) - 1;
        if (j == 0) return lo;
        const unsigned long long nlo = lo + (j - 1) * step + 1;
        hi = min(hi, lo + j * step);
        lo = nlo;
    }
    return lo;
}

// A run: records [start, end) of one source block with one key, placed at pos.
struct Run {
    unsigned long long start, end, pos;
    unsigned chunk, pad;
};

// Mark the run starts of every block (a record whose key differs from the
// previous one of its block, or a block's first record).
__global__ void __launch_bounds__(MERGE_THREADS) merge_runs(const hr_record* __restrict__ in, unsigned long long n,
                                                            const unsigned long long* __restrict__ starts,
                                                            unsigned n_chunks, Run* __restrict__ runs,
                                                            unsigned long long cap,
                                                            unsigned long long* __restrict__ n_runs)
{
    for (unsigned long long i = blockIdx.x * (unsigned long long)MERGE_THREADS + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * MERGE_THREADS) {
        unsigned lo = 0, hi = n_chunks;  // the block holding i: starts[c] <= i < starts[c + 1]
        while (hi - lo > 1) {
            const unsigned mid = (lo + hi) >> 1;
            if (starts[mid] <= i) lo = mid; else hi = mid;
        }
        if (i == starts[lo] || mkey(in, i) != mkey(in, i - 1)) {
            const unsigned long long r = atomicAdd(n_runs, 1ull);
            if (r < cap) {
                runs[r].start = i;
                runs[r].chunk = lo;
            }
        }
    }
}

// One warp per run: its end (the first later key of its block) and its place,
// the records of every block with a smaller key plus those of earlier blocks
// with the same key.  A key below the previous one in the same block (an
// unsorted block) gives HR_ERR_ORDER in *status.
__global__ void __launch_bounds__(MERGE_THREADS) merge_place(const hr_record* __restrict__ in,
                                                             const unsigned long long* __restrict__ starts,
                                                             unsigned n_chunks, Run* __restrict__ runs,
                                                             unsigned long long cap,
                                                             const unsigned long long* __restrict__ n_runs,
                                                             unsigned* __restrict__ status)
{
    const unsigned long long nr = min(*n_runs, cap);
    const unsigned lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x == 0 && *n_runs > cap) atomicCAS(status, 0u, (unsigned)HR_ERR_CAPACITY);
    for (unsigned long long r = (blockIdx.x * (unsigned long long)MERGE_THREADS + threadIdx.x) / 32; r < nr;
         r += (unsigned long long)gridDim.x * MERGE_THREADS / 32) {
        const unsigned c = runs[r].chunk;
        const unsigned long long s = runs[r].start, k = mkey(in, s);
        if (lane == 0 && s > starts[c] && mkey(in, s - 1) > k) atomicCAS(status, 0u, (unsigned)HR_ERR_ORDER);
        unsigned long long pos = 0, end = s;
        for (unsigned q = 0; q < n_chunks; ++q) {
            const unsigned long long a = starts[q], b = starts[q + 1];
            if (q < c) pos += warp_bound<true>(in, a, b, k) - a;
            else if (q > c) pos += warp_bound<false>(in, a, b, k) - a;
            else {
                pos += s - a;
                end = warp_bound<true>(in, s, b, k);
            }
        }
        if (lane == 0) {
            runs[r].end = end;
            runs[r].pos = pos;
        }
    }
}

// Copy every run to its place (one CTA per run at a time).
__global__ void __launch_bounds__(MERGE_THREADS) merge_copy(const hr_record* __restrict__ in, unsigned long long n,
                                                            const Run* __restrict__ runs, unsigned long long cap,
                                                            const unsigned long long* __restrict__ n_runs,
                                                            hr_record* __restrict__ out)
{
    const unsigned long long nr = min(*n_runs, cap);
    for (unsigned long long r = blockIdx.x; r < nr; r += gridDim.x) {
        const Run x = runs[r];
        // in bounds whatever the input (a block that is not wave-sorted has been reported)
        if (x.end < x.start || x.end > n || x.pos > n - (x.end - x.start)) continue;
        for (unsigned long long i = x.start + threadIdx.x; i < x.end; i += MERGE_THREADS)
            *reinterpret_cast<uint4*>(out + x.pos + (i - x.start)) = *reinterpret_cast<const uint4*>(in + i);
    }
}

inline size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" uint64_t hr_shard_partition_scratch_bytes(uint64_t n, uint32_t world)
{
    const unsigned long long tiles = (n + PT_TILE - 1) / PT_TILE;
    return a256((size_t)tiles * world * 8) + a256((size_t)(world + 1) * 8);
}

extern "C" hr_status hr_shard_partition(const hr_record* d_trace, uint64_t n, const uint64_t* d_bounds, uint32_t world,
                                        hr_record* d_out, uint64_t* d_counts, void* d_scratch, uint64_t scratch_bytes,
                                        hr_stream_t stream)
{
    if (world == 0 || world > HR_SHARD_MAX_WORLD || !d_bounds || !d_counts || (n > 0 && (!d_trace || !d_out)))
        return HR_ERR_INVALID;
    if (((uintptr_t)d_trace & 15u) || ((uintptr_t)d_out & 15u) || ((uintptr_t)d_scratch & 7u)) return HR_ERR_INVALID;
    if (n >= (1ull << 40) || scratch_bytes < hr_shard_partition_scratch_bytes(n, world) || !d_scratch)
        return HR_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    (void)cudaGetLastError();
    if (n == 0) return cudaMemsetAsync(d_counts, 0, world * 8, s) == cudaSuccess ? HR_OK : HR_ERR_CUDA;
    const unsigned tiles = (unsigned)((n + PT_TILE - 1) / PT_TILE);
    unsigned long long* cnt = (unsigned long long*)d_scratch;
    shard_count<<<tiles, PT_THREADS, 0, s>>>(d_trace, n, (const unsigned long long*)d_bounds, world, tiles, cnt);
    shard_scan<<<1, 1024, 0, s>>>(cnt, world, tiles, (unsigned long long*)d_counts);
    shard_place<<<tiles, PT_THREADS, 0, s>>>(d_trace, n, (const unsigned long long*)d_bounds, world, tiles, cnt,
                                             d_out);
    return cudaGetLastError() == cudaSuccess ? HR_OK : HR_ERR_CUDA;
}

extern "C" uint64_t hr_shard_merge_scratch_bytes(uint64_t max_runs)
{
    return a256(8) + a256(4) + a256((size_t)max_runs * sizeof(Run));
}

extern "C" hr_status hr_shard_merge(const hr_record* d_in, const uint64_t* d_starts, uint32_t n_chunks,
                                    uint64_t n, hr_record* d_out, void* d_scratch, uint64_t scratch_bytes,
                                    uint64_t max_runs, uint32_t* d_status, hr_stream_t stream)
{
    if (n_chunks == 0 || n_chunks > HR_SHARD_MAX_WORLD || !d_starts || !d_status || (n > 0 && (!d_in || !d_out)))
        return HR_ERR_INVALID;
    if (((uintptr_t)d_in & 15u) || ((uintptr_t)d_out & 15u) || ((uintptr_t)d_scratch & 255u)) return HR_ERR_INVALID;
    if (max_runs == 0 || !d_scratch || scratch_bytes < hr_shard_merge_scratch_bytes(max_runs) || n >= (1ull << 40))
        return HR_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    (void)cudaGetLastError();
    char* p = (char*)d_scratch;
    unsigned long long* n_runs = (unsigned long long*)p;
    Run* runs = (Run*)(p + a256(8) + a256(4));
    cudaError_t e = cudaMemsetAsync(d_scratch, 0, a256(8), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, 4, s);
    if (e != cudaSuccess) return HR_ERR_CUDA;
    if (n == 0) return HR_OK;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)(sms > 0 ? sms * 8 : 1024);
    merge_runs<<<grid, MERGE_THREADS, 0, s>>>(d_in, n, (const unsigned long long*)d_starts, n_chunks, runs, max_runs,
                                               n_runs);
    merge_place<<<grid, MERGE_THREADS, 0, s>>>(d_in, (const unsigned long long*)d_starts, n_chunks, runs, max_runs,
                                                n_runs, d_status);
    merge_copy<<<grid, MERGE_THREADS, 0, s>>>(d_in, n, runs, max_runs, n_runs, d_out);
    e = cudaGetLastError();
    return e == cudaSuccess ? HR_OK : HR_ERR_CUDA;
}
