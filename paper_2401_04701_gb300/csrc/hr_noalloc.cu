// hr_noalloc.cu - a trace check that allocates no device memory.
//
// hr_check_trace needs a context from hr_init, which allocates the shadow,
// the report ring and the scratch of the wave pre-pass.  Some callers must not
// allocate device memory at all: code that runs while another component owns
// the device memory budget (a framework's caching allocator or a fixed memory
// pool that has already claimed the free memory), and latency-critical paths
// where cudaMalloc / cudaFree would stall on an implicit device
// synchronisation.  hr_check_trace_noalloc serves them: the caller passes the
// trace, the shadow store, the race buffer and a result block, all in memory it
// already owns, and the pre-pass scratch lives in the file-scope array below.
//
// The array is part of the library image: every GPU that loads the library
// holds HR_NOALLOC_SCRATCH_BYTES of it until the process exits.  All calls on
// one device share it and it keeps the previous call's contents, so every call
// re-initialises the parts that must start at zero, and calls whose work
// overlaps on the GPU (different streams, or different host threads) race on
// it: serialise them.
#include <cuda_runtime.h>

#include <mutex>

#include "hr_internal.h"

namespace {

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// layout of the scratch array: region state, FSM table, then the pre-pass
// scratch of one job (job slot, interval counts, wave table, stages, control)
constexpr size_t OFF_REGION = 0;
constexpr size_t OFF_TABLE = OFF_REGION + align256(sizeof(hr_region_dev));
constexpr size_t OFF_WORK = OFF_TABLE + align256(2048);
constexpr size_t WORK_BYTES = align256(sizeof(hr_ctl)) + align256(sizeof(hr_jobd)) +
                              align256(HR_MAX_INTERVALS * sizeof(unsigned)) +
                              3 * align256(HR_NOALLOC_MAX_WAVES * sizeof(unsigned long long)) +
                              align256((2 * HR_NOALLOC_MAX_WAVES + 1) * sizeof(hr_stage));
constexpr size_t SCRATCH_BYTES = OFF_WORK + WORK_BYTES;
static_assert(SCRATCH_BYTES == HR_NOALLOC_SCRATCH_BYTES, "header size must match the layout");

static __device__ __align__(256) unsigned char hr_noalloc_scratch[SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch[kMaxDevices] = {};

// Once per device, with that device current: the array's device address (the
// host-side name is only a stand-in) and the FSM table copied into it.
cudaError_t setup_device(int dev, unsigned char** out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, hr_noalloc_scratch);
        if (e != cudaSuccess) return e;
        uint8_t table[2048];
        hr_fsm_table(table, nullptr);
        e = cudaMemcpy((unsigned char*)p + OFF_TABLE, table, sizeof table, cudaMemcpyHostToDevice);
        // a copy from pageable memory may return before it lands, and the caller's
        // stream may be one that does not wait for the legacy stream
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return e;
        g_scratch[dev] = (unsigned char*)p;
    }
    *out = g_scratch[dev];
    return cudaSuccess;
}

__global__ void hr_noalloc_begin(hr_region_dev* region, unsigned long long* shadow, unsigned long long n_words,
                                 hr_race* ring, unsigned long long ring_cap, hr_geom geom)
{
    region->shadow = shadow;
    region->ring = ring;
    region->n_words = n_words;
    region->ring_cap = ring_cap;
    region->n_races = 0;
    region->error = 0;
    region->flags = 0;
    // every call is a fresh check: kernel ordinals start over and the shadow is
    // cleared before the first wave, whatever an earlier call left in it
    region->last_key = 0;
    region->used = 2;
    region->region = 0;
    for (int i = 0; i < 4; ++i) region->counters[i] = 0;
    region->geom = geom;
    region->filter = hr_filter_all();
}

__global__ void hr_noalloc_end(const hr_region_dev* region, hr_result* result)
{
    result->n_races = region->n_races;
    result->error = region->error;
    result->flags = region->flags | (region->n_races > region->ring_cap ? HR_FLAG_TRUNCATED : 0u);
}

}  // namespace

extern "C" hr_status hr_check_trace_noalloc(const hr_record* d_trace, uint64_t n, uint64_t* d_shadow,
                                            uint64_t n_words, uint32_t block_dim, uint32_t warp_size,
                                            hr_race* d_races, uint64_t race_cap, hr_result* d_result,
                                            hr_stream_t stream)
{
    if ((n > 0 && !d_trace) || !d_shadow || !d_result || (race_cap > 0 && !d_races)) return HR_ERR_INVALID;
    if (((uintptr_t)d_trace & 15u) != 0) return HR_ERR_INVALID;
    if (n_words == 0 || n_words > (1ull << 32) || block_dim == 0 || warp_size == 0 || warp_size > 32 ||
        n >= (1ull << 40))
        return HR_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HR_ERR_CUDA;
    unsigned char* base = nullptr;
    if (setup_device(dev, &base) != cudaSuccess) return HR_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    hr_region_dev* region = (hr_region_dev*)(base + OFF_REGION);
    const hr_work w = hr_work_at(base + OFF_WORK, 1, HR_MAX_INTERVALS, HR_NOALLOC_MAX_WAVES);
    const hr_geom g = hr_make_geom(block_dim, warp_size);
    hr_noalloc_begin<<<1, 1, 0, s>>>(region, (unsigned long long*)d_shadow, n_words, d_races, race_cap, g);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && n > 0) {
        hr_jobd job{};
        job.trace = d_trace;
        job.n = n;
        job.region = 0;  // the region array is the single struct above
        hr_plan_intervals(n, HR_SMALL_INTERVALS, &job.G, &job.n_int);
        e = hr_launch_jobs(region, w, &job, 1, base + OFF_TABLE, 0u, s, nullptr);
    }
    if (e == cudaSuccess) {
        hr_noalloc_end<<<1, 1, 0, s>>>(region, d_result);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? HR_OK : HR_ERR_CUDA;
}
