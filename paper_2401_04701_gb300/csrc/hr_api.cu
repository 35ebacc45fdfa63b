// hr_api.cu - the C-ABI entry points declared in include/hirace.h.
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "hr_internal.h"

namespace {

// the Python binding mirrors these layouts (paper_2401_04701_gb300/hirace.py)
static_assert(sizeof(hr_filter) == 48 && sizeof(hr_view) == 168, "hr_filter / hr_view layouts");

struct RegionHost {
    hr_region_desc desc{};
    hr_region_dev* d = nullptr;           // element of the context's device region array
    unsigned long long* shadow = nullptr;
    hr_race* ring = nullptr;
    unsigned long long ring_cap = 0;
    unsigned long long capacity = 0;      // shadow words allocated (n_words may be reconfigured below it)
    void* work_mem = nullptr;
    hr_work work{};
    unsigned kernel = 0;                  // kernel ordinal seen by device views
    hr_filter filter = hr_filter_all();   // monitored accesses (hr_set_filter)
    bool owns_shadow = true;              // false: caller-owned (hr_init_with_buffers)
    bool owns_ring = true;
    cudaEvent_t done = nullptr;           // recorded after every call on the region
    bool captured = false;                // work was queued inside a stream capture
    bool views = false;                   // a device view was handed out (inline writes possible)
    void* bin_mem = nullptr;              // binned checker tables (allocated by its first check)
    hr_bin bin{};                         // carved out of bin_mem; bin.out is its own allocation
};

// Record the region's completion event, unless the stream is being captured
// into a CUDA graph (an event recorded there is only a graph edge); then
// hr_report falls back to a device-wide synchronisation.
cudaError_t mark_done(RegionHost& r, cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusNone) {
        r.captured = true;
        return cudaSuccess;
    }
    return cudaEventRecord(r.done, s);
}

hr_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return HR_OK;
    if (e == cudaErrorMemoryAllocation) return HR_ERR_OOM;
    return HR_ERR_CUDA;
}

unsigned max_waves_setting()
{
    const char* s = getenv("HR_MAX_WAVES");
    long v = s ? strtol(s, nullptr, 10) : 0;
    if (v < 1 || v > (1l << 24)) v = 1l << 16;
    return (unsigned)v;
}

}  // namespace

struct ProfiledCall {
    cudaEvent_t begin, mid, end;  // before the pre-pass, before the checker, after it
    unsigned launches;
};

struct hr_ctx {
    int device = 0;
    std::vector<RegionHost> regions;
    hr_region_dev* d_regions = nullptr;
    unsigned char* d_table = nullptr;
    bool profile = false;
    unsigned long long wait_ns = HR_DEFAULT_WAIT_NS;
    unsigned cas_cap = HR_DEFAULT_CAS_CAP;
    unsigned test_flags = 0;
    unsigned variant = 0;              // kernel variant of later checks (hr_set_variant / hr_autotune)
    cudaStream_t copies = nullptr;     // non-blocking stream for report copies (never waits on user streams)
    void* batch_mem = nullptr;         // scratch of hr_check_batch (allocated on first use)
    // hr_check_trace_host: two device staging buffers, a copy stream, and events
    // ordering each buffer's copy before its check and its check before its next copy
    hr_record* stage_buf[2] = {nullptr, nullptr};
    uint64_t stage_cap = 0;            // records per staging buffer
    cudaStream_t h2d = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr};
    cudaEvent_t used[2] = {nullptr, nullptr};
    hr_work batch{};
    unsigned batch_jobs = 0;
    std::vector<int> batch_map;        // last hr_check_batch: caller's job -> device job (-1: empty trace)
    unsigned long long batch_waves = 0;
    std::vector<ProfiledCall> calls;   // profiled calls not read yet
    std::vector<ProfiledCall> spare;   // event triples to reuse
};

static ProfiledCall take_events(hr_ctx* c)
{
    if (!c->spare.empty()) {
        ProfiledCall p = c->spare.back();
        c->spare.pop_back();
        return p;
    }
    ProfiledCall p{};
    cudaEventCreate(&p.begin);
    cudaEventCreate(&p.mid);
    cudaEventCreate(&p.end);
    return p;
}

static void free_ctx(hr_ctx* c)
{
    if (!c) return;
    for (auto& r : c->regions) {
        if (r.done) cudaEventDestroy(r.done);
        if (r.owns_shadow) cudaFree(r.shadow);
        if (r.owns_ring) cudaFree(r.ring);
        cudaFree(r.work_mem);
        cudaFree(r.bin_mem);
        cudaFree(r.bin.out);
    }
    for (auto* v : {&c->calls, &c->spare})
        for (auto& p : *v) {
            cudaEventDestroy(p.begin);
            cudaEventDestroy(p.mid);
            cudaEventDestroy(p.end);
        }
    if (c->copies) cudaStreamDestroy(c->copies);
    for (int b = 0; b < 2; ++b) {
        cudaFree(c->stage_buf[b]);
        if (c->copied[b]) cudaEventDestroy(c->copied[b]);
        if (c->used[b]) cudaEventDestroy(c->used[b]);
    }
    if (c->h2d) cudaStreamDestroy(c->h2d);
    cudaFree(c->batch_mem);
    cudaFree(c->d_regions);
    cudaFree(c->d_table);
    delete c;
}

static bool valid_region(hr_ctx* ctx, uint32_t region) { return ctx && region < ctx->regions.size(); }
static hr_status fetch_region(hr_ctx* ctx, uint32_t region, hr_region_dev* out);

static hr_status init_impl(hr_ctx** out, const hr_region_desc* regions, uint32_t n_regions, uint64_t report_capacity,
                           void* const* shadows, hr_race* const* rings, hr_stream_t stream)
{
    if (!out) return HR_ERR_INVALID;
    *out = nullptr;
    if (!regions || n_regions == 0 || n_regions > 65535 || report_capacity == 0) return HR_ERR_INVALID;
    for (uint32_t i = 0; i < n_regions; ++i) {
        const hr_region_desc& d = regions[i];
        if (d.n_words == 0 || d.n_words > (1ull << 32) || d.block_dim == 0 || d.warp_size == 0 ||
            d.warp_size > 32 || d.reserved != 0 || d.space > HR_SPACE_SHARED)
            return HR_ERR_INVALID;
        if (d.shadow_bytes != 0 && d.shadow_bytes != 4 && d.shadow_bytes != 8) return HR_ERR_INVALID;
        if (d.report_mode > HR_REPORT_EVERY_EPOCH || (d.report_mode == HR_REPORT_EVERY_EPOCH && d.shadow_bytes == 4))
            return HR_ERR_INVALID;
        if (d.shadow_bytes == 4) {
            const uint32_t t = hr_desc_tid_bits(d);
            if (t < 4 || t > 22 || d.block_dim > (1u << t)) return HR_ERR_INVALID;
        } else if (d.tid_bits != 0) {
            return HR_ERR_INVALID;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    hr_ctx* c = new (std::nothrow) hr_ctx;
    if (!c) return HR_ERR_OOM;
    cudaGetDevice(&c->device);
    c->regions.resize(n_regions);
    hr_status st = HR_OK;
    uint8_t table[2048];
    hr_fsm_table(table, nullptr);
    cudaError_t e = cudaStreamCreateWithFlags(&c->copies, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_table, sizeof table);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_table, table, sizeof table, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_regions, sizeof(hr_region_dev) * n_regions);
    const unsigned max_waves = max_waves_setting();
    std::vector<hr_region_dev> hdev(n_regions);
    for (uint32_t i = 0; i < n_regions && e == cudaSuccess; ++i) {
        RegionHost& r = c->regions[i];
        r.desc = regions[i];
        r.ring_cap = regions[i].report_capacity ? regions[i].report_capacity : report_capacity;
        r.d = c->d_regions + i;
        r.capacity = r.desc.n_words;
        r.owns_shadow = !(shadows && shadows[i]);
        r.owns_ring = !(rings && rings[i]);
        if (r.owns_shadow)
            e = cudaMalloc(&r.shadow, r.desc.n_words * hr_desc_shadow_bytes(r.desc));
        else
            r.shadow = (unsigned long long*)shadows[i];
        if (e == cudaSuccess) {
            if (r.owns_ring)
                e = cudaMalloc(&r.ring, r.ring_cap * sizeof(hr_race));
            else
                r.ring = rings[i];
        }
        // scratch of one trace check: job table, interval counts, wave table, stages, control block
        const size_t total = hr_work_bytes(1, HR_MAX_INTERVALS, max_waves);
        if (e == cudaSuccess) e = cudaMalloc(&r.work_mem, total);
        if (e == cudaSuccess) {
            r.work = hr_work_at(r.work_mem, 1, HR_MAX_INTERVALS, max_waves);
            e = cudaMemsetAsync(r.work_mem, 0, total, s);
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(r.shadow, 0, r.desc.n_words * hr_desc_shadow_bytes(r.desc), s);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming);
        hr_region_dev& h = hdev[i];
        memset(&h, 0, sizeof h);
        h.shadow = r.shadow;
        h.ring = r.ring;
        h.n_words = r.desc.n_words;
        h.ring_cap = r.ring_cap;
        h.region = i;
        h.geom = hr_desc_geom(r.desc);
        h.filter = hr_filter_all();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_regions, hdev.data(), sizeof(hr_region_dev) * n_regions, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        st = cuda_status(e);
        free_ctx(c);
        return st;
    }
    *out = c;
    return HR_OK;
}

extern "C" hr_status hr_init(hr_ctx** out, const hr_region_desc* regions, uint32_t n_regions,
                             uint64_t report_capacity, hr_stream_t stream)
{
    return init_impl(out, regions, n_regions, report_capacity, nullptr, nullptr, stream);
}

extern "C" hr_status hr_init_with_buffers(hr_ctx** out, const hr_region_desc* regions, uint32_t n_regions,
                                          uint64_t report_capacity, void* const* shadows, hr_race* const* rings,
                                          hr_stream_t stream)
{
    if (!shadows) return HR_ERR_INVALID;
    for (uint32_t i = 0; i < n_regions && regions; ++i) {
        if (!shadows[i] || ((uintptr_t)shadows[i] & 15u)) return HR_ERR_INVALID;  // 16-byte clears
        if (rings && rings[i] && ((uintptr_t)rings[i] & 15u)) return HR_ERR_INVALID;
    }
    return init_impl(out, regions, n_regions, report_capacity, shadows, rings, stream);
}

// The binned checker's tables for the region's current size and an access
// buffer of n records.  Growing them waits for the device (work in flight may
// still use the old buffers); the first binned check of a region allocates.
static hr_status ensure_bin(RegionHost& r, uint64_t n, cudaStream_t s)
{
    (void)s;
    const unsigned n_seg = (unsigned)((r.desc.n_words + HR_BIN_SEG - 1) / HR_BIN_SEG);
    cudaError_t e = cudaSuccess;
    if (!r.bin_mem || r.bin.seg_cap < n_seg) {
        const unsigned cap = (unsigned)((r.capacity + HR_BIN_SEG - 1) / HR_BIN_SEG);
        unsigned clusters = 0, sub = 0;
        hr_bin_shape(&clusters, &sub);
        const unsigned slices = clusters * sub;
        const unsigned part_cap = HR_BIN_MAX_WAVES + slices - 1;
        const size_t bytes = hr_bin_table_bytes(cap, part_cap);
        if (r.bin_mem) e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaFree(r.bin_mem);
        r.bin_mem = nullptr;
        r.bin.seg_cap = 0;
        if (e == cudaSuccess) e = cudaMalloc(&r.bin_mem, bytes);
        if (e != cudaSuccess) return cuda_status(e);
        auto a = [](size_t x) { return (x + 255) & ~size_t(255); };
        const size_t ent = (size_t)cap * part_cap;
        char* p = (char*)r.bin_mem;
        r.bin.table = (unsigned*)p;
        p += a(ent * 4);
        r.bin.sums = (unsigned*)p;
        p += a((ent / HR_BIN_SCAN + 1) * 4);
        r.bin.part_wave = (unsigned*)p;
        p += a((size_t)part_cap * 4);
        r.bin.clear = (unsigned char*)p;
        r.bin.seg_cap = cap;
        r.bin.part_cap = part_cap;
        r.bin.clusters = clusters;
        r.bin.sub = sub;
        r.bin.slices = slices;
    }
    if (r.bin.out_cap < n) {
        if (r.bin.out) e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaFree(r.bin.out);
        r.bin.out = nullptr;
        r.bin.out_cap = 0;
        if (e == cudaSuccess) e = cudaMalloc(&r.bin.out, n * sizeof(uint2) + 16);
        if (e != cudaSuccess) return cuda_status(e);
        r.bin.out_cap = n;
    }
    r.bin.n_seg = n_seg;
    r.bin.pow2 = hr_desc_geom(r.desc).bd_shift != ~0u ? 1u : 0u;
    return HR_OK;
}

static hr_status check_common(hr_ctx* ctx, uint32_t region, const hr_record* d_trace, uint64_t n,
                              uint32_t kernel_base, hr_stream_t stream, bool aggregate)
{
    if (!valid_region(ctx, region) || (n > 0 && !d_trace) || kernel_base > 0xFFFF) return HR_ERR_INVALID;
    if (((uintptr_t)d_trace & 15u) != 0) return HR_ERR_INVALID;  // records are copied in 16-byte units
    if (n >= (1ull << 40)) return HR_ERR_INVALID;
    if (n == 0) return HR_OK;
    (void)cudaGetLastError();  // report only errors of this call's launches
    RegionHost& r = ctx->regions[region];
    cudaStream_t s = (cudaStream_t)stream;
    hr_jobd job{};
    job.trace = d_trace;
    job.n = n;
    job.kb = (unsigned long long)kernel_base << 32;
    job.region = region;
    job.int_begin = 0;
    hr_plan_intervals(n, HR_SMALL_INTERVALS, &job.G, &job.n_int);
    ProfiledCall pc{};
    if (ctx->profile) pc = take_events(ctx);
    if (ctx->profile) cudaEventRecord(pc.begin, s);
    hr_work w = r.work;
    w.wait_ns = ctx->wait_ns;
    w.cas_cap = ctx->cas_cap;
    w.test_flags = ctx->test_flags;
    w.views = r.views ? 1u : 0u;
    unsigned variant = ctx->variant;
    if (!aggregate && variant < HR_N_SHAPES) variant |= 1u;  // odd ids do not aggregate (nor does the binned one)
    if (r.desc.report_mode == HR_REPORT_EVERY_EPOCH) variant = HR_EVERY_EPOCH_VARIANT;
    // 32-bit bucket offsets; segment histograms in shared memory
    if (variant == HR_BIN_VARIANT && (n >= (1ull << 32) || r.desc.n_words > (uint64_t)HR_BIN_MAX_SEGS * HR_BIN_SEG))
        variant = HR_BIN_FALLBACK;
    if (variant == HR_BIN_VARIANT) {
        const hr_status bs = ensure_bin(r, n, s);
        if (bs != HR_OK) return bs;
        w.bin = r.bin;
    }
    unsigned launches = 0;
    cudaError_t e = hr_launch_jobs(ctx->d_regions, w, &job, 1, ctx->d_table, variant, s,
                                   ctx->profile ? pc.mid : nullptr, &launches);
    if (ctx->profile) {
        cudaEventRecord(pc.end, s);
        pc.launches = launches;
        ctx->calls.push_back(pc);
    }
    if (e == cudaSuccess) e = mark_done(r, s);
    return cuda_status(e);
}

extern "C" hr_status hr_check_trace(hr_ctx* ctx, uint32_t region, const hr_record* d_trace, uint64_t n,
                                    hr_stream_t stream)
{
    return check_common(ctx, region, d_trace, n, 0, stream, true);
}

extern "C" hr_status hr_check_trace_host(hr_ctx* ctx, uint32_t region, const hr_record* h_trace, uint64_t n,
                                         uint64_t chunk_records, hr_stream_t stream)
{
    if (!valid_region(ctx, region) || (n > 0 && !h_trace) || n >= (1ull << 40)) return HR_ERR_INVALID;
    if (n == 0) return HR_OK;
    if (chunk_records == 0) chunk_records = 1ull << 24;  // 256 MB per staging buffer
    if (chunk_records > n) chunk_records = n;
    cudaStream_t s = (cudaStream_t)stream;
    (void)cudaGetLastError();
    cudaError_t e = cudaSuccess;
    if (!ctx->h2d) e = cudaStreamCreateWithFlags(&ctx->h2d, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        if (!ctx->copied[b]) e = cudaEventCreateWithFlags(&ctx->copied[b], cudaEventDisableTiming);
        if (e == cudaSuccess && !ctx->used[b]) e = cudaEventCreateWithFlags(&ctx->used[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess && chunk_records > ctx->stage_cap) {
        // earlier calls may still read the old buffers
        e = cudaDeviceSynchronize();
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            cudaFree(ctx->stage_buf[b]);
            ctx->stage_buf[b] = nullptr;
            e = cudaMalloc(&ctx->stage_buf[b], chunk_records * sizeof(hr_record));
        }
        ctx->stage_cap = e == cudaSuccess ? chunk_records : 0;
    }
    if (e != cudaSuccess) return cuda_status(e);
    hr_status st = HR_OK;
    uint64_t i = 0;
    for (uint64_t off = 0; off < n && st == HR_OK; off += chunk_records, ++i) {
        const int b = (int)(i & 1);
        const uint64_t m = n - off < chunk_records ? n - off : chunk_records;
        // the copy into buffer b waits for the check that last read it, the check for the copy
        e = cudaStreamWaitEvent(ctx->h2d, ctx->used[b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ctx->stage_buf[b], h_trace + off, m * sizeof(hr_record), cudaMemcpyHostToDevice,
                                ctx->h2d);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->copied[b], ctx->h2d);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ctx->copied[b], 0);
        if (e != cudaSuccess) return cuda_status(e);
        st = check_common(ctx, region, ctx->stage_buf[b], m, 0, stream, true);
        e = cudaEventRecord(ctx->used[b], s);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return st;
}

extern "C" hr_status hr_check_trace_kbase(hr_ctx* ctx, uint32_t region, const hr_record* d_trace, uint64_t n,
                                          uint32_t kernel_base, hr_stream_t stream)
{
    return check_common(ctx, region, d_trace, n, kernel_base, stream, true);
}

extern "C" hr_status hr_check_trace_plain(hr_ctx* ctx, uint32_t region, const hr_record* d_trace, uint64_t n,
                                          hr_stream_t stream)
{
    return check_common(ctx, region, d_trace, n, 0, stream, false);
}

extern "C" hr_status hr_batch_job_times(hr_ctx* ctx, uint64_t* ns_out, uint32_t n)
{
    if (!ctx || (n > 0 && !ns_out) || n > ctx->batch_map.size()) return HR_ERR_INVALID;
    if (n == 0) return HR_OK;
    cudaError_t e = cudaDeviceSynchronize();
    std::vector<hr_jobd> jobs(ctx->batch_jobs);
    hr_ctl ctl{};
    if (e == cudaSuccess && ctx->batch_mem)
        e = cudaMemcpy(jobs.data(), ctx->batch.jobs, jobs.size() * sizeof(hr_jobd), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && ctx->batch_mem) e = cudaMemcpy(&ctl, ctx->batch.ctl, sizeof ctl, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    for (uint32_t i = 0; i < n; ++i) {
        const int d = ctx->batch_map[i];
        const uint64_t t = d >= 0 && (size_t)d < jobs.size() ? jobs[d].done_ns : 0;
        ns_out[i] = t > ctl.t0_ns ? t - ctl.t0_ns : 0;
    }
    return HR_OK;
}

extern "C" hr_status hr_batch_reserve(hr_ctx* ctx, uint32_t max_jobs, uint64_t max_waves)
{
    if (!ctx || max_jobs == 0 || max_jobs > HR_MAX_BATCH || max_waves == 0 || max_waves > (1ull << 24))
        return HR_ERR_INVALID;
    if (ctx->batch_mem && ctx->batch_jobs >= max_jobs && ctx->batch_waves >= max_waves) return HR_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && ctx->batch_mem) e = cudaFree(ctx->batch_mem);
    ctx->batch_mem = nullptr;
    const unsigned mj = max_jobs > ctx->batch_jobs ? max_jobs : ctx->batch_jobs;
    const unsigned mw = (unsigned)(max_waves > ctx->batch_waves ? max_waves : ctx->batch_waves);
    const size_t bytes = hr_work_bytes(mj, HR_BATCH_INTERVALS, mw);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->batch_mem, bytes);
    if (e == cudaSuccess) e = cudaMemset(ctx->batch_mem, 0, bytes);
    if (e != cudaSuccess) {
        ctx->batch_mem = nullptr;
        ctx->batch_jobs = 0;
        ctx->batch_waves = 0;
        return cuda_status(e);
    }
    ctx->batch = hr_work_at(ctx->batch_mem, mj, HR_BATCH_INTERVALS, mw);
    ctx->batch_jobs = mj;
    ctx->batch_waves = mw;
    return HR_OK;
}

extern "C" hr_status hr_check_batch(hr_ctx* ctx, const hr_job* jobs, uint32_t n_jobs, hr_stream_t stream)
{
    if (!ctx || (n_jobs > 0 && !jobs)) return HR_ERR_INVALID;
    std::vector<hr_jobd> js;
    std::vector<int> map(n_jobs, -1);
    std::vector<char> seen(ctx->regions.size(), 0);
    for (uint32_t i = 0; i < n_jobs; ++i) {
        const hr_job& j = jobs[i];
        if (!valid_region(ctx, j.region) || j.reserved != 0 || (j.n > 0 && !j.trace) || j.n >= (1ull << 40) ||
            ((uintptr_t)j.trace & 15u) != 0)
            return HR_ERR_INVALID;
        if (seen[j.region]) return HR_ERR_INVALID;  // one job per region
        seen[j.region] = 1;
        if (j.n == 0) continue;
        hr_jobd d{};
        d.trace = j.trace;
        d.n = j.n;
        d.region = j.region;
        map[i] = (int)js.size();
        js.push_back(d);
    }
    ctx->batch_map = map;
    if (js.empty()) return HR_OK;
    if (js.size() > HR_MAX_BATCH) return HR_ERR_INVALID;
    if (!ctx->batch_mem || ctx->batch_jobs < js.size()) {
        hr_status st = hr_batch_reserve(ctx, (uint32_t)js.size() > ctx->batch_jobs ? (uint32_t)js.size() : ctx->batch_jobs,
                                        ctx->batch_waves ? ctx->batch_waves : (1ull << 18));
        if (st != HR_OK) return st;
    }
    // split the pre-pass interval budget across the jobs
    const unsigned budget = HR_BATCH_INTERVALS / (unsigned)js.size();
    unsigned at = 0;
    for (auto& d : js) {
        hr_plan_intervals(d.n, budget, &d.G, &d.n_int);
        d.int_begin = at;
        at += d.n_int;
    }
    cudaStream_t s = (cudaStream_t)stream;
    (void)cudaGetLastError();  // report only errors of this call's launches
    ProfiledCall pc{};
    if (ctx->profile) pc = take_events(ctx);
    if (ctx->profile) cudaEventRecord(pc.begin, s);
    hr_work w = ctx->batch;
    w.wait_ns = ctx->wait_ns;
    w.cas_cap = ctx->cas_cap;
    unsigned variant = ctx->variant == HR_BIN_VARIANT ? HR_BIN_FALLBACK : ctx->variant;  // not for batches
    for (const auto& d : js)
        if (ctx->regions[d.region].desc.report_mode == HR_REPORT_EVERY_EPOCH) variant = HR_EVERY_EPOCH_VARIANT;
    unsigned launches = 0;
    cudaError_t e = hr_launch_jobs(ctx->d_regions, w, js.data(), (unsigned)js.size(), ctx->d_table, variant, s,
                                   ctx->profile ? pc.mid : nullptr, &launches);
    if (ctx->profile) {
        cudaEventRecord(pc.end, s);
        pc.launches = launches;
        ctx->calls.push_back(pc);
    }
    for (auto& d : js)
        if (e == cudaSuccess) e = mark_done(ctx->regions[d.region], s);
    return cuda_status(e);
}

extern "C" hr_status hr_sync(hr_ctx* ctx, uint32_t region, uint32_t scope, hr_stream_t stream)
{
    if (!valid_region(ctx, region) || scope != HR_SYNC_KERNEL) return HR_ERR_INVALID;
    RegionHost& r = ctx->regions[region];
    cudaStream_t s = (cudaStream_t)stream;
    (void)cudaGetLastError();  // report only errors of this call's launches
    // device views (hand instrumentation) tag shadow values with kernel mod 8:
    // when the next kernel starts a new group of 8, clear the shadow
    cudaError_t e = cudaSuccess;
    if (((r.kernel + 1) >> 3) != (r.kernel >> 3))
        e = cudaMemsetAsync(r.shadow, 0, r.desc.n_words * hr_desc_shadow_bytes(r.desc), s);
    if (e == cudaSuccess) e = hr_launch_sync_kernel(r.d, s);
    if (e == cudaSuccess) e = mark_done(r, s);
    if (e == cudaSuccess) r.kernel++;
    return cuda_status(e);
}

static hr_status fetch_region(hr_ctx* ctx, uint32_t region, hr_region_dev* out)
{
    RegionHost& r = ctx->regions[region];
    cudaError_t e = r.captured ? cudaDeviceSynchronize() : cudaEventSynchronize(r.done);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, r.d, sizeof *out, cudaMemcpyDeviceToHost, ctx->copies);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->copies);
    return cuda_status(e);
}

extern "C" hr_status hr_report(hr_ctx* ctx, uint32_t region, hr_race* host_out, uint64_t cap, uint64_t* n_total,
                               uint32_t* flags)
{
    if (!valid_region(ctx, region) || (cap > 0 && !host_out)) return HR_ERR_INVALID;
    hr_region_dev h;
    hr_status st = fetch_region(ctx, region, &h);
    if (st != HR_OK) return st;
    const RegionHost& r = ctx->regions[region];
    unsigned long long avail = h.n_races < r.ring_cap ? h.n_races : r.ring_cap;
    unsigned long long ncopy = avail < cap ? avail : cap;
    if (ncopy) {
        cudaError_t e = cudaMemcpyAsync(host_out, r.ring, ncopy * sizeof(hr_race), cudaMemcpyDeviceToHost, ctx->copies);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->copies);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (n_total) *n_total = h.n_races;
    if (flags) *flags = h.flags | (h.n_races > cap ? HR_FLAG_TRUNCATED : 0u);
    return (hr_status)h.error;
}

extern "C" hr_status hr_counters(hr_ctx* ctx, uint32_t region, uint64_t out[4])
{
    if (!valid_region(ctx, region) || !out) return HR_ERR_INVALID;
    hr_region_dev h;
    hr_status st = fetch_region(ctx, region, &h);
    if (st != HR_OK) return st;
    for (int i = 0; i < 4; ++i) out[i] = h.counters[i];
    return HR_OK;
}

extern "C" hr_status hr_reset(hr_ctx* ctx, uint32_t region, hr_stream_t stream)
{
    if (!valid_region(ctx, region)) return HR_ERR_INVALID;
    RegionHost& r = ctx->regions[region];
    cudaStream_t s = (cudaStream_t)stream;
    (void)cudaGetLastError();  // report only errors of this call's launches
    cudaError_t e = hr_launch_reset(r.d, r.shadow, r.desc.n_words * hr_desc_shadow_bytes(r.desc), s);
    if (e == cudaSuccess) e = mark_done(r, s);
    r.kernel = 0;
    return cuda_status(e);
}

extern "C" hr_status hr_region_reconfigure(hr_ctx* ctx, uint32_t region, uint64_t n_words, uint32_t block_dim,
                                           uint32_t warp_size, hr_stream_t stream)
{
    if (!valid_region(ctx, region)) return HR_ERR_INVALID;
    RegionHost& r = ctx->regions[region];
    if (n_words == 0 || n_words > r.capacity || block_dim == 0 || warp_size == 0 || warp_size > 32)
        return HR_ERR_INVALID;
    if (r.desc.shadow_bytes == 4 && block_dim > (1u << hr_desc_tid_bits(r.desc))) return HR_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    (void)cudaGetLastError();  // report only errors of this call's launches
    r.desc.n_words = n_words;
    r.desc.block_dim = block_dim;
    r.desc.warp_size = warp_size;
    r.filter = hr_filter_all();
    cudaError_t e = hr_launch_reconfigure(r.d, n_words, hr_desc_geom(r.desc), s);
    if (e == cudaSuccess) e = hr_launch_reset(r.d, r.shadow, n_words * hr_desc_shadow_bytes(r.desc), s);
    if (e == cudaSuccess) e = mark_done(r, s);
    r.kernel = 0;
    return cuda_status(e);
}

extern "C" hr_status hr_set_filter(hr_ctx* ctx, uint32_t region, const hr_filter* filter, hr_stream_t stream)
{
    if (!valid_region(ctx, region)) return HR_ERR_INVALID;
    RegionHost& r = ctx->regions[region];
    const hr_filter f = filter ? *filter : hr_filter_all();
    if (f.reserved != 0 || f.lane_mask == 0) return HR_ERR_INVALID;
    if (f.word_hi == 0 ? f.word_lo != 0 : (f.word_hi <= f.word_lo || f.word_hi - f.word_lo > r.desc.n_words))
        return HR_ERR_INVALID;
    if (f.word_hi > (1ull << 32)) return HR_ERR_INVALID;  // record word indices are 32-bit
    if (f.block_hi != 0 && f.block_hi < f.block_lo) return HR_ERR_INVALID;
    if (f.sym_hi != 0 && f.sym_hi <= f.sym_lo) return HR_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    (void)cudaGetLastError();  // report only errors of this call's launches
    cudaError_t e = hr_launch_set_filter(r.d, f, s);
    if (e == cudaSuccess) {
        r.filter = f;
        e = mark_done(r, s);
    }
    return cuda_status(e);
}

extern "C" hr_status hr_destroy(hr_ctx* ctx)
{
    if (!ctx) return HR_ERR_INVALID;
    cudaError_t e = cudaDeviceSynchronize();
    free_ctx(ctx);
    return cuda_status(e);
}

extern "C" hr_status hr_device_view(hr_ctx* ctx, uint32_t region, hr_view* out)
{
    if (!valid_region(ctx, region) || !out) return HR_ERR_INVALID;
    RegionHost& r = ctx->regions[region];
    hr_region_dev* d = r.d;
    r.views = true;
    out->shadow = r.shadow;
    out->ring = r.ring;
    out->n_races = &d->n_races;
    out->error = &d->error;
    out->flags = &d->flags;
    out->table = ctx->d_table;
    out->n_words = r.desc.n_words;
    out->ring_cap = r.ring_cap;
    out->geom = hr_desc_geom(r.desc);
    out->filter = r.filter;
    out->kernel = r.kernel;
    out->region = region;
    return HR_OK;
}

extern "C" uint32_t hr_variant_count(void) { return HR_N_VARIANTS; }

extern "C" hr_status hr_variant_desc(uint32_t id, uint32_t* aggregate, uint32_t* records_per_lane,
                                     uint32_t* consumer_warps)
{
    if (id >= HR_N_VARIANTS) return HR_ERR_INVALID;
    const bool shape = id < HR_N_SHAPES;  // else the binned checker: all zero
    if (aggregate) *aggregate = shape ? (uint32_t)HR_VARIANTS[id].aggregate : 0u;
    if (records_per_lane) *records_per_lane = shape ? (uint32_t)HR_VARIANTS[id].rpl : 0u;
    if (consumer_warps) *consumer_warps = shape ? (uint32_t)HR_VARIANTS[id].consumers : 0u;
    return HR_OK;
}

extern "C" hr_status hr_set_variant(hr_ctx* ctx, uint32_t id)
{
    if (!ctx || id >= HR_N_VARIANTS) return HR_ERR_INVALID;
    ctx->variant = id;
    return HR_OK;
}

extern "C" hr_status hr_get_variant(hr_ctx* ctx, uint32_t* id)
{
    if (!ctx || !id) return HR_ERR_INVALID;
    *id = ctx->variant;
    return HR_OK;
}

extern "C" hr_status hr_autotune(hr_ctx* ctx, uint32_t region, const hr_record* d_trace, uint64_t n,
                                 hr_stream_t stream, uint32_t* best, float* ms, uint32_t ms_cap)
{
    if (!valid_region(ctx, region) || !d_trace || n == 0 || (ms_cap > 0 && !ms)) return HR_ERR_INVALID;
    // every-epoch regions always run their own checker; there is nothing to choose
    if (ctx->regions[region].desc.report_mode == HR_REPORT_EVERY_EPOCH) return HR_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    const unsigned saved = ctx->variant;
    const bool saved_profile = ctx->profile;
    ctx->profile = false;
    float best_ms = 0.0f;
    unsigned best_v = saved;
    bool have_best = false;
    hr_status st = HR_OK;
    for (unsigned v = 0; v < HR_N_VARIANTS && e == cudaSuccess && st == HR_OK; ++v) {
        ctx->variant = v;
        float t = 0.0f;
        for (int rep = 0; rep < 2 && st == HR_OK && e == cudaSuccess; ++rep) {  // warm-up, then timed
            st = hr_reset(ctx, region, stream);
            if (st == HR_OK) e = cudaEventRecord(a, s);
            if (st == HR_OK && e == cudaSuccess) st = check_common(ctx, region, d_trace, n, 0, stream, true);
            if (st == HR_OK && e == cudaSuccess) e = cudaEventRecord(b, s);
            if (st == HR_OK && e == cudaSuccess) e = cudaEventSynchronize(b);
            if (st == HR_OK && e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
        }
        hr_region_dev h;
        if (st == HR_OK && e == cudaSuccess) st = fetch_region(ctx, region, &h);
        bool usable = true;
        if (st == HR_OK && h.error != 0) {
            // a bounded retry or wait that ran out belongs to this variant: skip it;
            // any other error is the trace's own
            if (h.error == HR_ERR_CONTENTION || h.error == HR_ERR_TIMEOUT) {
                usable = false;
                t = -1.0f;
            } else {
                st = (hr_status)h.error;
            }
        }
        if (v < ms_cap) ms[v] = t;
        if (st == HR_OK && e == cudaSuccess && usable && (!have_best || t < best_ms)) {
            best_ms = t;
            best_v = v;
            have_best = true;
        }
    }
    ctx->profile = saved_profile;
    ctx->variant = (st == HR_OK && e == cudaSuccess) ? best_v : saved;
    if (best) *best = ctx->variant;
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (st == HR_OK) st = hr_reset(ctx, region, stream);
    return st != HR_OK ? st : cuda_status(e);
}

extern "C" hr_status hr_set_limits(hr_ctx* ctx, uint64_t wait_ns, uint32_t cas_retry_cap, uint32_t test_flags)
{
    if (!ctx || wait_ns == 0 || (test_flags & ~HR_TEST_HOLD_STAGE)) return HR_ERR_INVALID;
    ctx->wait_ns = wait_ns;
    ctx->cas_cap = cas_retry_cap;
    ctx->test_flags = test_flags;
    return HR_OK;
}

extern "C" hr_status hr_profile_enable(hr_ctx* ctx, int on)
{
    if (!ctx) return HR_ERR_INVALID;
    ctx->profile = on != 0;
    return HR_OK;
}

extern "C" hr_status hr_profile_read(hr_ctx* ctx, double* check_ms, double* prepass_ms, uint64_t* calls,
                                     uint64_t* launches)
{
    if (!ctx) return HR_ERR_INVALID;
    double ck = 0, pre = 0;
    uint64_t nl = 0;
    cudaError_t e = cudaSuccess;
    for (auto& p : ctx->calls) {
        float a = 0, b = 0;
        if (e == cudaSuccess) e = cudaEventSynchronize(p.end);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&a, p.begin, p.mid);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&b, p.mid, p.end);
        pre += a;
        ck += b;
        nl += p.launches;
    }
    if (check_ms) *check_ms = ck;
    if (prepass_ms) *prepass_ms = pre;
    if (calls) *calls = ctx->calls.size();
    if (launches) *launches = nl;
    ctx->spare.insert(ctx->spare.end(), ctx->calls.begin(), ctx->calls.end());
    ctx->calls.clear();
    return cuda_status(e);
}

extern "C" const char* hr_status_str(hr_status s)
{
    switch (s) {
    case HR_OK: return "ok";
    case HR_ERR_INVALID: return "invalid argument";
    case HR_ERR_OOM: return "out of memory";
    case HR_ERR_CUDA: return "CUDA runtime error";
    case HR_ERR_ORDER: return "trace not sorted by (kernel, bc, wc) or older than the region's last record";
    case HR_ERR_RANGE: return "word index out of range";
    case HR_ERR_CLOCK_OVERFLOW: return "clock overflow";
    case HR_ERR_CONTENTION: return "CAS retry cap reached";
    case HR_ERR_TIMEOUT: return "bounded device wait expired";
    case HR_ERR_UNSUPPORTED: return "unsupported record (partial-mask __syncwarp or unknown op)";
    case HR_ERR_CAPACITY: return "too many waves in one call";
    case HR_ERR_NOT_READY: return "region busy";
    }
    return "unknown status";
}

extern "C" const char* hr_version(void) { return "hirace-gb300 0.1 (sm_103a)"; }
