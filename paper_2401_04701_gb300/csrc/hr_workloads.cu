// hr_workloads.cu - hand-instrumented synthetic kernels (libhirace_workloads.so).
//
// Three small CUDA kernels written the way a user instruments code by hand
// with include/hirace_device.cuh: every monitored load, store or atomic is
// paired with hr_access(), and __syncthreads() is replaced by
// hr_syncthreads() so the thread's block clock advances at the barrier.
// Each kernel also runs uninstrumented (view == NULL) so the instrumented
// slowdown can be measured on identical work.  Optional race injection makes
// a chosen subset of threads misbehave.
//
// Monitored words of one region:
//   stencil    in[0..n) -> words [0, n), out[0..n) -> words [n, 2n)
//   histogram  bins[0..n_bins) -> words [0, n_bins)
//   reduction  data[0..n) -> words [0, n)
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/hirace_device.cuh"

namespace {

template <bool INSTR>
__global__ void stencil_kernel(hr_view v, const float* in, float* out, float* in_w, uint32_t n, uint32_t racy_stride)
{
    hr_clock c = hr_clock_init();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = in[i];
    if (INSTR) hr_access(v, i, HR_R, c);
    if (i > 0) {
        s += in[i - 1];
        if (INSTR) hr_access(v, i - 1, HR_R, c);
    }
    if (i + 1 < n) {
        s += in[i + 1];
        if (INSTR) hr_access(v, i + 1, HR_R, c);
    }
    out[i] = s;
    if (INSTR) hr_access(v, (unsigned long long)n + i, HR_W, c);
    if (racy_stride && i % racy_stride == 0) {  // injected bug: write back into the input
        in_w[i] = s;
        if (INSTR) hr_access(v, i, HR_W, c);
    }
}

template <bool INSTR>
__global__ void histogram_kernel(hr_view v, const uint32_t* keys, uint32_t n, uint32_t* bins, uint32_t racy_stride)
{
    hr_clock c = hr_clock_init();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t b = keys[i];
    if (racy_stride && i % racy_stride == 0) {  // injected bug: plain read-modify-write
        const uint32_t x = bins[b];
        if (INSTR) hr_access(v, b, HR_R, c);
        bins[b] = x + 1;
        if (INSTR) hr_access(v, b, HR_W, c);
    } else {
        atomicAdd(bins + b, 1u);
        if (INSTR) hr_access(v, b, HR_A, c);
    }
}

// Block-level tree reduction over data[2*blockDim*blockIdx ...]: at each level
// thread t < s adds element t+s into element t, with a barrier between levels.
// drop_level >= 0 removes the barrier after that level in every block.
template <bool INSTR>
__global__ void reduce_kernel(hr_view v, float* data, uint32_t n, int drop_level)
{
    hr_clock c = hr_clock_init();
    const uint32_t base = 2u * blockDim.x * blockIdx.x;
    const uint32_t t = threadIdx.x;
    int level = 0;
    for (uint32_t s = blockDim.x; s > 0; s >>= 1, ++level) {
        if (t < s && base + t + s < n) {
            const float a = data[base + t];
            if (INSTR) hr_access(v, base + t, HR_R, c);
            const float b = data[base + t + s];
            if (INSTR) hr_access(v, base + t + s, HR_R, c);
            data[base + t] = a + b;
            if (INSTR) hr_access(v, base + t, HR_W, c);
        }
        if (level != drop_level) {
            if (INSTR)
                hr_syncthreads(c);
            else
                __syncthreads();
        }
    }
}

// Block reduction through a __shared__ buffer of blockDim floats: every thread
// stores its element, then at level L threads t < s = blockDim >> (L + 1) add
// buf[t + s] into buf[t] with a barrier after each level (the one after level
// drop_level removed), and thread 0 writes the block's sum.  MODE 0: plain;
// 1: monitored through the region's global shadow (word = block * blockDim + t);
// 2: monitored through a shadow in shared memory beside the buffer.
template <int MODE>
__global__ void smem_reduce_kernel(hr_view v, const float* in, float* out, uint32_t n, int drop_level)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const uint32_t bd = blockDim.x;
    float* buf = reinterpret_cast<float*>(sm);
    unsigned long long* sh = reinterpret_cast<unsigned long long*>(sm + ((bd * 4 + 15) & ~15u));
    hr_clock c = hr_clock_init();
    hr_smem_view sv{};
    if (MODE == 2) sv = hr_smem_begin(sh, bd);
    const uint32_t t = threadIdx.x;
    const uint32_t i = blockIdx.x * bd + t;
    auto mon = [&](uint32_t word, uint32_t op) {
        if (MODE == 1) hr_access(v, (unsigned long long)blockIdx.x * bd + word, op, c);
        if (MODE == 2) hr_access_shared(v, sv, word, op, c);
    };
    auto barrier = [&]() {
        if (MODE) hr_syncthreads(c);
        else __syncthreads();
    };
    buf[t] = i < n ? in[i] : 0.f;
    mon(t, HR_W);
    barrier();
    int level = 0;
    for (uint32_t s = bd >> 1; s > 0; s >>= 1, ++level) {
        if (t < s) {
            const float a = buf[t];
            mon(t, HR_R);
            const float b2 = buf[t + s];
            mon(t + s, HR_R);
            buf[t] = a + b2;
            mon(t, HR_W);
        }
        if (level != drop_level) barrier();
    }
    if (t == 0) {
        out[blockIdx.x] = buf[0];
        mon(0, HR_R);
    }
}

hr_view null_view()
{
    hr_view v{};
    return v;
}

}  // namespace

extern "C" int hrw_stencil(const hr_view* view, const float* in, float* out, uint32_t n, uint32_t block,
                           uint32_t racy_stride, hr_stream_t stream)
{
    if (!in || !out || n == 0 || block == 0 || block > 1024) return 1;
    const uint32_t grid = (n + block - 1) / block;
    cudaStream_t s = (cudaStream_t)stream;
    if (view)
        stencil_kernel<true><<<grid, block, 0, s>>>(*view, in, out, const_cast<float*>(in), n, racy_stride);
    else
        stencil_kernel<false><<<grid, block, 0, s>>>(null_view(), in, out, const_cast<float*>(in), n, racy_stride);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

extern "C" int hrw_histogram(const hr_view* view, const uint32_t* keys, uint32_t n, uint32_t* bins, uint32_t block,
                             uint32_t racy_stride, hr_stream_t stream)
{
    if (!keys || !bins || n == 0 || block == 0 || block > 1024) return 1;
    const uint32_t grid = (n + block - 1) / block;
    cudaStream_t s = (cudaStream_t)stream;
    if (view)
        histogram_kernel<true><<<grid, block, 0, s>>>(*view, keys, n, bins, racy_stride);
    else
        histogram_kernel<false><<<grid, block, 0, s>>>(null_view(), keys, n, bins, racy_stride);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

extern "C" int hrw_reduce(const hr_view* view, float* data, uint32_t n, uint32_t block, int drop_level,
                          hr_stream_t stream)
{
    if (!data || n == 0 || block == 0 || block > 1024 || (block & (block - 1))) return 1;
    const uint32_t grid = (n + 2 * block - 1) / (2 * block);
    cudaStream_t s = (cudaStream_t)stream;
    if (view)
        reduce_kernel<true><<<grid, block, 0, s>>>(*view, data, n, drop_level);
    else
        reduce_kernel<false><<<grid, block, 0, s>>>(null_view(), data, n, drop_level);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

// Shared-memory block reduction over in[0..n) into out[0..grid): mode 0 plain,
// 1 global shadow (view required), 2 shared-memory shadow (view required).
// block must be a power of two <= 1024.  Returns 0, 1 for bad arguments.
extern "C" int hrw_smem_reduce(const hr_view* view, int mode, const float* in, float* out, uint32_t n,
                               uint32_t block, int drop_level, hr_stream_t stream)
{
    if (!in || !out || n == 0 || block == 0 || block > 1024 || (block & (block - 1)) || mode < 0 || mode > 2 ||
        (mode && !view))
        return 1;
    const uint32_t grid = (n + block - 1) / block;
    const size_t smem = ((block * 4 + 15) & ~15u) + (mode == 2 ? block * 8 : 0);
    cudaStream_t s = (cudaStream_t)stream;
    if (mode == 0)
        smem_reduce_kernel<0><<<grid, block, smem, s>>>(null_view(), in, out, n, drop_level);
    else if (mode == 1)
        smem_reduce_kernel<1><<<grid, block, smem, s>>>(*view, in, out, n, drop_level);
    else
        smem_reduce_kernel<2><<<grid, block, smem, s>>>(*view, in, out, n, drop_level);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}
