// mcd_peaks.cu -- microbenchmarks of this GPU's shared-memory bandwidth and
// FP32 / FP64 FMA throughput, the denominators of the collide kernel's
// rooflines (the paper has no counterpart: this is measurement only).
//
// Shared memory: every SM runs two CTAs of 1024 threads; each warp reads
// 16 bytes per lane per load from consecutive addresses (four 128-byte
// wavefronts, no bank conflict) and folds the words with one three-input XOR,
// so the shared-memory pipe, not the issue slots, sets the pace.  FMA: eight
// independent FMA chains per thread, four CTAs of 512 threads per SM.  Each
// kernel runs once to warm up and three times timed with CUDA events on the
// given stream; the median counts.
#include "mcd_internal.cuh"

namespace {

constexpr int kSmemThreads = 1024, kFmaThreads = 512;

// the kernels' sinks are written only on values they never reach; a small
// static array gives them a valid address without an allocation
__device__ double g_sink[4096];

__global__ void __launch_bounds__(kSmemThreads) k_smem_read(int iters, unsigned *sink)
{
    __shared__ uint4 buf[kSmemThreads];
    buf[threadIdx.x] = make_uint4(threadIdx.x, threadIdx.x * 3u, threadIdx.x ^ 5u, 7u);
    __syncthreads();
    unsigned a = 0, b = 0;
    unsigned idx = threadIdx.x;
#pragma unroll 8
    for (int it = 0; it < iters; ++it) {
        const uint4 v = buf[idx];
        asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(a) : "r"(a), "r"(v.x), "r"(v.y));
        asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(b) : "r"(b), "r"(v.z), "r"(v.w));
        idx = (idx + 32u) & (kSmemThreads - 1);
    }
    if ((a ^ b) == 0x9E3779B9u) sink[blockIdx.x] = a;  // (keeps the loads; practically never taken)
}

template <class T>
__global__ void __launch_bounds__(kFmaThreads) k_fma(int iters, T x, T *sink)
{
    T a0 = x, a1 = x + (T)1, a2 = x + (T)2, a3 = x + (T)3, a4 = x + (T)4, a5 = x + (T)5, a6 = x + (T)6,
      a7 = x + (T)7;
    const T m = (T)0.999999, c = (T)1e-7;
#pragma unroll 4
    for (int it = 0; it < iters; ++it) {
        a0 = fma(a0, m, c);
        a1 = fma(a1, m, c);
        a2 = fma(a2, m, c);
        a3 = fma(a3, m, c);
        a4 = fma(a4, m, c);
        a5 = fma(a5, m, c);
        a6 = fma(a6, m, c);
        a7 = fma(a7, m, c);
    }
    const T s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
    if (s == (T)-1) sink[blockIdx.x] = s;  // (keeps the chains; never taken)
}

template <class F>
cudaError_t median_ms(F launch, cudaStream_t st, float *out)
{
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float ms[4] = {};
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(a, st);
        if (e == cudaSuccess) launch();
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[rep], a, b);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    // the median of the three timed runs (the first warms up)
    float x = ms[1], y = ms[2], z = ms[3];
    *out = x > y ? (y > z ? y : (x > z ? z : x)) : (x > z ? x : (y > z ? z : y));
    return e;
}

}  // namespace

extern "C" int mcd_probe_peaks(mcd_peaks *out, void *cuda_stream)
{
    if (!out) return MCD_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, nsm = 0, clk = 0, l2 = 0, smsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smsm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e != cudaSuccess) return MCD_ECUDA;
    void *sp = nullptr;
    if (cudaGetSymbolAddress(&sp, g_sink) != cudaSuccess) return MCD_ECUDA;
    const int smem_iters = 1 << 14, fma_iters = 1 << 14;
    const unsigned g_smem = (unsigned)nsm * 2, g_fma = (unsigned)nsm * 4;
    float t_smem = 0, t32 = 0, t64 = 0;
    e = median_ms([&] { k_smem_read<<<g_smem, kSmemThreads, 0, st>>>(smem_iters, (unsigned *)sp); }, st, &t_smem);
    if (e == cudaSuccess)
        e = median_ms([&] { k_fma<float><<<g_fma, kFmaThreads, 0, st>>>(fma_iters, 1.0f, (float *)sp); }, st, &t32);
    if (e == cudaSuccess)
        e = median_ms([&] { k_fma<double><<<g_fma, kFmaThreads, 0, st>>>(fma_iters / 16, 1.0, (double *)sp); }, st,
                      &t64);
    if (e != cudaSuccess) return MCD_ECUDA;
    const double smem_bytes = (double)g_smem * kSmemThreads * smem_iters * 16.0;
    const double f32 = (double)g_fma * kFmaThreads * fma_iters * 8.0 * 2.0;
    const double f64 = (double)g_fma * kFmaThreads * (fma_iters / 16) * 8.0 * 2.0;
    out->smem_gbs = smem_bytes / (t_smem * 1e-3) / 1e9;
    out->fp32_tflops = f32 / (t32 * 1e-3) / 1e12;
    out->fp64_tflops = f64 / (t64 * 1e-3) / 1e12;
    out->sm_count = nsm;
    out->sm_clock_mhz = clk / 1000;
    out->l2_bytes = l2;
    out->smem_per_sm_bytes = smsm;
    out->ms_smem = t_smem;
    out->ms_fp32 = t32;
    out->ms_fp64 = t64;
    return MCD_OK;
}
