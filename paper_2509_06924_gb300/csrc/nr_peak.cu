// nr_peak.cu -- throughput probes of the arithmetic pipes that bound the
// reflectivity kernels: scalar FP32 FMA, paired FP32 FMA (fma.rn.f32x2, two
// FP32 FMAs per thread instruction), FP64 FMA and the special-function unit
// (ex2.approx).  The measured rates are the denominators of the kernels'
// roofline fractions; the nominal figures (lanes x clock) only say what the
// hardware is meant to do.
//
// Every thread runs CH independent dependency chains, unrolled, so that each
// SM sub-partition always has an independent instruction to issue; the
// chains are contractions (|b| < 1) that stay finite and normal for any
// length.  Each thread writes its sum once, so that nothing is optimised
// away; the store is one word per thread against thousands of operations.
//
// Built into its own library (libnr_peak.so), used by the benchmark only.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 16;

template <int CH>
__global__ void __launch_bounds__(kThreads) peak_ffma(float *out, float b, float c, int iters)
{
    float a[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) a[i] = 1e-3f * (float)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int i = 0; i < CH; ++i) a[i] = fmaf(a[i], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int CH>
__global__ void __launch_bounds__(kThreads) peak_ffma2(float *out, float b, float c, int iters)
{
    float2 a[CH];
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, 0.5f * c);
#pragma unroll
    for (int i = 0; i < CH; ++i) a[i] = make_float2(1e-3f * (float)(threadIdx.x + i), 2e-3f * (float)i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int i = 0; i < CH; ++i) a[i] = __ffma2_rn(a[i], b2, c2);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += a[i].x + a[i].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int CH>
__global__ void __launch_bounds__(kThreads) peak_dfma(float *out, float b, float c, int iters)
{
    double a[CH];
    const double bd = b, cd = c;
#pragma unroll
    for (int i = 0; i < CH; ++i) a[i] = 1e-3 * (double)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int i = 0; i < CH; ++i) a[i] = fma(a[i], bd, cd);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

// x -> 2^(-x): maps (0, inf) into (0, 1), so the chain stays bounded
__device__ __forceinline__ float ex2_neg(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
    return y;
}

template <int CH>
__global__ void __launch_bounds__(kThreads) peak_ex2(float *out, float, float, int iters)
{
    float a[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) a[i] = 1e-3f * (float)(threadIdx.x + i) + 0.25f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int i = 0; i < CH; ++i) a[i] = ex2_neg(a[i]);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

constexpr int kChains = 8;

using PeakKernel = void (*)(float *, float, float, int);

PeakKernel kernel_of(int kind)
{
    switch (kind) {
    case 0: return peak_ffma<kChains>;
    case 1: return peak_ffma2<kChains>;
    case 2: return peak_dfma<kChains>;
    case 3: return peak_ex2<kChains>;
    default: return nullptr;
    }
}

// operations one thread performs per loop iteration: flops for the FMA
// kinds (an FMA is 2, a paired FMA 4), results for ex2
double ops_per_iter(int kind)
{
    switch (kind) {
    case 0: return 2.0 * kUnroll * kChains;
    case 1: return 4.0 * kUnroll * kChains;
    case 2: return 2.0 * kUnroll * kChains;
    case 3: return 1.0 * kUnroll * kChains;
    default: return 0.0;
    }
}

} // namespace

extern "C" {

// Threads per CTA of every probe; `out` must hold grid x 256 floats.
int nr_peak_threads(void) { return kThreads; }

// Runs probe `kind` (0 FP32 FMA, 1 paired FP32 FMA, 2 FP64 FMA, 3 ex2) on
// the current device: `ctas_per_sm` x SM-count CTAs of 256 threads, `iters`
// loop iterations per thread, launched `reps` times back to back on the
// legacy default stream after one warm-up launch.  `out` is a device buffer
// of at least ctas_per_sm x SMs x 256 floats.  On success writes the elapsed
// time of the `reps` launches (CUDA events, ms) and the operations they
// performed (flops for the FMA kinds, results for ex2) and returns 0;
// otherwise returns the CUDA error code (or -1 for a bad argument).
int nr_peak_run(int kind, int ctas_per_sm, int iters, int reps, float *out, double *ms_out, double *ops_out)
{
    PeakKernel k = kernel_of(kind);
    if (!k || ctas_per_sm < 1 || iters < 1 || reps < 1 || !out || !ms_out || !ops_out) return -1;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    const int grid = sms * ctas_per_sm;
    const float b = 0.999f, c = 1e-3f;
    k<<<grid, kThreads>>>(out, b, c, iters);
    if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return (int)e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return (int)e;
    }
    cudaEventRecord(e0, 0);
    for (int r = 0; r < reps; ++r) k<<<grid, kThreads>>>(out, b, c, iters);
    cudaEventRecord(e1, 0);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return (int)e;
    *ms_out = ms;
    *ops_out = ops_per_iter(kind) * (double)iters * (double)reps * (double)grid * kThreads;
    return 0;
}

} // extern "C"
