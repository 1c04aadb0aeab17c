// fp32_peak.cu -- FP32 fused multiply-add throughput of the current device, measured.
//
// Measurement support for the roofline of the force kernel (which is bound by FP32
// arithmetic issue, not by HBM or tensor cores): every thread runs kChains independent
// multiply-add chains, so no instruction waits on its predecessor, over a grid of
// several waves of CTAs per SM.  Two forms: scalar fma.rn.f32 (FFMA) and packed
// fma.rn.f32x2 (two lanes' worth per instruction).  FLOP/s = 2 per lane per multiply-add.
// Host entry points enqueue one launch, time it with CUDA events on the given stream and
// synchronise that stream; nothing is allocated.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

__device__ float g_sink;  // written only if a chain's sum hits a value it never takes

__global__ void __launch_bounds__(kThreads) k_ffma(int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = __fmaf_rn(x[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) g_sink = s;  // keeps the chains live; never true for these inputs
}

__global__ void __launch_bounds__(kThreads) k_ffma2(int iters, float a, float b)
{
    unsigned long long x[kChains];
    unsigned long long av, bv;
    asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        const float lo = (float)(threadIdx.x + c), hi = lo + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(lo), "f"(hi));
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(av), "l"(bv));
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    if (s == 12345.678f) g_sink = s;
}

}  // namespace

extern "C" {

// SMs of the current device (cudaDeviceProp::multiProcessorCount), or -1.
int mdp_sm_count(void)
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    return n;
}

// One timed launch: `packed` 0 = FFMA, 1 = FFMA2; grid = blocks_per_sm x SMs CTAs of 256
// threads, `iters` iterations of kChains chains.  Writes the event-timed milliseconds and
// the FP32 operations executed (2 per lane per multiply-add); returns 0 or a CUDA error.
int mdp_fma_run(int packed, int blocks_per_sm, int iters, void *stream, double *ms_out,
                double *flop_out)
{
    const int sms = mdp_sm_count();
    if (sms <= 0 || blocks_per_sm <= 0 || iters <= 0 || !ms_out || !flop_out) return -1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const dim3 grid((unsigned)(blocks_per_sm * sms));
    cudaEventRecord(a, s);
    if (packed)
        k_ffma2<<<grid, kThreads, 0, s>>>(iters, 0.999999f, 1e-7f);
    else
        k_ffma<<<grid, kThreads, 0, s>>>(iters, 0.999999f, 1e-7f);
    cudaEventRecord(b, s);
    e = cudaEventSynchronize(b);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return (int)e;
    *ms_out = ms;
    *flop_out = 2.0 * (packed ? 2.0 : 1.0) * kChains * (double)iters * kThreads * (double)grid.x;
    return 0;
}

}  // extern "C"
