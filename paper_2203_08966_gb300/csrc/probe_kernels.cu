// Measurement aid (no counterpart in the paper): the FP32 fused multiply-add rate this GPU
// sustains, the denominator against which the walk's useful FP32 rate is read besides the
// nominal SMs x 128 lanes x 2 flop x clock.
#include "nbody_internal.cuh"

namespace nb {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;  // independent chains per thread (cover the FMA latency)

// Every thread runs kProbeChains independent chains x <- x * a + b for `iters` rounds; a and b
// keep x bounded and normal, and the sum is stored only when it is impossible (x never reaches
// -1), so the arithmetic cannot be removed.
__global__ void __launch_bounds__(kProbeThreads) ffma_probe_kernel(int iters, float a, float b,
                                                                    float *sink)
{
    float x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = 0.5f + 0.01f * (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int c = 0; c < kProbeChains; ++c) x[c] = fmaf(x[c], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
    if (s == -1.f) sink[blockIdx.x] = s;
}

// The same with FP64 chains (GB300's FP64 rate is a small fraction of its FP32 rate, so the
// caller runs fewer rounds).
__global__ void __launch_bounds__(kProbeThreads) dfma_probe_kernel(int iters, double a, double b,
                                                                    double *sink)
{
    double x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = 0.5 + 0.01 * (double)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int c = 0; c < kProbeChains; ++c) x[c] = fma(x[c], a, b);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
    if (s == -1.0) sink[blockIdx.x] = s;
}

// Times `kernel(iters, ...)` on 8 blocks per SM after a warm-up launch: FMA rate in TFLOP/s.
template <class T, class K>
cudaError_t time_fma(K kernel, int iters, T a, T b, cudaStream_t s, double *tflops)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    T *sink = nullptr;
    e = cudaMalloc(&sink, sizeof(T) * (size_t)sms * 8);
    if (e != cudaSuccess) return e;
    const int blocks = sms * 8;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    kernel<<<blocks, kProbeThreads, 0, s>>>(iters, a, b, sink);  // warm-up
    cudaEventRecord(e0, s);
    kernel<<<blocks, kProbeThreads, 0, s>>>(iters, a, b, sink);
    cudaEventRecord(e1, s);
    count_launches(2);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * (double)blocks * kProbeThreads * iters * 16 * kProbeChains;
    if (e == cudaSuccess) *tflops = ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    return e;
}

}  // namespace

cudaError_t measure_fp64_rate(cudaStream_t s, double *tflops)
{
    return time_fma<double>(dfma_probe_kernel, 64, 0.9999, 1e-4, s, tflops);
}

cudaError_t measure_fp32_rate(cudaStream_t s, double *tflops)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    float *sink = nullptr;
    e = cudaMalloc(&sink, sizeof(float) * (size_t)sms * 8);
    if (e != cudaSuccess) return e;
    const int blocks = sms * 8, iters = 4096;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    ffma_probe_kernel<<<blocks, kProbeThreads, 0, s>>>(iters, 0.9999f, 1e-4f, sink);  // warm-up
    cudaEventRecord(e0, s);
    ffma_probe_kernel<<<blocks, kProbeThreads, 0, s>>>(iters, 0.9999f, 1e-4f, sink);
    cudaEventRecord(e1, s);
    count_launches(2);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * (double)blocks * kProbeThreads * iters * 16 * kProbeChains;
    if (e == cudaSuccess) *tflops = ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    return e;
}

}  // namespace nb
