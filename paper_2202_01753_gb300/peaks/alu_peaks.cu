// alu_peaks.cu -- measured arithmetic peaks of the device, the denominators
// of the sampling kernel's roofline: fused multiply-add throughput in single
// and double precision, from long independent FMA chains in every thread of a
// full grid, timed with CUDA events.
#include <cstdio>

#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chains(T* sink, T a, T b, int iters)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
        }
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)-1.2345) sink[blockIdx.x] = s;  // keeps the chains alive; never true
}

template <typename T>
int measure(int blocks_per_sm, int iters, double* fma_per_s, float* ms_out)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    T* sink = nullptr;
    if (cudaMalloc(&sink, sizeof(T) * sms * blocks_per_sm) != cudaSuccess) return 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int grid = sms * blocks_per_sm;
    fma_chains<T><<<grid, kThreads>>>(sink, (T)0.9999999, (T)1e-7, iters / 8);  // warm
    cudaEventRecord(e0);
    fma_chains<T><<<grid, kThreads>>>(sink, (T)0.9999999, (T)1e-7, iters);
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess) return 2;
    const double fmas = (double)grid * kThreads * iters * kUnroll * kChains;
    *fma_per_s = fmas / (ms * 1e-3);
    *ms_out = ms;
    return 0;
}

}  // namespace

// FMA/s in single and double precision over the whole device (one FMA = 2
// flops) and the duration of each timed launch.  Returns 0 on success.
extern "C" int mcpeaks_fma(int device, double* ffma_per_s, double* dfma_per_s, float* ms_f32, float* ms_f64)
{
    if (cudaSetDevice(device) != cudaSuccess) return 3;
    int r = measure<float>(8, 2048, ffma_per_s, ms_f32);
    if (r) return r;
    return measure<double>(8, 64, dfma_per_s, ms_f64);
}
