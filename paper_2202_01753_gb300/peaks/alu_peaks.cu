// alu_peaks.cu -- measured arithmetic peaks of the device, the denominators
// of the sampling kernel's roofline: fused multiply-add throughput in single
// and double precision, and the double-precision add and multiply, from long
// independent chains in every thread of a full grid, timed with CUDA events.
#include <cstdio>

#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

// OP 0: x = fma(x, a, b); 1: x = x + b; 2: x = x * a
template <typename T, int OP>
__global__ void __launch_bounds__(kThreads) fma_chains(T* sink, T a, T b, int iters)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                if constexpr (OP == 0) x[c] = fma(x[c], a, b);
                else if constexpr (OP == 1) x[c] = x[c] + b;
                else x[c] = x[c] * a;
            }
        }
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)-1.2345) sink[blockIdx.x] = s;  // keeps the chains alive; never true
}

template <typename T, int OP = 0>
int measure(int blocks_per_sm, int iters, double* ops_per_s, float* ms_out)
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
    fma_chains<T, OP><<<grid, kThreads>>>(sink, (T)0.9999999, (T)1e-7, iters / 8);  // warm
    cudaEventRecord(e0);
    fma_chains<T, OP><<<grid, kThreads>>>(sink, (T)0.9999999, (T)1e-7, iters);
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess) return 2;
    const double ops = (double)grid * kThreads * iters * kUnroll * kChains;
    *ops_per_s = ops / (ms * 1e-3);
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

// Double-precision additions and multiplications per second over the whole
// device (the other instructions of the FP64 pipe).  Returns 0 on success.
extern "C" int mcpeaks_fp64_addmul(int device, double* dadd_per_s, double* dmul_per_s)
{
    if (cudaSetDevice(device) != cudaSuccess) return 3;
    float ms = 0.f;
    int r = measure<double, 1>(8, 64, dadd_per_s, &ms);
    if (r) return r;
    return measure<double, 2>(8, 64, dmul_per_s, &ms);
}
