// fxtest.cu -- test entry points: element-wise evaluation of the library's
// log/exp (fixed-point series) and single-precision cosine, and of CUDA's,
// over a device array, for accuracy tests; and one axis's Adjust-Bin-Bounds
// on a given histogram, for parity tests of the device rebinning.
#include <algorithm>

#include "refine_dev.cuh"

namespace {

// the fixed factor of selftest 6: (kScaleM / 2^63) 2^kScaleE, a significand
// above 1.5 so that products with most exponentials reach [2, 4) and take the
// renormalising step
constexpr uint64_t kScaleM = 0xD3C21BCECCEDA100ull;
constexpr int kScaleE = 40;

__global__ void fxmath_kernel(int which, long long n, const double* in, double* out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double x = in[i];
        double y;
        switch (which) {
        case 0: y = mc::fx::fx_log(x); break;
        case 1: y = mc::fx::fx_exp(x); break;
        case 2: y = log(x); break;
        case 3: y = exp(x); break;
        case 4: y = (double)mc::fx::fx_cosf((float)x); break;
        case 5: y = (double)cosf((float)x); break;
        default: y = mc::fx::fx_exp_neg_scaled(x, kScaleM, kScaleE); break;
        }
        out[i] = y;
    }
}

__device__ int g_rebin_flags[2];  // error, done

__global__ void __launch_bounds__(mc::kRefineThreads)
rebin_kernel(int nb, double alpha, double* C, double* B, double* Blo)
{
    __shared__ double scratch[33];
    // the histogram is its own single partial; its sum is written back in place
    mc::refine_detail::rebin_axis(C, 0, 1, false, nb, alpha, B, Blo, C, &g_rebin_flags[0], &g_rebin_flags[1],
                                  scratch);
}

}  // namespace

extern "C" mcubes_status mcubes_selftest_rebin(int nb, double alpha, double* d_C, double* d_B, double* d_Blo,
                                              void* cuda_stream)
{
    if (nb < 2 || nb > MCUBES_NBMAX || !(alpha > 0.0) || !d_C || !d_B || !d_Blo) return MCUBES_EINVAL;
    const cudaStream_t s = (cudaStream_t)cuda_stream;
    const int zero[2] = {0, 0};
    int flags[2] = {0, 0};
    if (cudaMemcpyToSymbolAsync(g_rebin_flags, zero, sizeof zero, 0, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return MCUBES_ECUDA;
    rebin_kernel<<<1, mc::kRefineThreads, 0, s>>>(nb, alpha, d_C, d_B, d_Blo);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyFromSymbolAsync(flags, g_rebin_flags, sizeof flags, 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return MCUBES_ECUDA;
    return flags[0] ? (mcubes_status)flags[0] : MCUBES_OK;
}

extern "C" mcubes_status mcubes_selftest_fxmath(int which, long long n, const double* d_in, double* d_out,
                                               void* cuda_stream)
{
    if (which < 0 || which > 6 || n < 0 || (n > 0 && (!d_in || !d_out))) return MCUBES_EINVAL;
    if (n == 0) return MCUBES_OK;
    fxmath_kernel<<<(int)std::min<long long>((n + 255) / 256, 65535), 256, 0, (cudaStream_t)cuda_stream>>>(
        which, n, d_in, d_out);
    return cudaGetLastError() == cudaSuccess ? MCUBES_OK : MCUBES_ECUDA;
}
