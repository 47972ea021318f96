// fxtest.cu -- element-wise evaluation of the library's log/exp (fixed-point
// series) and single-precision cosine, and of CUDA's, over a device array,
// for accuracy tests.
#include <algorithm>

#include "mc_device.cuh"

namespace {

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
        default: y = (double)cosf((float)x); break;
        }
        out[i] = y;
    }
}

}  // namespace

extern "C" mcubes_status mcubes_selftest_fxmath(int which, long long n, const double* d_in, double* d_out,
                                               void* cuda_stream)
{
    if (which < 0 || which > 5 || n < 0 || (n > 0 && (!d_in || !d_out))) return MCUBES_EINVAL;
    if (n == 0) return MCUBES_OK;
    fxmath_kernel<<<(int)std::min<long long>((n + 255) / 256, 65535), 256, 0, (cudaStream_t)cuda_stream>>>(
        which, n, d_in, d_out);
    return cudaGetLastError() == cudaSuccess ? MCUBES_OK : MCUBES_ECUDA;
}
