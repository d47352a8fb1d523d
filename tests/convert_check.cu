// Test harness for csrc/convert.cuh: the integer-pipe conversions and the
// GPU's own conversions of the same inputs, side by side.
#include <cuda_runtime.h>

#include "convert.cuh"

__global__ void k_convert_check(long long n, const double *x, float *sw32, float *hw32,
                                const float *f, double *sw64, double *hw64) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        sw32[i] = emin::f64_to_f32_rn(x[i]);
        hw32[i] = __double2float_rn(x[i]);
        sw64[i] = emin::f32_to_f64(f[i]);
        hw64[i] = (double)f[i];
    }
}

extern "C" int convert_check(long long n, const double *x, float *sw32, float *hw32,
                             const float *f, double *sw64, double *hw64) {
    if (n <= 0) return 0;
    k_convert_check<<<1024, 256>>>(n, x, sw32, hw32, f, sw64, hw64);
    return (int)cudaDeviceSynchronize();
}
