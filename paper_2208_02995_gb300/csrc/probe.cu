// Throughput of the fused multiply-add pipe, the ceiling of the products
// whose arithmetic, not their memory traffic, bounds them (the FP64 masked
// products: GB300 issues about 2 FP64 FMAs per SM and clock).  Every thread
// runs kChains independent FMA chains so that the pipe, not the latency of
// one chain, sets the rate; the grid fills every SM with full occupancy.
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "emin_internal.cuh"

namespace emin {
namespace {

constexpr int kChains = 8;
constexpr int kProbeBlock = 256;

// written only when a chain ends on a value it cannot reach, so that the
// compiler keeps every FMA
static __device__ double g_fma_sink;

template <class T>
__global__ void __launch_bounds__(kProbeBlock) k_fma_rate(int iters, T b, T c) {
    T a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = T(threadIdx.x + j) * T(1e-3);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fmat(a[j], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == T(-1.2345e30)) g_fma_sink = (double)s;
}

template <class T>
int fma_rate(int nsm, cudaStream_t s, double *rate, double *ms_out) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_rate<T>, kProbeBlock, 0) !=
            cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int grid = nsm * per_sm;
    // about 20 ms on GB300: FP64 ~0.5e12 FMA/s, float ~64 times more
    const int iters = sizeof(T) == 8 ? 4096 : 131072;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return EMIN_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return EMIN_ERR_CUDA;
    }
    // b slightly below 1 and c small keep every chain finite and non-trivial
    const T b = T(0.999999), c = T(1e-7);
    k_fma_rate<T><<<grid, kProbeBlock, 0, s>>>(iters / 8, b, c);  // warm-up
    note_launch();
    cudaEventRecord(e0, s);
    k_fma_rate<T><<<grid, kProbeBlock, 0, s>>>(iters, b, c);
    note_launch();
    cudaEventRecord(e1, s);
    float ms = 0.f;
    cudaError_t err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess || ms <= 0.f) {
        cudaGetLastError();
        return EMIN_ERR_CUDA;
    }
    const double fmas = (double)grid * kProbeBlock * kChains * (double)iters;
    *rate = fmas / (ms * 1e-3);
    if (ms_out) *ms_out = ms;
    return EMIN_OK;
}

}  // namespace
}  // namespace emin

extern "C" int emin_fma_rate(int precision, double *fma_per_s, double *ms, void *stream) {
    using namespace emin;
    if (!fma_per_s || (precision != EMIN_FP64 && precision != EMIN_MIXED)) return EMIN_ERR_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return EMIN_ERR_CUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return precision == EMIN_FP64 ? fma_rate<double>(nsm, s, fma_per_s, ms)
                                  : fma_rate<float>(nsm, s, fma_per_s, ms);
}
