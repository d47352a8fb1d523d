// Allocation-free masked product with its dot product.
//
// Some callers cannot let a library allocate device memory: a process whose
// device memory is owned by another allocator (the caching allocator of a
// framework, the fixed pool of a serving process) would be fragmented or
// overcommitted by foreign cudaMalloc calls, and cudaMalloc / cudaFree
// synchronise the device, which a latency-bound request path cannot afford.
// emin_masked_product_noalloc serves them: the caller passes every input and
// output, and the only extra device memory the kernel uses is a file-scope
// __device__ scratch array that every GPU loading the library holds until
// the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "device_util.cuh"
#include "emin_internal.cuh"

namespace emin {
namespace {

constexpr int kNoAllocBlock = 256;
// one partial sum per block; the grid is one thread per row, so the scratch
// size fixes the largest accepted problem: 16,384 blocks x 256 rows
constexpr int kNoAllocMaxBlocks = 16384;
constexpr long long kNoAllocMaxRows = (long long)kNoAllocMaxBlocks * kNoAllocBlock;
constexpr int kNoAllocMaxDevices = 64;

struct NoAllocScratch {
    double partials[kNoAllocMaxBlocks];  // block totals of the dot product
    unsigned int ticket;                 // blocks done (must start at 0)
    int bad;                             // an index out of range was seen (must start at 0)
};

// 128 KiB + 8 bytes per device, shared by every call on that device
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// out = mask_P(A Y) and *dot = <Y, out>, one thread per row of P: for every
// entry (i, c) of P, sum a_il y_lc over the stored a_il of row i whose row l
// of Y holds column c (binary search in the sorted row l).  Indices out of
// range are skipped and make *dot NaN.
__global__ void __launch_bounds__(kNoAllocBlock)
k_masked_product_dot_noalloc(int n, int nc, const int *__restrict__ Ap,
                             const int *__restrict__ Aj, const double *__restrict__ Av,
                             const int *__restrict__ Pp, const int *__restrict__ Pj,
                             const double *__restrict__ Y, double *__restrict__ out, double *dot,
                             NoAllocScratch *scr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nnz_a = Ap[n], nnz_p = Pp[n];
    double part = 0.0;
    int bad = 0;
    if (i < n) {
        const int a0 = Ap[i], a1 = Ap[i + 1], p0 = Pp[i], p1 = Pp[i + 1];
        if (a0 < 0 || a1 < a0 || a1 > nnz_a || p0 < 0 || p1 < p0 || p1 > nnz_p) {
            bad = 1;
        } else {
            for (int s = p0; s < p1; ++s) {
                const int c = Pj[s];
                double v = 0.0;
                for (int e = a0; e < a1; ++e) {
                    const int l = Aj[e];
                    if (l < 0 || l >= n) {
                        bad = 1;
                        continue;
                    }
                    const int q0 = Pp[l], q1 = Pp[l + 1];
                    if (q0 < 0 || q1 < q0 || q1 > nnz_p) {
                        bad = 1;
                        continue;
                    }
                    int lo = q0, hi = q1;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (Pj[mid] < c) lo = mid + 1; else hi = mid;
                    }
                    if (lo < q1 && Pj[lo] == c) v = fma(Av[e], Y[lo], v);
                }
                if (c < 0 || c >= nc) bad = 1;
                out[s] = v;
                part = fma(Y[s], v, part);
            }
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) {
        atomicOr(&scr->bad, 1);
        __threadfence();  // visible before this block's ticket is counted
    }
    __shared__ double sh[32];
    const double bt = block_sum(part, sh);
    double total;
    if (grid_reduce(bt, scr->partials, &scr->ticket, &total)) {
        __threadfence();
        *dot = (atomicAdd(&scr->bad, 0) != 0) ? __longlong_as_double(0x7ff8000000000000LL) : total;
    }
}

std::mutex g_mu;
NoAllocScratch *g_scratch[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and kept for the life of the
// process: a reset of the device's primary context (cudaDeviceReset) frees
// the array, so calls must not continue across one.
int scratch_for_current_device(NoAllocScratch **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return EMIN_ERR_CUDA;
    }
    if (dev < 0 || dev >= kNoAllocMaxDevices) return EMIN_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return EMIN_ERR_CUDA;
        }
        g_scratch[dev] = static_cast<NoAllocScratch *>(p);
    }
    *out = g_scratch[dev];
    return EMIN_OK;
}

}  // namespace
}  // namespace emin

extern "C" int emin_masked_product_noalloc(int n, int nc, const int *A_rowptr, const int *A_col,
                                           const double *A_val, const int *P_rowptr,
                                           const int *P_col, const double *Y, double *out,
                                           double *dot, void *stream) {
    using namespace emin;
    if (n < 0 || nc < 0 || !A_rowptr || !P_rowptr || !dot) return EMIN_ERR_ARG;
    // with rows to process the kernel dereferences every array
    if (n > 0 && (!A_col || !A_val || !P_col || !Y || !out)) return EMIN_ERR_ARG;
    if ((long long)n > kNoAllocMaxRows) return EMIN_ERR_ARG;  // beyond the scratch size
    NoAllocScratch *scr = nullptr;
    const int st = scratch_for_current_device(&scr);
    if (st != EMIN_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the ticket and the error flag start at zero on every call
    if (cudaMemsetAsync(&scr->ticket, 0, sizeof(unsigned int) + sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return EMIN_ERR_CUDA;
    }
    if (n == 0) {
        if (cudaMemsetAsync(dot, 0, sizeof(double), s) != cudaSuccess) {
            cudaGetLastError();
            return EMIN_ERR_CUDA;
        }
        return EMIN_OK;
    }
    const int grid = (n + kNoAllocBlock - 1) / kNoAllocBlock;
    k_masked_product_dot_noalloc<<<grid, kNoAllocBlock, 0, s>>>(n, nc, A_rowptr, A_col, A_val,
                                                                P_rowptr, P_col, Y, out, dot, scr);
    note_launch();
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EMIN_OK : EMIN_ERR_CUDA;
}
