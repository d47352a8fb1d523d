// Kernels of the implicit adjoint (derived from the saddle-point system
// (sadsys)): the masked outer product mask_A(U V^T) and the per-row least
// squares mu_i = G_i^{-1} B_i^T x_i.
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "emin_internal.cuh"

namespace emin {
namespace {

inline int grid_for(long long work, int cap) {
    long long g = (work + kBlock - 1) / kBlock;
    if (g < 1) g = 1;
    return (int)(g < cap ? g : cap);
}

__device__ __forceinline__ int tri(int a, int b) { return a * (a + 1) / 2 + b; }

// out_e = scale * sum_c U(a,c) V(b,c) for every stored (a, b) = entry e of A.
// One warp per row a: row a of U is staged in shared memory; each lane takes
// entries b of the row and walks row b of V, finding each column in J_a by
// binary search.
__global__ void __launch_bounds__(kBlock)
k_outer_warp(int n, const int *__restrict__ Ap, const int *__restrict__ Aj,
             const int *__restrict__ Pp, const int *__restrict__ Pj, const double *__restrict__ U,
             const double *__restrict__ V, double scale, double *__restrict__ out, int mcap) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *sU = reinterpret_cast<double *>(smem) + (size_t)w * mcap;
    int *sJ = reinterpret_cast<int *>(smem + (size_t)nw * mcap * sizeof(double)) + (size_t)w * mcap;
    for (int a = blockIdx.x * nw + w; a < n; a += gridDim.x * nw) {
        const int p0 = Pp[a], m = Pp[a + 1] - p0;
        for (int s = lane; s < m; s += 32) {
            sJ[s] = Pj[p0 + s];
            sU[s] = U[p0 + s];
        }
        __syncwarp();
        for (int e = Ap[a] + lane; e < Ap[a + 1]; e += 32) {
            const int b = Aj[e];
            double v = 0.0;
            for (int q = Pp[b]; q < Pp[b + 1]; ++q) {
                const int cc = Pj[q];
                int lo = 0, hi = m;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (sJ[mid] < cc) lo = mid + 1; else hi = mid;
                }
                if (lo < m && sJ[lo] == cc) v = fma(sU[lo], V[q], v);
            }
            out[e] = scale * v;
        }
        __syncwarp();
    }
}

// mu_i = G_i^{-1} B_i^T x_i (least squares of B_i mu = x_i), one thread per row.
template <int K>
__global__ void k_lsq(int n, const int *__restrict__ Pp, const int *__restrict__ Pj,
                      const double *__restrict__ Bc, const double *__restrict__ Ginv,
                      const double *__restrict__ x, double *__restrict__ mu) {
    constexpr int KK = K * (K + 1) / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double t[K];
#pragma unroll
        for (int a = 0; a < K; ++a) t[a] = 0.0;
        for (int s = Pp[i]; s < Pp[i + 1]; ++s) {
            const double v = x[s];
            const double *b = Bc + (size_t)Pj[s] * K;
#pragma unroll
            for (int a = 0; a < K; ++a) t[a] = fma(b[a], v, t[a]);
        }
        const double *g = Ginv + (size_t)i * KK;
#pragma unroll
        for (int a = 0; a < K; ++a) {
            double v = 0.0;
#pragma unroll
            for (int b = 0; b < K; ++b) v = fma(g[a >= b ? tri(a, b) : tri(b, a)], t[b], v);
            mu[(size_t)i * K + a] = v;
        }
    }
}

__global__ void k_axpby(long long count, double a, const double *__restrict__ x, double b,
                        double *__restrict__ y) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
         q += (long long)gridDim.x * blockDim.x)
        y[q] = fma(a, x[q], b * y[q]);
}

// <x, y> into st->aux (deterministic last-block reduction).
__global__ void __launch_bounds__(kBlock)
k_dot_aux(long long count, const double *__restrict__ x, const double *__restrict__ y,
          DevState *st, double *partials) {
    double v = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
         q += (long long)gridDim.x * blockDim.x)
        v = fma(x[q], y[q], v);
    __shared__ double sh[32];
    const double bt = block_sum(v, sh);
    double total;
    if (grid_reduce(bt, partials, &st->ticket[2], &total)) st->aux = total;
}

// out[i] += scale * d_i^(-pw/2) * sum over row i of P of u v  (d_i^(-1/2) = dsq[i])
__global__ void k_row_dot_acc(int n, const int *__restrict__ Pp, const double *__restrict__ u,
                              const double *__restrict__ v, const double *__restrict__ dsq,
                              int pw, double scale, double *__restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int s = Pp[i]; s < Pp[i + 1]; ++s) t = fma(u[s], v[s], t);
        double g = 1.0;
        for (int q = 0; q < pw; ++q) g *= dsq[i];
        out[i] += scale * g * t;
    }
}

// Chain rule from A^ = D^{-1/2} A D^{-1/2} (d = diag A) to the stored values
// of A, one thread per row i: with ghat the gradient with respect to A^,
//   dL/da_e = ghat_e d_i^{-1/2} d_l^{-1/2}                   (e = (i, l))
//   dL/dd_i = dext_i - 1/2 d_i^{-1} sum over the entries e of row i and
//             their mirrors e' = (l, i) of ghat A^ (row and column factor),
// and dL/dd_i is added to the diagonal entry.  A is symmetric with sorted
// columns, so the mirror of (i, l) is found in row l by binary search.
__global__ void k_grad_a(int n, const int *__restrict__ Ap, const int *__restrict__ Aj,
                         const double *__restrict__ Av, const double *__restrict__ dsq,
                         const double *__restrict__ ghat, const double *__restrict__ dext,
                         double *__restrict__ gA) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double di = dsq[i];
        double t = 0.0;
        for (int e = Ap[i]; e < Ap[i + 1]; ++e) {
            const int l = Aj[e];
            const double ahat = di * Av[e] * dsq[l];
            t = fma(ghat[e], ahat, t);
            int lo = Ap[l], hi = Ap[l + 1];
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (Aj[mid] < i) lo = mid + 1; else hi = mid;
            }
            if (lo < Ap[l + 1] && Aj[lo] == i) t = fma(ghat[lo], ahat, t);
        }
        const double dbar = dext[i] - 0.5 * di * di * t;
        for (int e = Ap[i]; e < Ap[i + 1]; ++e) {
            const int l = Aj[e];
            gA[e] = ghat[e] * di * dsq[l] + (l == i ? dbar : 0.0);
        }
    }
}

}  // namespace

void launch_outer(const Launch &L, int n, const int *Ap, const int *Aj, const int *Pp,
                  const int *Pj, const double *U, const double *V, double scale, double *out,
                  int maxrow) {
    if (n <= 0) return;
    const int mcap = staging_cap(maxrow);
    const size_t smem = (size_t)(kBlock / 32) * mcap * (sizeof(double) + sizeof(int));
    k_outer_warp<<<grid_for((long long)n * 32, L.grid_warps), kBlock, smem, L.stream>>>(
        n, Ap, Aj, Pp, Pj, U, V, scale, out, mcap); note_launch();
}

void launch_lsq(const Launch &L, int n, int k, const int *Pp, const int *Pj, const double *Bc,
                const double *Ginv, const double *x, double *mu) {
    if (n <= 0) return;
    const int g = grid_for(n, L.grid_rows);
    switch (k) {
#define EMIN_LSQ(KV) \
    case KV: k_lsq<KV><<<g, kBlock, 0, L.stream>>>(n, Pp, Pj, Bc, Ginv, x, mu); note_launch(); break;
        EMIN_LSQ(1) EMIN_LSQ(2) EMIN_LSQ(3) EMIN_LSQ(4)
        EMIN_LSQ(5) EMIN_LSQ(6) EMIN_LSQ(7) EMIN_LSQ(8)
#undef EMIN_LSQ
        default: break;
    }
}

void launch_axpby(const Launch &L, long long count, double a, const double *x, double b,
                  double *y) {
    if (count <= 0) return;
    k_axpby<<<grid_for(count, L.grid_rows), kBlock, 0, L.stream>>>(count, a, x, b, y); note_launch();
}

void launch_dot_aux(const Launch &L, long long count, const double *x, const double *y,
                    DevState *st, double *partials) {
    k_dot_aux<<<grid_for(count > 0 ? count : 1, L.grid_rows), kBlock, 0, L.stream>>>(
        count, x, y, st, partials);
    note_launch();
}

void launch_row_dot_acc(const Launch &L, int n, const int *Pp, const double *u, const double *v,
                        const double *dsq, int pw, double scale, double *out) {
    if (n <= 0) return;
    k_row_dot_acc<<<grid_for(n, L.grid_rows), kBlock, 0, L.stream>>>(n, Pp, u, v, dsq, pw, scale,
                                                                      out);
    note_launch();
}

void launch_grad_a(const Launch &L, int n, const int *Ap, const int *Aj, const double *Av,
                   const double *dsq, const double *ghat, const double *dext, double *gA) {
    if (n <= 0) return;
    k_grad_a<<<grid_for(n, L.grid_rows), kBlock, 0, L.stream>>>(n, Ap, Aj, Av, dsq, ghat, dext,
                                                                 gA);
    note_launch();
}

void set_adjoint_attributes() {
    const int bytes = (kBlock / 32) * kMaxRowP * (int)(sizeof(double) + sizeof(int));
    cudaFuncSetAttribute(k_outer_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace emin
