// Set-up kernels: input validation, the Jacobi diagonal, the per-row Gram
// factorisation and the constraint-restoring correction of Algorithm 2.
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

// CSR sanity: monotone row pointers inside [0, nnz], columns in [0, ncols),
// strictly ascending per row.  Also the longest row.
__global__ void k_validate_csr(int nrows, int ncols, const int *__restrict__ rowptr, int nnz,
                               const int *__restrict__ col, int *flags, int *maxrow) {
    int bad = 0, mx = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nrows; i += gridDim.x * blockDim.x) {
        const int a = rowptr[i], b = rowptr[i + 1];
        if (a < 0 || b < a || b > nnz) {
            bad |= F_ROWPTR;
            continue;
        }
        mx = max(mx, b - a);
        int prev = -1;
        for (int e = a; e < b; ++e) {
            const int c = col[e];
            if (c < 0 || c >= ncols) bad |= F_COL;
            if (c <= prev) bad |= F_ORDER;
            prev = c;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        bad |= __shfl_down_sync(0xffffffffu, bad, o);
        mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicOr(flags, bad);
        atomicMax(maxrow, mx);
    }
}

__global__ void k_check_finite(const double *__restrict__ v, long long count, int *flags) {
    int bad = 0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
         q += (long long)gridDim.x * blockDim.x)
        if (!isfinite(v[q])) bad = 1;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, F_NONFINITE);
}

// Jacobi preconditioner M_J = diag(K): row i of P is scaled by 1 / A(i,i)
// (Theorem 1).  Binary search of the diagonal in the sorted row.
__global__ void k_diag(int n, const int *__restrict__ Ap, const int *__restrict__ Aj,
                       const double *__restrict__ Av, double *dinv64, float *dinv32,
                       int *flags) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int lo = Ap[i], hi = Ap[i + 1];
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (Aj[mid] < i) lo = mid + 1; else hi = mid;
        }
        double d = (lo < Ap[i + 1] && Aj[lo] == i) ? Av[lo] : 0.0;
        if (!(d > 0.0) || !isfinite(d)) {
            atomicOr(flags, F_DIAG);
            d = 1.0;
        }
        const double inv = 1.0 / d;
        dinv64[i] = inv;
        dinv32[i] = (float)inv;
    }
}

__device__ __forceinline__ int tri(int a, int b) { return a * (a + 1) / 2 + b; }  // a >= b

// Symmetric pseudo-inverse by cyclic Jacobi rotations (K <= 8): the
// eigenvalues of G_i are the squared singular values of B_i, so dropping
// lambda <= tol * lambda_max is the SVD branch of Algorithm 2.
template <int K>
__device__ void pinv_sym(double (&G)[K * K], double (&out)[K * K]) {
    double V[K * K];
#pragma unroll
    for (int a = 0; a < K; ++a)
#pragma unroll
        for (int b = 0; b < K; ++b) V[a * K + b] = (a == b) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 30; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int p = 0; p < K; ++p) {
            diag += G[p * K + p] * G[p * K + p];
            for (int q = p + 1; q < K; ++q) off += G[p * K + q] * G[p * K + q];
        }
        if (off <= 1e-32 * diag || off == 0.0) break;
        for (int p = 0; p < K; ++p)
            for (int q = p + 1; q < K; ++q) {
                const double apq = G[p * K + q];
                if (apq == 0.0) continue;
                const double theta = (G[q * K + q] - G[p * K + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int r = 0; r < K; ++r) {  // G <- G J
                    const double gp = G[r * K + p], gq = G[r * K + q];
                    G[r * K + p] = c * gp - s * gq;
                    G[r * K + q] = s * gp + c * gq;
                }
                for (int r = 0; r < K; ++r) {  // G <- J^T G
                    const double gp = G[p * K + r], gq = G[q * K + r];
                    G[p * K + r] = c * gp - s * gq;
                    G[q * K + r] = s * gp + c * gq;
                }
                for (int r = 0; r < K; ++r) {
                    const double vp = V[r * K + p], vq = V[r * K + q];
                    V[r * K + p] = c * vp - s * vq;
                    V[r * K + q] = s * vp + c * vq;
                }
            }
    }
    double lmax = 0.0;
    for (int a = 0; a < K; ++a) lmax = fmax(lmax, G[a * K + a]);
    for (int a = 0; a < K * K; ++a) out[a] = 0.0;
    for (int j = 0; j < K; ++j) {
        const double lam = G[j * K + j];
        if (!(lam > kRankTol * lmax) || !(lam > 0.0)) continue;
        for (int a = 0; a < K; ++a)
            for (int b = 0; b < K; ++b) out[a * K + b] += V[a * K + j] * V[b * K + j] / lam;
    }
}

// Per row: G_i = B_i^T B_i (B_i = Bc(J_i,:)) in double, Cholesky G = L L^T
// with the rank test L_jj^2 <= tol * max diag(G_i), then G_i^{-1} = L^{-T}
// L^{-1} stored packed.  Rank-deficient rows: error (strict) or the
// pseudo-inverse (counted).
template <int K>
__global__ void k_gram(int n, const int *__restrict__ Pp, const int *__restrict__ Pj,
                       const double *__restrict__ Bc, double *Ginv, float *Ginv32, int policy,
                       int *flags, int *ndef) {
    constexpr int KK = K * (K + 1) / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double G[K * K];
#pragma unroll
        for (int a = 0; a < K * K; ++a) G[a] = 0.0;
        const int p0 = Pp[i], p1 = Pp[i + 1];
        for (int s = p0; s < p1; ++s) {
            const double *b = Bc + (size_t)Pj[s] * K;
            double bv[K];
#pragma unroll
            for (int a = 0; a < K; ++a) bv[a] = b[a];
#pragma unroll
            for (int a = 0; a < K; ++a)
#pragma unroll
                for (int c = 0; c <= a; ++c) G[a * K + c] = fma(bv[a], bv[c], G[a * K + c]);
        }
        double maxd = 0.0;
#pragma unroll
        for (int a = 0; a < K; ++a) maxd = fmax(maxd, G[a * K + a]);
        double L[K * K];
#pragma unroll
        for (int a = 0; a < K * K; ++a) L[a] = 0.0;
        bool ok = (p1 - p0 >= K) && maxd > 0.0;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            double d = G[j * K + j];
#pragma unroll
            for (int q = 0; q < j; ++q) d -= L[j * K + q] * L[j * K + q];
            if (!(d > kRankTol * maxd)) ok = false;
            const double ljj = sqrt(fmax(d, 1e-300));
            L[j * K + j] = ljj;
#pragma unroll
            for (int r = j + 1; r < K; ++r) {
                double v = G[r * K + j];
#pragma unroll
                for (int q = 0; q < j; ++q) v -= L[r * K + q] * L[j * K + q];
                L[r * K + j] = v / ljj;
            }
        }
        double out[K * K];
        if (ok) {
            // Li = L^{-1} (lower), then G^{-1} = Li^T Li
            double Li[K * K];
#pragma unroll
            for (int a = 0; a < K * K; ++a) Li[a] = 0.0;
#pragma unroll
            for (int c = 0; c < K; ++c)
#pragma unroll
                for (int a = c; a < K; ++a) {
                    double v = (a == c) ? 1.0 : 0.0;
#pragma unroll
                    for (int q = c; q < a; ++q) v -= L[a * K + q] * Li[q * K + c];
                    Li[a * K + c] = v / L[a * K + a];
                }
#pragma unroll
            for (int a = 0; a < K; ++a)
#pragma unroll
                for (int b = 0; b <= a; ++b) {
                    double v = 0.0;
#pragma unroll
                    for (int q = a; q < K; ++q) v += Li[q * K + a] * Li[q * K + b];
                    out[a * K + b] = v;
                }
        } else if (policy == EMIN_RANK_PINV) {
#pragma unroll
            for (int a = 0; a < K; ++a)
#pragma unroll
                for (int b = 0; b < a; ++b) G[b * K + a] = G[a * K + b];
            pinv_sym<K>(G, out);
            atomicAdd(ndef, 1);
        } else {
            atomicOr(flags, F_RANK);
#pragma unroll
            for (int a = 0; a < K * K; ++a) out[a] = 0.0;
        }
#pragma unroll
        for (int a = 0; a < K; ++a)
#pragma unroll
            for (int b = 0; b <= a; ++b) {
                Ginv[(size_t)i * KK + tri(a, b)] = out[a * K + b];
                Ginv32[(size_t)i * KK + tri(a, b)] = (float)out[a * K + b];
            }
    }
}

// Least-norm constraint correction of one row (Algorithm 2, Eq. (resEq)):
//   p = base + add;  r = B(i,:)^T - B_i^T p;  p += B_i G_i^{-1} r.
template <int K>
__global__ void k_restore(int n, const int *__restrict__ Pp, const int *__restrict__ Pj,
                          const double *__restrict__ Bc, const double *__restrict__ B,
                          const double *__restrict__ Ginv, const double *base,
                          const double *__restrict__ add64, const float *__restrict__ add32,
                          double *P) {
    constexpr int KK = K * (K + 1) / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p0 = Pp[i], p1 = Pp[i + 1];
        double r[K];
#pragma unroll
        for (int a = 0; a < K; ++a) r[a] = B[(size_t)i * K + a];
        for (int s = p0; s < p1; ++s) {
            double p = base[s];
            if (add64) p += add64[s];
            if (add32) p += (double)add32[s];
            const double *b = Bc + (size_t)Pj[s] * K;
#pragma unroll
            for (int a = 0; a < K; ++a) r[a] = fma(-b[a], p, r[a]);
        }
        double c[K];
        const double *g = Ginv + (size_t)i * KK;
#pragma unroll
        for (int a = 0; a < K; ++a) {
            double v = 0.0;
#pragma unroll
            for (int b = 0; b < K; ++b) v = fma(g[a >= b ? tri(a, b) : tri(b, a)], r[b], v);
            c[a] = v;
        }
        for (int s = p0; s < p1; ++s) {
            double p = base[s];
            if (add64) p += add64[s];
            if (add32) p += (double)add32[s];
            const double *b = Bc + (size_t)Pj[s] * K;
#pragma unroll
            for (int a = 0; a < K; ++a) p = fma(b[a], c[a], p);
            P[s] = p;
        }
    }
}

__global__ void k_to_float(const double *__restrict__ s, float *__restrict__ d, long long count) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
         q += (long long)gridDim.x * blockDim.x)
        d[q] = (float)s[q];
}

__global__ void k_to_double(const float *__restrict__ s, double *__restrict__ d, long long count) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
         q += (long long)gridDim.x * blockDim.x)
        d[q] = (double)s[q];
}

}  // namespace

void launch_validate_csr(const Launch &L, int nrows, int ncols, const int *rowptr, int nnz,
                         const int *col, int *flags, int *maxrow) {
    if (nrows <= 0) return;
    k_validate_csr<<<grid_for(nrows, L.grid_rows), kBlock, 0, L.stream>>>(nrows, ncols, rowptr, nnz,
                                                                          col, flags, maxrow); note_launch();
}

void launch_check_finite(const Launch &L, const double *v, long long count, int *flags) {
    if (count <= 0) return;
    k_check_finite<<<grid_for(count, L.grid_rows), kBlock, 0, L.stream>>>(v, count, flags); note_launch();
}

void launch_diag(const Launch &L, int n, const int *Ap, const int *Aj, const double *Av,
                 double *dinv64, float *dinv32, int *flags) {
    if (n <= 0) return;
    k_diag<<<grid_for(n, L.grid_rows), kBlock, 0, L.stream>>>(n, Ap, Aj, Av, dinv64, dinv32, flags); note_launch();
}

void launch_gram(const Launch &L, int n, int k, const int *Pp, const int *Pj, const double *Bc,
                 double *Ginv, float *Ginv32, int policy, int *flags, int *ndef) {
    if (n <= 0) return;
    const int g = grid_for(n, L.grid_rows);
    switch (k) {
#define EMIN_GRAM(KV) \
    case KV: k_gram<KV><<<g, kBlock, 0, L.stream>>>(n, Pp, Pj, Bc, Ginv, Ginv32, policy, flags, ndef); note_launch(); break;
        EMIN_GRAM(1) EMIN_GRAM(2) EMIN_GRAM(3) EMIN_GRAM(4)
        EMIN_GRAM(5) EMIN_GRAM(6) EMIN_GRAM(7) EMIN_GRAM(8)
#undef EMIN_GRAM
        default: break;
    }
}

void launch_restore(const Launch &L, int n, int k, const int *Pp, const int *Pj,
                    const double *Bc, const double *B, const double *Ginv, const double *base,
                    const double *add64, const float *add32, double *P) {
    if (n <= 0) return;
    const int g = grid_for(n, L.grid_rows);
    switch (k) {
#define EMIN_RESTORE(KV)                                                                      \
    case KV:                                                                                  \
        k_restore<KV><<<g, kBlock, 0, L.stream>>>(n, Pp, Pj, Bc, B, Ginv, base, add64, add32, P); note_launch(); \
        break;
        EMIN_RESTORE(1) EMIN_RESTORE(2) EMIN_RESTORE(3) EMIN_RESTORE(4)
        EMIN_RESTORE(5) EMIN_RESTORE(6) EMIN_RESTORE(7) EMIN_RESTORE(8)
#undef EMIN_RESTORE
        default: break;
    }
}

void launch_to_float(const Launch &L, const double *src, float *dst, long long count) {
    if (count <= 0) return;
    k_to_float<<<grid_for(count, L.grid_rows), kBlock, 0, L.stream>>>(src, dst, count); note_launch();
}

void launch_to_double(const Launch &L, const float *src, double *dst, long long count) {
    if (count <= 0) return;
    k_to_double<<<grid_for(count, L.grid_rows), kBlock, 0, L.stream>>>(src, dst, count); note_launch();
}

}  // namespace emin
