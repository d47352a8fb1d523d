// Set-up kernels: input validation, the Jacobi diagonal, the per-row Gram
// factorisation and the constraint-restoring correction of Algorithm 2.
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "convert.cuh"
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

// G_i = B_i^T B_i (B_i = Bc(J_i,:)), full, for the rank-deficient rows
template <int K>
__device__ __forceinline__ void gram_full(int p0, int p1, const int *__restrict__ Pj,
                                          const double *__restrict__ Bc, double (&G)[K * K]) {
#pragma unroll
    for (int a = 0; a < K * K; ++a) G[a] = 0.0;
    for (int s = p0; s < p1; ++s) {
        const double *b = Bc + (size_t)Pj[s] * K;
#pragma unroll
        for (int a = 0; a < K; ++a)
#pragma unroll
            for (int c = 0; c < K; ++c) G[a * K + c] = fma(b[a], b[c], G[a * K + c]);
    }
}

// The rows whose G_i failed the rank test: the pseudo-inverse (counted) or
// an error and a zero factor.  Kept out of line: it is rare, and its
// dense arrays would otherwise weigh on the registers of every row.
template <int K>
__device__ __noinline__ void gram_rank_deficient(int i, int rep, int p0, int p1,
                                                 const int *__restrict__ Pj,
                                                 const double *__restrict__ Bc, double *Ginv,
                                                 float *Ginv32, int policy, int *flags,
                                                 int *ndef) {
    constexpr int KK = K * (K + 1) / 2;
    double out[K * K];
    if (policy == EMIN_RANK_PINV) {
        double G[K * K];
        gram_full<K>(p0, p1, Pj, Bc, G);
        pinv_sym<K>(G, out);
        atomicAdd(ndef, rep);
    } else {
        atomicOr(flags, F_RANK);
        for (int a = 0; a < K * K; ++a) out[a] = 0.0;
    }
    for (int r = 0; r < rep; ++r)
        for (int a = 0; a < K; ++a)
            for (int b = 0; b <= a; ++b) {
                Ginv[(size_t)(i + r) * KK + tri(a, b)] = out[a * K + b];
                Ginv32[(size_t)(i + r) * KK + tri(a, b)] = (float)out[a * K + b];
            }
}

// Per row: G_i = B_i^T B_i (B_i = Bc(J_i,:)) in double, Cholesky G = L L^T
// with the rank test L_jj^2 <= tol * max diag(G_i), then G_i^{-1} = L^{-T}
// L^{-1} stored packed.  Rank-deficient rows: error (strict) or the
// pseudo-inverse (counted).  Every matrix is held as its packed lower
// triangle, the factor overwriting G, with one reciprocal per pivot.
template <int K>
__global__ void __launch_bounds__(kBlock, K >= 6 ? 3 : 1)
k_gram(int n, const int *__restrict__ Pp, const int *__restrict__ Pj,
                       const double *__restrict__ Bc, double *Ginv, float *Ginv32, int policy,
                       int *flags, int *ndef, int rep) {
    // rep consecutive rows share their columns of P (rep = 3 for the rows of
    // a node of a node-blocked problem), hence G_i: computed once per group
    constexpr int KK = K * (K + 1) / 2;
    const int ngr = n / rep;
    for (int gi = blockIdx.x * blockDim.x + threadIdx.x; gi < ngr; gi += gridDim.x * blockDim.x) {
        const int i = gi * rep;
        double G[KK];
#pragma unroll
        for (int a = 0; a < KK; ++a) G[a] = 0.0;
        const int p0 = Pp[i], p1 = Pp[i + 1];
        for (int s = p0; s < p1; ++s) {
            const double *b = Bc + (size_t)Pj[s] * K;
            double bv[K];
#pragma unroll
            for (int a = 0; a < K; ++a) bv[a] = b[a];
#pragma unroll
            for (int a = 0; a < K; ++a)
#pragma unroll
                for (int c = 0; c <= a; ++c) G[tri(a, c)] = fma(bv[a], bv[c], G[tri(a, c)]);
        }
        double maxd = 0.0;
#pragma unroll
        for (int a = 0; a < K; ++a) maxd = fmax(maxd, G[tri(a, a)]);
        bool ok = (p1 - p0 >= K) && maxd > 0.0;
        double rinv[K];  // 1 / L_jj
#pragma unroll
        for (int j = 0; j < K; ++j) {
            double d = G[tri(j, j)];
#pragma unroll
            for (int q = 0; q < j; ++q) d -= G[tri(j, q)] * G[tri(j, q)];
            if (!(d > kRankTol * maxd)) ok = false;
            const double ljj = sqrt(fmax(d, 1e-300));
            rinv[j] = 1.0 / ljj;
            G[tri(j, j)] = ljj;
#pragma unroll
            for (int r = j + 1; r < K; ++r) {
                double v = G[tri(r, j)];
#pragma unroll
                for (int q = 0; q < j; ++q) v -= G[tri(r, q)] * G[tri(j, q)];
                G[tri(r, j)] = v * rinv[j];
            }
        }
        if (!ok) {
            gram_rank_deficient<K>(i, rep, p0, p1, Pj, Bc, Ginv, Ginv32, policy, flags, ndef);
            continue;
        }
        // Li = L^{-1} (lower), then G^{-1} = Li^T Li
        double Li[KK];
#pragma unroll
        for (int c = 0; c < K; ++c)
#pragma unroll
            for (int a = c; a < K; ++a) {
                double v = (a == c) ? 1.0 : 0.0;
#pragma unroll
                for (int q = c; q < a; ++q) v -= G[tri(a, q)] * Li[tri(q, c)];
                Li[tri(a, c)] = v * rinv[a];
            }
#pragma unroll
        for (int a = 0; a < K; ++a)
#pragma unroll
            for (int b = 0; b <= a; ++b) {
                double v = 0.0;
#pragma unroll
                for (int q = a; q < K; ++q) v += Li[tri(q, a)] * Li[tri(q, b)];
                for (int r = 0; r < rep; ++r) {
                    Ginv[(size_t)(i + r) * KK + tri(a, b)] = v;
                    Ginv32[(size_t)(i + r) * KK + tri(a, b)] = (float)v;
                }
            }
    }
}

// Least-norm constraint correction of one row (Algorithm 2, Eq. (resEq)):
//   p = base + f_i add;  r = B(i,:)^T - B_i^T p;  p += B_i G_i^{-1} r.
// With correct == 0 only p = base + f_i add is formed.
template <int K>
__global__ void k_restore(int n, const int *__restrict__ Pp, const int *__restrict__ Pj,
                          const double *__restrict__ Bc, const double *__restrict__ B,
                          const double *__restrict__ Ginv, const double *base,
                          const double *__restrict__ add64, const float *__restrict__ add32,
                          const double *__restrict__ f, int correct, double *P) {
    constexpr int KK = K * (K + 1) / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p0 = Pp[i], p1 = Pp[i + 1];
        const double fi = f ? f[i] : 1.0;
        double c[K];
#pragma unroll
        for (int a = 0; a < K; ++a) c[a] = 0.0;
        if (correct) {
            double r[K];
#pragma unroll
            for (int a = 0; a < K; ++a) r[a] = B[(size_t)i * K + a];
            for (int s = p0; s < p1; ++s) {
                double p = base[s];
                if (add64) p = fma(fi, add64[s], p);
                if (add32) p = fma(fi, (double)add32[s], p);
                const double *b = Bc + (size_t)Pj[s] * K;
#pragma unroll
                for (int a = 0; a < K; ++a) r[a] = fma(-b[a], p, r[a]);
            }
            const double *g = Ginv + (size_t)i * KK;
#pragma unroll
            for (int a = 0; a < K; ++a) {
                double v = 0.0;
#pragma unroll
                for (int b = 0; b < K; ++b) v = fma(g[a >= b ? tri(a, b) : tri(b, a)], r[b], v);
                c[a] = v;
            }
        }
        for (int s = p0; s < p1; ++s) {
            double p = base[s];
            if (add64) p = fma(fi, add64[s], p);
            if (add32) p = fma(fi, (double)add32[s], p);
            if (correct) {
                const double *b = Bc + (size_t)Pj[s] * K;
#pragma unroll
                for (int a = 0; a < K; ++a) p = fma(b[a], c[a], p);
            }
            P[s] = p;
        }
    }
}

// ---------------------------------------------------------------------------
// Whole k = 1 set-up of one row (rows of P with at most 4 entries), fused:
//   Jacobi scaling from d = A(i,i) (Theorem 1: M_J scales row i by 1/d):
//     D^{-1/2} = s = 1/sqrt(d), D^{1/2} = d s (float on the float path,
//     double on the FP64 path);
//   Gram factor of the 1 x m_i block b = Bc(J_i), in double: G = b^T b,
//     rn = 1/|b| (Newton), G^{-1} = rn^2; projection vector q = b rn in the
//     iteration type (Pi_B = I - q q^T); G = 0 is rank deficient (error, or
//     a zero factor under the PINV policy);
//   least-norm correction of P0 (Algorithm 2), in double:
//     p += b G^{-1} (B_i - b^T p);
//   the iteration's start vector x0 = D^{1/2} p in the iteration type.
// ---------------------------------------------------------------------------
// One row of the fused k = 1 set-up with at most M entries (M >= the row's m).
template <class Tit, int M>
__device__ __forceinline__ void setup_row_k1(int i, const int *__restrict__ dpos,
                                             const double *__restrict__ Av,
                                             const int *__restrict__ Pp,
                                             const int *__restrict__ Pj,
                                             const double *__restrict__ Bc,
                                             const double *__restrict__ B,
                                             const double *__restrict__ P0_in, int policy,
                                             int *flags, int *ndef, double *dsq, double *dhalf,
                                             float *dsq32, double *Ginv, Tit *qv, double *P0,
                                             Tit *x0) {
    const int p0 = Pp[i], m = Pp[i + 1] - p0;
    double b[M], p[M];
#pragma unroll
    for (int s = 0; s < M; ++s) {
        const bool h = s < m;
        b[s] = h ? Bc[Pj[p0 + s]] : 0.0;
        p[s] = h ? P0_in[p0 + s] : 0.0;
    }
    const double Bi = B[i];
    const int dp = dpos[i];
    double d = (dp >= 0) ? Av[dp] : 0.0;
    if (!(d > 0.0) || !isfinite(d)) {
        atomicOr(flags, F_DIAG);
        d = 1.0;
    }
    // the scaling is a change of variables of the iteration: the float
    // path takes it in float (exactly representable in double, so every
    // later use sees the same value), the FP64 path in double
    double sq, dh;
    if constexpr (sizeof(Tit) == 4) {
        // conversions on the integer pipe (convert.cuh): the FP64 pipe is
        // this kernel's bound
        const float df = f64_to_f32_rn(d);
        const float sf = (df > 0.f && isfinite(df)) ? rsqrtf(df) : 1.f;
        if (!(df > 0.f) || !isfinite(df)) atomicOr(flags, F_DIAG);
        sq = f32_to_f64(sf);
        dh = f32_to_f64(df * sf);
        if (dsq32) dsq32[i] = sf;
    } else {
        sq = rsqrt_newton(d);
        dh = d * sq;
    }
    dsq[i] = sq;
    dhalf[i] = dh;
    double G = 0.0;
#pragma unroll
    for (int s = 0; s < M; ++s) G = fma(b[s], b[s], G);
    double r = 0.0, gi = 0.0;
    if (sizeof(Tit) == 4 && G >= 1e-30 && G <= 1e30) {
        // float path: q = b / |b| is stored in float, so 1/|b| is taken in
        // float; 1/G (for the least-norm correction and the final FP64
        // restore) by two Newton-Raphson steps for the reciprocal,
        // x <- x + x (1 - G x), from the float seed 1/|b|^2, each step
        // squaring the relative error (about 1e-7 -> 1e-14 -> 1e-28)
        const float rf = rsqrtf(f64_to_f32_rn(G));
        r = f32_to_f64(rf);
        gi = f32_to_f64(rf * rf);
        gi = fma(gi, fma(-G, gi, 1.0), gi);
        gi = fma(gi, fma(-G, gi, 1.0), gi);
    } else if (G > 0.0) {
        r = rsqrt_newton(G);
        gi = r * r;
    } else if (policy == EMIN_RANK_PINV) {
        atomicAdd(ndef, 1);
    } else {
        atomicOr(flags, F_RANK);
    }
    Ginv[i] = gi;
    double res = Bi;
#pragma unroll
    for (int s = 0; s < M; ++s) res = fma(-b[s], p[s], res);
    const double c = gi * res;
#pragma unroll
    for (int s = 0; s < M; ++s)
        if (s < m) {
            const double pc = fma(b[s], c, p[s]);
            P0[p0 + s] = pc;
            if constexpr (sizeof(Tit) == 4) {
                x0[p0 + s] = f64_to_f32_rn(dh) * f64_to_f32_rn(pc);
                qv[p0 + s] = f64_to_f32_rn(b[s]) * f64_to_f32_rn(r);
            } else {
                x0[p0 + s] = dh * pc;
                qv[p0 + s] = b[s] * r;
            }
        }
}

template <class Tit>
__global__ void k_setup_k1(int n, const int *__restrict__ dpos, const double *__restrict__ Av,
                           const int *__restrict__ Pp, const int *__restrict__ Pj,
                           const double *__restrict__ Bc, const double *__restrict__ B,
                           const double *__restrict__ P0_in, int policy, int *flags, int *ndef,
                           double *dsq, double *dhalf, float *dsq32, double *Ginv, Tit *qv,
                           double *P0, Tit *x0) {
    // rows in warp-uniform passes, so that each warp runs the body for the
    // largest row of P among its 32 rows (no FP64 work on absent slots)
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < n;
         base += nwarps * 32) {
        const int i = base + lane;
        const bool row = i < n;
        const int m = row ? Pp[i + 1] - Pp[i] : 0;
        const unsigned mw = __reduce_max_sync(0xffffffffu, (unsigned)m);
        if (!row) continue;
        switch (mw) {
            case 0:
            case 1:
                setup_row_k1<Tit, 1>(i, dpos, Av, Pp, Pj, Bc, B, P0_in, policy, flags, ndef, dsq,
                                     dhalf, dsq32, Ginv, qv, P0, x0);
                break;
            case 2:
                setup_row_k1<Tit, 2>(i, dpos, Av, Pp, Pj, Bc, B, P0_in, policy, flags, ndef, dsq,
                                     dhalf, dsq32, Ginv, qv, P0, x0);
                break;
            case 3:
                setup_row_k1<Tit, 3>(i, dpos, Av, Pp, Pj, Bc, B, P0_in, policy, flags, ndef, dsq,
                                     dhalf, dsq32, Ginv, qv, P0, x0);
                break;
            default:
                setup_row_k1<Tit, 4>(i, dpos, Av, Pp, Pj, Bc, B, P0_in, policy, flags, ndef, dsq,
                                     dhalf, dsq32, Ginv, qv, P0, x0);
        }
    }
}

// Final prolongation for k = 1 (rows of P with at most 4 entries):
// p = P0 + D^{-1/2} dW~ and, when `correct`, the least-norm constraint
// correction in double p += b G^{-1} (B_i - b^T p) (b = Bc(J_i)).
// One row of the k = 1 final P with at most M entries (M >= the row's m).
template <class Tx, int M>
__device__ __forceinline__ void final_row_k1(int i, const int *__restrict__ Pp,
                                             const int *__restrict__ Pj,
                                             const double *__restrict__ Bc,
                                             const double *__restrict__ Ginv,
                                             const double *__restrict__ P0,
                                             const Tx *__restrict__ X,
                                             const double *__restrict__ dsq,
                                             const double *__restrict__ B, int correct,
                                             double *__restrict__ P) {
    const int p0 = Pp[i], m = Pp[i + 1] - p0;
    const double f = dsq[i];
    double p[M], b[M];
#pragma unroll
    for (int s = 0; s < M; ++s) {
        const bool h = s < m;
        p[s] = h ? fma(f, as_f64(X[p0 + s]), P0[p0 + s]) : 0.0;
        b[s] = (h && correct) ? Bc[Pj[p0 + s]] : 0.0;
    }
    if (correct) {
        double r = B[i];
#pragma unroll
        for (int s = 0; s < M; ++s) r = fma(-b[s], p[s], r);
        const double c = Ginv[i] * r;
#pragma unroll
        for (int s = 0; s < M; ++s) p[s] = fma(b[s], c, p[s]);
    }
#pragma unroll
    for (int s = 0; s < M; ++s)
        if (s < m) P[p0 + s] = p[s];
}

template <class Tx>
__global__ void k_final_k1(int n, const int *__restrict__ Pp, const int *__restrict__ Pj,
                           const double *__restrict__ Bc, const double *__restrict__ Ginv,
                           const double *__restrict__ P0, const Tx *__restrict__ X,
                           const double *__restrict__ dsq, const double *__restrict__ B,
                           int correct, double *__restrict__ P) {
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < n;
         base += nwarps * 32) {
        const int i = base + lane;
        const bool row = i < n;
        const int m = row ? Pp[i + 1] - Pp[i] : 0;
        const unsigned mw = __reduce_max_sync(0xffffffffu, (unsigned)m);
        if (!row) continue;
        switch (mw) {
            case 0:
            case 1: final_row_k1<Tx, 1>(i, Pp, Pj, Bc, Ginv, P0, X, dsq, B, correct, P); break;
            case 2: final_row_k1<Tx, 2>(i, Pp, Pj, Bc, Ginv, P0, X, dsq, B, correct, P); break;
            case 3: final_row_k1<Tx, 3>(i, Pp, Pj, Bc, Ginv, P0, X, dsq, B, correct, P); break;
            default: final_row_k1<Tx, 4>(i, Pp, Pj, Bc, Ginv, P0, X, dsq, B, correct, P);
        }
    }
}

// Longest row of A in every slice of 32 rows.
__global__ void k_sell_len(int n, const int *__restrict__ Ap, int *slen) {
    const int ns = (n + 31) / 32;
    for (int sl = blockIdx.x * blockDim.x + threadIdx.x; sl < ns; sl += gridDim.x * blockDim.x) {
        int mx = 0;
        for (int i = sl * 32; i < min(n, sl * 32 + 32); ++i) mx = max(mx, Ap[i + 1] - Ap[i]);
        slen[sl] = mx;
    }
}

// slice lengths -> slice starts in place (exclusive prefix sum of 32 len),
// one block of 1024 threads over tiles of 4096 slices: each tile is read
// with coalesced loads, every thread scans 4 consecutive slices, the thread
// totals are scanned across the block (warp shuffles, then the 32 warp
// totals), and the running total carries to the next tile; *total receives
// the plan's entry count (64-bit, so that the host can reject a plan beyond
// int32 positions)
__global__ void __launch_bounds__(1024) k_sell_scan(int ns, int *sptr, long long *total) {
    __shared__ long long wsum[32];
    __shared__ long long carry_s;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    long long carry = 0;
    for (int base = 0; base < ns; base += 4096) {
        long long v[4], run = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int s = base + 4 * t + k;
            v[k] = s < ns ? 32LL * sptr[s] : 0;
            run += v[k];
        }
        long long inc = run;  // inclusive scan of the thread totals in the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        if (lane == 31) wsum[w] = inc;
        __syncthreads();
        if (w == 0) {
            long long x = wsum[lane], xi = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long u = __shfl_up_sync(0xffffffffu, xi, o);
                if (lane >= o) xi += u;
            }
            wsum[lane] = xi - x;  // exclusive over the warps
            if (lane == 31) carry_s = xi;
        }
        __syncthreads();
        long long acc = carry + wsum[w] + inc - run;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int s = base + 4 * t + k;
            // positions past int32 are never used: the host rejects such a plan
            if (s < ns) sptr[s] = (int)(acc < 0x7fffffffLL ? acc : 0x7fffffffLL);
            acc += v[k];
        }
        carry += carry_s;
        __syncthreads();  // wsum and carry_s are rewritten by the next tile
    }
    if (t == 0) {
        sptr[ns] = (int)(carry < 0x7fffffffLL ? carry : 0x7fffffffLL);
        *total = carry;
    }
}

// The k = 1 plan of the fixed pattern (the adjacency of Section 4, built
// once) in SELL-32 order: for every stored (i, l) of A, the offset of row l
// of P and, for each slot s < 4 of row i, the position q of the same column
// in row l (3 bits, 7 if absent).  Padding entries carry no slot (map 0xFFF)
// and offset 0; that includes every entry of the lanes past row n - 1 in a
// ragged last slice, so that no entry of the plan is left unwritten.
// The packed word of an entry (sw, optional) holds the offset relative to
// the entry's own row, (o - p0_i) << 12 | map, and *wide is set if some
// difference falls outside [-2^19, 2^19).  Requires rows of P with at most
// 4 entries.
__global__ void k_sell_plan(int n, const int *__restrict__ Ap, const int *__restrict__ Aj,
                            const int *__restrict__ Pp, const int *__restrict__ Pj,
                            const int *__restrict__ sell_ptr, int *soff, unsigned short *smap,
                            unsigned int *sw, int *wide, int *dpos, long long nsell, int *chk) {
    // chk (bounds checks on): every position written lies in the plan and
    // every row l it refers to in [0, n); a violation is skipped and flagged
    int too_wide = 0, bad = 0;
    const int nlanes = ((n + 31) >> 5) << 5;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nlanes; i += gridDim.x * blockDim.x) {
        const int sl = i >> 5, lane = i & 31;
        const int base = sell_ptr[sl], len = (sell_ptr[sl + 1] - base) >> 5;
        const bool row = i < n;
        const int p0 = row ? Pp[i] : 0, m = row ? Pp[i + 1] - p0 : 0;
        const int e0 = row ? Ap[i] : 0, rl = row ? Ap[i + 1] - e0 : 0;
        int J[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) J[s] = (s < m) ? Pj[p0 + s] : -1;
        int dp = -1;
        for (int j = 0; j < rl; ++j)
            if (Aj[e0 + j] == i) dp = e0 + j;
        if (row) dpos[i] = dp;  // position of A(i,i) in the CSR arrays (-1: missing)
        for (int j = 0; j < len; ++j) {
            const int pos = base + j * 32 + lane;
            if (chk && (pos < 0 || pos >= nsell)) {
                bad = 1;
                continue;
            }
            unsigned int map = 0xFFFu;
            int off = 0;
            if (j < rl) {
                int l = Aj[e0 + j];
                if (chk && (l < 0 || l >= n)) {
                    bad = 1;
                    l = 0;
                }
                const int q0 = Pp[l], ml = Pp[l + 1] - q0;
                for (int q = 0; q < ml && q < 4; ++q) {
                    const int c = Pj[q0 + q];
#pragma unroll
                    for (int s = 0; s < 4; ++s)
                        if (c == J[s]) map = (map & ~(7u << (3 * s))) | ((unsigned)q << (3 * s));
                }
                off = q0;
            }
            soff[pos] = off;
            smap[pos] = (unsigned short)map;
            if (sw) {
                const int rel = (j < rl) ? off - p0 : 0;
                if (rel < -(1 << 19) || rel >= (1 << 19)) too_wide = 1;
                sw[pos] = ((unsigned int)rel << 12) | map;
            }
        }
    }
    if (__any_sync(0xffffffffu, too_wide) && (threadIdx.x & 31) == 0) atomicOr(wide, 1);
    if (chk && __any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(chk, 1);
}

// A^ = D^{-1/2} A D^{-1/2} in SELL-32 order (padding 0).  One warp per
// slice: the slice's CSR range (contiguous) is read coalesced into shared
// memory, then each lane writes its row's entries in slice order.
template <class T>
__global__ void __launch_bounds__(kBlock)
k_sell_values(int n, const int *__restrict__ Ap, const int *__restrict__ Aj,
              const double *__restrict__ Av, const double *__restrict__ dsq,
              const float *__restrict__ dsq32, const int *__restrict__ sell_ptr, T *sa,
              const unsigned int *__restrict__ sw, uint2 *spk) {
    constexpr int CAP = 256;
    __shared__ double sv[kBlock / 32][CAP];
    __shared__ int sc[kBlock / 32][CAP];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nslices = (n + 31) >> 5;
    for (int sl = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < nslices;
         sl += (gridDim.x * blockDim.x) >> 5) {
        const int i0 = sl * 32, i1 = min(i0 + 32, n);
        const int eb = Ap[i0], cnt = Ap[i1] - eb;
        const int base = sell_ptr[sl], len = (sell_ptr[sl + 1] - base) >> 5;
        const int i = i0 + lane;
        const bool valid = i < n;
        const int e0 = valid ? Ap[i] : eb, rl = valid ? Ap[i + 1] - e0 : 0;
        const double di = (valid && !dsq32) ? dsq[i] : 0.0;
        const float di32 = (valid && dsq32) ? dsq32[i] : 0.f;
        const bool staged = cnt <= CAP;
        if (staged)
            for (int t = lane; t < cnt; t += 32) {
                sv[w][t] = Av[eb + t];
                sc[w][t] = Aj[eb + t];
            }
        __syncwarp();
        for (int j = 0; j < len; ++j) {
            T v = T(0);
            if (j < rl) {
                const double a = staged ? sv[w][e0 - eb + j] : Av[e0 + j];
                const int l = staged ? sc[w][e0 - eb + j] : Aj[e0 + j];
                if constexpr (sizeof(T) == 4)
                    v = dsq32 ? di32 * f64_to_f32_rn(a) * dsq32[l]
                              : f64_to_f32_rn(di) * f64_to_f32_rn(a) * f64_to_f32_rn(dsq[l]);
                else
                    v = di * a * dsq[l];
            }
            const int pos = base + j * 32 + lane;
            if constexpr (sizeof(T) == 4) {
                if (spk) {
                    spk[pos] = make_uint2(__float_as_uint(v), sw[pos]);
                    continue;
                }
            }
            sa[pos] = v;
        }
        __syncwarp();
    }
}

// Row scales of the symmetric Jacobi scaling: D^{-1/2} and D^{1/2}.
__global__ void k_diag_scales(int n, const double *__restrict__ dinv, double *dsq, double *dhalf) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double s = sqrt(dinv[i]);
        dsq[i] = s;
        dhalf[i] = 1.0 / s;
    }
}

// A^ = D^{-1/2} A D^{-1/2} (in double, stored as T).
template <class T>
__global__ void k_scale_a(int n, const int *__restrict__ Ap, const int *__restrict__ Aj,
                          const double *__restrict__ Av, const double *__restrict__ dsq, T *Ahat) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double di = dsq[i];
        for (int e = Ap[i]; e < Ap[i + 1]; ++e) Ahat[e] = (T)(di * Av[e] * dsq[Aj[e]]);
    }
}

// k = 1: q = b / |b| per row (b = Bc(J_i)), so that Pi_B = I - q q^T.
template <class T>
__global__ void k_qvec_k1(int n, const int *__restrict__ Pp, const int *__restrict__ Pj,
                          const double *__restrict__ Bc, T *qv) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p0 = Pp[i], p1 = Pp[i + 1];
        double g = 0.0;
        for (int s = p0; s < p1; ++s) g = fma(Bc[Pj[s]], Bc[Pj[s]], g);
        const double inv = g > 0.0 ? 1.0 / sqrt(g) : 0.0;
        for (int s = p0; s < p1; ++s) qv[s] = (T)(Bc[Pj[s]] * inv);
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
                 double *Ginv, float *Ginv32, int policy, int *flags, int *ndef, int rep) {
    if (n <= 0) return;
    if (rep < 1 || n % rep) rep = 1;
    const int g = grid_for(n / rep, L.grid_rows);
    switch (k) {
#define EMIN_GRAM(KV) \
    case KV: k_gram<KV><<<g, kBlock, 0, L.stream>>>(n, Pp, Pj, Bc, Ginv, Ginv32, policy, flags, ndef, rep); note_launch(); break;
        EMIN_GRAM(1) EMIN_GRAM(2) EMIN_GRAM(3) EMIN_GRAM(4)
        EMIN_GRAM(5) EMIN_GRAM(6) EMIN_GRAM(7) EMIN_GRAM(8)
#undef EMIN_GRAM
        default: break;
    }
}

void launch_restore(const Launch &L, int n, int k, const int *Pp, const int *Pj,
                    const double *Bc, const double *B, const double *Ginv, const double *base,
                    const double *add64, const float *add32, const double *f, int correct,
                    double *P) {
    if (n <= 0) return;
    const int g = grid_for(n, L.grid_rows);
    switch (k) {
#define EMIN_RESTORE(KV)                                                                   \
    case KV:                                                                               \
        k_restore<KV><<<g, kBlock, 0, L.stream>>>(n, Pp, Pj, Bc, B, Ginv, base, add64, add32, \
                                                  f, correct, P);                          \
        note_launch();                                                                     \
        break;
        EMIN_RESTORE(1) EMIN_RESTORE(2) EMIN_RESTORE(3) EMIN_RESTORE(4)
        EMIN_RESTORE(5) EMIN_RESTORE(6) EMIN_RESTORE(7) EMIN_RESTORE(8)
#undef EMIN_RESTORE
        default: break;
    }
}

template <class Tit>
void launch_setup_k1(const Launch &L, int n, const int *dpos, const double *Av, const int *Pp,
                     const int *Pj, const double *Bc, const double *B, const double *P0_in,
                     int policy, int *flags, int *ndef, double *dsq, double *dhalf, float *dsq32,
                     double *Ginv, Tit *qv, double *P0, Tit *x0) {
    if (n <= 0) return;
    k_setup_k1<Tit><<<grid_for(n, L.grid_rows), kBlock, 0, L.stream>>>(
        n, dpos, Av, Pp, Pj, Bc, B, P0_in, policy, flags, ndef, dsq, dhalf, dsq32, Ginv, qv, P0,
        x0);
    note_launch();
}
template void launch_setup_k1<float>(const Launch &, int, const int *, const double *,
                                     const int *, const int *, const double *, const double *,
                                     const double *, int, int *, int *, double *, double *,
                                     float *, double *, float *, double *, float *);
template void launch_setup_k1<double>(const Launch &, int, const int *, const double *,
                                      const int *, const int *, const double *, const double *,
                                      const double *, int, int *, int *, double *, double *,
                                      float *, double *, double *, double *, double *);

template <class Tx>
void launch_final_k1(const Launch &L, int n, const int *Pp, const int *Pj, const double *Bc,
                     const double *Ginv, const double *P0, const Tx *X, const double *dsq,
                     const double *B, int correct, double *P) {
    if (n <= 0) return;
    k_final_k1<Tx><<<grid_for(n, L.grid_rows), kBlock, 0, L.stream>>>(n, Pp, Pj, Bc, Ginv, P0, X,
                                                                       dsq, B, correct, P);
    note_launch();
}
template void launch_final_k1<float>(const Launch &, int, const int *, const int *,
                                     const double *, const double *, const double *,
                                     const float *, const double *, const double *, int,
                                     double *);
template void launch_final_k1<double>(const Launch &, int, const int *, const int *,
                                      const double *, const double *, const double *,
                                      const double *, const double *, const double *, int,
                                      double *);

void launch_sell_scan(const Launch &L, int ns, int *sptr, long long *total) {
    k_sell_scan<<<1, 1024, 0, L.stream>>>(ns, sptr, total);
    note_launch();
}

void launch_sell_len(const Launch &L, int n, const int *Ap, int *slen) {
    if (n <= 0) return;
    k_sell_len<<<grid_for((n + 31) / 32, L.grid_rows), kBlock, 0, L.stream>>>(n, Ap, slen);
    note_launch();
}

void launch_sell_plan(const Launch &L, int n, const int *Ap, const int *Aj, const int *Pp,
                      const int *Pj, const int *sell_ptr, int *soff, unsigned short *smap,
                      unsigned int *sw, int *wide, int *dpos, long long nsell, int *chk) {
    if (n <= 0) return;
    k_sell_plan<<<grid_for(n, L.grid_rows), kBlock, 0, L.stream>>>(
        n, Ap, Aj, Pp, Pj, sell_ptr, soff, smap, sw, wide, dpos, nsell, chk);
    note_launch();
}

template <class T>
void launch_sell_values(const Launch &L, int n, const int *Ap, const int *Aj, const double *Av,
                        const double *dsq, const int *sell_ptr, T *sa, const unsigned int *sw,
                        uint2 *spk, const float *dsq32) {
    if (n <= 0) return;
    k_sell_values<T><<<grid_for((long long)((n + 31) / 32) * 32, L.grid_rows), kBlock, 0,
                       L.stream>>>(n, Ap, Aj, Av, dsq, dsq32, sell_ptr, sa, sw, spk);
    note_launch();
}
template void launch_sell_values<float>(const Launch &, int, const int *, const int *,
                                        const double *, const double *, const int *, float *,
                                        const unsigned int *, uint2 *, const float *);
template void launch_sell_values<double>(const Launch &, int, const int *, const int *,
                                         const double *, const double *, const int *, double *,
                                         const unsigned int *, uint2 *, const float *);

void launch_diag_scales(const Launch &L, int n, const double *dinv, double *dsq, double *dhalf) {
    if (n <= 0) return;
    k_diag_scales<<<grid_for(n, L.grid_rows), kBlock, 0, L.stream>>>(n, dinv, dsq, dhalf);
    note_launch();
}

template <class T>
void launch_scale_a(const Launch &L, int n, const int *Ap, const int *Aj, const double *Av,
                    const double *dsq, T *Ahat) {
    if (n <= 0) return;
    k_scale_a<T><<<grid_for(n, L.grid_rows), kBlock, 0, L.stream>>>(n, Ap, Aj, Av, dsq, Ahat);
    note_launch();
}

template <class T>
void launch_qvec_k1(const Launch &L, int n, const int *Pp, const int *Pj, const double *Bc, T *qv) {
    if (n <= 0) return;
    k_qvec_k1<T><<<grid_for(n, L.grid_rows), kBlock, 0, L.stream>>>(n, Pp, Pj, Bc, qv);
    note_launch();
}

template void launch_scale_a<double>(const Launch &, int, const int *, const int *, const double *,
                                     const double *, double *);
template void launch_scale_a<float>(const Launch &, int, const int *, const int *, const double *,
                                    const double *, float *);
template void launch_qvec_k1<double>(const Launch &, int, const int *, const int *, const double *,
                                     double *);
template void launch_qvec_k1<float>(const Launch &, int, const int *, const int *, const double *,
                                    float *);

void launch_to_float(const Launch &L, const double *src, float *dst, long long count) {
    if (count <= 0) return;
    k_to_float<<<grid_for(count, L.grid_rows), kBlock, 0, L.stream>>>(src, dst, count); note_launch();
}

void launch_to_double(const Launch &L, const float *src, double *dst, long long count) {
    if (count <= 0) return;
    k_to_double<<<grid_for(count, L.grid_rows), kBlock, 0, L.stream>>>(src, dst, count); note_launch();
}

}  // namespace emin
