// Kernels of one restricted PCG iteration (Algorithm 3):
//   K y as the fixed-pattern masked product mask_P(A Y) (Section 4) with the
//   projection Pi_B (Section 3.1) and the y^T y_ reduction fused in;
//   the Jacobi-preconditioned direction update and the vector updates with
//   the r^T M^{-1} r reduction.
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "emin_internal.cuh"

namespace emin {
namespace {

__device__ __forceinline__ int tri(int a, int b) { return a * (a + 1) / 2 + b; }  // a >= b

// ---------------------------------------------------------------------------
// Masked product, one thread per row of P, k = 1, at most MAXS entries per
// row of P.  For row i and every stored a_il of A, every entry (c, y_lc) of
// row l of Y whose column c is in J_i adds a_il y_lc to that slot.  The slot
// is found by comparing c with the row's (register-held) columns; one FMA is
// issued per in-pattern product, into an accumulator picked by selects.
// Epilogue: Pi_B for k = 1, x -= b (b^T x) / (b^T b) with b = Bc(J_i), and
// the partial y^T y_.
// ---------------------------------------------------------------------------
template <class T, int MAXS>
__global__ void __launch_bounds__(kBlock)
k_kprod_row_k1(int n, const int *__restrict__ Ap, const int *__restrict__ Aj,
               const T *__restrict__ Av, const int *__restrict__ Pp, const int *__restrict__ Pj,
               const T *__restrict__ Y, T *__restrict__ out, const T *__restrict__ Bc,
               const T *__restrict__ Ginv, int project, int dot_mode, DevState *st,
               double *partials, double *hist, int cap, int check_stop) {
    if (check_stop && st->stop) return;
    Dot<T> dot;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p0 = Pp[i], m = Pp[i + 1] - p0;
        int c[MAXS];
        T acc[MAXS];
#pragma unroll
        for (int s = 0; s < MAXS; ++s) {
            c[s] = (s < m) ? Pj[p0 + s] : -1;
            acc[s] = T(0);
        }
        const int e1 = Ap[i + 1];
        for (int e = Ap[i]; e < e1; ++e) {
            const int l = Aj[e];
            const T a = Av[e];
            const int q1 = Pp[l + 1];
            for (int q = Pp[l]; q < q1; ++q) {
                const int cc = Pj[q];
                int sl = -1;
#pragma unroll
                for (int s = 0; s < MAXS; ++s) sl = (cc == c[s]) ? s : sl;
                if (sl >= 0) {
                    T cur = acc[0];
#pragma unroll
                    for (int s = 1; s < MAXS; ++s) cur = (sl == s) ? acc[s] : cur;
                    cur = fmat(a, Y[q], cur);
#pragma unroll
                    for (int s = 0; s < MAXS; ++s) acc[s] = (sl == s) ? cur : acc[s];
                }
            }
        }
        if (project) {
            T b[MAXS], t = T(0);
#pragma unroll
            for (int s = 0; s < MAXS; ++s) {
                b[s] = (s < m) ? Bc[c[s]] : T(0);
                t = fmat(b[s], acc[s], t);
            }
            const T cf = t * Ginv[i];
#pragma unroll
            for (int s = 0; s < MAXS; ++s) acc[s] = fmat(-b[s], cf, acc[s]);
        }
#pragma unroll
        for (int s = 0; s < MAXS; ++s)
            if (s < m) {
                out[p0 + s] = acc[s];
                if (dot_mode) dot.add(Y[p0 + s], acc[s]);
            }
    }
    if (dot_mode) {
        __shared__ double sh[32];
        double bt = block_dot_total(dot, sh);
        double total;
        if (grid_reduce(bt, partials, &st->ticket[0], &total)) {
            if (dot_mode == DOT_ALPHA) finalize_alpha(st, total, hist, cap);
            else st->aux = total;
        }
    }
}

// ---------------------------------------------------------------------------
// Masked product, one warp per row of P, any k <= 8, rows up to kMaxRowP
// entries.  The row's columns J_i and accumulators sit in shared memory; for
// each stored a_il the lanes walk row l of Y (coalesced), find each column
// in J_i by binary search, and add a_il y_lc to that slot (distinct columns
// of row l hit distinct slots, so no two lanes of one step collide).
// Epilogue: Pi_B x = x - B_i G_i^{-1} B_i^T x with the warp-reduced k-vector
// B_i^T x, and the partial y^T y_.
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(kBlock)
k_kprod_warp(int n, int k, const int *__restrict__ Ap, const int *__restrict__ Aj,
             const T *__restrict__ Av, const int *__restrict__ Pp, const int *__restrict__ Pj,
             const T *__restrict__ Y, T *__restrict__ out, const T *__restrict__ Bc,
             const T *__restrict__ Ginv, int project, int dot_mode, DevState *st,
             double *partials, double *hist, int cap, int check_stop, int mcap) {
    if (check_stop && st->stop) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *sA = reinterpret_cast<T *>(smem) + (size_t)w * mcap;
    int *sJ = reinterpret_cast<int *>(smem + (size_t)nw * mcap * sizeof(T)) + (size_t)w * mcap;
    const int kk = k * (k + 1) / 2;
    Dot<T> dot;
    for (int i = blockIdx.x * nw + w; i < n; i += gridDim.x * nw) {
        const int p0 = Pp[i], m = Pp[i + 1] - p0;
        for (int s = lane; s < m; s += 32) {
            sJ[s] = Pj[p0 + s];
            sA[s] = T(0);
        }
        __syncwarp();
        const int e1 = Ap[i + 1];
        for (int e = Ap[i]; e < e1; ++e) {
            const int l = Aj[e];
            const T a = Av[e];
            const int q1 = Pp[l + 1];
            for (int q = Pp[l] + lane; q < q1; q += 32) {
                const int cc = Pj[q];
                int lo = 0, hi = m;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (sJ[mid] < cc) lo = mid + 1; else hi = mid;
                }
                if (lo < m && sJ[lo] == cc) sA[lo] = fmat(a, Y[q], sA[lo]);
            }
            __syncwarp();
        }
        if (project) {
            T t[kMaxK];
#pragma unroll
            for (int a = 0; a < kMaxK; ++a) t[a] = T(0);
            for (int s = lane; s < m; s += 32) {
                const T x = sA[s];
                const T *b = Bc + (size_t)sJ[s] * k;
#pragma unroll
                for (int a = 0; a < kMaxK; ++a)
                    if (a < k) t[a] = fmat(b[a], x, t[a]);
            }
#pragma unroll
            for (int a = 0; a < kMaxK; ++a)
                if (a < k)
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) t[a] += __shfl_xor_sync(0xffffffffu, t[a], o);
            T cv[kMaxK];
            const T *g = Ginv + (size_t)i * kk;
#pragma unroll
            for (int a = 0; a < kMaxK; ++a) {
                T v = T(0);
                if (a < k) {
#pragma unroll
                    for (int b = 0; b < kMaxK; ++b)
                        if (b < k) v = fmat(g[a >= b ? tri(a, b) : tri(b, a)], t[b], v);
                }
                cv[a] = v;
            }
            for (int s = lane; s < m; s += 32) {
                T x = sA[s];
                const T *b = Bc + (size_t)sJ[s] * k;
#pragma unroll
                for (int a = 0; a < kMaxK; ++a)
                    if (a < k) x = fmat(-b[a], cv[a], x);
                sA[s] = x;
            }
        }
        for (int s = lane; s < m; s += 32) {
            const T x = sA[s];
            out[p0 + s] = x;
            if (dot_mode) dot.add(Y[p0 + s], x);
        }
        __syncwarp();
    }
    if (dot_mode) {
        __shared__ double sh[32];
        double bt = block_dot_total(dot, sh);
        double total;
        if (grid_reduce(bt, partials, &st->ticket[0], &total)) {
            if (dot_mode == DOT_ALPHA) finalize_alpha(st, total, hist, cap);
            else st->aux = total;
        }
    }
}

// Stand-alone x = scale * Pi_B x (one warp per row; any k).
template <class T>
__global__ void __launch_bounds__(kBlock)
k_project_warp(int n, int k, const int *__restrict__ Pp, const int *__restrict__ Pj,
               const T *__restrict__ Bc, const T *__restrict__ Ginv, T *x, T scale) {
    const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kk = k * (k + 1) / 2;
    for (int i = blockIdx.x * nw + w; i < n; i += gridDim.x * nw) {
        const int p0 = Pp[i], p1 = Pp[i + 1];
        T t[kMaxK];
#pragma unroll
        for (int a = 0; a < kMaxK; ++a) t[a] = T(0);
        for (int s = p0 + lane; s < p1; s += 32) {
            const T v = x[s];
            const T *b = Bc + (size_t)Pj[s] * k;
#pragma unroll
            for (int a = 0; a < kMaxK; ++a)
                if (a < k) t[a] = fmat(b[a], v, t[a]);
        }
#pragma unroll
        for (int a = 0; a < kMaxK; ++a)
            if (a < k)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) t[a] += __shfl_xor_sync(0xffffffffu, t[a], o);
        T cv[kMaxK];
        const T *g = Ginv + (size_t)i * kk;
#pragma unroll
        for (int a = 0; a < kMaxK; ++a) {
            T v = T(0);
            if (a < k) {
#pragma unroll
                for (int b = 0; b < kMaxK; ++b)
                    if (b < k) v = fmat(g[a >= b ? tri(a, b) : tri(b, a)], t[b], v);
            }
            cv[a] = v;
        }
        for (int s = p0 + lane; s < p1; s += 32) {
            T v = x[s];
            const T *b = Bc + (size_t)Pj[s] * k;
#pragma unroll
            for (int a = 0; a < kMaxK; ++a)
                if (a < k) v = fmat(-b[a], cv[a], v);
            x[s] = scale * v;
        }
    }
}

// ---------------------------------------------------------------------------
// Direction update of Algorithm 3 with the Jacobi preconditioner:
// y = z + beta y with z = M_J^{-1} r = r / A(i,i) row by row (beta = 0 before
// the first step).  G lanes per row of P.  The projection after M^{-1} is
// skipped: by Theorem 1 and its corollary the row scaling keeps r in
// range(Pi_B).
// ---------------------------------------------------------------------------
template <class T, int G>
__global__ void __launch_bounds__(kBlock)
k_ydir(int n, const int *__restrict__ Pp, const T *__restrict__ dinv, const T *__restrict__ R,
       T *__restrict__ Y, const DevState *st) {
    if (st->stop) return;
    const T beta = (T)st->beta;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int sub = gid % G, groups = gridDim.x * blockDim.x / G;
    for (int i = gid / G; i < n; i += groups) {
        const int p0 = Pp[i], p1 = Pp[i + 1];
        const T d = dinv[i];
        for (int s = p0 + sub; s < p1; s += G) Y[s] = fmat(d, R[s], beta * Y[s]);
    }
}

// Vector updates dW += alpha y, r -= alpha y_ (UPD_STEP), then
// gamma = r^T M_J^{-1} r; UPD_INIT only forms gamma, UPD_FLOOR sets the
// convergence floor from the (unprojected) r.
template <class T, int G>
__global__ void __launch_bounds__(kBlock)
k_update(int n, const int *__restrict__ Pp, const T *__restrict__ dinv, T *__restrict__ R,
         const T *__restrict__ Y, const T *__restrict__ Yb, T *__restrict__ X, DevState *st,
         double *partials, int mode) {
    if (mode != UPD_FLOOR && st->stop) return;
    const T alpha = (T)st->alpha;
    Dot<T> dot;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int sub = gid % G, groups = gridDim.x * blockDim.x / G;
    for (int i = gid / G; i < n; i += groups) {
        const int p0 = Pp[i], p1 = Pp[i + 1];
        const T d = dinv[i];
        for (int s = p0 + sub; s < p1; s += G) {
            T r = R[s];
            if (mode == UPD_STEP) {
                X[s] = fmat(alpha, Y[s], X[s]);
                r = fmat(-alpha, Yb[s], r);
                R[s] = r;
            }
            dot.add(r, d * r);
        }
    }
    __shared__ double sh[32];
    double bt = block_dot_total(dot, sh);
    double total;
    if (grid_reduce(bt, partials, &st->ticket[1], &total))
        finalize_gamma(st, total, mode, GammaFloor<T>::value);
}

__global__ void k_state_reset(DevState *st) {
    DevState z = {};
    *st = z;
}

__global__ void k_state_begin(DevState *st, double tau) { st->tau = tau; }

inline int grid_for(long long work, int cap) {
    long long g = (work + kBlock - 1) / kBlock;
    if (g < 1) g = 1;
    return (int)(g < cap ? g : cap);
}

}  // namespace

template <class T>
void launch_kprod(const Launch &L, const Ops<T> &o, const T *Y, T *out, int project, int dot_mode,
                  Work<T> &w, int check_stop) {
    if (o.n <= 0) return;
    if (o.k == 1 && o.maxrow <= 4) {
        k_kprod_row_k1<T, 4><<<grid_for(o.n, L.grid_rows), kBlock, 0, L.stream>>>(
            o.n, o.Ap, o.Aj, o.Av, o.Pp, o.Pj, Y, out, o.Bc, o.Ginv, project, dot_mode, w.st,
            w.partials, w.hist, w.hist_cap, check_stop); note_launch();
    } else if (o.k == 1 && o.maxrow <= 8) {
        k_kprod_row_k1<T, 8><<<grid_for(o.n, L.grid_rows), kBlock, 0, L.stream>>>(
            o.n, o.Ap, o.Aj, o.Av, o.Pp, o.Pj, Y, out, o.Bc, o.Ginv, project, dot_mode, w.st,
            w.partials, w.hist, w.hist_cap, check_stop); note_launch();
    } else {
        const int mcap = staging_cap(o.maxrow);
        const size_t smem = (size_t)(kBlock / 32) * mcap * (sizeof(T) + sizeof(int));
        const int g = grid_for((long long)o.n * 32, L.grid_warps);
        k_kprod_warp<T><<<g, kBlock, smem, L.stream>>>(o.n, o.k, o.Ap, o.Aj, o.Av, o.Pp, o.Pj, Y,
                                                       out, o.Bc, o.Ginv, project, dot_mode, w.st,
                                                       w.partials, w.hist, w.hist_cap, check_stop,
                                                       mcap); note_launch();
    }
}

template <class T>
void launch_project(const Launch &L, const Ops<T> &o, T *x, T scale) {
    if (o.n <= 0) return;
    k_project_warp<T><<<grid_for((long long)o.n * 32, L.grid_rows), kBlock, 0, L.stream>>>(
        o.n, o.k, o.Pp, o.Pj, o.Bc, o.Ginv, x, scale); note_launch();
}

template <class T>
void launch_ydir(const Launch &L, const Ops<T> &o, Work<T> &w) {
    if (o.n <= 0) return;
    if (o.lanes == 1)
        k_ydir<T, 1><<<grid_for(o.n, L.grid_rows), kBlock, 0, L.stream>>>(o.n, o.Pp, o.dinv, w.R,
                                                                         w.Y, w.st);
    else
        k_ydir<T, 32><<<grid_for((long long)o.n * 32, L.grid_rows), kBlock, 0, L.stream>>>(
            o.n, o.Pp, o.dinv, w.R, w.Y, w.st);
    note_launch();
}

template <class T>
void launch_update(const Launch &L, const Ops<T> &o, Work<T> &w, int mode) {
    if (o.n <= 0) return;
    if (o.lanes == 1)
        k_update<T, 1><<<grid_for(o.n, L.grid_rows), kBlock, 0, L.stream>>>(
            o.n, o.Pp, o.dinv, w.R, w.Y, w.Yb, w.X, w.st, w.partials, mode);
    else
        k_update<T, 32><<<grid_for((long long)o.n * 32, L.grid_rows), kBlock, 0, L.stream>>>(
            o.n, o.Pp, o.dinv, w.R, w.Y, w.Yb, w.X, w.st, w.partials, mode);
    note_launch();
}

void set_iter_attributes() {
    const int bytes = (kBlock / 32) * kMaxRowP * (int)(sizeof(double) + sizeof(int));
    cudaFuncSetAttribute(k_kprod_warp<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_kprod_warp<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

void launch_state_reset(const Launch &L, DevState *st) { k_state_reset<<<1, 1, 0, L.stream>>>(st); note_launch(); }

void launch_state_begin(const Launch &L, DevState *st, double tau) {
    k_state_begin<<<1, 1, 0, L.stream>>>(st, tau); note_launch();
}

template void launch_kprod<double>(const Launch &, const Ops<double> &, const double *, double *,
                                   int, int, Work<double> &, int);
template void launch_kprod<float>(const Launch &, const Ops<float> &, const float *, float *, int,
                                  int, Work<float> &, int);
template void launch_project<double>(const Launch &, const Ops<double> &, double *, double);
template void launch_project<float>(const Launch &, const Ops<float> &, float *, float);
template void launch_ydir<double>(const Launch &, const Ops<double> &, Work<double> &);
template void launch_ydir<float>(const Launch &, const Ops<float> &, Work<float> &);
template void launch_update<double>(const Launch &, const Ops<double> &, Work<double> &, int);
template void launch_update<float>(const Launch &, const Ops<float> &, Work<float> &, int);

}  // namespace emin
