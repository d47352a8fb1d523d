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
// k = 1 masked product on the SELL-32 plan: one warp per slice of 32 rows,
// one lane per row.  Step j loads entry j of the 32 rows (a^_il, the offset
// of row l of Y, the slot map) as three contiguous 128/64-byte runs, then
// gathers y_lq for every slot s of row i that row l holds; one FMA per
// in-pattern product.  Epilogue per row: x -= q (q^T x), store, y^T y_.
// ---------------------------------------------------------------------------
template <bool CK, class T>
__device__ __forceinline__ void sell_step(T a, int off, unsigned int im, const T *__restrict__ Y,
                                          T &a0, T &a1, T &a2, T &a3, long long ny, int &bad) {
    const unsigned int q0 = im & 7u, q1 = (im >> 3) & 7u, q2 = (im >> 6) & 7u, q3 = (im >> 9) & 7u;
    if (q0 < 4u) a0 = fmat(a, Y[chk_index<CK>(off + (int)q0, ny, bad)], a0);
    if (q1 < 4u) a1 = fmat(a, Y[chk_index<CK>(off + (int)q1, ny, bad)], a1);
    if (q2 < 4u) a2 = fmat(a, Y[chk_index<CK>(off + (int)q2, ny, bad)], a2);
    if (q3 < 4u) a3 = fmat(a, Y[chk_index<CK>(off + (int)q3, ny, bad)], a3);
}

// The first 8 entries of every row are loaded in one round (three coalesced
// runs per entry) before any gather of Y is issued, so that a slice costs
// two memory round trips; longer rows continue in a loop.
template <class T, bool CK = false>
__global__ void __launch_bounds__(kBlock)
k_kprod_k1_sell(int n, const int *__restrict__ sell_ptr, const T *__restrict__ sa,
                const int *__restrict__ soff, const unsigned short *__restrict__ smap,
                const int *__restrict__ Pp, const T *__restrict__ qv, const T *__restrict__ Y,
                T *__restrict__ out, int project, int dot_mode, DevState *st, double *partials,
                double *hist, int cap, int check_stop, int *chk, long long ny) {
    if (check_stop && st->stop) return;
    int bad = 0;
    constexpr int U = 8;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int nslices = (n + 31) >> 5;
    Dot<T> dot;
    // slice pointers and row pointers of the next slice are fetched one
    // iteration ahead
    int sl = warp;
    int nb0 = 0, nb1 = 0, np0 = 0, np1 = 0;
    if (sl < nslices) {
        nb0 = sell_ptr[sl];
        nb1 = sell_ptr[sl + 1];
        const int i = sl * 32 + lane;
        if (i < n) {
            np0 = Pp[i];
            np1 = Pp[i + 1];
        }
    }
    for (; sl < nslices; sl += nwarps) {
        // lanes past the last row (ragged last slice) take no entries
        const int base = nb0, len = (sl * 32 + lane < n) ? (nb1 - nb0) >> 5 : 0;
        const int p0 = np0, m = np1 - np0;
        const T *pa = sa + base + lane;
        const int *po = soff + base + lane;
        const unsigned short *pm = smap + base + lane;
        T av[U];
        int ov[U];
        unsigned int mv[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            if (j < len) {
                av[j] = __ldcs(pa + j * 32);
                ov[j] = __ldcs(po + j * 32);
                mv[j] = __ldcs(pm + j * 32);
            } else {
                av[j] = T(0);
                ov[j] = 0;
                mv[j] = 0xFFFu;
            }
        }
        const int nsl = sl + nwarps;
        if (nsl < nslices) {
            nb0 = sell_ptr[nsl];
            nb1 = sell_ptr[nsl + 1];
            const int ni = nsl * 32 + lane;
            if (ni < n) {
                np0 = Pp[ni];
                np1 = Pp[ni + 1];
            } else {
                np0 = np1 = 0;
            }
        }
        // the row's own values (projection vector, y for the dot) meanwhile
        T q[4], yown[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const bool h = s < m;
            q[s] = (h && project) ? __ldcs(qv + p0 + s) : T(0);
            yown[s] = (h && dot_mode) ? Y[p0 + s] : T(0);
        }
        T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
#pragma unroll
        for (int j = 0; j < U; ++j) sell_step<CK>(av[j], ov[j], mv[j], Y, a0, a1, a2, a3, ny, bad);
        for (int j = U; j < len; ++j)
            sell_step<CK>(__ldcs(pa + j * 32), __ldcs(po + j * 32), (unsigned int)__ldcs(pm + j * 32),
                          Y, a0, a1, a2, a3, ny, bad);
        T x[4] = {a0, a1, a2, a3};
        if (project) {
            T t = T(0);
#pragma unroll
            for (int s = 0; s < 4; ++s) t = fmat(q[s], x[s], t);
#pragma unroll
            for (int s = 0; s < 4; ++s) x[s] = fmat(-q[s], t, x[s]);
        }
#pragma unroll
        for (int s = 0; s < 4; ++s)
            if (s < m) {
                out[p0 + s] = x[s];
                if (dot_mode) dot.add(yown[s], x[s]);
            }
    }
    chk_report<CK>(bad, chk);
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
// The same product (float) with the plan staged through shared memory.
// A block owns groups of 8 consecutive slices (one warp per slice); the plan
// of a group is one contiguous run of the three SELL arrays, copied with
// 16-byte cp.async into one of two shared buffers while the block works on
// the previous group, so the only memory latency left in a slice is the
// gather of Y.  A group whose plan exceeds the buffer (rows longer than 8)
// is read from global memory directly.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned int s = (unsigned int)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

constexpr int kStageWarps = kBlock / 32;
constexpr int kStageCap = kStageWarps * 8 * 32;  // plan entries per buffer

template <bool CK = false>
__global__ void __launch_bounds__(kBlock)
k_kprod_k1_staged(int n, const int *__restrict__ sell_ptr, const float *__restrict__ sa,
                  const int *__restrict__ soff, const unsigned short *__restrict__ smap,
                  const int *__restrict__ Pp, const float *__restrict__ qv,
                  const float *__restrict__ Y, float *__restrict__ out, int project, int dot_mode,
                  DevState *st, double *partials, double *hist, int cap, int check_stop, int *chk,
                  long long ny) {
    if (check_stop && st->stop) return;
    int bad = 0;
    __shared__ __align__(16) float sA[2][kStageCap];
    __shared__ __align__(16) int sO[2][kStageCap];
    __shared__ __align__(16) unsigned short sM[2][kStageCap];
    __shared__ int sPtr[2][kStageWarps + 1];
    __shared__ int sFit[2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nslices = (n + 31) >> 5;
    const int ngroups = (nslices + kStageWarps - 1) / kStageWarps;

    // issue the copies of group g into buffer b (always commits one group)
    auto prefetch = [&](int g, int b) {
        const int s0 = g * kStageWarps, s1 = min(s0 + kStageWarps, nslices);
        const int pb = sell_ptr[s0], pe = sell_ptr[s1];
        const int cnt = pe - pb;  // a multiple of 32
        if (threadIdx.x <= kStageWarps) sPtr[b][threadIdx.x] = sell_ptr[min(s0 + (int)threadIdx.x, s1)];
        const bool fit = cnt <= kStageCap;
        if (threadIdx.x == 0) sFit[b] = fit ? 1 : 0;
        if (fit) {
            for (int c = threadIdx.x; c < cnt / 4; c += blockDim.x) {
                cp_async16(&sA[b][4 * c], sa + pb + 4 * c);
                cp_async16(&sO[b][4 * c], soff + pb + 4 * c);
            }
            for (int c = threadIdx.x; c < cnt / 8; c += blockDim.x)
                cp_async16(&sM[b][8 * c], smap + pb + 8 * c);
        }
        cp_async_commit();
    };

    Dot<float> dot;
    int b = 0;
    if ((int)blockIdx.x < ngroups) prefetch(blockIdx.x, 0);
    else cp_async_commit();
    for (int g = blockIdx.x; g < ngroups; g += gridDim.x, b ^= 1) {
        const int gn = g + gridDim.x;
        if (gn < ngroups) prefetch(gn, b ^ 1);
        else cp_async_commit();
        const int sl = g * kStageWarps + warp;
        const bool have = sl < nslices;
        const int i = sl * 32 + lane;
        const bool valid = have && i < n;
        int p0 = 0, m = 0;
        if (valid) {
            p0 = Pp[i];
            m = Pp[i + 1] - p0;
        }
        float q[4], yown[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const bool h = s < m;
            q[s] = (h && project) ? __ldcs(qv + p0 + s) : 0.f;
            yown[s] = (h && dot_mode) ? Y[p0 + s] : 0.f;
        }
        cp_async_wait1();
        __syncthreads();
        if (have) {
            const int gb = sPtr[b][warp];
            const int len = valid ? (sPtr[b][warp + 1] - gb) >> 5 : 0;
            const int lb = gb - sPtr[b][0];
            const bool fit = sFit[b] != 0;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
            if (fit) {
                float av[8];
                int ov[8];
                unsigned int mv[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (j < len) {
                        av[j] = sA[b][lb + j * 32 + lane];
                        ov[j] = sO[b][lb + j * 32 + lane];
                        mv[j] = sM[b][lb + j * 32 + lane];
                    } else {
                        av[j] = 0.f;
                        ov[j] = 0;
                        mv[j] = 0xFFFu;
                    }
                }
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    sell_step<CK>(av[j], ov[j], mv[j], Y, a0, a1, a2, a3, ny, bad);
            } else {
                for (int j = 0; j < len; ++j)
                    sell_step<CK>(__ldcs(sa + gb + j * 32 + lane), __ldcs(soff + gb + j * 32 + lane),
                                  (unsigned int)__ldcs(smap + gb + j * 32 + lane), Y, a0, a1, a2,
                                  a3, ny, bad);
            }
            float x[4] = {a0, a1, a2, a3};
            if (project) {
                float t = 0.f;
#pragma unroll
                for (int s = 0; s < 4; ++s) t = fmaf(q[s], x[s], t);
#pragma unroll
                for (int s = 0; s < 4; ++s) x[s] = fmaf(-q[s], t, x[s]);
            }
#pragma unroll
            for (int s = 0; s < 4; ++s)
                if (s < m) {
                    out[p0 + s] = x[s];
                    if (dot_mode) dot.add(yown[s], x[s]);
                }
        }
        __syncthreads();  // buffer b is refilled two groups later
    }
    cp_async_wait0();
    chk_report<CK>(bad, chk);
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
// The same product on the packed plan: one 8-byte record per entry for float
// ({a^_il, word}) or a double value plus a word, read straight from global
// memory (coalesced, streaming), one warp per slice, one lane per row.  The
// word gives row l's offset relative to the lane's own row and the slot map,
// so that one load per entry replaces the three of the plain plan.  A slice's
// length and the largest row of P among its 32 rows are uniform over the
// warp; the loop body is specialised for both (exact entry count, only the
// slots that some row of the slice has), so no instruction is spent on
// padding steps or on slots no row holds.
// ---------------------------------------------------------------------------
template <class T>
struct PkPlan;
template <>
struct PkPlan<float> {
    const uint2 *e;
    __device__ __forceinline__ void get(int pos, float &a, unsigned int &w) const {
        const uint2 v = __ldcs(e + pos);
        a = __uint_as_float(v.x);
        w = v.y;
    }
};
template <>
struct PkPlan<double> {
    const double *a;
    const unsigned int *w;
    __device__ __forceinline__ void get(int pos, double &av, unsigned int &wv) const {
        av = __ldcs(a + pos);
        wv = __ldcs(w + pos);
    }
};

// L consecutive entries (positions pos, pos + 32, ...) of one lane's row:
// all records first, then every gather of Y, then the products.  The gathers
// carry no branch: a slot with no match in row l loads Y[0] (valid whenever
// a row of the warp has entries of P, the only case that gets here) and a
// select keeps its accumulator, so the loads of all L entries issue back to
// back instead of one divergent branch per slot.
template <class T, int L, int M, bool CK>
__device__ __forceinline__ void pk_entries(const PkPlan<T> &pl, int pos, int p0,
                                           const T *__restrict__ Y, T *acc, long long ny,
                                           int &bad) {
    T a[L];
    unsigned int w[L];
#pragma unroll
    for (int j = 0; j < L; ++j) pl.get(pos + 32 * j, a[j], w[j]);
    T v[L][M];
#pragma unroll
    for (int j = 0; j < L; ++j) {
        const int off = p0 + ((int)w[j] >> 12);
#pragma unroll
        for (int s = 0; s < M; ++s) {
            const unsigned int q = (w[j] >> (3 * s)) & 7u;
            v[j][s] = Y[chk_index<CK>(q < 4u ? off + (int)q : 0, ny, bad)];
        }
    }
#pragma unroll
    for (int j = 0; j < L; ++j)
#pragma unroll
        for (int s = 0; s < M; ++s) {
            const unsigned int q = (w[j] >> (3 * s)) & 7u;
            acc[s] = (q < 4u) ? fmat(a[j], v[j][s], acc[s]) : acc[s];
        }
}

template <class T, int M, bool CK>
__device__ __forceinline__ void pk_row(const PkPlan<T> &pl, int pos, int len, int p0,
                                       const T *__restrict__ Y, T *acc, long long ny, int &bad) {
    switch (len) {
        case 7: pk_entries<T, 7, M, CK>(pl, pos, p0, Y, acc, ny, bad); break;
        case 6: pk_entries<T, 6, M, CK>(pl, pos, p0, Y, acc, ny, bad); break;
        case 5: pk_entries<T, 5, M, CK>(pl, pos, p0, Y, acc, ny, bad); break;
        case 4: pk_entries<T, 4, M, CK>(pl, pos, p0, Y, acc, ny, bad); break;
        case 8: pk_entries<T, 8, M, CK>(pl, pos, p0, Y, acc, ny, bad); break;
        default: {
            int j = 0;
            for (; j + 4 <= len; j += 4) pk_entries<T, 4, M, CK>(pl, pos + 32 * j, p0, Y, acc, ny, bad);
            for (; j < len; ++j) pk_entries<T, 1, M, CK>(pl, pos + 32 * j, p0, Y, acc, ny, bad);
        }
    }
}

// 512 threads: the 16 warps of a block take 16 consecutive slices per pass, so
// more of a slice's neighbours in the second grid direction (4 slices away in
// the 3D workloads) are gathered by a sibling warp of the same SM; 768 threads
// (2 blocks per SM) measured slower
constexpr int kPkBlock = 512;
// DM, the reduction (one instantiation each, so that the product of the
// iteration, DOT_ALPHA, carries nothing else): DOT_NONE, DOT_ALPHA
// (y^T y_ -> alpha), DOT_AUX (y^T y_ -> aux), or DOT_START: out = -Pi(A^ x0)
// with the floor's <r, r> taken before the projection and (gamma0) gamma_0
// = <r~, r~> after it, reduced together.
template <class T, int DM, bool CK = false>
__global__ void __launch_bounds__(kPkBlock)
k_kprod_k1_pk(int n, const int *__restrict__ sell_ptr, PkPlan<T> pl, const int *__restrict__ Pp,
              const T *__restrict__ qv, const T *__restrict__ Y, T *__restrict__ out, int project,
              int gamma0, DevState *st, double *partials, double *hist, int cap,
              int check_stop, int *chk, long long ny) {
    constexpr bool dot_mode = (DM == DOT_ALPHA || DM == DOT_AUX);
    Dot<T> dot0, dot1;  // DOT_START: the sums before and after the projection
    if (check_stop && st->stop) return;
    const int lane = threadIdx.x & 31;
    const int nslices = (n + 31) >> 5;
    int bad = 0;
    Dot<T> dot;
    // the loop is uniform over the warp (one slice per warp and pass)
    for (int sl = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < nslices;
         sl += (gridDim.x * blockDim.x) >> 5) {
        const int i = sl * 32 + lane;
        const bool row = i < n;  // lanes past the last row take no entries
        const int base = sell_ptr[sl];
        const int len = row ? (sell_ptr[sl + 1] - base) >> 5 : 0;
        int p0 = 0, m = 0;
        if (row) {
            p0 = Pp[i];
            m = Pp[i + 1] - p0;
        }
        const unsigned int mw = __reduce_max_sync(0xffffffffu, (unsigned int)m);
        T q[4], yown[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const bool h = s < m;
            q[s] = (h && project) ? __ldcs(qv + p0 + s) : T(0);
            yown[s] = (h && dot_mode) ? Y[p0 + s] : T(0);
        }
        T x[4] = {T(0), T(0), T(0), T(0)};
        const int pos = base + lane;
        switch (mw) {
            case 0: break;  // no row of the slice has an entry of P
            case 1: pk_row<T, 1, CK>(pl, pos, len, p0, Y, x, ny, bad); break;
            case 2: pk_row<T, 2, CK>(pl, pos, len, p0, Y, x, ny, bad); break;
            case 3: pk_row<T, 3, CK>(pl, pos, len, p0, Y, x, ny, bad); break;
            default: pk_row<T, 4, CK>(pl, pos, len, p0, Y, x, ny, bad); break;
        }
        if constexpr (DM == DOT_START) {
#pragma unroll
            for (int s = 0; s < 4; ++s)
                if (s < m) dot0.add(x[s], x[s]);
        }
        if (project) {
            T t = T(0);
#pragma unroll
            for (int s = 0; s < 4; ++s) t = fmat(q[s], x[s], t);
#pragma unroll
            for (int s = 0; s < 4; ++s) x[s] = fmat(-q[s], t, x[s]);
        }
#pragma unroll
        for (int s = 0; s < 4; ++s)
            if (s < m) {
                if constexpr (DM == DOT_START) {
                    out[p0 + s] = -x[s];
                    if (gamma0) dot1.add(x[s], x[s]);
                } else {
                    out[p0 + s] = x[s];
                }
                if constexpr (dot_mode) dot.add(yown[s], x[s]);
            }
    }
    chk_report<CK>(bad, chk);
    if constexpr (dot_mode) {
        __shared__ double sh[32];
        double bt = block_dot_total(dot, sh);
        double total;
        if (grid_reduce(bt, partials, &st->ticket[0], &total)) {
            if (DM == DOT_ALPHA) finalize_alpha(st, total, hist, cap);
            else st->aux = total;
        }
    } else if constexpr (DM == DOT_START) {
        __shared__ double sh[32];
        const double b0 = block_dot_total(dot0, sh);
        __syncthreads();
        const double b1 = block_dot_total(dot1, sh);
        double s0, s1;
        if (grid_reduce2(b0, b1, partials, &st->ticket[0], &s0, &s1)) {
            finalize_gamma(st, s0, UPD_FLOOR, GammaFloor<T>::value);
            if (gamma0) finalize_gamma(st, s1, UPD_INIT, GammaFloor<T>::value);
        }
    }
}

// k = 1 stand-alone x = scale * (x - q (q^T x)), one thread per row.
template <class T>
__global__ void __launch_bounds__(kBlock)
k_project_k1(int n, const int *__restrict__ Pp, const T *__restrict__ qv, T *x, T scale) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p0 = Pp[i], p1 = Pp[i + 1];
        T t = T(0);
        for (int s = p0; s < p1; ++s) t = fmat(qv[s], x[s], t);
        for (int s = p0; s < p1; ++s) x[s] = scale * fmat(-qv[s], t, x[s]);
    }
}

// ---------------------------------------------------------------------------
// Vector steps of Algorithm 3 in the symmetrically scaled variables
// r~ = D^{-1/2} r, y~ = D^{1/2} y, dW~ = D^{1/2} dW (Jacobi M = D, Theorem 1):
// z = M^{-1} r becomes D^{-1/2} r~, so y = z + beta y is y~ = r~ + beta y~ and
// gamma = r^T M^{-1} r = <r~, r~>.  Every step is then a flat stream over the
// value arrays, 16-byte vectorised.
// ---------------------------------------------------------------------------
template <class T>
struct Vec;
template <>
struct Vec<float> {
    using V = float4;
    static constexpr int W = 4;
};
template <>
struct Vec<double> {
    using V = double2;
    static constexpr int W = 2;
};

__device__ __forceinline__ float4 axpy4(float b, float4 y, float4 r) {
    return make_float4(fmaf(b, y.x, r.x), fmaf(b, y.y, r.y), fmaf(b, y.z, r.z), fmaf(b, y.w, r.w));
}
__device__ __forceinline__ double2 axpy4(double b, double2 y, double2 r) {
    return make_double2(fma(b, y.x, r.x), fma(b, y.y, r.y));
}

// y~ = z~ + beta y~ (z~ = r~ for Jacobi; R is z~)
// the flat streams ask for 8 resident blocks (2048 threads) per SM and are
// launched as one resident wave (Launch::grid_flat*)
template <class T>
__global__ void __launch_bounds__(kBlock, 8)
k_ydir_flat(long long count, const T *__restrict__ R, T *__restrict__ Y, const DevState *st) {
    if (st->stop) return;
    const T beta = (T)st->beta;
    using V = typename Vec<T>::V;
    constexpr int W = Vec<T>::W;
    // 32-bit unsigned indices: value arrays on P's pattern have fewer than
    // 2^31 entries (int32 row pointers), so no index or step passes 2^32
    const unsigned nv = (unsigned)(count / W), cnt = (unsigned)count;
    const unsigned stride = gridDim.x * blockDim.x;
    const V *R4 = reinterpret_cast<const V *>(R);
    V *Y4 = reinterpret_cast<V *>(Y);
    for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride)
        Y4[v] = axpy4(beta, Y4[v], R4[v]);
    for (unsigned q = nv * W + blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += stride)
        Y[q] = fmat(beta, Y[q], R[q]);
}

// dW~ += alpha y~, r~ -= alpha y_~ (UPD_STEP, UPD_XR), then gamma = <r~, r~>
// (UPD_STEP, UPD_INIT) or <r~, z~> (UPD_GZ_*, Z given); UPD_FLOOR sets the
// convergence floor from <r~, r~>.
template <class T, int MODE>
__device__ __forceinline__ void upd1(T &r, T &x, T y, T yb, T alpha, Dot<T> &dot) {
    x = fmat(alpha, y, x);
    r = fmat(-alpha, yb, r);
    if constexpr (MODE == UPD_STEP) dot.add(r, r);
}

// one instantiation per mode, so that each carries only its own path
template <class T, int MODE>
__global__ void __launch_bounds__(kBlock, 8)
k_update_flat(long long count, T *__restrict__ R, const T *__restrict__ Y,
              const T *__restrict__ Yb, T *__restrict__ X, DevState *st, double *partials,
              const T *__restrict__ Z) {
    constexpr int mode = MODE;
    if (mode != UPD_FLOOR && st->stop) return;
    const T alpha = (T)st->alpha;
    using V = typename Vec<T>::V;
    constexpr int W = Vec<T>::W;
    // 32-bit unsigned indices (see k_ydir_flat)
    const unsigned nv = (unsigned)(count / W), cnt = (unsigned)count;
    const unsigned stride = gridDim.x * blockDim.x;
    Dot<T> dot;
    constexpr bool step = (mode == UPD_STEP || mode == UPD_XR);
    constexpr bool gz = (mode == UPD_GZ_INIT || mode == UPD_GZ_STEP);
    for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) {
        V r = reinterpret_cast<V *>(R)[v];
        if constexpr (gz) {
            const V z = reinterpret_cast<const V *>(Z)[v];
            dot.add(r.x, z.x);
            dot.add(r.y, z.y);
            if constexpr (W == 4) {
                dot.add(r.z, z.z);
                dot.add(r.w, z.w);
            }
        } else if constexpr (step) {
            V x = reinterpret_cast<V *>(X)[v];
            const V y = reinterpret_cast<const V *>(Y)[v];
            const V yb = reinterpret_cast<const V *>(Yb)[v];
            upd1<T, MODE>(r.x, x.x, y.x, yb.x, alpha, dot);
            upd1<T, MODE>(r.y, x.y, y.y, yb.y, alpha, dot);
            if constexpr (W == 4) {
                upd1<T, MODE>(r.z, x.z, y.z, yb.z, alpha, dot);
                upd1<T, MODE>(r.w, x.w, y.w, yb.w, alpha, dot);
            }
            reinterpret_cast<V *>(X)[v] = x;
            reinterpret_cast<V *>(R)[v] = r;
        } else {
            dot.add(r.x, r.x);
            dot.add(r.y, r.y);
            if constexpr (W == 4) {
                dot.add(r.z, r.z);
                dot.add(r.w, r.w);
            }
        }
    }
    for (unsigned q = nv * W + blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += stride) {
        T r = R[q];
        if constexpr (gz) {
            dot.add(r, Z[q]);
        } else if constexpr (step) {
            T x = X[q];
            upd1<T, MODE>(r, x, Y[q], Yb[q], alpha, dot);
            X[q] = x;
            R[q] = r;
        } else {
            dot.add(r, r);
        }
    }
    if constexpr (mode == UPD_XR) return;  // no reduction: gamma follows the preconditioner
    __shared__ double sh[32];
    double bt = block_dot_total(dot, sh);
    double total;
    if (grid_reduce(bt, partials, &st->ticket[1], &total))
        finalize_gamma(st, total,
                       mode == UPD_GZ_INIT ? UPD_INIT : (mode == UPD_GZ_STEP ? UPD_STEP : mode),
                       GammaFloor<T>::value);
}

// out[s] = (Tout)(scale * f[i] * in[s]) on the entries of row i (G lanes per row)
template <class Tin, class Tout, int G>
__global__ void __launch_bounds__(kBlock)
k_row_scale(int n, const int *__restrict__ Pp, const double *__restrict__ f, double scale,
            const Tin *in, Tout *out) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int sub = gid % G, groups = gridDim.x * blockDim.x / G;
    for (int i = gid / G; i < n; i += groups) {
        const double fi = scale * f[i];
        for (int s = Pp[i] + sub; s < Pp[i + 1]; s += G) out[s] = (Tout)(fi * (double)in[s]);
    }
}

__global__ void k_state_reset(DevState *st) {
    DevState z = {};
    *st = z;
}

__global__ void k_state_begin(DevState *st, double tau, int n_iters) {
    st->tau = tau;
    st->loop_left = n_iters;
}

// End of one iteration of the captured while-loop: one iteration fewer
// left; the loop goes on while some are left and the stop test has not
// fired (a stopped state makes every kernel of the body return at once, so
// at most one empty pass follows the stop).
__global__ void k_loop_control(DevState *st, cudaGraphConditionalHandle h) {
    const int left = --st->loop_left;
    cudaGraphSetConditional(h, (left > 0 && st->stop == 0) ? 1u : 0u);
}

inline int grid_for(long long work, int cap) {
    long long g = (work + kBlock - 1) / kBlock;
    if (g < 1) g = 1;
    return (int)(g < cap ? g : cap);
}

}  // namespace

// Resident blocks per SM of one instantiation of the packed product (the
// instantiations hold different register counts), queried once.
template <class T, int DM>
int pk_per_sm() {
    static const int per_sm = [] {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_kprod_k1_pk<T, DM>, kPkBlock,
                                                          0) != cudaSuccess) {
            cudaGetLastError();
            nb = 1;
        }
        return nb > 0 ? nb : 1;
    }();
    return per_sm;
}

template <class T>
void launch_kprod(const Launch &L, const Ops<T> &o, const T *Y, T *out, int project, int dot_mode,
                  Work<T> &w, int check_stop) {
    if (o.n <= 0) return;
    if (o.boff && o.blen && o.bmap) {
        launch_kprod_blk<T>(L, o, Y, out, project, dot_mode, w, check_stop);
        return;
    }
    if (o.k == 1 && o.sell_ptr && o.sw && o.qv && o.maxrow <= 4 &&
        (sizeof(T) == 4 ? o.spk != nullptr : o.sa != nullptr)) {
        PkPlan<T> pl;
        if constexpr (sizeof(T) == 4) {
            pl.e = o.spk;
        } else {
            pl.a = o.sa;
            pl.w = o.sw;
        }
        const long long warps = (o.n + 31) / 32;
        const long long need = (warps * 32 + kPkBlock - 1) / kPkBlock;
        // one resident wave of the instantiation that runs (queried at create)
        switch (dot_mode) {
#define EMIN_PK(DMV)                                                                         \
    case DMV: {                                                                              \
        long long cap = (long long)L.nsm * pk_per_sm<T, DMV>();                              \
        if (cap > kMaxGrid) cap = kMaxGrid;                                                  \
        const int g = (int)(need < cap ? (need > 0 ? need : 1) : cap);                      \
        if (o.chk)                                                                           \
            k_kprod_k1_pk<T, DMV, true><<<g, kPkBlock, 0, L.stream>>>(                       \
                o.n, o.sell_ptr, pl, o.Pp, o.qv, Y, out, project, 0, w.st, w.partials,       \
                w.hist, w.hist_cap, check_stop, o.chk, o.nnz_p);                             \
        else                                                                                 \
            k_kprod_k1_pk<T, DMV><<<g, kPkBlock, 0, L.stream>>>(                             \
                o.n, o.sell_ptr, pl, o.Pp, o.qv, Y, out, project, 0, w.st, w.partials,       \
                w.hist, w.hist_cap, check_stop, nullptr, o.nnz_p);                           \
    } break;
            EMIN_PK(DOT_NONE)
            EMIN_PK(DOT_ALPHA)
            EMIN_PK(DOT_AUX)
#undef EMIN_PK
            default: return;
        }
    } else if (o.k == 1 && o.sell_ptr && o.sa && o.qv && o.maxrow <= 4) {
        if constexpr (sizeof(T) == 4) {
            // one block per group of 8 slices, at most the resident grid
            const long long groups = ((o.n + 31) / 32 + kStageWarps - 1) / kStageWarps;
            const int g = (int)(groups < L.grid_staged ? groups : L.grid_staged);
            if (o.chk)
                k_kprod_k1_staged<true><<<g, kBlock, 0, L.stream>>>(
                    o.n, o.sell_ptr, o.sa, o.soff, o.smap, o.Pp, o.qv, Y, out, project, dot_mode,
                    w.st, w.partials, w.hist, w.hist_cap, check_stop, o.chk, o.nnz_p);
            else
                k_kprod_k1_staged<<<g, kBlock, 0, L.stream>>>(
                    o.n, o.sell_ptr, o.sa, o.soff, o.smap, o.Pp, o.qv, Y, out, project, dot_mode,
                    w.st, w.partials, w.hist, w.hist_cap, check_stop, nullptr, o.nnz_p);
        } else {
            const int g = grid_for((long long)((o.n + 31) / 32) * 32, L.grid_rows);
            if (o.chk)
                k_kprod_k1_sell<T, true><<<g, kBlock, 0, L.stream>>>(
                    o.n, o.sell_ptr, o.sa, o.soff, o.smap, o.Pp, o.qv, Y, out, project, dot_mode,
                    w.st, w.partials, w.hist, w.hist_cap, check_stop, o.chk, o.nnz_p);
            else
                k_kprod_k1_sell<T><<<g, kBlock, 0, L.stream>>>(
                    o.n, o.sell_ptr, o.sa, o.soff, o.smap, o.Pp, o.qv, Y, out, project, dot_mode,
                    w.st, w.partials, w.hist, w.hist_cap, check_stop, nullptr, o.nnz_p);
        }
    } else if (o.k == 1 && o.maxrow <= 4) {
        k_kprod_row_k1<T, 4><<<grid_for(o.n, L.grid_rows), kBlock, 0, L.stream>>>(
            o.n, o.Ap, o.Aj, o.Av, o.Pp, o.Pj, Y, out, o.Bc, o.Ginv, project, dot_mode, w.st,
            w.partials, w.hist, w.hist_cap, check_stop);
    } else if (o.k == 1 && o.maxrow <= 8) {
        k_kprod_row_k1<T, 8><<<grid_for(o.n, L.grid_rows), kBlock, 0, L.stream>>>(
            o.n, o.Ap, o.Aj, o.Av, o.Pp, o.Pj, Y, out, o.Bc, o.Ginv, project, dot_mode, w.st,
            w.partials, w.hist, w.hist_cap, check_stop);
    } else {
        const int mcap = staging_cap(o.maxrow);
        const size_t smem = (size_t)(kBlock / 32) * mcap * (sizeof(T) + sizeof(int));
        const int g = grid_for((long long)o.n * 32, L.grid_warps);
        k_kprod_warp<T><<<g, kBlock, smem, L.stream>>>(o.n, o.k, o.Ap, o.Aj, o.Av, o.Pp, o.Pj, Y,
                                                       out, o.Bc, o.Ginv, project, dot_mode, w.st,
                                                       w.partials, w.hist, w.hist_cap, check_stop,
                                                       mcap);
    }
    note_launch();
}

template <class T>
void launch_project(const Launch &L, const Ops<T> &o, T *x, T scale) {
    if (o.n <= 0) return;
    if (o.k == 1 && o.qv)
        k_project_k1<T><<<grid_for(o.n, L.grid_rows), kBlock, 0, L.stream>>>(o.n, o.Pp, o.qv, x,
                                                                             scale);
    else
        k_project_warp<T><<<grid_for((long long)o.n * 32, L.grid_rows), kBlock, 0, L.stream>>>(
            o.n, o.k, o.Pp, o.Pj, o.Bc, o.Ginv, x, scale);
    note_launch();
}

template <class T>
bool launch_kprod_start(const Launch &L, const Ops<T> &o, const T *x0, T *R, Work<T> &w,
                        int gamma0) {
    if (o.n <= 0) return false;
    if (o.nbs.ntiles > 0 && o.nbs_blob) {  // the staged node-block product
        launch_kprod_nbs<T>(L, o.nbs, o.nbs_blob, x0, R, 1, DOT_START, w, 0, o.chk, o.nnz_p,
                            gamma0);
        return true;
    }
    if (o.boff && o.blen && o.bmap) return false;
    if (!(o.k == 1 && o.sell_ptr && o.sw && o.qv && o.maxrow <= 4 &&
          (sizeof(T) == 4 ? o.spk != nullptr : o.sa != nullptr)))
        return false;
    PkPlan<T> pl;
    if constexpr (sizeof(T) == 4) {
        pl.e = o.spk;
    } else {
        pl.a = o.sa;
        pl.w = o.sw;
    }
    const long long warps = (o.n + 31) / 32;
    const long long need = (warps * 32 + kPkBlock - 1) / kPkBlock;
    // one resident wave of this instantiation (it holds more registers than
    // the iteration's product)
    const long long cap = (long long)L.nsm * pk_per_sm<T, DOT_START>();
    int g = (int)(need < cap ? (need > 0 ? need : 1) : cap);
    if (2 * g > kMaxGrid) g = kMaxGrid / 2;  // two partial sums per block
    if (o.chk)
        k_kprod_k1_pk<T, DOT_START, true><<<g, kPkBlock, 0, L.stream>>>(
            o.n, o.sell_ptr, pl, o.Pp, o.qv, x0, R, 1, gamma0, w.st, w.partials, w.hist,
            w.hist_cap, 0, o.chk, o.nnz_p);
    else
        k_kprod_k1_pk<T, DOT_START><<<g, kPkBlock, 0, L.stream>>>(
            o.n, o.sell_ptr, pl, o.Pp, o.qv, x0, R, 1, gamma0, w.st, w.partials, w.hist,
            w.hist_cap, 0, nullptr, o.nnz_p);
    note_launch();
    return true;
}

template <class T>
void launch_ydir(const Launch &L, long long count, Work<T> &w) {
    if (count <= 0) return;
    const int g = grid_for((count + Vec<T>::W - 1) / Vec<T>::W,
                           sizeof(T) == 4 ? L.grid_flat32 : L.grid_flat64);
    k_ydir_flat<T><<<g, kBlock, 0, L.stream>>>(count, w.Z ? w.Z : w.R, w.Y, w.st);
    note_launch();
}

template <class T>
void launch_update(const Launch &L, long long count, Work<T> &w, int mode) {
    if (count <= 0) return;
    const int g = grid_for((count + Vec<T>::W - 1) / Vec<T>::W,
                           sizeof(T) == 4 ? L.grid_flat32 : L.grid_flat64);
    switch (mode) {
#define EMIN_UPD(M)                                                                           \
    case M:                                                                                   \
        k_update_flat<T, M><<<g, kBlock, 0, L.stream>>>(count, w.R, w.Y, w.Yb, w.X, w.st,    \
                                                        w.partials, w.Z);                     \
        break;
        EMIN_UPD(UPD_INIT)
        EMIN_UPD(UPD_STEP)
        EMIN_UPD(UPD_FLOOR)
        EMIN_UPD(UPD_XR)
        EMIN_UPD(UPD_GZ_INIT)
        EMIN_UPD(UPD_GZ_STEP)
#undef EMIN_UPD
        default: return;
    }
    note_launch();
}

// Resident grid of the flat streams (direction and update kernels): the
// blocks per SM of the hot update (and of the direction kernel, whichever is
// smaller), so that a launch is one full wave.
int flat_blocks_per_sm(int double_precision) {
    int a = 0, b = 0;
    cudaError_t e1, e2;
    if (double_precision) {
        e1 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_update_flat<double, UPD_STEP>,
                                                           kBlock, 0);
        e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_ydir_flat<double>, kBlock, 0);
    } else {
        e1 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_update_flat<float, UPD_STEP>,
                                                           kBlock, 0);
        e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_ydir_flat<float>, kBlock, 0);
    }
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    const int nb = a < b ? a : b;
    return nb > 0 ? nb : 1;
}

template <class Tin, class Tout>
void launch_row_scale(const Launch &L, int n, const int *Pp, int lanes, const double *f,
                      double scale, const Tin *in, Tout *out) {
    if (n <= 0) return;
    if (lanes == 1)
        k_row_scale<Tin, Tout, 1><<<grid_for(n, L.grid_rows), kBlock, 0, L.stream>>>(
            n, Pp, f, scale, in, out);
    else
        k_row_scale<Tin, Tout, 32><<<grid_for((long long)n * 32, L.grid_rows), kBlock, 0,
                                      L.stream>>>(n, Pp, f, scale, in, out);
    note_launch();
}

int staged_blocks_per_sm() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_kprod_k1_staged<false>, kBlock, 0) !=
        cudaSuccess) {
        cudaGetLastError();
        nb = 1;
    }
    return nb > 0 ? nb : 1;
}

int pk_blocks_per_sm(int double_precision) {
    // every instantiation's query is made here, at create, and not first
    // inside a graph capture; the iteration's product is DOT_ALPHA
    if (double_precision) {
        pk_per_sm<double, DOT_NONE>();
        pk_per_sm<double, DOT_AUX>();
        pk_per_sm<double, DOT_START>();
        return pk_per_sm<double, DOT_ALPHA>();
    }
    pk_per_sm<float, DOT_NONE>();
    pk_per_sm<float, DOT_AUX>();
    pk_per_sm<float, DOT_START>();
    return pk_per_sm<float, DOT_ALPHA>();
}

void set_iter_attributes() {
    const int bytes = (kBlock / 32) * kMaxRowP * (int)(sizeof(double) + sizeof(int));
    cudaFuncSetAttribute(k_kprod_warp<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_kprod_warp<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

void launch_state_reset(const Launch &L, DevState *st) {
    k_state_reset<<<1, 1, 0, L.stream>>>(st);
    note_launch();
}

void launch_loop_control(const Launch &L, DevState *st, cudaGraphConditionalHandle h) {
    k_loop_control<<<1, 1, 0, L.stream>>>(st, h);
    note_launch();
}

void launch_state_begin(const Launch &L, DevState *st, double tau, int n_iters) {
    k_state_begin<<<1, 1, 0, L.stream>>>(st, tau, n_iters);
    note_launch();
}

template void launch_kprod<double>(const Launch &, const Ops<double> &, const double *, double *,
                                   int, int, Work<double> &, int);
template void launch_kprod<float>(const Launch &, const Ops<float> &, const float *, float *, int,
                                  int, Work<float> &, int);
template void launch_project<double>(const Launch &, const Ops<double> &, double *, double);
template void launch_project<float>(const Launch &, const Ops<float> &, float *, float);
template bool launch_kprod_start<double>(const Launch &, const Ops<double> &, const double *,
                                         double *, Work<double> &, int);
template bool launch_kprod_start<float>(const Launch &, const Ops<float> &, const float *,
                                        float *, Work<float> &, int);
template void launch_ydir<double>(const Launch &, long long, Work<double> &);
template void launch_ydir<float>(const Launch &, long long, Work<float> &);
template void launch_update<double>(const Launch &, long long, Work<double> &, int);
template void launch_update<float>(const Launch &, long long, Work<float> &, int);
template void launch_row_scale<double, double>(const Launch &, int, const int *, int,
                                               const double *, double, const double *, double *);
template void launch_row_scale<double, float>(const Launch &, int, const int *, int,
                                              const double *, double, const double *, float *);
template void launch_row_scale<float, double>(const Launch &, int, const int *, int,
                                              const double *, double, const float *, double *);

}  // namespace emin
