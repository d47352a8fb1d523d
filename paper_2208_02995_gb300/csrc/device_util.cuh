// Device helpers: typed fused multiply-add, compensated float accumulation
// and deterministic block / grid reductions to double.
#pragma once
#include <cuda_runtime.h>

#include "emin_internal.cuh"

namespace emin {

__device__ __forceinline__ double fmat(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmat(float a, float b, float c) { return fmaf(a, b, c); }

// ---------------------------------------------------------------------------
// Dot-product accumulators.  Dot<double> is a plain FMA chain.  Dot<float>
// (mixed path) sums the float products of one thread in float - a thread
// holds a few dozen of them at most - and every further level (warp, block,
// grid) is summed in double.
// ---------------------------------------------------------------------------
template <class T>
struct Dot;

template <>
struct Dot<double> {
    double v = 0.0;
    __device__ __forceinline__ void add(double a, double b) { v = fma(a, b, v); }
    __device__ __forceinline__ double warp_total() {
        double s = v;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        return s;  // lane 0 holds the warp sum
    }
};

template <>
struct Dot<float> {
    float v = 0.f;
    __device__ __forceinline__ void add(float a, float b) { v = fmaf(a, b, v); }
    __device__ __forceinline__ double warp_total() {
        double s = (double)v;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        return s;
    }
};

// Sum of one double per thread over the block, fixed order; result valid in
// thread 0.  `sh` holds at least 32 doubles.
__device__ __forceinline__ double block_sum(double v, double *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    return s;
}

// Deterministic grid reduction: every block passes its total (valid in
// thread 0); the last block to arrive sums the block totals in block order.
// Returns true in thread 0 of that last block, with *total set.
__device__ __forceinline__ bool grid_reduce(double block_total, double *partials,
                                            unsigned int *ticket, double *total) {
    __shared__ bool am_last;
    __shared__ double sh[32];
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = block_total;
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += __ldcg(partials + b);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        *total = s;
        *ticket = 0u;
    }
    return threadIdx.x == 0;
}

// Two sums reduced at once, deterministically (as grid_reduce): partials
// holds 2 gridDim.x doubles; returns true in thread 0 of the last block,
// with *ta and *tb set.
__device__ __forceinline__ bool grid_reduce2(double a, double b, double *partials,
                                             unsigned int *ticket, double *ta, double *tb) {
    __shared__ bool am_last;
    __shared__ double sh[32];
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = a;
        partials[gridDim.x + blockIdx.x] = b;
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    double sa = 0.0, sb = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
        sa += __ldcg(partials + k);
        sb += __ldcg(partials + gridDim.x + k);
    }
    sa = block_sum(sa, sh);
    __syncthreads();
    sb = block_sum(sb, sh);
    if (threadIdx.x == 0) {
        *ta = sa;
        *tb = sb;
        *ticket = 0u;
    }
    return threadIdx.x == 0;
}

// Warp totals of a Dot accumulator gathered into one double per block.
template <class T>
__device__ __forceinline__ double block_dot_total(Dot<T> &d, double *sh) {
    double wt = d.warp_total();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = wt;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    return s;
}

// 1/sqrt(x) for positive, finite, normal x by Newton-Raphson on
// f(r) = r^-2 - x (r <- r (3 - x r^2) / 2), from a float seed on the
// mantissa: the seed has about 23 correct bits, each step doubles them, so
// two steps reach double precision up to a few ulps.  The exponent is
// handled exactly (even power of two split off), so no FP64 division or
// square root is issued.  Subnormal or non-positive x fall back to 1/sqrt.
__device__ __forceinline__ double rsqrt_newton(double x) {
    if (!(x >= 2.2250738585072014e-308) || !(x <= 1.7976931348623157e308)) return 1.0 / sqrt(x);
    const long long b = __double_as_longlong(x);
    int ex = (int)((b >> 52) & 0x7ff) - 1023;
    double m = __longlong_as_double((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);  // [1, 2)
    if (ex & 1) {
        m *= 2.0;
        ex -= 1;
    }
    double r = (double)rsqrtf((float)m);
    r = r * fma(-0.5 * m, r * r, 1.5);
    r = r * fma(-0.5 * m, r * r, 1.5);
    return r * __longlong_as_double((long long)(1023 - ex / 2) << 52);
}

// ---- bounds checks of the gather kernels (emin_opts.checks = 1) ----
// With CK, an index outside [0, len) is replaced by 0 (a valid position, so
// the access stays in bounds) and the thread records the fault; chk_report,
// called by whole warps at the end of a kernel, ORs the warp's faults into
// the context's check word, which the host reads after the call and reports
// as EMIN_ERR_PATTERN.  Without CK both compile to nothing.
template <bool CK>
__device__ __forceinline__ int chk_index(int i, long long len, int &bad) {
    if constexpr (CK) {
        if (i < 0 || (long long)i >= len) {
            bad = 1;
            return 0;
        }
    }
    return i;
}
template <bool CK>
__device__ __forceinline__ void chk_report(int bad, int *word) {
    if constexpr (CK) {
        if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(word, 1);
    }
}

// ---- scalar steps of Algorithm 3, run by one thread after a reduction ----

// After y^T y_ is known: alpha, dE_k = gamma alpha (Eq. (CG_dEa)), the stop
// test dE_k < tau dE_1 of Eq. (relRed) (the step is then not applied).
__device__ __forceinline__ void finalize_alpha(DevState *st, double ydy, double *hist, int cap) {
    st->ydy = ydy;
    const double g = st->gamma;
    if (!(ydy > 0.0) || !isfinite(ydy) || !isfinite(g)) {
        st->stop = 2;
        st->status = EMIN_ERR_BREAKDOWN;
        return;
    }
    const double alpha = g / ydy;
    const double dE = g * alpha;
    const int kk = st->k;
    st->k = kk + 1;
    if (kk < cap) hist[kk] = dE;
    if (kk == 0) st->dE1 = dE;
    st->dE_last = dE;
    st->alpha = alpha;
    if (dE < st->tau * st->dE1) st->stop = 1;
}

// Convergence floor of gamma relative to the unprojected <b, M^{-1} b>:
// (100 eps)^2 of the working precision (the residual cannot shrink further
// than about 100 ulps relative to the right-hand side).
template <class T>
struct GammaFloor;
template <>
struct GammaFloor<double> {
    static constexpr double value = kGammaFloor;  // (100 * 2^-53)^2 ~ 1.2e-28
};
template <>
struct GammaFloor<float> {
    static constexpr double value = 3.6e-11;      // (100 * 2^-24)^2 ~ 3.6e-11
};

// After the new gamma = r^T M^{-1} r is known.
__device__ __forceinline__ void finalize_gamma(DevState *st, double gnew, int mode,
                                               double floor_factor) {
    if (mode == UPD_FLOOR) {
        st->gamma_floor = floor_factor * gnew;
        return;
    }
    if (!isfinite(gnew)) {
        st->stop = 2;
        st->status = EMIN_ERR_BREAKDOWN;
        return;
    }
    if (mode == UPD_INIT) {
        st->gamma = gnew;
        st->gamma_old = 0.0;
        st->beta = 0.0;
    } else {
        st->applied += 1;
        st->beta = gnew / st->gamma;
        st->gamma_old = st->gamma;
        st->gamma = gnew;
    }
    if (!(gnew > st->gamma_floor)) st->stop = 1;
}

}  // namespace emin
