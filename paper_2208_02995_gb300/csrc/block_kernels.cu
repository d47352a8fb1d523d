// Masked product for node-blocked problems (3D elasticity: 3 dofs per node,
// k = 6 coarse dofs per aggregate).  The fixed pattern is then a pattern of
// 3 x 3 blocks of A between nodes and 3 x 6 blocks of P between a node and
// an aggregate, so the product works on blocks:
//   Y_(v,g) = sum over neighbours b of v with g in aggs(b) of A_vb Y_(b,g)
// for every aggregate g of node v (Section 4's fixed-pattern product, read
// at node level).  A node plan, built once per context, gives for every
// stored block (v,b) the offset and row length of node b's rows of P and,
// for each aggregate slot s of node v, the slot q of the same aggregate in
// node b (4 bits, 15 = none).
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "emin_internal.cuh"

namespace emin {
namespace {

constexpr int NB = 3;           // dofs per node
constexpr int KB = 6;           // columns of P per aggregate (= k)
constexpr int kMaxSlots = 8;    // aggregates per node (qmap holds 8 slots of 4 bits)
constexpr int kMaxDeg = 32;     // neighbours per node staged in shared memory

inline int grid_for(long long work, int cap) {
    long long g = (work + kBlock - 1) / kBlock;
    if (g < 1) g = 1;
    return (int)(g < cap ? g : cap);
}

__device__ __forceinline__ int tri(int a, int b) { return a * (a + 1) / 2 + b; }  // a >= b

// Block structure test, one thread per node: the NB rows of a node share
// their column pattern in A and in P; A's columns come in whole aligned
// node triples, P's in whole aligned groups of KB; at most kMaxSlots
// aggregates and kMaxDeg neighbours per node.
__global__ void k_detect_blocks(int nn, const int *__restrict__ Ap, const int *__restrict__ Aj,
                                const int *__restrict__ Pp, const int *__restrict__ Pj, int *bad) {
    int fail = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nn; v += gridDim.x * blockDim.x) {
        const int a0 = Ap[NB * v], la = Ap[NB * v + 1] - a0;
        const int p0 = Pp[NB * v], lp = Pp[NB * v + 1] - p0;
        if (la % NB || lp % KB || la / NB > kMaxDeg || lp / KB > kMaxSlots) {
            fail = 1;
            continue;
        }
        for (int r = 1; r < NB && !fail; ++r) {
            const int ar = Ap[NB * v + r], pr = Pp[NB * v + r];
            if (Ap[NB * v + r + 1] - ar != la || Pp[NB * v + r + 1] - pr != lp) {
                fail = 1;
                break;
            }
            for (int e = 0; e < la && !fail; ++e)
                if (Aj[ar + e] != Aj[a0 + e]) fail = 1;
            for (int e = 0; e < lp && !fail; ++e)
                if (Pj[pr + e] != Pj[p0 + e]) fail = 1;
        }
        for (int j = 0; j < la / NB && !fail; ++j) {
            const int c = Aj[a0 + NB * j];
            if (c % NB) fail = 1;
            for (int t = 1; t < NB; ++t)
                if (Aj[a0 + NB * j + t] != c + t) fail = 1;
        }
        for (int q = 0; q < lp / KB && !fail; ++q) {
            const int c = Pj[p0 + KB * q];
            if (c % KB) fail = 1;
            for (int t = 1; t < KB; ++t)
                if (Pj[p0 + KB * q + t] != c + t) fail = 1;
        }
    }
    if (__any_sync(0xffffffffu, fail) && (threadIdx.x & 31) == 0) atomicOr(bad, 1);
}

// Node plan: for node v and its j-th neighbour b (node entry Ap[NB v]/NB^2 + j):
// offset of node b's first row of P, the length of its rows, and for every
// aggregate slot s of v the slot q of that aggregate in b (15 = none).
__global__ void k_block_plan(int nn, const int *__restrict__ Ap, const int *__restrict__ Aj,
                             const int *__restrict__ Pp, const int *__restrict__ Pj, int *boff,
                             unsigned short *blen, unsigned int *bmap, long long nentries,
                             int *chk) {
    // chk (bounds checks on): every entry written lies in the plan and every
    // neighbour node in [0, nn); a violation is skipped and flagged
    int bad = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nn; v += gridDim.x * blockDim.x) {
        const int a0 = Ap[NB * v], deg = (Ap[NB * v + 1] - a0) / NB;
        const int p0 = Pp[NB * v], na = (Pp[NB * v + 1] - p0) / KB;
        const int ne0 = a0 / NB;  // a0 / (NB*NB) node entries before v, times NB
        for (int j = 0; j < deg; ++j) {
            const int b = Aj[a0 + NB * j] / NB;
            if (chk && (b < 0 || b >= nn || (long long)(ne0 / NB + j) >= nentries)) {
                bad = 1;
                continue;
            }
            const int q0 = Pp[NB * b], nbq = (Pp[NB * b + 1] - q0) / KB;
            unsigned int map = 0xFFFFFFFFu;
            for (int s = 0; s < na; ++s) {
                const int g = Pj[p0 + KB * s];
                for (int q = 0; q < nbq; ++q)
                    if (Pj[q0 + KB * q] == g) map = (map & ~(0xFu << (4 * s))) | ((unsigned)q << (4 * s));
            }
            const int idx = ne0 / NB + j;
            boff[idx] = q0;
            blen[idx] = (unsigned short)(KB * nbq);
            bmap[idx] = map;
        }
    }
    if (chk && __any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(chk, 1);
}

// ---------------------------------------------------------------------------
// One warp per node v.  Lane (s, t) = (lane / 6 + 5 pass, lane % 6), lanes
// 0..29, owns column t of aggregate slot s of v for the node's three rows;
// two passes cover up to 10 slots.  For every neighbour b: the 3 x 3 block
// A^_vb comes from shared memory (the node's rows of A are one contiguous
// run of the CSR arrays, staged once), the lane gathers the three values
// Y(b rows, column 6 g_s + t) if b holds g_s, and accumulates A_vb times
// that column.  Epilogue per dof row: B_i^T x reduced over the warp (k = 6
// values), c = G_i^{-1} t from the staged packed factor, x -= B_i c, store,
// and the partial y^T y_.
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(kBlock)
k_kprod_blk(int nn, const int *__restrict__ Ap, const T *__restrict__ Av,
            const int *__restrict__ Pp, const int *__restrict__ Pj, const int *__restrict__ boff,
            const unsigned short *__restrict__ blen, const unsigned int *__restrict__ bmap,
            const T *__restrict__ Bc, const T *__restrict__ Ginv, const T *__restrict__ Y,
            T *__restrict__ out, int project, int dot_mode, DevState *st, double *partials,
            double *hist, int cap, int check_stop) {
    if (check_stop && st->stop) return;
    constexpr int KK = KB * (KB + 1) / 2;
    constexpr int NW = kBlock / 32;
    __shared__ T sA[NW][NB * NB * kMaxDeg];
    __shared__ int sOff[NW][kMaxDeg];
    __shared__ int sLen[NW][kMaxDeg];
    __shared__ unsigned int sMap[NW][kMaxDeg];
    __shared__ T sG[NW][NB * KK];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s_in = lane / KB, t = lane % KB;
    Dot<T> dot;
    for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < nn;
         v += (gridDim.x * blockDim.x) >> 5) {
        const int a0 = Ap[NB * v], deg = (Ap[NB * v + 1] - a0) / NB;
        const int p0 = Pp[NB * v], mrow = Pp[NB * v + 1] - p0, na = mrow / KB;
        const int ne0 = a0 / (NB * NB);
        // stage the node's blocks of A (row r, neighbour j, column c at
        // r*NB*deg + NB*j + c), its plan and its three packed factors
        for (int e = lane; e < NB * NB * deg; e += 32) sA[w][e] = Av[a0 + e];
        for (int j = lane; j < deg; j += 32) {
            sOff[w][j] = boff[ne0 + j];
            sLen[w][j] = blen[ne0 + j];
            sMap[w][j] = bmap[ne0 + j];
        }
        if (project)
            for (int e = lane; e < NB * KK; e += 32) sG[w][e] = Ginv[(size_t)NB * v * KK + e];
        __syncwarp();
        T x[2][NB];
        int col[2];
        bool act[2];
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
            const int s = s_in + 5 * pass;
            act[pass] = lane < 30 && s < na;
            col[pass] = act[pass] ? Pj[p0 + KB * s + t] : 0;
#pragma unroll
            for (int r = 0; r < NB; ++r) x[pass][r] = T(0);
        }
        const bool two = na > 5;  // warp-uniform
        const int rs = NB * deg;
        // neighbours in rounds of U: every gather of a round is issued before
        // its products, so a round costs one memory latency
        constexpr int U = 4;
        for (int j0 = 0; j0 < deg; j0 += U) {
            T y[U][2][NB];
            bool ok[U][2];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int j = j0 + u;
                const bool inr = j < deg;
                const unsigned int mp = inr ? sMap[w][j] : 0xFFFFFFFFu;
                const int off = inr ? sOff[w][j] : 0, yl = inr ? sLen[w][j] : 0;
#pragma unroll
                for (int pass = 0; pass < 2; ++pass) {
                    const int s = s_in + 5 * pass;
                    const unsigned int q = (act[pass] && (pass == 0 || two)) ? (mp >> (4 * s)) & 0xFu : 0xFu;
                    ok[u][pass] = q < (unsigned)kMaxSlots;
                    if (ok[u][pass]) {
                        const int yb = off + KB * q + t;
                        y[u][pass][0] = Y[yb];
                        y[u][pass][1] = Y[yb + yl];
                        y[u][pass][2] = Y[yb + 2 * yl];
                    } else {
                        y[u][pass][0] = y[u][pass][1] = y[u][pass][2] = T(0);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int j = j0 + u;
                if (j < deg) {
                    const T *ab = &sA[w][NB * j];
#pragma unroll
                    for (int pass = 0; pass < 2; ++pass)
                        if (ok[u][pass]) {
#pragma unroll
                            for (int r = 0; r < NB; ++r)
                                x[pass][r] = fmat(ab[r * rs], y[u][pass][0],
                                                  fmat(ab[r * rs + 1], y[u][pass][1],
                                                       fmat(ab[r * rs + 2], y[u][pass][2], x[pass][r])));
                        }
                }
            }
        }
        if (project) {
            // t_r = B_i^T x_r for each of the node's rows (B_i = Bc(J_i,:))
            T b[2][KB];
#pragma unroll
            for (int pass = 0; pass < 2; ++pass)
#pragma unroll
                for (int a = 0; a < KB; ++a)
                    b[pass][a] = act[pass] ? Bc[(size_t)col[pass] * KB + a] : T(0);
#pragma unroll
            for (int r = 0; r < NB; ++r) {
                T tv[KB];
#pragma unroll
                for (int a = 0; a < KB; ++a) {
                    T v = fmat(b[0][a], x[0][r], b[1][a] * x[1][r]);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    tv[a] = v;
                }
                const T *g = &sG[w][r * KK];
                T cv[KB];
#pragma unroll
                for (int a = 0; a < KB; ++a) {
                    T v = T(0);
#pragma unroll
                    for (int c = 0; c < KB; ++c) v = fmat(g[a >= c ? tri(a, c) : tri(c, a)], tv[c], v);
                    cv[a] = v;
                }
#pragma unroll
                for (int pass = 0; pass < 2; ++pass)
#pragma unroll
                    for (int a = 0; a < KB; ++a) x[pass][r] = fmat(-b[pass][a], cv[a], x[pass][r]);
            }
        }
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
            const int s = s_in + 5 * pass;
            if (act[pass]) {
#pragma unroll
                for (int r = 0; r < NB; ++r) {
                    const int o = p0 + r * mrow + KB * s + t;
                    out[o] = x[pass][r];
                    if (dot_mode) dot.add(Y[o], x[pass][r]);
                }
            }
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

// ---------------------------------------------------------------------------
// Output-block kernel: one lane per output block (node v, aggregate slot s)
// = the 3 x 6 block of P rows 3v..3v+2, columns 6 g_s .. 6 g_s + 5.  Warps
// hold whole nodes (a tile map, built once, lists the blocks of each warp
// with -1 padding), so the per-row projection reduces over the lanes of one
// node through shared memory.  Per neighbour b holding g_s the lane loads
// the 3 x 3 block A^_vb (lanes of one node load the same addresses) and the
// 3 x 6 block Y_(b, g_s) as 8-byte pairs (rows of P have multiples of 6
// entries, so every block column pair is 8-byte aligned), then does the 54
// products of A_vb Y_(b, g_s).
// ---------------------------------------------------------------------------
template <class T>
struct Pair;
template <>
struct Pair<float> {
    using V = float2;
};
template <>
struct Pair<double> {
    using V = double2;
};

template <class T, int MINB, bool CK = false>
__global__ void __launch_bounds__(kBlock, MINB)
k_kprod_blk2(int ntiles, const int *__restrict__ tile_map, const int *__restrict__ Ap,
             const T *__restrict__ Av, const int *__restrict__ Pp, const int *__restrict__ Pj,
             const int *__restrict__ boff, const unsigned short *__restrict__ blen,
             const unsigned int *__restrict__ bmap, const T *__restrict__ Bc,
             const T *__restrict__ Ginv, const T *__restrict__ Y, T *__restrict__ out,
             int project, int dot_mode, DevState *st, double *partials, double *hist, int cap,
             int check_stop, int *chk, long long ny) {
    if (check_stop && st->stop) return;
    int bad = 0;
    using V = typename Pair<T>::V;
    constexpr int KK = KB * (KB + 1) / 2;
    constexpr int NW = kBlock / 32;
    constexpr int R = NB * KB;  // 18 partial sums per lane: t_r[a]
    __shared__ T sT[NW][32][R + 1];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Dot<T> dot;
    for (int tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile < ntiles;
         tile += (gridDim.x * blockDim.x) >> 5) {
        const int code = tile_map[tile * 32 + lane];
        const bool valid = code >= 0;
        const int v = valid ? code >> 3 : 0, s = code & 7;
        int a0 = 0, deg = 0, p0 = 0, mrow = 0, c0 = 0;
        if (valid) {
            a0 = Ap[NB * v];
            deg = (Ap[NB * v + 1] - a0) / NB;
            p0 = Pp[NB * v];
            mrow = Pp[NB * v + 1] - p0;
            c0 = Pj[p0 + KB * s];
        }
        const int ne0 = a0 / (NB * NB), rs = NB * deg;
        T acc[NB][KB];
#pragma unroll
        for (int r = 0; r < NB; ++r)
#pragma unroll
            for (int t = 0; t < KB; ++t) acc[r][t] = T(0);
#pragma unroll 2
        for (int j = 0; j < deg; ++j) {
            const unsigned int q = (bmap[ne0 + j] >> (4 * s)) & 0xFu;
            if (q < (unsigned)kMaxSlots) {
                const int yb = boff[ne0 + j] + KB * (int)q, yl = blen[ne0 + j];
                T a[NB][NB];
#pragma unroll
                for (int r = 0; r < NB; ++r)
#pragma unroll
                    for (int c = 0; c < NB; ++c) a[r][c] = Av[a0 + r * rs + NB * j + c];
                T y[NB][KB];
#pragma unroll
                for (int c = 0; c < NB; ++c) {
                    // a row segment of KB values: its first index in [0, ny - KB]
                    const V *yp = reinterpret_cast<const V *>(
                        Y + chk_index<CK>(yb + c * yl, ny - KB + 1, bad));
#pragma unroll
                    for (int h = 0; h < KB / 2; ++h) {
                        const V u = yp[h];
                        y[c][2 * h] = u.x;
                        y[c][2 * h + 1] = u.y;
                    }
                }
#pragma unroll
                for (int r = 0; r < NB; ++r)
#pragma unroll
                    for (int t = 0; t < KB; ++t)
                        acc[r][t] = fmat(a[r][0], y[0][t],
                                         fmat(a[r][1], y[1][t], fmat(a[r][2], y[2][t], acc[r][t])));
            }
        }
        if (project) {
            // B_i restricted to this block's columns is rows c0..c0+5 of B_c;
            // they are streamed one row at a time (L1-resident) rather than
            // held, which keeps the epilogue's register footprint near that
            // of the accumulators.  This block's share of t_r = B_i^T x_r:
            const T *bcp = Bc + (size_t)c0 * KB;
            T tr[NB][KB];
#pragma unroll
            for (int r = 0; r < NB; ++r)
#pragma unroll
                for (int a = 0; a < KB; ++a) tr[r][a] = T(0);
            if (valid) {
#pragma unroll
                for (int t = 0; t < KB; ++t) {
                    T b[KB];
#pragma unroll
                    for (int a = 0; a < KB; ++a) b[a] = bcp[t * KB + a];
#pragma unroll
                    for (int r = 0; r < NB; ++r)
#pragma unroll
                        for (int a = 0; a < KB; ++a) tr[r][a] = fmat(b[a], acc[r][t], tr[r][a]);
                }
            }
#pragma unroll
            for (int r = 0; r < NB; ++r)
#pragma unroll
                for (int a = 0; a < KB; ++a) sT[w][lane][r * KB + a] = tr[r][a];
            __syncwarp();
            // the sum over the node's lanes (consecutive: first lane = lane - s)
            const int first = lane - s;
#pragma unroll
            for (int r = 0; r < NB; ++r)
#pragma unroll
                for (int a = 0; a < KB; ++a) tr[r][a] = T(0);
            if (valid) {
                const int nslot = mrow / KB;
                for (int u = 0; u < nslot; ++u)
#pragma unroll
                    for (int r = 0; r < NB; ++r)
#pragma unroll
                        for (int a = 0; a < KB; ++a) tr[r][a] += sT[w][first + u][r * KB + a];
            }
            __syncwarp();
            if (valid) {
                // c_r = G^{-1} t_r (the node's three rows share J_i, hence G_i),
                // overwriting t_r row by row
                const T *gp = Ginv + (size_t)NB * v * KK;
#pragma unroll
                for (int r = 0; r < NB; ++r) {
                    T cv[KB];
#pragma unroll
                    for (int a = 0; a < KB; ++a) {
                        T v2 = T(0);
#pragma unroll
                        for (int c = 0; c < KB; ++c)
                            v2 = fmat(gp[a >= c ? tri(a, c) : tri(c, a)], tr[r][c], v2);
                        cv[a] = v2;
                    }
#pragma unroll
                    for (int a = 0; a < KB; ++a) tr[r][a] = cv[a];
                }
                // x_r -= B_i c_r, streaming the rows of B_i again
#pragma unroll
                for (int t = 0; t < KB; ++t) {
                    T b[KB];
#pragma unroll
                    for (int a = 0; a < KB; ++a) b[a] = bcp[t * KB + a];
#pragma unroll
                    for (int r = 0; r < NB; ++r) {
                        T x = acc[r][t];
#pragma unroll
                        for (int a = 0; a < KB; ++a) x = fmat(-b[a], tr[r][a], x);
                        acc[r][t] = x;
                    }
                }
            }
        }
        if (valid) {
#pragma unroll
            for (int r = 0; r < NB; ++r) {
                const int o = p0 + r * mrow + KB * s;
                V *op = reinterpret_cast<V *>(out + o);
                const V *yo = reinterpret_cast<const V *>(Y + o);
#pragma unroll
                for (int h = 0; h < KB / 2; ++h) {
                    V u;
                    u.x = acc[r][2 * h];
                    u.y = acc[r][2 * h + 1];
                    op[h] = u;
                    if (dot_mode) {
                        const V yv = yo[h];
                        dot.add(yv.x, u.x);
                        dot.add(yv.y, u.y);
                    }
                }
            }
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

// aggregate slots per node (for the host-side tile packing)
__global__ void k_node_slots(int nn, const int *__restrict__ Pp, int *na) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nn; v += gridDim.x * blockDim.x)
        na[v] = (Pp[NB * v + 1] - Pp[NB * v]) / KB;
}

}  // namespace

int launch_detect_blocks(const Launch &L, int n, int k, const int *Ap, const int *Aj,
                         const int *Pp, const int *Pj, int *bad) {
    if (k != KB || n <= 0 || n % NB) return 0;
    const int nn = n / NB;
    k_detect_blocks<<<grid_for(nn, L.grid_rows), kBlock, 0, L.stream>>>(nn, Ap, Aj, Pp, Pj, bad);
    note_launch();
    return 1;
}

void launch_block_plan(const Launch &L, int n, const int *Ap, const int *Aj, const int *Pp,
                       const int *Pj, int *boff, unsigned short *blen, unsigned int *bmap,
                       long long nentries, int *chk) {
    const int nn = n / NB;
    if (nn <= 0) return;
    k_block_plan<<<grid_for(nn, L.grid_rows), kBlock, 0, L.stream>>>(nn, Ap, Aj, Pp, Pj, boff, blen,
                                                                    bmap, nentries, chk);
    note_launch();
}

void launch_node_slots(const Launch &L, int n, const int *Pp, int *na) {
    const int nn = n / NB;
    if (nn <= 0) return;
    k_node_slots<<<grid_for(nn, L.grid_rows), kBlock, 0, L.stream>>>(nn, Pp, na);
    note_launch();
}

// the output-block kernel on its resident grid (blocks per SM from the
// occupancy of this instantiation), at most one tile per warp
template <class T, int MINB>
void launch_blk2(const Launch &L, const Ops<T> &o, const T *Y, T *out, int project, int dot_mode,
                 Work<T> &w, int check_stop) {
    static const int per_sm = [] {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_kprod_blk2<T, MINB, false>, kBlock, 0) !=
            cudaSuccess) {
            cudaGetLastError();
            nb = 1;
        }
        return nb > 0 ? nb : 1;
    }();
    long long cap = (long long)L.nsm * per_sm;
    if (cap > kMaxGrid) cap = kMaxGrid;
    const int g = grid_for((long long)o.ntiles * 32, (int)cap);
    if (o.chk)
        k_kprod_blk2<T, MINB, true><<<g, kBlock, 0, L.stream>>>(
            o.ntiles, o.tile_map, o.Ap, o.Av, o.Pp, o.Pj, o.boff, o.blen, o.bmap, o.Bc, o.Ginv, Y,
            out, project, dot_mode, w.st, w.partials, w.hist, w.hist_cap, check_stop, o.chk,
            o.nnz_p);
    else
        k_kprod_blk2<T, MINB><<<g, kBlock, 0, L.stream>>>(
            o.ntiles, o.tile_map, o.Ap, o.Av, o.Pp, o.Pj, o.boff, o.blen, o.bmap, o.Bc, o.Ginv, Y,
            out, project, dot_mode, w.st, w.partials, w.hist, w.hist_cap, check_stop, nullptr,
            o.nnz_p);
}

template <class T>
void launch_kprod_blk(const Launch &L, const Ops<T> &o, const T *Y, T *out, int project,
                      int dot_mode, Work<T> &w, int check_stop) {
    const int nn = o.n / NB;
    if (nn <= 0) return;
    if (o.nbs.ntiles > 0 && o.nbs_blob) {
        launch_kprod_nbs<T>(L, o.nbs, o.nbs_blob, Y, out, project, dot_mode, w, check_stop, o.chk,
                            o.nnz_p);
        return;
    }
    if (o.tile_map && o.ntiles > 0) {
        // register caps without spills: 80 per thread (float), 128 (double)
        launch_blk2<T, sizeof(T) == 4 ? 3 : 2>(L, o, Y, out, project, dot_mode, w, check_stop);
        note_launch();
        return;
    }
    const int g = grid_for((long long)nn * 32, L.grid_warps);
    k_kprod_blk<T><<<g, kBlock, 0, L.stream>>>(nn, o.Ap, o.Av, o.Pp, o.Pj, o.boff, o.blen, o.bmap,
                                                o.Bc, o.Ginv, Y, out, project, dot_mode, w.st,
                                                w.partials, w.hist, w.hist_cap, check_stop);
    note_launch();
}

template void launch_kprod_blk<float>(const Launch &, const Ops<float> &, const float *, float *,
                                      int, int, Work<float> &, int);
template void launch_kprod_blk<double>(const Launch &, const Ops<double> &, const double *,
                                       double *, int, int, Work<double> &, int);

long long block_plan_entries(long long nnz_a) { return nnz_a / (NB * NB); }

}  // namespace emin
