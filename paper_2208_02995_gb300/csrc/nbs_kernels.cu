// Staged masked product for node-blocked problems (3D elasticity: 3 dofs per
// node, k = 6 coarse dofs per aggregate), Section 4's fixed-pattern product
// Y_(v,g) = sum over neighbours b of v holding g of A_vb Y_(b,g), with the
// projection Pi_B of Section 3.1 fused into its epilogue.
//
// Why staged: with one lane per 3 x 6 output block (node v, aggregate slot s)
// the lanes of a warp gather 3 x 6 blocks of Y from many nodes, and every
// warp-wide load touches about ten 128-byte lines; the L1 data pipe, which
// returns one line-sized wavefront per cycle, saturates long before HBM or
// the FMA pipes do.  Here a CTA works on a tile of whole nodes grown over the
// node graph (compact in space, so that the tile's neighbours are few), and
// one thread brings in, with TMA bulk copies that bypass the load pipe:
//   - the tile's blob: per-lane and per-node records, the pair plan (for
//     every two neighbours of a node: the shared-memory offset and row length
//     of each neighbour's rows of Y and its slot map), the 3 x 3 blocks of A^
//     in pairs, the nodes' inverse Gram factors and the tile's B_c rows;
//   - every node the tile's nodes touch: its rows of Y, copied as contiguous
//     runs of consecutive nodes.
// The gathers then read shared memory, where a warp-wide load costs bank
// cycles, not lines.  A neighbour that does not hold a lane's aggregate is
// read from a zero block (the product adds A x 0), so every lane runs the
// same loop with no branch per neighbour.
#include <cuda_runtime.h>

#include <algorithm>
#include <deque>
#include <vector>

#include "bulk_copy.cuh"
#include "device_util.cuh"
#include "emin_internal.cuh"

namespace emin {
namespace {

constexpr int NB = 3;      // dofs per node
constexpr int KB = 6;      // columns of P per aggregate (k)
constexpr int KK = KB * (KB + 1) / 2;
constexpr int kSlots = 8;  // aggregates per node (4-bit slot codes in a 32-bit map)
constexpr int kZero = 24;  // elements of the zero block at the start of the Y area
constexpr int kNbsWaitLimit = 1 << 22;  // bounded wait for a tile's copies
constexpr int kGRow = 22;               // staged Ginv: 21 values per row, padded
constexpr int kGStride = NB * kGRow;    // per node
constexpr int kBStride = KB * KB + 2;   // staged B_c table per aggregate

__device__ __forceinline__ int tri(int a, int b) { return a * (a + 1) / 2 + b; }

// Per-tile blob regions, in 16-byte units from the tile's start:
//   lanes   W*32 ints: node-in-tile | slot << 10 | aggregate-in-tile << 13, -1 padding
//   nodes   int4: {first pair | pairs << 20, p0, mrow | first lane << 8 | slots << 16,
//                  shared-memory offset of the node's own rows of Y}
//   plan    uint4 per pair: {offset0 | slots0 << 28, offset1 | slots1 << 28, map0, map1}
//   A       18 T per pair: A^(r, c) of both neighbours, [r*3 + c][h]
//   Ginv    66 T per node: the three rows' packed inverse Gram factors, 21 values
//           padded to 22 per row (rows start 8-byte aligned for paired loads)
//   Bc      38 T per aggregate of the tile: B_c rows 6 g .. 6 g + 5, padded
//           by 2 (an odd number of pairs per aggregate, so that the tables of
//           different aggregates start in different banks)
struct TileView {
    int npairs, nnodes, naggs;
    long long plan16, a16, g16, bc16;  // region starts
};

template <class T>
__host__ __device__ __forceinline__ TileView tile_view(int W, int npairs, int nnodes, int naggs) {
    TileView v;
    v.npairs = npairs;
    v.nnodes = nnodes;
    v.naggs = naggs;
    const long long lanes16 = (long long)W * 32 * 4 / 16;
    v.plan16 = lanes16 + nnodes;
    v.a16 = v.plan16 + npairs;
    v.g16 = v.a16 + ((long long)npairs * 18 * sizeof(T) + 15) / 16;
    v.bc16 = v.g16 + ((long long)nnodes * kGStride * sizeof(T) + 15) / 16;
    return v;
}

template <class T>
__host__ __device__ __forceinline__ long long tile_len16(int W, int npairs, int nnodes, int naggs) {
    const TileView v = tile_view<T>(W, npairs, nnodes, naggs);
    return v.bc16 + ((long long)naggs * kBStride * sizeof(T) + 15) / 16;
}

// a pair of T (8 or 16 bytes), the unit of the blob's paired values
template <class T>
struct PairOf;
template <>
struct PairOf<float> {
    using V = float2;
};
template <>
struct PairOf<double> {
    using V = double2;
};

// ---------------------------------------------------------------------------
// Values of the blob, refreshed at every set-up: A^ = D^-1/2 A D^-1/2 (dsq
// null: A itself) in pairs, Ginv and B_c in the working precision.
// fill_pair {v, j0, dst, has second}, fill_node {v, dst}, fill_agg {g, dst};
// dst in elements of T from the blob's start.
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(kBlock)
k_nbs_fill(long long npairs, const int4 *__restrict__ fp, long long nnodes,
           const int2 *__restrict__ fnode, long long naggs, const int2 *__restrict__ fagg,
           const int *__restrict__ Ap, const int *__restrict__ Aj, const double *__restrict__ Av,
           const double *__restrict__ dsq, const double *__restrict__ Ginv,
           const double *__restrict__ Bc, T *blob) {
    const long long total = npairs + nnodes + naggs;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        if (q < npairs) {
            // a node-blocked row stores neighbour j's 3 x 3 block at columns
            // NB j .. NB j + 2 of each of the node's rows, all in the column
            // node b: one read of Aj per neighbour, D^-1/2 of b's three dofs
            // shared by the three rows
            const int4 f = fp[q];
            const int v = f.x, j0 = f.y;
            const int a0 = Ap[NB * v], rs = Ap[NB * v + 1] - a0;
            using V = typename PairOf<T>::V;
            V *dst = reinterpret_cast<V *>(blob + (unsigned)f.z);
            double dv[NB], db[2][NB], a[2][NB][NB];
#pragma unroll
            for (int r = 0; r < NB; ++r) dv[r] = dsq ? dsq[NB * v + r] : 1.0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = j0 + h;
                const bool has = h == 0 || f.w;
                const int cb = has ? Aj[a0 + NB * j] : 0;  // first column of node b
#pragma unroll
                for (int c = 0; c < NB; ++c) db[h][c] = (has && dsq) ? dsq[cb + c] : 1.0;
#pragma unroll
                for (int r = 0; r < NB; ++r)
#pragma unroll
                    for (int c = 0; c < NB; ++c)
                        a[h][r][c] = has ? Av[a0 + r * rs + NB * j + c] : 0.0;
            }
#pragma unroll
            for (int r = 0; r < NB; ++r)
#pragma unroll
                for (int c = 0; c < NB; ++c) {
                    V u;
                    u.x = (T)(dv[r] * a[0][r][c] * db[0][c]);
                    u.y = (T)(dv[r] * a[1][r][c] * db[1][c]);
                    dst[r * NB + c] = u;
                }
        } else if (q < npairs + nnodes) {
            const int2 f = fnode[q - npairs];
            const double *g = Ginv + (size_t)NB * f.x * KK;
            T *dst = blob + (unsigned)f.y;
            for (int r = 0; r < NB; ++r)
                for (int e = 0; e < kGRow; ++e) dst[r * kGRow + e] = e < KK ? (T)g[r * KK + e] : T(0);
        } else {
            const int2 f = fagg[q - npairs - nnodes];
            const double *b = Bc + (size_t)KB * f.x * KB;
            T *dst = blob + (unsigned)f.y;
            for (int e = 0; e < kBStride; ++e) dst[e] = e < KB * KB ? (T)b[e] : T(0);
        }
    }
}

// six consecutive elements of a row of Y in shared memory (8-byte aligned
// for float, 16-byte aligned for double)
__device__ __forceinline__ void lds_row6(const float *p, float (&y)[KB]) {
    const float2 *q = reinterpret_cast<const float2 *>(p);
#pragma unroll
    for (int h = 0; h < 3; ++h) {
        const float2 u = q[h];
        y[2 * h] = u.x;
        y[2 * h + 1] = u.y;
    }
}
__device__ __forceinline__ void lds_row6(const double *p, double (&y)[KB]) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
    for (int h = 0; h < 3; ++h) {
        const double2 u = q[h];
        y[2 * h] = u.x;
        y[2 * h + 1] = u.y;
    }
}


// ---------------------------------------------------------------------------
// The staged product.  Dynamic shared memory: [blob cap][Y cap][scratch
// W*32*19 T]; one mbarrier counts the bytes of a tile's copies.
// ---------------------------------------------------------------------------
template <class T, int W, bool CK = false>
__global__ void __launch_bounds__(W * 32)
k_kprod_nbs(int ntiles, const int4 *__restrict__ thdr, const uint4 *__restrict__ blob,
            const int4 *__restrict__ runs, int stage_cap16, const T *__restrict__ Y,
            T *__restrict__ out, int project, int dot_mode, DevState *st, double *partials,
            double *hist, int cap, int check_stop, int *chk, long long ny, long long blob16,
            int gamma0) {
    // dot_mode DOT_START (the start of Algorithm 3): out = -Pi(A^ x), the
    // convergence floor from <x, x> before the projection and, with gamma0,
    // gamma_0 = <Pi x, Pi x> after it, reduced together
    using V = typename PairOf<T>::V;
    if (check_stop && st->stop) return;
    int bad = 0;
    // with checks: copies that would leave the blob, Y (16-byte rounded) or
    // the staging area are skipped and flagged
    const long long y16 = (ny * (long long)sizeof(T) + 15) / 16;
    auto run_ok = [&](const int4 &rn, int blen16) {
        return rn.x >= 0 && rn.y >= 0 && (long long)rn.x + rn.y <= y16 &&
               rn.z >= kZero * (int)sizeof(T) / 16 && (long long)blen16 + rn.z + rn.y <= stage_cap16;
    };
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int s_abort, s_skip;
    unsigned char *sBlob = smem;
    T(*sT)[NB * KB + 1] = reinterpret_cast<T(*)[NB * KB + 1]>(smem + (size_t)stage_cap16 * 16);
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        fence_proxy_async();
        s_abort = 0;
        s_skip = 0;
    }
    __syncthreads();
    Dot<T> dot, dot1;  // DOT_START: dot before the projection, dot1 after
    unsigned phase = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int4 h0 = thdr[2 * tile], h1 = thdr[2 * tile + 1];
        // h0 = {blob offset16, blob len16, first run, runs}; h1 = {pairs, nodes, aggs, Y len16};
        // the tile's rows of Y follow its blob, after a zero block
        T *sY = reinterpret_cast<T *>(smem + (size_t)h0.y * 16);
        for (int i = tid; i < kZero; i += W * 32) sY[i] = T(0);
        if (tid < 32) {
            // with checks, a tile whose header does not describe a blob inside
            // the blob array and the staging area is skipped whole
            bool tile_ok = true;
            if constexpr (CK)
                tile_ok = h0.x >= 0 && h0.y >= 0 && h1.x >= 0 && h1.y >= 0 && h1.z >= 0 &&
                          h1.w >= 0 && h0.z >= 0 && h0.w >= 0 &&
                          (long long)h0.x + h0.y <= blob16 &&
                          tile_len16<T>(W, h1.x, h1.y, h1.z) == h0.y && h1.y <= W * 32 &&
                          (long long)h0.y + kZero * (int)sizeof(T) / 16 + h1.w <= stage_cap16;
            if (tid == 0) {
                fence_proxy_async();  // earlier generic reads of this memory come first
                unsigned bytes = (unsigned)(h0.y + h1.w) * 16u;
                if constexpr (CK) {
                    bytes = 0u;
                    if (tile_ok) {
                        bytes = (unsigned)h0.y * 16u;
                        for (int r = 0; r < h0.w; ++r) {
                            const int4 rn = runs[h0.z + r];
                            if (run_ok(rn, h0.y)) bytes += (unsigned)rn.y * 16u;
                            else bad = 1;
                        }
                    } else {
                        bad = 1;
                        s_skip = 1;
                    }
                }
                mbar_expect_tx(&bar, bytes);
            }
            __syncwarp();
            if (tid == 0 && tile_ok) bulk_g2s(sBlob, blob + h0.x, (unsigned)h0.y * 16u, &bar);
            for (int r = tid; r < (tile_ok ? h0.w : 0); r += 32) {
                const int4 rn = runs[h0.z + r];  // {src16, len16, dst16}
                if (CK && !run_ok(rn, h0.y)) continue;
                bulk_g2s(reinterpret_cast<unsigned char *>(sY) + (size_t)rn.z * 16,
                         reinterpret_cast<const unsigned char *>(Y) + (size_t)rn.x * 16,
                         (unsigned)rn.y * 16u, &bar);
            }
        }
        if (tid == 0) {
            if (!mbar_wait_bounded(&bar, phase, kNbsWaitLimit)) {
                st->status = EMIN_ERR_TIMEOUT;
                st->stop = 2;
                mbar_wait_bounded(&bar, phase, kNbsWaitLimit);  // the copies in flight, bounded again
                s_abort = 1;
            }
        }
        phase ^= 1u;
        __syncthreads();
        if (s_abort) break;
        if (CK && s_skip) {
            __syncthreads();  // every thread has read the flag
            if (tid == 0) s_skip = 0;
            __syncthreads();
            continue;
        }

        const TileView tv = tile_view<T>(W, h1.x, h1.y, h1.z);
        const int *sLane = reinterpret_cast<const int *>(sBlob);
        const int4 *sNode = reinterpret_cast<const int4 *>(sBlob) + (size_t)W * 32 * 4 / 16;
        const uint4 *sPlan = reinterpret_cast<const uint4 *>(sBlob) + tv.plan16;
        const T *sA = reinterpret_cast<const T *>(reinterpret_cast<const uint4 *>(sBlob) + tv.a16);
        const T *sG = reinterpret_cast<const T *>(reinterpret_cast<const uint4 *>(sBlob) + tv.g16);
        const T *sB = reinterpret_cast<const T *>(reinterpret_cast<const uint4 *>(sBlob) + tv.bc16);

        const int rec = sLane[tid];
        const bool valid = rec >= 0;
        // (padding lanes, rec = -1, take no entries and index nothing)
        const int ni = valid ? chk_index<CK>(rec & 1023, h1.y, bad) : 0, s = (rec >> 10) & 7;
        const int ai = valid ? chk_index<CK>(rec >> 13, h1.z, bad) : 0;
        int4 nd = make_int4(0, 0, 0, 0);
        if (valid) nd = sNode[ni];
        int pair0 = nd.x & 0xFFFFF, ng = valid ? (nd.x >> 20) : 0;
        if (CK && (long long)pair0 + ng > h1.x) {
            bad = 1;
            pair0 = ng = 0;
        }
        const int p0 = nd.y, mrow = nd.z & 255, first = tid - s, nslot = (nd.z >> 16) & 255;
        // the Y area of this tile, in elements (a row segment reads KB of them)
        const long long ylim = ((long long)stage_cap16 - h0.y) * 16 / (long long)sizeof(T) - KB + 1;
        T acc[NB][KB];
#pragma unroll
        for (int r = 0; r < NB; ++r)
#pragma unroll
            for (int t = 0; t < KB; ++t) acc[r][t] = T(0);
#pragma unroll 2
        for (int g = 0; g < ng; ++g) {
            const uint4 pe = sPlan[pair0 + g];
            const V *ap = reinterpret_cast<const V *>(sA + (size_t)(pair0 + g) * 18);
            V a2[NB * NB];
#pragma unroll
            for (int e = 0; e < NB * NB; ++e) a2[e] = ap[e];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const unsigned bo = h ? pe.y : pe.x, bm = h ? pe.w : pe.z;
                const unsigned q = (bm >> (4 * s)) & 0xFu;
                const bool ok = q < (unsigned)kSlots;
                const int yl = ok ? KB * (int)(bo >> 28) : 0;
                const int yb = ok ? (int)(bo & 0x0FFFFFFFu) + KB * (int)q : 0;
                T y[NB][KB];
#pragma unroll
                for (int c = 0; c < NB; ++c) lds_row6(sY + chk_index<CK>(yb + c * yl, ylim, bad), y[c]);
#pragma unroll
                for (int r = 0; r < NB; ++r) {
                    const T a0 = h ? a2[r * NB].y : a2[r * NB].x;
                    const T a1 = h ? a2[r * NB + 1].y : a2[r * NB + 1].x;
                    const T a3 = h ? a2[r * NB + 2].y : a2[r * NB + 2].x;
#pragma unroll
                    for (int t = 0; t < KB; ++t)
                        acc[r][t] = fmat(a0, y[0][t], fmat(a1, y[1][t], fmat(a3, y[2][t], acc[r][t])));
                }
            }
        }
        if (dot_mode == DOT_START && valid) {
#pragma unroll
            for (int r = 0; r < NB; ++r)
#pragma unroll
                for (int t = 0; t < KB; ++t) dot.add(acc[r][t], acc[r][t]);
        }
        if (project) {
            // t_r = sum over the node's lanes of B_s^T x_r (B_s = B_c rows of
            // this lane's aggregate), c_r = G_i^-1 t_r, x_r -= B_s c_r
            T bq[KB * KB];  // B_s, loaded once as pairs
            if (valid) {
                const V *bp = reinterpret_cast<const V *>(sB + (size_t)ai * kBStride);
#pragma unroll
                for (int e = 0; e < KB * KB / 2; ++e) {
                    const V u = bp[e];
                    bq[2 * e] = u.x;
                    bq[2 * e + 1] = u.y;
                }
            } else {
#pragma unroll
                for (int e = 0; e < KB * KB; ++e) bq[e] = T(0);
            }
            T tr[NB][KB];
#pragma unroll
            for (int r = 0; r < NB; ++r)
#pragma unroll
                for (int a = 0; a < KB; ++a) {
                    T v2 = T(0);
#pragma unroll
                    for (int t = 0; t < KB; ++t) v2 = fmat(bq[t * KB + a], acc[r][t], v2);
                    tr[r][a] = v2;
                }
#pragma unroll
            for (int r = 0; r < NB; ++r)
#pragma unroll
                for (int a = 0; a < KB; ++a) sT[tid][r * KB + a] = tr[r][a];
            __syncwarp();
#pragma unroll
            for (int r = 0; r < NB; ++r)
#pragma unroll
                for (int a = 0; a < KB; ++a) tr[r][a] = T(0);
            if (valid) {
                for (int u = 0; u < nslot; ++u)
#pragma unroll
                    for (int r = 0; r < NB; ++r)
#pragma unroll
                        for (int a = 0; a < KB; ++a) tr[r][a] += sT[first + u][r * KB + a];
#pragma unroll
                for (int r = 0; r < NB; ++r) {
                    T g[kGRow];
                    const V *gp = reinterpret_cast<const V *>(sG + (size_t)ni * kGStride + r * kGRow);
#pragma unroll
                    for (int e = 0; e < kGRow / 2; ++e) {
                        const V u = gp[e];
                        g[2 * e] = u.x;
                        g[2 * e + 1] = u.y;
                    }
                    T cv[KB];
#pragma unroll
                    for (int a = 0; a < KB; ++a) {
                        T v2 = T(0);
#pragma unroll
                        for (int c = 0; c < KB; ++c)
                            v2 = fmat(g[a >= c ? tri(a, c) : tri(c, a)], tr[r][c], v2);
                        cv[a] = v2;
                    }
#pragma unroll
                    for (int a = 0; a < KB; ++a) tr[r][a] = cv[a];
                }
#pragma unroll
                for (int t = 0; t < KB; ++t)
#pragma unroll
                    for (int r = 0; r < NB; ++r) {
                        T x = acc[r][t];
#pragma unroll
                        for (int a = 0; a < KB; ++a) x = fmat(-bq[t * KB + a], tr[r][a], x);
                        acc[r][t] = x;
                    }
            }
        }
        if (valid) {
            const int own = nd.w;  // the node's own rows of Y in shared memory
#pragma unroll
            for (int r = 0; r < NB; ++r) {
                const int o = p0 + r * mrow + KB * s;
                V *op = reinterpret_cast<V *>(out + chk_index<CK>(o, ny - KB + 1, bad));
                const V *yo = reinterpret_cast<const V *>(
                    sY + chk_index<CK>(own + r * mrow + KB * s, ylim, bad));
#pragma unroll
                for (int h = 0; h < KB / 2; ++h) {
                    V u;
                    u.x = acc[r][2 * h];
                    u.y = acc[r][2 * h + 1];
                    if (dot_mode == DOT_START) {
                        dot1.add(u.x, u.x);
                        dot1.add(u.y, u.y);
                        u.x = -u.x;
                        u.y = -u.y;
                    } else if (dot_mode) {
                        const V yv = yo[h];
                        dot.add(yv.x, u.x);
                        dot.add(yv.y, u.y);
                    }
                    op[h] = u;
                }
            }
        }
        __syncthreads();  // the next tile's copies overwrite the blob and Y areas
    }
    chk_report<CK>(bad, chk);
    if (dot_mode == DOT_START) {
        __shared__ double sh[32];
        const double b0 = block_dot_total(dot, sh);
        __syncthreads();
        const double b1 = block_dot_total(dot1, sh);
        double s0, s1;
        if (grid_reduce2(b0, b1, partials, &st->ticket[0], &s0, &s1)) {
            finalize_gamma(st, s0, UPD_FLOOR, GammaFloor<T>::value);
            if (gamma0) finalize_gamma(st, s1, UPD_INIT, GammaFloor<T>::value);
        }
    } else if (dot_mode) {
        __shared__ double sh[32];
        double bt = block_dot_total(dot, sh);
        double total;
        if (grid_reduce(bt, partials, &st->ticket[0], &total)) {
            if (dot_mode == DOT_ALPHA) finalize_alpha(st, total, hist, cap);
            else st->aux = total;
        }
    }
}

}  // namespace

long long tile_len16_host(int esize, int W, int npairs, int nnodes, int naggs) {
    return esize == 4 ? tile_len16<float>(W, npairs, nnodes, naggs)
                      : tile_len16<double>(W, npairs, nnodes, naggs);
}

// ---------------------------------------------------------------------------
// Host plan: tiles of whole nodes grown breadth-first over the node graph,
// at most W warps of output blocks (whole nodes per warp) and at most
// `budget` bytes of blob plus staged rows of Y per tile.
// ---------------------------------------------------------------------------
int build_nbs_plan(int n, const int *Ap, const int *Aj, const int *Pp, const int *Pj, int esize,
                   int W, long long budget, NbsHost &h) {
    if (n % NB || n <= 0) return EMIN_ERR_ARG;
    const int nn = n / NB;
    h = NbsHost();
    h.W = W;
    h.esize = esize;
    std::vector<int> deg(nn), na(nn), agg(nn * (size_t)kSlots, -1);
    std::vector<long long> ybytes(nn);
    for (int v = 0; v < nn; ++v) {
        deg[v] = (Ap[NB * v + 1] - Ap[NB * v]) / NB;
        const int p0 = Pp[NB * v], m = Pp[NB * v + 1] - p0;
        na[v] = m / KB;
        if (na[v] > kSlots || na[v] < 1) return EMIN_ERR_ARG;
        for (int s = 0; s < na[v]; ++s) agg[(size_t)v * kSlots + s] = Pj[p0 + KB * s] / KB;
        ybytes[v] = (long long)NB * m * esize;
        if ((long long)Pp[NB * v] >= (1LL << 28)) return EMIN_ERR_ARG;  // offsets in 28 bits
    }
    auto nbr = [&](int v, int j) { return Aj[Ap[NB * v] + NB * j] / NB; };
    const int nagg_total = [&] {
        int m = 0;
        for (int v = 0; v < nn; ++v)
            for (int s = 0; s < na[v]; ++s) m = std::max(m, agg[(size_t)v * kSlots + s] + 1);
        return m;
    }();
    std::vector<int> assigned(nn, 0), inq(nn, -1), inU(nn, -1), aggStamp(nagg_total, -1);
    std::deque<int> Q;
    const int zero16 = kZero * esize / 16;
    int tile = 0;
    long long blob16 = 0;
    for (int seed = 0; seed < nn; ++seed) {
        if (assigned[seed]) continue;
        std::vector<int> members, warp_of, U, aggs;
        int cur_warp = 0, cur_fill = 0, npairs = 0;
        long long ybyt = (long long)kZero * esize;
        Q.clear();
        Q.push_back(seed);
        inq[seed] = tile;
        while (!Q.empty()) {
            const int v = Q.front();
            Q.pop_front();
            if (assigned[v]) continue;
            int w = cur_warp, f = cur_fill;
            if (f + na[v] > 32) {
                ++w;
                f = 0;
            }
            if (w >= W) break;
            // bytes the node adds: its rows of Y it brings into the union, its
            // blob records and values, new aggregates
            long long addY = 0;
            for (int j = 0; j < deg[v]; ++j) {
                const int b = nbr(v, j);
                if (inU[b] != tile) addY += ybytes[b] + 16;
            }
            int newagg = 0;
            for (int s = 0; s < na[v]; ++s)
                if (aggStamp[agg[(size_t)v * kSlots + s]] != tile) ++newagg;
            const int ng = (deg[v] + 1) / 2;
            const long long blob_bytes =
                16 * (tile_len16_host(esize, W, npairs + ng, (int)members.size() + 1,
                                      (int)aggs.size() + newagg) + 4);
            if (!members.empty() && blob_bytes + ybyt + addY > budget) break;
            // admit v
            assigned[v] = 1;
            members.push_back(v);
            warp_of.push_back(w);
            cur_warp = w;
            cur_fill = f + na[v];
            npairs += ng;
            ybyt += addY;
            for (int j = 0; j < deg[v]; ++j) {
                const int b = nbr(v, j);
                if (inU[b] != tile) {
                    inU[b] = tile;
                    U.push_back(b);
                }
                if (!assigned[b] && inq[b] != tile) {
                    inq[b] = tile;
                    Q.push_back(b);
                }
            }
            for (int s = 0; s < na[v]; ++s) {
                const int g = agg[(size_t)v * kSlots + s];
                if (aggStamp[g] != tile) {
                    aggStamp[g] = tile;
                    aggs.push_back(g);
                }
            }
        }
        if (members.empty()) return EMIN_ERR_ARG;
        // a node of a tile must appear in its own neighbour list (A has the
        // diagonal block), so that its rows of Y are staged for the dot
        for (int v : members)
            if (inU[v] != tile) return EMIN_ERR_ARG;
        // runs of consecutive nodes of the union
        std::sort(U.begin(), U.end());
        std::vector<long long> sboff(U.size());
        const int first_run = (int)h.runs.size();
        long long dst16 = zero16;
        for (size_t i = 0; i < U.size();) {
            size_t k = i;
            while (k + 1 < U.size() && U[k + 1] == U[k] + 1) ++k;
            const long long b0 = Pp[NB * U[i]], b1 = Pp[NB * U[k] + NB];
            const long long src16 = b0 * esize / 16, end16 = (b1 * esize + 15) / 16;
            for (size_t m = i; m <= k; ++m)
                sboff[m] = dst16 * (16 / esize) + (Pp[NB * U[m]] - src16 * (16 / esize));
            h.runs.push_back(int4{(int)src16, (int)(end16 - src16), (int)dst16, 0});
            dst16 += end16 - src16;
            i = k + 1;
        }
        auto off_of = [&](int b) -> long long {
            const size_t i = std::lower_bound(U.begin(), U.end(), b) - U.begin();
            return sboff[i];
        };
        const int nnodes = (int)members.size(), naggs = (int)aggs.size();
        const long long len16 = tile_len16_host(esize, W, npairs, nnodes, naggs);
        // static blob records (values are zero until the fill kernel runs)
        const size_t base = h.blob.size();
        h.blob.resize(base + (size_t)len16, uint4{0, 0, 0, 0});
        int *lanes = reinterpret_cast<int *>(&h.blob[base]);
        for (int l = 0; l < W * 32; ++l) lanes[l] = -1;
        int4 *nodes = reinterpret_cast<int4 *>(&h.blob[base]) + (size_t)W * 32 * 4 / 16;
        const long long plan16 = (long long)W * 32 * 4 / 16 + nnodes;
        const long long a16 = plan16 + npairs;
        const long long g16 = a16 + ((long long)npairs * 18 * esize + 15) / 16;
        const long long bc16 = g16 + ((long long)nnodes * kGStride * esize + 15) / 16;
        uint4 *plan = &h.blob[base + (size_t)plan16];
        std::vector<int> wfill(W, 0);
        int pair = 0;
        const long long blob_elem0 = (blob16 * 16) / esize;
        for (int m = 0; m < nnodes; ++m) {
            const int v = members[m], w = warp_of[m];
            const int fl = w * 32 + wfill[w];
            wfill[w] += na[v];
            const int ng = (deg[v] + 1) / 2;
            for (int s = 0; s < na[v]; ++s) {
                const int g = agg[(size_t)v * kSlots + s];
                const int ai = (int)(std::find(aggs.begin(), aggs.end(), g) - aggs.begin());
                lanes[fl + s] = m | (s << 10) | (ai << 13);
            }
            nodes[m] = int4{pair | (ng << 20), Pp[NB * v], (Pp[NB * v + 1] - Pp[NB * v]) | (fl << 8) | (na[v] << 16),
                            (int)off_of(v)};
            for (int p = 0; p < ng; ++p) {
                unsigned wd[2] = {0u, 0u}, mp[2] = {0xFFFFFFFFu, 0xFFFFFFFFu};
                for (int hh = 0; hh < 2; ++hh) {
                    const int j = 2 * p + hh;
                    if (j >= deg[v]) continue;
                    const int b = nbr(v, j);
                    wd[hh] = (unsigned)off_of(b) | ((unsigned)na[b] << 28);
                    unsigned map = 0xFFFFFFFFu;
                    for (int s = 0; s < na[v]; ++s) {
                        const int g = agg[(size_t)v * kSlots + s];
                        for (int q = 0; q < na[b]; ++q)
                            if (agg[(size_t)b * kSlots + q] == g)
                                map = (map & ~(0xFu << (4 * s))) | ((unsigned)q << (4 * s));
                    }
                    mp[hh] = map;
                }
                plan[pair + p] = uint4{wd[0], wd[1], mp[0], mp[1]};
                h.fill_pair.push_back(int4{v, 2 * p,
                                           (int)(blob_elem0 + (a16 * 16 + (long long)(pair + p) * 18 * esize) / esize),
                                           2 * p + 1 < deg[v] ? 1 : 0});
            }
            h.fill_node.push_back(int2{v, (int)(blob_elem0 + (g16 * 16 + (long long)m * kGStride * esize) / esize)});
            pair += ng;
        }
        for (int a = 0; a < naggs; ++a)
            h.fill_agg.push_back(int2{aggs[a], (int)(blob_elem0 + (bc16 * 16 + (long long)a * kBStride * esize) / esize)});
        h.hdr.push_back(int4{(int)blob16, (int)len16, first_run, (int)h.runs.size() - first_run});
        h.hdr.push_back(int4{npairs, nnodes, naggs, (int)(dst16 - zero16)});
        h.stage_cap16 = std::max(h.stage_cap16, (int)(len16 + dst16));
        blob16 += len16;
        if (blob16 * 16 / esize >= (1LL << 31)) return EMIN_ERR_ARG;
        ++tile;
    }
    h.ntiles = tile;
    return EMIN_OK;
}

template <class T>
void launch_nbs_fill(const Launch &L, const NbsOps &nb, const int *Ap, const int *Aj,
                     const double *Av, const double *dsq, const double *Ginv, const double *Bc,
                     T *blob) {
    const long long total = nb.nfill_pair + nb.nfill_node + nb.nfill_agg;
    if (total <= 0) return;
    long long g = (total + kBlock - 1) / kBlock;
    if (g > L.grid_rows) g = L.grid_rows;
    k_nbs_fill<T><<<(int)g, kBlock, 0, L.stream>>>(nb.nfill_pair, nb.fill_pair, nb.nfill_node,
                                                   nb.fill_node, nb.nfill_agg, nb.fill_agg, Ap, Aj,
                                                   Av, dsq, Ginv, Bc, blob);
    note_launch();
}

template <class T>
size_t nbs_smem_bytes(const NbsOps &nb) {
    return (size_t)nb.stage_cap16 * 16 + (size_t)nb.W * 32 * (NB * KB + 1) * sizeof(T);
}

template <class T, int W>
static int nbs_blocks_per_sm(size_t smem) {
    if (cudaFuncSetAttribute(k_kprod_nbs<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_kprod_nbs<T, W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_kprod_nbs<T, W>, W * 32, smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

// resident CTAs per SM of the staged product for this plan (0: it cannot
// launch, e.g. too much shared memory); also sets the kernel's shared-memory
// attribute, so call it at create, outside any graph capture
template <class T>
int nbs_prepare(const NbsOps &nb) {
    const size_t smem = nbs_smem_bytes<T>(nb);
    switch (nb.W) {
        case 2: return nbs_blocks_per_sm<T, 2>(smem);
        case 3: return nbs_blocks_per_sm<T, 3>(smem);
        case 4: return nbs_blocks_per_sm<T, 4>(smem);
        case 8: return nbs_blocks_per_sm<T, 8>(smem);
        default: return 0;
    }
}

template <class T>
void launch_kprod_nbs(const Launch &L, const NbsOps &nb, const T *blob, const T *Y, T *out,
                      int project, int dot_mode, Work<T> &w, int check_stop, int *chk,
                      long long ny, int gamma0) {
    const size_t smem = nbs_smem_bytes<T>(nb);
    long long g = (long long)L.nsm * (nb.per_sm > 0 ? nb.per_sm : 1);
    if (g > nb.ntiles) g = nb.ntiles;
    if (g > kMaxGrid / 2) g = kMaxGrid / 2;  // DOT_START reduces two partial sums per block
    if (g < 1) g = 1;
    const uint4 *bl = reinterpret_cast<const uint4 *>(blob);
    switch (nb.W) {
#define EMIN_NBS(WV)                                                                          \
    case WV:                                                                                  \
        if (chk)                                                                              \
            k_kprod_nbs<T, WV, true><<<(int)g, WV * 32, smem, L.stream>>>(                    \
                nb.ntiles, nb.hdr, bl, nb.runs, nb.stage_cap16, Y, out, project, dot_mode,   \
                w.st, w.partials, w.hist, w.hist_cap, check_stop, chk, ny, nb.blob16, gamma0);\
        else                                                                                  \
            k_kprod_nbs<T, WV><<<(int)g, WV * 32, smem, L.stream>>>(                          \
                nb.ntiles, nb.hdr, bl, nb.runs, nb.stage_cap16, Y, out, project, dot_mode,   \
                w.st, w.partials, w.hist, w.hist_cap, check_stop, nullptr, ny, nb.blob16,     \
                gamma0);                                                                      \
        break;
        EMIN_NBS(2)
        EMIN_NBS(3)
        EMIN_NBS(4)
        EMIN_NBS(8)
#undef EMIN_NBS
        default: return;
    }
    note_launch();
}

template void launch_nbs_fill<float>(const Launch &, const NbsOps &, const int *, const int *,
                                     const double *, const double *, const double *,
                                     const double *, float *);
template void launch_nbs_fill<double>(const Launch &, const NbsOps &, const int *, const int *,
                                      const double *, const double *, const double *,
                                      const double *, double *);
template int nbs_prepare<float>(const NbsOps &);
template int nbs_prepare<double>(const NbsOps &);
template void launch_kprod_nbs<float>(const Launch &, const NbsOps &, const float *,
                                      const float *, float *, int, int, Work<float> &, int, int *,
                                      long long, int);
template void launch_kprod_nbs<double>(const Launch &, const NbsOps &, const double *,
                                       const double *, double *, int, int, Work<double> &, int,
                                       int *, long long, int);

}  // namespace emin
