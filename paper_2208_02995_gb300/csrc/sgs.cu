// Projected block symmetric Gauss-Seidel preconditioner (M_2 of Section 3.4).
//
// K is block diagonal by columns of P: the block of column j is the
// principal submatrix A(I_j, I_j), I_j the rows of P that hold column j, and
// in the row-wise order of p its rows come in increasing row index.  The
// preconditioner applies M_SGS^{-1} = (L + D)^{-T} D (L + D)^{-1} block by
// block and then Pi_B.  The iteration runs in the symmetrically scaled
// variables (A^ = D^{-1/2} A D^{-1/2}, unit diagonal), where the same
// preconditioner is (L^ + I)^{-T} (L^ + I)^{-1}: a forward and a backward
// unit-diagonal triangular sweep per block.
//
// Plan (built once per context on the host): columns with identical row
// sets (the k columns of one aggregate in a node-blocked problem) form one
// group and share one block.  One-column groups of identical structure (the
// interior aggregates of a structured grid) form classes and are swept in
// batches of 32, one lane per group, by a CTA whose warps share the rows of
// each dependency level (the batched path); the other groups are swept one
// per warp, level by level (the level path).
//
// The batched path stores one value per coupling of L^, in forward order;
// the backward sweep reads the same values transposed, which is the L^T of
// (L^ + I)^{-T}.  It also forms gamma = r~^T M^{-1} r~ = |(L^ + I)^{-1} r~|^2
// after the forward sweep: r~ is kept in the range of Pi (every update of
// it is projected), so <r~, Pi M^{-1} r~> = <r~, M^{-1} r~>, and the
// projection of z~ is applied in the next direction update instead of a
// pass of its own.
#include <cuda_runtime.h>

#include <algorithm>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bulk_copy.cuh"
#include "device_util.cuh"
#include "convert.cuh"
#include "emin_internal.cuh"

namespace emin {
namespace {

constexpr int kSgsMaxCols = 8;        // columns per group
constexpr int kSgsMaxRows = 65535;    // rows per group (16-bit local indices)
constexpr int kBatchRows = 1024;      // rows of a batched group (10-bit local rows)
constexpr int kBatchRowCpl = 63;      // couplings of one row in one sweep (6-bit counts)
constexpr int kBatchMin = 8;          // groups of one structure before it is batched
constexpr int kBatchTail = 1024;      // rarer structures batched too while this few groups have them
constexpr long long kBatchSmem = 100 * 1024;  // float bytes of one batch (u, values, structure)
constexpr int kSgsWaitLimit = 1 << 22;        // bounded wait for a batch's copies
constexpr int kGatherRows = 16;               // rows per warp whose loads are issued together

inline int grid_for(long long work, int cap) {
    long long g = (work + kBlock - 1) / kBlock;
    if (g < 1) g = 1;
    return (int)(g < cap ? g : cap);
}

// A^ at the plan's couplings: val[o] = d_i a_il d_l for the entry e = aent[o]
// of row i = own[o] (A symmetric, so a_il = a_li serves both sweeps).
template <class T>
__global__ void k_sgs_values(long long nops, const int *__restrict__ own,
                             const int *__restrict__ aent, const int *__restrict__ Aj,
                             const double *__restrict__ Av, const double *__restrict__ dsq,
                             T *__restrict__ val) {
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < nops;
         o += (long long)gridDim.x * blockDim.x) {
        if (own[o] < 0) {  // an empty lane of a batch
            val[o] = T(0);
            continue;
        }
        const int e = aent[o];
        const double di = dsq[own[o]], a = Av[e], dl = dsq[Aj[e]];
        if constexpr (sizeof(T) == 4)  // narrowing on the integer pipe (convert.cuh)
            val[o] = f64_to_f32_rn(di) * f64_to_f32_rn(a) * f64_to_f32_rn(dl);
        else
            val[o] = di * a * dl;
    }
}

// With the packed k = 1 plan (SELL-32 order of A), A^ is already formed in
// plan order at every set-up; the batched couplings then read it there.
// Their A entries become plan positions once per context: entry e of row i
// sits at the slice start + 32 (e - Ap[i]) + i mod 32.  Lanes without a
// group (own < 0) are left as they are.
__global__ void k_sgs_sell_pos(long long nops, const int *__restrict__ own, int *ent,
                               const int *__restrict__ Ap, const int *__restrict__ sell_ptr) {
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < nops;
         o += (long long)gridDim.x * blockDim.x) {
        const int i = own[o];
        if (i < 0) continue;
        ent[o] = sell_ptr[i >> 5] + 32 * (ent[o] - Ap[i]) + (i & 31);
    }
}

// A^ at the batched couplings from A^ in plan order: the value half of a
// packed record (float, spk) or the plain array (sa); 0 on empty lanes
template <class T>
__global__ void k_sgs_values_sell(long long nops, const int *__restrict__ own,
                                  const int *__restrict__ pos, const T *__restrict__ sa,
                                  const uint2 *__restrict__ spk, T *__restrict__ val) {
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < nops;
         o += (long long)gridDim.x * blockDim.x) {
        T v = T(0);
        if (own[o] >= 0) {
            if constexpr (sizeof(T) == 4)
                v = spk ? __uint_as_float(spk[pos[o]].x) : sa[pos[o]];
            else
                v = sa[pos[o]];
        }
        val[o] = v;
    }
}

// Group header (12 ints): rows m, columns G, first plan row r0, index blob
// offset and length (16-byte units), first forward / backward value,
// forward / backward couplings nf / nb, forward / backward levels.
constexpr int kHdr = 12;

// The index blob of a group (uint16): flvl[nlf+1] frow[m] foptr[m+1]
// blvl[nlb+1] brow[m] boptr[m+1] fidx[nf] bidx[nb], padded to 16 bytes.
// Level bounds and coupling pointers are relative to the group.
struct SgsView {
    const unsigned short *flvl, *frow, *foptr, *fidx, *blvl, *brow, *boptr, *bidx;
};
__device__ __forceinline__ SgsView sgs_view(const unsigned short *b, int m, int nlf, int nlb,
                                            int nf) {
    SgsView v;
    v.flvl = b;
    v.frow = v.flvl + nlf + 1;
    v.foptr = v.frow + m;
    v.blvl = v.foptr + m + 1;
    v.brow = v.blvl + nlb + 1;
    v.boptr = v.brow + m;
    v.fidx = v.boptr + m + 1;
    v.bidx = v.fidx + nf;
    return v;
}

// One level-ordered unit-diagonal triangular sweep of a group held in u
// (row t, column c at u[t * G + c]) by the LPG lanes of a lane group: for
// the rows of each level, u_t -= sum over the row's couplings (t', v) v u_t'.
template <class T, int GM, int LPG, bool CK>
__device__ __forceinline__ void sgs_sweep_levels(T *u, int G, int nl, const unsigned short *lvl,
                                                 const unsigned short *row,
                                                 const unsigned short *optr,
                                                 const unsigned short *idx, const T *val,
                                                 int sub, unsigned mask, int m, int &bad) {
    for (int lv = 0; lv < nl; ++lv) {
        const int a = lvl[lv], b = lvl[lv + 1];
        for (int x = a + sub; x < b; x += LPG) {
            const int t = chk_index<CK>(row[x], m, bad);
            T acc[GM];
#pragma unroll
            for (int c = 0; c < GM; ++c) acc[c] = (c < G) ? u[t * G + c] : T(0);
            const int o1 = optr[x + 1];
            for (int o = optr[x]; o < o1; ++o) {
                const int tl = chk_index<CK>(idx[o], m, bad);
                const T v = val[o];
#pragma unroll
                for (int c = 0; c < GM; ++c)
                    if (c < G) acc[c] = fmat(-v, u[tl * G + c], acc[c]);
            }
#pragma unroll
            for (int c = 0; c < GM; ++c)
                if (c < G) u[t * G + c] = acc[c];
        }
        __syncwarp(mask);  // the next level reads this level's rows
    }
}

// z~ = (L^ + I)^{-T} (L^ + I)^{-1} r~ over the groups, LPG lanes per group
// (32 / LPG groups per warp at a time, grid-stride).  Each lane group owns
// `slot` bytes of shared memory: u (m * G values) and, for a group whose u,
// index blob and coupling values fit the slot, the blob and the values,
// copied in with coalesced loads so that the sweeps touch shared memory
// only; a larger group's blob and values are read from global memory.
template <class T, int GM, int LPG, bool CK = false>
__global__ void k_sgs_sweep(int ngroups, const int *__restrict__ hdr, const int *__restrict__ rpos,
                            const uint4 *__restrict__ blob, const T *__restrict__ fval,
                            const T *__restrict__ bval, const T *__restrict__ R,
                            T *__restrict__ Z, const DevState *st, int slot, int *chk,
                            long long ny) {
    if (st->stop) return;
    int bad = 0;
    extern __shared__ __align__(16) unsigned char sgs_smem[];
    constexpr int GPW = 32 / LPG;  // lane groups per warp
    const int lane = threadIdx.x & 31, sub = lane % LPG, half = lane / LPG;
    const unsigned mask = (LPG == 32) ? 0xffffffffu : (((1u << LPG) - 1u) << (half * LPG));
    unsigned char *mine = sgs_smem + (size_t)((threadIdx.x >> 5) * GPW + half) * slot;
    const int ntask = (gridDim.x * blockDim.x) / LPG;
    for (int g = (blockIdx.x * blockDim.x + threadIdx.x) / LPG; g < ngroups; g += ntask) {
        const int *h = hdr + (size_t)kHdr * g;
        const int m = h[0], G = h[1], r0 = h[2], boff = h[3], blen = h[4];
        const int fo0 = h[5], bo0 = h[6], nf = h[7], nb = h[8], nlf = h[9], nlb = h[10];
        T *u = reinterpret_cast<T *>(mine);
        const unsigned short *ib;
        const T *fv, *bv;
        const int ubytes = ((m * G * (int)sizeof(T)) + 15) & ~15;
        if (ubytes + 16 * blen + (nf + nb) * (int)sizeof(T) <= slot) {
            // u, then the blob (16-byte aligned), then the values
            uint4 *sb = reinterpret_cast<uint4 *>(mine + ubytes);
            for (int q = sub; q < blen; q += LPG) sb[q] = blob[boff + q];
            T *sv = reinterpret_cast<T *>(mine + ubytes + 16 * blen);
            for (int o = sub; o < nf; o += LPG) sv[o] = fval[fo0 + o];
            for (int o = sub; o < nb; o += LPG) sv[nf + o] = bval[bo0 + o];
            ib = reinterpret_cast<const unsigned short *>(sb);
            fv = sv;
            bv = sv + nf;
        } else {
            ib = reinterpret_cast<const unsigned short *>(blob + boff);
            fv = fval + fo0;
            bv = bval + bo0;
        }
        // the block's entries of r~: row t, column c at rpos[r0 + t] + c
        for (int x = sub; x < m * G; x += LPG) {
            const int t = x / G, c = x - t * G;
            u[x] = R[chk_index<CK>(rpos[r0 + t] + c, ny, bad)];
        }
        __syncwarp(mask);
        const SgsView v = sgs_view(ib, m, nlf, nlb, nf);
        sgs_sweep_levels<T, GM, LPG, CK>(u, G, nlf, v.flvl, v.frow, v.foptr, v.fidx, fv, sub,
                                         mask, m, bad);
        sgs_sweep_levels<T, GM, LPG, CK>(u, G, nlb, v.blvl, v.brow, v.boptr, v.bidx, bv, sub,
                                         mask, m, bad);
        for (int x = sub; x < m * G; x += LPG) {
            const int t = x / G, c = x - t * G;
            Z[chk_index<CK>(rpos[r0 + t] + c, ny, bad)] = u[x];
        }
        __syncwarp(mask);  // the slot is refilled by the next group
    }
    chk_report<CK>(bad, chk);
}

// 4-byte (float) or 8-byte (double) asynchronous copy global -> shared,
// completed by cp_async_wait_all in the issuing thread
template <class T>
__device__ __forceinline__ void cp_async4(T *dst, const T *src) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "cp.async of 4 or 8 bytes");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_addr(dst)), "l"(src),
                 "n"((int)sizeof(T))
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

__host__ __device__ __forceinline__ int pad4(int x) { return (x + 3) & ~3; }

// The C coupling terms of one row: acc - sum_k v_k u_(src_k), with the
// coupling words (local row | value index << 16) already in registers; ul
// and svl are u and the values offset by the lane.
template <class T, int C, bool CK>
__device__ __forceinline__ T row_terms(const unsigned (&w)[C], const T *ul, const T *svl, T acc,
                                       int m, int nv, int &bad) {
    T va[C], ua[C];
#pragma unroll
    for (int k = 0; k < C; ++k) {
        va[k] = svl[32 * chk_index<CK>((int)(w[k] >> 16), nv, bad)];
        ua[k] = ul[32 * chk_index<CK>((int)(w[k] & 0xffffu), m, bad)];
    }
#pragma unroll
    for (int k = 0; k < C; ++k) acc = fmat(-va[k], ua[k], acc);
    return acc;
}

// One level-ordered unit-diagonal triangular sweep of a batch held in u
// (row t of lane L at u[32 t + L], conflict-free) with the coupling values
// in sv (coupling o of lane L at sv[32 o + L]) and the class's sweep
// structure in shared memory.  The rows of a level are spread over the
// CTA's warps; a row's record is one 16-byte word, the same for every lane
// (a broadcast load): t | count << 10 | first coupling << 16, then its first
// three couplings (local row | value index << 16); a row with more reads the
// rest from the spill words, from the record's first-coupling index on.  Rows without couplings are not listed.  One CTA
// barrier per level.
template <class T, int NW, bool CK>
__device__ __forceinline__ void batch_sweep(T *u, const T *sv, int nl, const unsigned *lvl,
                                            const uint4 *rec, const unsigned *cpl, int nr,
                                            int nspill, int m, int nv, int warp, int lane,
                                            int &bad) {
    T *ul = u + lane;
    const T *svl = sv + lane;
    for (int l = 0; l < nl; ++l) {
        int a = (int)lvl[l], e = (int)lvl[l + 1];
        if (CK && (a < 0 || e > nr || a > e)) {
            bad = 1;
            a = e = 0;
        }
        for (int x = a + warp; x < e; x += NW) {
            const uint4 r = rec[x];
            const int cnt = (int)((r.x >> 10) & 63u), c0 = (int)(r.x >> 16);
            if (CK && cnt > 3 && c0 + cnt - 3 > nspill) {
                bad = 1;
                continue;
            }
            const int t = chk_index<CK>((int)(r.x & 1023u), m, bad);
            T acc = ul[32 * t];
            switch (cnt) {  // warp-uniform: exact unrolled paths for short rows
                case 1: {
                    const unsigned w[1] = {r.y};
                    acc = row_terms<T, 1, CK>(w, ul, svl, acc, m, nv, bad);
                    break;
                }
                case 2: {
                    const unsigned w[2] = {r.y, r.z};
                    acc = row_terms<T, 2, CK>(w, ul, svl, acc, m, nv, bad);
                    break;
                }
                default: {
                    const unsigned w[3] = {r.y, r.z, r.w};
                    acc = row_terms<T, 3, CK>(w, ul, svl, acc, m, nv, bad);
                    for (int k = 3; k < cnt; ++k) {
                        const unsigned wk[1] = {cpl[c0 + k - 3]};
                        acc = row_terms<T, 1, CK>(wk, ul, svl, acc, m, nv, bad);
                    }
                }
            }
            ul[32 * t] = acc;
        }
        __syncthreads();  // the next level reads this level's rows
    }
}

// gamma modes of the batched sweep: none; this launch's block totals only
// (an earlier bucket); block totals, then the grid total and the scalar step
enum { SG_NONE = 0, SG_PART = 1, SG_LAST = 2 };

// The batched sweep: one CTA per batch of 32 structurally identical
// one-column groups (grid-stride over the bucket's batches).  Thread 0 posts
// the batch's values (32 nv of them, contiguous) and, when the class
// changes, the class's sweep structure on an mbarrier and brings both into
// shared memory with TMA bulk copies while the warps gather r~ into u; then
// the forward sweep, |u|^2 into gamma (SG_*), the backward sweep, and the
// scatter of z~.  A lane without a group has positions -1, values 0 and
// stays 0.
template <class T, int NW, bool CK>
__global__ void __launch_bounds__(NW * 32)
k_sgs_batch(int b0, int b1, const int *__restrict__ bat_hdr, const int *__restrict__ cls_hdr,
            const unsigned *__restrict__ cls_blob, const int *__restrict__ rpos,
            const T *__restrict__ vals, const T *__restrict__ R, T *__restrict__ Z, DevState *st,
            double *partials, int pbase, int gmode, int init, int umax, int vmax, int wmax,
            int *chk, long long ny, long long nrpos, long long nval, long long nblob) {
    if (st->stop) return;
    int bad = 0;
    extern __shared__ __align__(16) unsigned char sgs_smem[];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int s_abort;
    __shared__ double sh[32];
    T *u = reinterpret_cast<T *>(sgs_smem);
    T *sv = u + 32 * (size_t)umax;
    unsigned *sb = reinterpret_cast<unsigned *>(sv + 32 * (size_t)vmax);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int cur_cls = -1;
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    double g = 0.0;
    unsigned phase = 0;
    for (int b = b0 + blockIdx.x; b < b1; b += gridDim.x) {
        const int *h = bat_hdr + 4 * (size_t)b;
        const int c = h[0], r0 = h[1], v0 = h[2];
        const int *ch = cls_hdr + 8 * (size_t)c;
        const int m = ch[0], nv = ch[1], nlf = ch[2] & 0xffff, nlb = ch[2] >> 16,
                  nsf = ch[3] & 0xffff, nsb = ch[3] >> 16, off = ch[4], nrf = ch[5], nrb = ch[6],
                  wpad = ch[7];
        if constexpr (CK) {
            // a batch whose header or class does not fit the arrays and the
            // shared memory is skipped whole (the same test in every thread)
            const long long words = pad4(nlf + 1) + 4LL * nrf + pad4(nsf) + pad4(nlb + 1) +
                                    4LL * nrb + pad4(nsb);
            if (m < 0 || nv < 0 || nlf < 0 || nlb < 0 || nrf < 0 || nrb < 0 || off < 0 ||
                (off & 3) || wpad < words || (wpad & 3) || wpad > wmax || r0 < 0 || v0 < 0 ||
                m > umax || nv > vmax || off + wpad > nblob ||
                (long long)r0 + 32LL * m > nrpos || (long long)v0 + 32LL * nv > nval) {
                bad = 1;
                continue;
            }
        }
        // the class's sweep structure is copied only when it changes
        const bool new_cls = c != cur_cls;
        cur_cls = c;
        if (tid == 0) {
            fence_proxy_async();  // the previous batch's reads of sv and sb come first
            const unsigned vbytes = 32u * (unsigned)nv * (unsigned)sizeof(T);
            const unsigned wbytes = new_cls ? 4u * (unsigned)wpad : 0u;
            mbar_expect_tx(&bar, vbytes + wbytes);
            if (vbytes) bulk_g2s(sv, vals + v0, vbytes, &bar);
            if (wbytes) bulk_g2s(sb, cls_blob + off, wbytes, &bar);
        }
        // the gather of r~: each warp's rows in groups of kGatherRows, all
        // their position loads in flight at once, then asynchronous copies
        // of r~ straight into u (no register round trip, all in flight)
        for (int t0 = warp; t0 < m; t0 += kGatherRows * NW) {
            int p[kGatherRows];
#pragma unroll
            for (int k = 0; k < kGatherRows; ++k) {
                const int t = t0 + k * NW;
                p[k] = t < m ? rpos[r0 + 32 * t + lane] : -2;
            }
#pragma unroll
            for (int k = 0; k < kGatherRows; ++k) {
                T *dst = u + 32 * (t0 + k * NW) + lane;
                if (p[k] >= 0)
                    cp_async4(dst, R + chk_index<CK>(p[k], ny, bad));
                else if (p[k] == -1)
                    *dst = T(0);  // a lane without a group
            }
        }
        cp_async_wait_all();
        if (tid == 0 && !mbar_wait_bounded(&bar, phase, kSgsWaitLimit)) {
            st->status = EMIN_ERR_TIMEOUT;
            st->stop = 2;
            mbar_wait_bounded(&bar, phase, kSgsWaitLimit);  // the copies in flight, bounded again
            s_abort = 1;
        }
        phase ^= 1u;
        __syncthreads();
        if (s_abort) break;
        const unsigned *fl = sb;
        const uint4 *fr = reinterpret_cast<const uint4 *>(fl + pad4(nlf + 1));
        const unsigned *fc = reinterpret_cast<const unsigned *>(fr + nrf);
        const unsigned *bl = fc + pad4(nsf);
        const uint4 *br = reinterpret_cast<const uint4 *>(bl + pad4(nlb + 1));
        const unsigned *bc = reinterpret_cast<const unsigned *>(br + nrb);
        batch_sweep<T, NW, CK>(u, sv, nlf, fl, fr, fc, nrf, nsf, m, nv, warp, lane, bad);
        if (gmode != SG_NONE) {
            // a thread's squares of one batch in T (a few dozen terms; the
            // FP64 pipe is slow), then one double addition per batch
            T gb = T(0);
            for (int t = warp; t < m; t += NW) gb = fmat(u[32 * t + lane], u[32 * t + lane], gb);
            g += (double)gb;
            __syncthreads();  // every warp has read u before the backward sweep rewrites it
        }
        batch_sweep<T, NW, CK>(u, sv, nlb, bl, br, bc, nrb, nsb, m, nv, warp, lane, bad);
        for (int t0 = warp; t0 < m; t0 += kGatherRows * NW) {
            int p[kGatherRows];
#pragma unroll
            for (int k = 0; k < kGatherRows; ++k) {
                const int t = t0 + k * NW;
                p[k] = t < m ? rpos[r0 + 32 * t + lane] : -2;
            }
#pragma unroll
            for (int k = 0; k < kGatherRows; ++k)
                if (p[k] >= 0) Z[chk_index<CK>(p[k], ny, bad)] = u[32 * (t0 + k * NW) + lane];
        }
        __syncthreads();  // u, sv and sb are refilled by the next batch
    }
    chk_report<CK>(bad, chk);
    if (gmode == SG_NONE) return;
    const double bt = block_sum(g, sh);
    if (gmode == SG_PART) {
        if (tid == 0) partials[pbase + blockIdx.x] = bt;
        return;
    }
    // the last bucket: the grid total over every bucket's block totals, in
    // block order (deterministic), then gamma_0 or beta
    __shared__ bool am_last;
    if (tid == 0) {
        partials[pbase + blockIdx.x] = bt;
        __threadfence();
        const unsigned t = atomicAdd(&st->ticket[1], 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double sum = 0.0;
    for (int k = tid; k < pbase + (int)gridDim.x; k += blockDim.x) sum += __ldcg(partials + k);
    sum = block_sum(sum, sh);
    if (tid == 0) {
        st->ticket[1] = 0u;
        finalize_gamma(st, sum, init ? UPD_INIT : UPD_STEP, GammaFloor<T>::value);
    }
}

// k = 1, fused SGS path: y~ = Pi z~ + beta y~ = z~ - q (q^T z~) + beta y~
// per row (M >= the longest row of P held in registers; M = 0: any row).
template <class T, int M>
__global__ void __launch_bounds__(kBlock)
k_ydir_proj_k1(int n, const int *__restrict__ Pp, const T *__restrict__ qv,
               const T *__restrict__ Z, T *__restrict__ Y, const DevState *st) {
    if (st->stop) return;
    const T beta = (T)st->beta;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p0 = Pp[i], p1 = Pp[i + 1];
        if constexpr (M > 0) {
            T q[M], z[M], y[M];
            T t = T(0);
#pragma unroll
            for (int k = 0; k < M; ++k)
                if (p0 + k < p1) {
                    q[k] = qv[p0 + k];
                    z[k] = Z[p0 + k];
                    y[k] = Y[p0 + k];
                    t = fmat(q[k], z[k], t);
                }
#pragma unroll
            for (int k = 0; k < M; ++k)
                if (p0 + k < p1) Y[p0 + k] = fmat(beta, y[k], fmat(-q[k], t, z[k]));
        } else {
            T t = T(0);
            for (int s = p0; s < p1; ++s) t = fmat(qv[s], Z[s], t);
            for (int s = p0; s < p1; ++s) Y[s] = fmat(beta, Y[s], fmat(-qv[s], t, Z[s]));
        }
    }
}

// k = 1: z~ <- Pi z~ = z~ - q (q^T z~) per row and gamma = <r~, z~> in one
// pass, then the scalar step of Algorithm 3 (gamma_0 or beta).
template <class T>
__global__ void __launch_bounds__(kBlock)
k_project_gamma_k1(int n, const int *__restrict__ Pp, const T *__restrict__ qv,
                   const T *__restrict__ R, T *__restrict__ Z, DevState *st, double *partials,
                   int mode) {
    if (st->stop) return;
    Dot<T> dot;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p0 = Pp[i], p1 = Pp[i + 1];
        T t = T(0);
        for (int s = p0; s < p1; ++s) t = fmat(qv[s], Z[s], t);
        for (int s = p0; s < p1; ++s) {
            const T z = fmat(-qv[s], t, Z[s]);
            Z[s] = z;
            dot.add(R[s], z);
        }
    }
    __shared__ double sh[32];
    double bt = block_dot_total(dot, sh);
    double total;
    if (grid_reduce(bt, partials, &st->ticket[1], &total))
        finalize_gamma(st, total, mode, GammaFloor<T>::value);
}

// ---------------------------------------------------------------------------
// host plan
// ---------------------------------------------------------------------------
struct GroupOut {
    std::vector<int> hdr, rpos, fown, fa, bown, ba;
    std::vector<unsigned short> blob;
};

// one sweep of a group: levels (relative row bounds), rows in level order,
// relative coupling pointers, couplings (local index), and per coupling its
// row and A entry for the value refill
void emit_sweep(const std::vector<int> &level, const std::vector<std::vector<int>> &cpl,
                const std::vector<std::vector<int>> &ent, const std::vector<int> &rows,
                std::vector<unsigned short> &lvl, std::vector<unsigned short> &orow,
                std::vector<unsigned short> &optr, std::vector<unsigned short> &idx,
                std::vector<int> &own, std::vector<int> &aent) {
    const int m = (int)rows.size();
    int maxl = -1;
    for (int t = 0; t < m; ++t) maxl = std::max(maxl, level[t]);
    const int nlev = maxl + 1;
    std::vector<int> cnt(nlev + 1, 0);
    for (int t = 0; t < m; ++t) cnt[level[t] + 1]++;
    for (int l = 0; l < nlev; ++l) cnt[l + 1] += cnt[l];
    std::vector<int> order(m);
    {
        std::vector<int> fill(cnt.begin(), cnt.end() - 1);
        for (int t = 0; t < m; ++t) order[fill[level[t]]++] = t;  // stable within a level
    }
    for (int l = 0; l <= nlev; ++l) lvl.push_back((unsigned short)cnt[l]);
    for (int x = 0; x < m; ++x) {
        const int t = order[x];
        orow.push_back((unsigned short)t);
        optr.push_back((unsigned short)idx.size());
        for (size_t q = 0; q < cpl[t].size(); ++q) {
            idx.push_back((unsigned short)cpl[t][q]);
            own.push_back(rows[t]);
            aent.push_back(ent[t][q]);
        }
    }
    optr.push_back((unsigned short)idx.size());
}

}  // namespace

int build_sgs_plan(int n, int nc, const int *Ap, const int *Aj, const int *Pp, const int *Pj,
                   SgsHost &out) {
    const long long nnz = Pp[n];
    // rows of every column (increasing) and their positions in the values
    std::vector<int> colp(nc + 1, 0), crow(nnz), cpos(nnz);
    for (long long q = 0; q < nnz; ++q) {
        if (Pj[q] < 0 || Pj[q] >= nc) return EMIN_ERR_PATTERN;
        colp[Pj[q] + 1]++;
    }
    for (int j = 0; j < nc; ++j) colp[j + 1] += colp[j];
    {
        std::vector<int> fill(colp.begin(), colp.end() - 1);
        for (int i = 0; i < n; ++i)
            for (int q = Pp[i]; q < Pp[i + 1]; ++q) {
                const int t = fill[Pj[q]]++;
                crow[t] = i;
                cpos[t] = q;
            }
    }
    // groups: runs of consecutive columns with the same rows whose entries
    // sit next to each other in every row
    std::vector<int> gcol, gsize;
    for (int j = 0; j < nc;) {
        const int m = colp[j + 1] - colp[j];
        int G = 1;
        while (m > 0 && j + G < nc && G < kSgsMaxCols && colp[j + G + 1] - colp[j + G] == m) {
            bool same = true;
            for (int t = 0; t < m && same; ++t)
                same = crow[colp[j + G] + t] == crow[colp[j] + t] &&
                       cpos[colp[j + G] + t] == cpos[colp[j] + t] + G;
            if (!same) break;
            ++G;
        }
        if (m > 0) {
            if (m > kSgsMaxRows) return EMIN_ERR_ARG;
            gcol.push_back(j);
            gsize.push_back(G);
        }
        j += G;
    }
    const int ng = (int)gcol.size();
    unsigned nth = std::thread::hardware_concurrency();
    nth = std::max(1u, std::min(nth, 32u));
    if (ng < 1024) nth = 1;
    auto run = [&](auto &&fn) {
        if (nth == 1) {
            fn(0);
        } else {
            std::vector<std::thread> th;
            for (unsigned t = 0; t < nth; ++t) th.emplace_back(fn, (int)t);
            for (auto &t : th) t.join();
        }
    };
    // the couplings of group g inside its block (local indices, A entries)
    struct Lists {
        std::vector<int> rows;
        std::vector<std::vector<int>> lo, lo_e, up, up_e;
        long long nf = 0, nb = 0;
    };
    auto lists = [&](int g, std::vector<int> &loc, Lists &L) {
        const int j = gcol[g], m = colp[j + 1] - colp[j];
        L.rows.assign(crow.begin() + colp[j], crow.begin() + colp[j + 1]);
        L.lo.assign(m, {});
        L.lo_e.assign(m, {});
        L.up.assign(m, {});
        L.up_e.assign(m, {});
        L.nf = L.nb = 0;
        for (int t = 0; t < m; ++t) loc[L.rows[t]] = t;
        for (int t = 0; t < m; ++t) {
            const int i = L.rows[t];
            for (int e = Ap[i]; e < Ap[i + 1]; ++e) {
                const int l = Aj[e];
                if (l == i || l < 0 || l >= n) continue;
                const int tl = loc[l];
                if (tl < 0) continue;
                if (tl < t) {
                    L.lo[t].push_back(tl);
                    L.lo_e[t].push_back(e);
                    ++L.nf;
                } else {
                    L.up[t].push_back(tl);
                    L.up_e[t].push_back(e);
                    ++L.nb;
                }
            }
        }
        for (int t = 0; t < m; ++t) loc[L.rows[t]] = -1;
    };
    // phase 1: a structure hash of every group that could be batched (one
    // column, local rows and per-row coupling counts that fit the batched
    // records, u, the values of 32 lanes and the sweep structure within
    // kBatchSmem in float)
    std::vector<unsigned long long> ghash(ng, 0);
    std::vector<char> gelig(ng, 0);
    run([&](int tid) {
        const int g0 = (int)((long long)ng * tid / nth), g1 = (int)((long long)ng * (tid + 1) / nth);
        std::vector<int> loc(n, -1);
        Lists L;
        for (int g = g0; g < g1; ++g) {
            const int m = colp[gcol[g] + 1] - colp[gcol[g]];
            if (gsize[g] != 1 || m > kBatchRows) continue;
            lists(g, loc, L);
            if (128LL * (m + L.nf) + 4LL * (10LL * m + 2 * L.nf + 16) > kBatchSmem || L.nf > 65535)
                continue;
            std::vector<int> tcnt(m, 0);
            bool fits = true;
            for (int t = 0; t < m && fits; ++t) {
                fits = (int)L.lo[t].size() <= kBatchRowCpl;
                for (int v : L.lo[t]) fits = fits && ++tcnt[v] <= kBatchRowCpl;
            }
            if (!fits) continue;
            unsigned long long h = 1469598103934665603ULL;
            auto mix = [&](unsigned long long v) { h = (h ^ v) * 1099511628211ULL; };
            mix((unsigned long long)m);
            for (int t = 0; t < m; ++t) {
                mix(0x100000000ULL + L.lo[t].size());
                for (int v : L.lo[t]) mix((unsigned long long)v);
                mix(0x200000000ULL + L.up[t].size());
                for (int v : L.up[t]) mix((unsigned long long)v);
            }
            ghash[g] = h;
            gelig[g] = 1;
        }
    });
    // phase 2: classes of structurally identical groups; a class with at
    // least kBatchMin members is batched, and so is every eligible class
    // when the groups of the rarer ones are few (they then run beside the
    // others instead of in a level-path launch of their own)
    out = SgsHost();
    std::unordered_map<unsigned long long, int> cls_of_hash;
    std::vector<int> gcls(ng, -1), cls_rep, cls_count;
    for (int g = 0; g < ng; ++g) {
        if (!gelig[g]) continue;
        auto it = cls_of_hash.find(ghash[g]);
        int c;
        if (it == cls_of_hash.end()) {
            c = (int)cls_rep.size();
            cls_of_hash.emplace(ghash[g], c);
            cls_rep.push_back(g);
            cls_count.push_back(0);
        } else {
            c = it->second;
        }
        gcls[g] = c;
        cls_count[c]++;
    }
    long long rare = 0;
    for (size_t c = 0; c < cls_rep.size(); ++c)
        if (cls_count[c] < kBatchMin) rare += cls_count[c];
    const int min_count = rare <= kBatchTail ? 1 : kBatchMin;
    std::vector<int> bcls(cls_rep.size(), -1);  // class -> batched class index
    std::vector<Lists> canon;
    std::vector<int> gbatch(ng, -1), glane(ng, -1);
    {
        std::vector<int> loc(n, -1);
        std::vector<int> next(cls_rep.size(), 0);
        std::vector<int> bc_src;  // batched class -> class
        for (size_t c = 0; c < cls_rep.size(); ++c) {
            if (cls_count[c] < min_count) continue;
            bcls[c] = (int)canon.size();
            bc_src.push_back((int)c);
            canon.emplace_back();
            lists(cls_rep[c], loc, canon.back());
        }
        const int nbc = (int)canon.size();
        // class sweep structures: levels of the rows with couplings, row
        // records and coupling words (see batch_sweep), 16-byte aligned and
        // padded; value o of a class is its o-th lower coupling in row order
        for (int b = 0; b < nbc; ++b) {
            const Lists &L = canon[b];
            const int m = (int)L.rows.size();
            std::vector<int> fstart(m + 1, 0);
            for (int t = 0; t < m; ++t) fstart[t + 1] = fstart[t] + (int)L.lo[t].size();
            const int nv = fstart[m];
            // the transpose: row t is coupled to the later rows u with t in lo[u]
            std::vector<std::vector<std::pair<int, int>>> tr(m);
            for (int t2 = 0; t2 < m; ++t2)
                for (size_t x = 0; x < L.lo[t2].size(); ++x)
                    tr[L.lo[t2][x]].push_back({t2, fstart[t2] + (int)x});
            std::vector<int> fl(m, 0), bl(m, 0);
            for (int t = 0; t < m; ++t)
                for (int v : L.lo[t]) fl[t] = std::max(fl[t], fl[v] + 1);
            for (int t = m - 1; t >= 0; --t)
                for (auto &pr : tr[t]) bl[t] = std::max(bl[t], bl[pr.first] + 1);
            while (out.cls_blob.size() % 4) out.cls_blob.push_back(0u);
            const int off = (int)out.cls_blob.size();
            int nl[2] = {0, 0}, nr[2] = {0, 0}, ns[2] = {0, 0};
            for (int sw = 0; sw < 2; ++sw) {
                const std::vector<int> &lev = sw == 0 ? fl : bl;
                int maxl = 0;
                for (int t = 0; t < m; ++t) maxl = std::max(maxl, lev[t]);
                std::vector<std::vector<int>> rows_at(maxl + 1);
                for (int t = 0; t < m; ++t)
                    if (lev[t] > 0) rows_at[lev[t]].push_back(t);
                std::vector<unsigned> lvl, rec, cpl;
                lvl.push_back(0);
                for (int l = 1; l <= maxl; ++l) {
                    for (int t : rows_at[l]) {
                        const int cnt = sw == 0 ? (int)L.lo[t].size() : (int)tr[t].size();
                        unsigned r4[4] = {(unsigned)t | (unsigned)cnt << 10 | (unsigned)cpl.size() << 16,
                                          0u, 0u, 0u};
                        for (int x = 0; x < cnt; ++x) {
                            const int src = sw == 0 ? L.lo[t][x] : tr[t][x].first;
                            const int vi = sw == 0 ? fstart[t] + x : tr[t][x].second;
                            const unsigned w = (unsigned)src | (unsigned)vi << 16;
                            if (x < 3) r4[1 + x] = w;
                            else cpl.push_back(w);  // spill: couplings past the third
                        }
                        rec.insert(rec.end(), r4, r4 + 4);
                    }
                    lvl.push_back((unsigned)(rec.size() / 4));
                }
                nl[sw] = maxl;
                nr[sw] = (int)(rec.size() / 4);
                ns[sw] = (int)cpl.size();
                // 16-byte aligned regions: level bounds, records, coupling words
                while (lvl.size() % 4) lvl.push_back(0u);
                while (cpl.size() % 4) cpl.push_back(0u);
                for (auto *v : {&lvl, &rec, &cpl}) out.cls_blob.insert(out.cls_blob.end(), v->begin(), v->end());
            }
            while (out.cls_blob.size() % 4) out.cls_blob.push_back(0u);
            const int wpad = (int)out.cls_blob.size() - off;
            // level counts (< 1024) and spill counts (< 65536) packed in pairs
            const int h[8] = {m, nv, nl[0] | nl[1] << 16, ns[0] | ns[1] << 16, off, nr[0], nr[1], wpad};
            out.cls_hdr.insert(out.cls_hdr.end(), h, h + 8);
        }
        // buckets: the classes whose batch fits as many CTAs per SM as the
        // class with the most groups, then the rest
        auto foot = [&](int b) {  // u, values and the class's sweep structure
            return 128LL * ((long long)canon[b].rows.size() + canon[b].nf) +
                   4LL * out.cls_hdr[8 * (size_t)b + 7];
        };
        auto per_sm = [](long long bytes) {
            const long long cap = 228LL * 1024, per = bytes + 1024 + 512;
            return std::min<long long>(2048 / (32 * kSgsWarps), cap / per);
        };
        std::vector<int> bucket_of(nbc, 0);
        if (nbc > 0) {
            int dom = 0;
            for (int b = 1; b < nbc; ++b)
                if (cls_count[bc_src[b]] > cls_count[bc_src[dom]]) dom = b;
            long long fa = 0;
            for (int b = 0; b < nbc; ++b)
                if (per_sm(foot(b)) >= per_sm(foot(dom))) fa = std::max(fa, foot(b));
            for (int b = 0; b < nbc; ++b) bucket_of[b] = foot(b) <= fa ? 0 : 1;
        }
        // batches by bucket, then by class, groups in column order
        std::vector<int> cls_first_batch(nbc, 0);
        int nb_total = 0;
        for (int bk = 0; bk < kSgsBuckets; ++bk) {
            SgsBucket &B = out.bucket[bk];
            B.b0 = nb_total;
            for (int b = 0; b < nbc; ++b) {
                if (bucket_of[b] != bk) continue;
                cls_first_batch[b] = nb_total;
                nb_total += (cls_count[bc_src[b]] + 31) / 32;
                B.umax = std::max(B.umax, (int)canon[b].rows.size());
                B.vmax = std::max(B.vmax, (int)canon[b].nf);
                B.wmax = std::max(B.wmax, out.cls_hdr[8 * (size_t)b + 7]);
            }
            B.b1 = nb_total;
        }
        out.nbucket = out.bucket[1].b1 > out.bucket[1].b0 ? 2 : (nb_total > 0 ? 1 : 0);
        for (int g = 0; g < ng; ++g) {
            const int c = gcls[g];
            if (c < 0 || bcls[c] < 0) continue;
            const int k = next[c]++;
            gbatch[g] = cls_first_batch[bcls[c]] + k / 32;
            glane[g] = k % 32;
        }
        // batch headers and the lane arrays (empty lanes: position -1)
        std::vector<int> bhdr(4LL * nb_total, 0);
        long long rp = 0, fv = 0;
        for (int bk = 0; bk < kSgsBuckets; ++bk)
            for (int b = 0; b < nbc; ++b) {
                if (bucket_of[b] != bk) continue;
                const int nbat = (cls_count[bc_src[b]] + 31) / 32;
                for (int k = 0; k < nbat; ++k) {
                    int *hb = &bhdr[4 * (size_t)(cls_first_batch[b] + k)];
                    hb[0] = b;
                    hb[1] = (int)rp;
                    hb[2] = (int)fv;
                    rp += 32LL * (long long)canon[b].rows.size();
                    fv += 32LL * canon[b].nf;
                    if (rp > 0x7fffffffLL || fv > 0x7fffffffLL) return EMIN_ERR_ARG;
                }
            }
        out.bat_hdr.swap(bhdr);
        out.nbatch = nb_total;
        out.bat_rpos.assign(rp, -1);
        out.bat_own.assign(fv, -1);
        out.bat_ent.assign(fv, 0);
    }
    // phase 3: batched groups fill their lane (after checking their lists
    // against the class's, so that equal hashes never stand in for equal
    // structure); the other groups get a level plan
    std::vector<GroupOut> part(nth);
    std::vector<int> bad(nth, 0);
    run([&](int tid) {
        GroupOut &o = part[tid];
        const int g0 = (int)((long long)ng * tid / nth), g1 = (int)((long long)ng * (tid + 1) / nth);
        std::vector<int> loc(n, -1);
        Lists L;
        for (int g = g0; g < g1 && !bad[tid]; ++g) {
            const int j = gcol[g], G = gsize[g], m = colp[j + 1] - colp[j];
            lists(g, loc, L);
            if (gbatch[g] >= 0) {
                const Lists &C = canon[bcls[gcls[g]]];
                if (C.lo == L.lo && C.up == L.up) {
                    const int *h = &out.bat_hdr[4 * (size_t)gbatch[g]];
                    const int lane = glane[g];
                    for (int t = 0; t < m; ++t) out.bat_rpos[h[1] + 32LL * t + lane] = cpos[colp[j] + t];
                    long long q = 0;
                    for (int t = 0; t < m; ++t)
                        for (size_t x = 0; x < L.lo[t].size(); ++x, ++q) {
                            out.bat_own[h[2] + 32 * q + lane] = L.rows[t];
                            out.bat_ent[h[2] + 32 * q + lane] = L.lo_e[t][x];
                        }
                    continue;
                }
            }
            if (L.nf > 65535 || L.nb > 65535) {  // 16-bit coupling pointers
                bad[tid] = 1;
                break;
            }
            std::vector<int> fl(m, 0), bl(m, 0);
            for (int t = 0; t < m; ++t)
                for (int tl : L.lo[t]) fl[t] = std::max(fl[t], fl[tl] + 1);
            for (int t = m - 1; t >= 0; --t)
                for (int tu : L.up[t]) bl[t] = std::max(bl[t], bl[tu] + 1);
            std::vector<unsigned short> flvl, frow, foptr, fidx, blvl, brow, boptr, bidx;
            const int fo0 = (int)o.fa.size(), bo0 = (int)o.ba.size();
            emit_sweep(fl, L.lo, L.lo_e, L.rows, flvl, frow, foptr, fidx, o.fown, o.fa);
            emit_sweep(bl, L.up, L.up_e, L.rows, blvl, brow, boptr, bidx, o.bown, o.ba);
            const int b0 = (int)o.blob.size();
            for (auto *v : {&flvl, &frow, &foptr, &blvl, &brow, &boptr, &fidx, &bidx})
                o.blob.insert(o.blob.end(), v->begin(), v->end());
            while (o.blob.size() % 8) o.blob.push_back(0);  // 16-byte units
            const int r0 = (int)o.rpos.size();
            for (int t = 0; t < m; ++t) o.rpos.push_back(cpos[colp[j] + t]);
            const int h[kHdr] = {m, G, r0, b0 / 8, (int)(o.blob.size() - b0) / 8, fo0, bo0,
                                 (int)L.nf, (int)L.nb, (int)flvl.size() - 1,
                                 (int)blvl.size() - 1, j};
            o.hdr.insert(o.hdr.end(), h, h + kHdr);
        }
    });
    for (unsigned t = 0; t < nth; ++t)
        if (bad[t]) return EMIN_ERR_ARG;
    // concatenate the level-plan parts, shifting their offsets
    long long row_off = 0, blob_off = 0, fo_off = 0, bo_off = 0;
    for (unsigned t = 0; t < nth; ++t) {
        GroupOut &o = part[t];
        if (row_off + (long long)o.rpos.size() > 0x7fffffffLL ||
            (blob_off + (long long)o.blob.size()) / 8 > 0x7fffffffLL ||
            fo_off + (long long)o.fa.size() > 0x7fffffffLL ||
            bo_off + (long long)o.ba.size() > 0x7fffffffLL)
            return EMIN_ERR_ARG;
        for (size_t g = 0; g < o.hdr.size(); g += kHdr) {
            int h[kHdr];
            std::copy(o.hdr.begin() + g, o.hdr.begin() + g + kHdr, h);
            h[2] += (int)row_off;
            h[3] += (int)(blob_off / 8);
            h[5] += (int)fo_off;
            h[6] += (int)bo_off;
            out.cap = std::max(out.cap, h[0] * h[1]);
            out.gmax = std::max(out.gmax, h[1]);
            const long long ub = ((long long)h[0] * h[1] * 4 + 15) / 16 * 16;
            out.stage32 = std::max(out.stage32, ub + 16LL * h[4] + 4LL * (h[7] + h[8]));
            const long long ub8 = ((long long)h[0] * h[1] * 8 + 15) / 16 * 16;
            out.stage64 = std::max(out.stage64, ub8 + 16LL * h[4] + 8LL * (h[7] + h[8]));
            out.hdr.insert(out.hdr.end(), h, h + kHdr);
        }
        out.rpos.insert(out.rpos.end(), o.rpos.begin(), o.rpos.end());
        out.blob.insert(out.blob.end(), o.blob.begin(), o.blob.end());
        out.fown.insert(out.fown.end(), o.fown.begin(), o.fown.end());
        out.fa.insert(out.fa.end(), o.fa.begin(), o.fa.end());
        out.bown.insert(out.bown.end(), o.bown.begin(), o.bown.end());
        out.ba.insert(out.ba.end(), o.ba.begin(), o.ba.end());
        row_off += (long long)o.rpos.size();
        blob_off += (long long)o.blob.size();
        fo_off += (long long)o.fa.size();
        bo_off += (long long)o.ba.size();
        o = GroupOut();
    }
    out.ngroups = (int)(out.hdr.size() / kHdr);
    return EMIN_OK;
}

template <class T>
void launch_sgs_values(const Launch &L, const int *fown, const int *fa, long long nf,
                       const int *bown, const int *ba, long long nb, const int *Aj,
                       const double *Av, const double *dsq, T *fval, T *bval) {
    if (nf > 0) {
        k_sgs_values<T><<<grid_for(nf, L.grid_rows), kBlock, 0, L.stream>>>(nf, fown, fa, Aj, Av,
                                                                           dsq, fval);
        note_launch();
    }
    if (nb > 0) {
        k_sgs_values<T><<<grid_for(nb, L.grid_rows), kBlock, 0, L.stream>>>(nb, bown, ba, Aj, Av,
                                                                           dsq, bval);
        note_launch();
    }
}

void launch_sgs_sell_pos(const Launch &L, long long nops, const int *own, int *ent,
                         const int *Ap, const int *sell_ptr) {
    if (nops <= 0) return;
    k_sgs_sell_pos<<<grid_for(nops, L.grid_rows), kBlock, 0, L.stream>>>(nops, own, ent, Ap,
                                                                          sell_ptr);
    note_launch();
}

template <class T>
void launch_sgs_values_sell(const Launch &L, long long nops, const int *own, const int *pos,
                            const T *sa, const uint2 *spk, T *val) {
    if (nops <= 0) return;
    k_sgs_values_sell<T><<<grid_for(nops, L.grid_rows), kBlock, 0, L.stream>>>(nops, own, pos,
                                                                              sa, spk, val);
    note_launch();
}
template void launch_sgs_values_sell<float>(const Launch &, long long, const int *, const int *,
                                            const float *, const uint2 *, float *);
template void launch_sgs_values_sell<double>(const Launch &, long long, const int *,
                                             const int *, const double *, const uint2 *,
                                             double *);

namespace {
// a kernel instantiation with its launch shape: `slot` bytes of shared
// memory per lane group of LPG lanes, up to 8 warps per block
template <class T, int GM, int LPG>
void sweep_with(const Launch &L, const SgsOps<T> &s, const T *R, T *Z, const DevState *st,
                long long slot) {
    auto kern = k_sgs_sweep<T, GM, LPG>;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_sgs_sweep<T, GM, LPG, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaGetLastError();
        attr = true;
    }
    const long long per_warp = slot * (32 / LPG);
    long long wpb = (96 * 1024) / (per_warp > 0 ? per_warp : 1);
    wpb = std::max(1LL, std::min(8LL, wpb));
    const int threads = (int)(32 * wpb);
    const size_t smem = (size_t)(wpb * per_warp);
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) !=
            cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const long long tasks_per_block = wpb * (32 / LPG);
    long long blocks = ((long long)s.ngroups + tasks_per_block - 1) / tasks_per_block;
    blocks = std::min(blocks, (long long)L.nsm * per_sm);
    if (s.chk)
        k_sgs_sweep<T, GM, LPG, true><<<(int)blocks, threads, smem, L.stream>>>(
            s.ngroups, s.hdr, s.rpos, s.blob, s.fval, s.bval, R, Z, st, (int)slot, s.chk, s.ny);
    else
        kern<<<(int)blocks, threads, smem, L.stream>>>(s.ngroups, s.hdr, s.rpos, s.blob, s.fval,
                                                       s.bval, R, Z, st, (int)slot, nullptr, s.ny);
}
}  // namespace

namespace {
// dynamic shared memory of a bucket's batched sweep: u and the values of 32
// lanes, and the largest class sweep structure
template <class T>
size_t batch_smem(const SgsBucket &B) {
    return (size_t)32 * (size_t)(B.umax + B.vmax) * sizeof(T) + 4 * (size_t)B.wmax;
}

// dynamic shared memory a batched sweep may use: a float batch is kept
// within kBatchSmem, a double one within twice that (and the structure)
constexpr int kBatchSmemOptIn = 2 * (int)kBatchSmem + 16 * 1024;

template <class T>
bool batch_attributes() {
    static int done = 0;  // 1 set, -1 refused
    if (!done) {
        const bool ok = cudaFuncSetAttribute(k_sgs_batch<T, kSgsWarps, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kBatchSmemOptIn) == cudaSuccess &&
                        cudaFuncSetAttribute(k_sgs_batch<T, kSgsWarps, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kBatchSmemOptIn) == cudaSuccess;
        cudaGetLastError();
        done = ok ? 1 : -1;
    }
    return done > 0;
}

// CTAs of one bucket (at most its batches, at most what fits every SM);
// -1 when the shared-memory opt-in was refused
template <class T>
int batch_grid(int nsm, const SgsBucket &B) {
    const int nb = B.b1 - B.b0;
    if (nb <= 0) return 0;
    if (!batch_attributes<T>()) return -1;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sgs_batch<T, kSgsWarps, false>,
                                                      32 * kSgsWarps, batch_smem<T>(B)) !=
            cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return -1;
    }
    return (int)std::min<long long>(nb, (long long)nsm * per_sm);
}
}  // namespace

// CTAs of every bucket for both value types (the plan keeps a float batch
// within kBatchSmem, so the double one, twice as large, fits one CTA too)
int sgs_prepare(int nsm, SgsHost &h) {
    for (int b = 0; b < h.nbucket; ++b) {
        SgsBucket &B = h.bucket[b];
        if (batch_smem<double>(B) > (size_t)kBatchSmemOptIn) return EMIN_ERR_ARG;
        B.grid32 = batch_grid<float>(nsm, B);
        B.grid64 = batch_grid<double>(nsm, B);
        if (B.b1 > B.b0 && (B.grid32 < 1 || B.grid64 < 1)) return EMIN_ERR_CUDA;
    }
    return EMIN_OK;
}

// The batched buckets first (with s.fused, gamma over all of them: block
// totals of the earlier buckets in the partials, the grid total and the
// scalar step in the last), then the level path.
template <class T>
void launch_sgs_sweep(const Launch &L, const SgsOps<T> &s, const T *R, T *Z, DevState *st,
                      double *partials, int init) {
    int pbase = 0;
    for (int b = 0; b < s.nbucket; ++b) {
        const SgsBucket &B = s.bucket[b];
        const int grid = sizeof(T) == 4 ? B.grid32 : B.grid64;
        if (grid <= 0) continue;
        const int gmode = !s.fused ? SG_NONE : (b == s.nbucket - 1 ? SG_LAST : SG_PART);
        const size_t smem = batch_smem<T>(B);
        if (s.chk)
            k_sgs_batch<T, kSgsWarps, true><<<grid, 32 * kSgsWarps, smem, L.stream>>>(
                B.b0, B.b1, s.bat_hdr, s.cls_hdr, s.cls_blob, s.bat_rpos, s.bat_val, R, Z, st,
                partials, pbase, gmode, init, B.umax, B.vmax, B.wmax, s.chk, s.ny, s.nbat_rpos,
                s.nbat_val, s.ncls_blob);
        else
            k_sgs_batch<T, kSgsWarps, false><<<grid, 32 * kSgsWarps, smem, L.stream>>>(
                B.b0, B.b1, s.bat_hdr, s.cls_hdr, s.cls_blob, s.bat_rpos, s.bat_val, R, Z, st,
                partials, pbase, gmode, init, B.umax, B.vmax, B.wmax, nullptr, s.ny,
                s.nbat_rpos, s.nbat_val, s.ncls_blob);
        note_launch();
        pbase += grid;
    }
    if (s.ngroups > 0) {
        const long long ubytes = ((long long)s.cap * sizeof(T) + 15) / 16 * 16;
        const long long slot = std::max(ubytes, (long long)(sizeof(T) == 4 ? 4096 : 8192));
        if (s.gmax <= 1)
            sweep_with<T, 1, 32>(L, s, R, Z, st, slot);
        else
            sweep_with<T, kSgsMaxCols, 32>(L, s, R, Z, st, slot);
        note_launch();
    }
}

template <class T>
void launch_ydir_proj_k1(const Launch &L, int n, int maxrow, const int *Pp, const T *qv,
                         const T *Z, T *Y, const DevState *st) {
    if (n <= 0) return;
    const int g = grid_for(n, L.grid_rows);
    if (maxrow <= 4)
        k_ydir_proj_k1<T, 4><<<g, kBlock, 0, L.stream>>>(n, Pp, qv, Z, Y, st);
    else if (maxrow <= 8)
        k_ydir_proj_k1<T, 8><<<g, kBlock, 0, L.stream>>>(n, Pp, qv, Z, Y, st);
    else
        k_ydir_proj_k1<T, 0><<<g, kBlock, 0, L.stream>>>(n, Pp, qv, Z, Y, st);
    note_launch();
}

// k = 1: projection and gamma in one pass; otherwise projection, then gamma
template <class T>
void launch_sgs_finish(const Launch &L, const Ops<T> &o, Work<T> &w, int init, long long nnz_p) {
    if (o.k == 1 && o.qv) {
        k_project_gamma_k1<T><<<grid_for(o.n, L.grid_rows), kBlock, 0, L.stream>>>(
            o.n, o.Pp, o.qv, w.R, w.Z, w.st, w.partials, init ? UPD_INIT : UPD_STEP);
        note_launch();
    } else {
        launch_project<T>(L, o, w.Z, T(1));
        launch_update<T>(L, nnz_p, w, init ? UPD_GZ_INIT : UPD_GZ_STEP);
    }
}

template void launch_sgs_values<float>(const Launch &, const int *, const int *, long long,
                                       const int *, const int *, long long, const int *,
                                       const double *, const double *, float *, float *);
template void launch_sgs_values<double>(const Launch &, const int *, const int *, long long,
                                        const int *, const int *, long long, const int *,
                                        const double *, const double *, double *, double *);
template void launch_sgs_sweep<float>(const Launch &, const SgsOps<float> &, const float *,
                                      float *, DevState *, double *, int);
template void launch_sgs_sweep<double>(const Launch &, const SgsOps<double> &, const double *,
                                       double *, DevState *, double *, int);
template void launch_ydir_proj_k1<float>(const Launch &, int, int, const int *, const float *,
                                         const float *, float *, const DevState *);
template void launch_ydir_proj_k1<double>(const Launch &, int, int, const int *, const double *,
                                          const double *, double *, const DevState *);
template void launch_sgs_finish<float>(const Launch &, const Ops<float> &, Work<float> &, int,
                                       long long);
template void launch_sgs_finish<double>(const Launch &, const Ops<double> &, Work<double> &, int,
                                        long long);

}  // namespace emin
