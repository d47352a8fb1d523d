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
// group and share one block; for every row of a group the coupled rows of
// the same group below it (forward sweep) and above it (backward sweep),
// with their A entries; the rows of a group ordered by dependency level for
// each sweep, so that a level's rows are independent.  One warp sweeps one
// group in shared memory, level by level.
#include <cuda_runtime.h>

#include <algorithm>
#include <thread>
#include <unordered_map>
#include <vector>

#include "device_util.cuh"
#include "convert.cuh"
#include "emin_internal.cuh"

namespace emin {
namespace {

constexpr int kSgsMaxCols = 8;        // columns per group
constexpr int kSgsMaxRows = 65535;    // rows per group (16-bit local indices)
constexpr int kBatchRows = 96;        // rows of a group swept by one lane (batched path)
constexpr int kBatchMin = 8;          // groups of one structure before it is batched
constexpr int kBatchCouplings = 256;  // couplings per sweep of a batched group

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

// 16-byte asynchronous copies of `bytes` (a multiple of 16, both addresses
// 16-byte aligned) from global to shared memory by the 32 lanes of a warp
__device__ __forceinline__ void stage_async(void *dst, const void *src, int bytes, int lane) {
    const unsigned base = (unsigned)__cvta_generic_to_shared(dst);
    const char *s = static_cast<const char *>(src);
    for (int q = lane; 16 * q < bytes; q += 32)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(base + 16 * q),
                     "l"(s + 16 * q)
                     : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void async_wait_all() {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// The batched sweep: 32 structurally identical groups of one column per
// warp, one lane each.  The class structure (coupling pointers and local
// indices, in row order) is the same for every lane and read as uniform
// loads; each lane's u and coupling values sit in shared memory interleaved
// by lane (row t of lane L at [32 t + L], conflict-free), the values of one
// sweep at a time.  Each lane then sweeps its own block row by row, forward
// and backward, with no synchronisation: no lane reads another lane's data.
template <class T, bool CK = false>
__global__ void k_sgs_batch(int nbatch, const int *__restrict__ bat_hdr,
                            const int *__restrict__ cls_hdr,
                            const unsigned short *__restrict__ cls_ptr,
                            const unsigned short *__restrict__ cls_idx,
                            const int *__restrict__ rpos, const T *__restrict__ fval,
                            const T *__restrict__ bval, const T *__restrict__ R,
                            T *__restrict__ Z, const DevState *st, int umax, int vmax, int *chk,
                            long long ny) {
    if (st->stop) return;
    int bad = 0;
    extern __shared__ __align__(16) unsigned char sgs_smem[];
    const int lane = threadIdx.x & 31;
    T *u = reinterpret_cast<T *>(sgs_smem) + (size_t)(threadIdx.x >> 5) * 32 * (umax + vmax);
    T *sv = u + 32 * umax;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nbatch; b += nwarps) {
        const int *h = bat_hdr + 4 * (size_t)b;
        const int *ch = cls_hdr + 8 * (size_t)h[0];
        const int m = ch[0], nf = ch[1], nb = ch[2];
        const unsigned short *fp = cls_ptr + ch[3], *fi = cls_idx + ch[4];
        const unsigned short *bp = cls_ptr + ch[5], *bi = cls_idx + ch[6];
        const int *rp = rpos + h[1];
        // the forward values in flight (16-byte asynchronous copies), then
        // the gather of r~, then one wait
        stage_async(sv, fval + h[2], 32 * nf * (int)sizeof(T), lane);
#pragma unroll 8
        for (int t = 0; t < m; ++t) {
            const int p = rp[32 * t + lane];
            u[32 * t + lane] = p >= 0 ? R[chk_index<CK>(p, ny, bad)] : T(0);
        }
        async_wait_all();
        __syncwarp();
        for (int t = 0; t < m; ++t) {
            T acc = u[32 * t + lane];
            const int o1 = fp[t + 1];
            for (int o = fp[t]; o < o1; ++o)
                acc = fmat(-sv[32 * o + lane], u[32 * chk_index<CK>(fi[o], m, bad) + lane], acc);
            u[32 * t + lane] = acc;
        }
        __syncwarp();
        stage_async(sv, bval + h[3], 32 * nb * (int)sizeof(T), lane);
        async_wait_all();
        __syncwarp();
        for (int t = m - 1; t >= 0; --t) {
            T acc = u[32 * t + lane];
            const int o1 = bp[t + 1];
            for (int o = bp[t]; o < o1; ++o)
                acc = fmat(-sv[32 * o + lane], u[32 * chk_index<CK>(bi[o], m, bad) + lane], acc);
            u[32 * t + lane] = acc;
        }
        for (int t = 0; t < m; ++t) {
            const int p = rp[32 * t + lane];
            if (p >= 0) Z[chk_index<CK>(p, ny, bad)] = u[32 * t + lane];
        }
        __syncwarp();  // the buffers are refilled by the warp's next batch
    }
    chk_report<CK>(bad, chk);
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
    // column, at most kBatchRows rows)
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
            if (L.nf > kBatchCouplings || L.nb > kBatchCouplings) continue;
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
    // least kBatchMin members is swept in batches of 32 (one lane a group)
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
    std::vector<int> bcls(cls_rep.size(), -1);  // class -> batched class index
    std::vector<Lists> canon;
    std::vector<int> gbatch(ng, -1), glane(ng, -1);
    {
        std::vector<int> loc(n, -1);
        std::vector<int> next(cls_rep.size(), 0);
        for (size_t c = 0; c < cls_rep.size(); ++c) {
            if (cls_count[c] < kBatchMin) continue;
            bcls[c] = (int)canon.size();
            canon.emplace_back();
            lists(cls_rep[c], loc, canon.back());
        }
        // batches in group order within each class
        std::vector<int> cls_first_batch(canon.size(), 0);
        int nb_total = 0;
        for (size_t c = 0; c < cls_rep.size(); ++c)
            if (bcls[c] >= 0) {
                cls_first_batch[bcls[c]] = nb_total;
                nb_total += (cls_count[c] + 31) / 32;
            }
        for (int g = 0; g < ng; ++g) {
            const int c = gcls[g];
            if (c < 0 || bcls[c] < 0) continue;
            const int k = next[c]++;
            gbatch[g] = cls_first_batch[bcls[c]] + k / 32;
            glane[g] = k % 32;
        }
        // class structure: coupling pointers and local indices of both sweeps
        for (size_t b = 0; b < canon.size(); ++b) {
            const Lists &L = canon[b];
            const int m = (int)L.rows.size();
            const int h[8] = {m, (int)L.nf, (int)L.nb, (int)out.cls_ptr.size(), 0, 0, 0, 0};
            out.cls_hdr.insert(out.cls_hdr.end(), h, h + 8);
            int cp0 = (int)out.cls_ptr.size();
            out.cls_hdr[8 * b + 3] = cp0;
            out.cls_hdr[8 * b + 4] = (int)out.cls_idx.size();
            int o = 0;
            for (int t = 0; t < m; ++t) {
                out.cls_ptr.push_back((unsigned short)o);
                for (int v : L.lo[t]) out.cls_idx.push_back((unsigned short)v), ++o;
            }
            out.cls_ptr.push_back((unsigned short)o);
            out.cls_hdr[8 * b + 5] = (int)out.cls_ptr.size();
            out.cls_hdr[8 * b + 6] = (int)out.cls_idx.size();
            o = 0;
            for (int t = 0; t < m; ++t) {
                out.cls_ptr.push_back((unsigned short)o);
                for (int v : L.up[t]) out.cls_idx.push_back((unsigned short)v), ++o;
            }
            out.cls_ptr.push_back((unsigned short)o);
            out.bmax_u = std::max(out.bmax_u, m);
            out.bmax_v = std::max(out.bmax_v, (int)std::max(L.nf, L.nb));
        }
        // batch headers and the lane arrays (empty lanes: position -1)
        long long rp = 0, fv = 0, bv = 0;
        for (size_t c = 0; c < cls_rep.size(); ++c) {
            if (bcls[c] < 0) continue;
            const Lists &L = canon[bcls[c]];
            const int nbat = (cls_count[c] + 31) / 32;
            for (int k = 0; k < nbat; ++k) {
                const int h[4] = {bcls[c], (int)rp, (int)fv, (int)bv};
                out.bat_hdr.insert(out.bat_hdr.end(), h, h + 4);
                rp += 32LL * (long long)L.rows.size();
                fv += 32LL * L.nf;
                bv += 32LL * L.nb;
            }
        }
        if (rp > 0x7fffffffLL || fv > 0x7fffffffLL || bv > 0x7fffffffLL) return EMIN_ERR_ARG;
        out.nbatch = (int)(out.bat_hdr.size() / 4);
        out.bat_rpos.assign(rp, -1);
        out.bat_fown.assign(fv, -1);
        out.bat_fa.assign(fv, 0);
        out.bat_bown.assign(bv, -1);
        out.bat_ba.assign(bv, 0);
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
                            out.bat_fown[h[2] + 32 * q + lane] = L.rows[t];
                            out.bat_fa[h[2] + 32 * q + lane] = L.lo_e[t][x];
                        }
                    q = 0;
                    for (int t = 0; t < m; ++t)
                        for (size_t x = 0; x < L.up[t].size(); ++x, ++q) {
                            out.bat_bown[h[3] + 32 * q + lane] = L.rows[t];
                            out.bat_ba[h[3] + 32 * q + lane] = L.up_e[t][x];
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

// Every warp owns a slot of at least 4 KB (8 KB for double) and at least the
// largest u; groups that fit their slot whole are staged.  (Two groups per
// warp on 16 lanes each was measured slower: different groups' level and
// coupling counts make the two halves diverge.)
template <class T>
void launch_sgs_sweep(const Launch &L, const SgsOps<T> &s, const T *R, T *Z, const DevState *st) {
    if (s.nbatch > 0) {
        // u and one sweep's values of 32 lanes per warp
        const long long per_warp = 32LL * (s.bmax_u + s.bmax_v) * sizeof(T);
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_sgs_batch<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024);
            cudaFuncSetAttribute(k_sgs_batch<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024);
            cudaGetLastError();
            attr = true;
        }
        long long wpb = (96 * 1024) / per_warp;
        wpb = std::max(1LL, std::min(8LL, wpb));
        const int threads = (int)(32 * wpb);
        const size_t smem = (size_t)(wpb * per_warp);
        int per_sm = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sgs_batch<T>, threads, smem) !=
                cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        long long blocks = ((long long)s.nbatch + wpb - 1) / wpb;
        blocks = std::min(blocks, (long long)L.nsm * per_sm);
        if (s.chk)
            k_sgs_batch<T, true><<<(int)blocks, threads, smem, L.stream>>>(
                s.nbatch, s.bat_hdr, s.cls_hdr, s.cls_ptr, s.cls_idx, s.bat_rpos, s.bat_fval,
                s.bat_bval, R, Z, st, s.bmax_u, s.bmax_v, s.chk, s.ny);
        else
            k_sgs_batch<T><<<(int)blocks, threads, smem, L.stream>>>(
                s.nbatch, s.bat_hdr, s.cls_hdr, s.cls_ptr, s.cls_idx, s.bat_rpos, s.bat_fval,
                s.bat_bval, R, Z, st, s.bmax_u, s.bmax_v, nullptr, s.ny);
        note_launch();
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
                                      float *, const DevState *);
template void launch_sgs_sweep<double>(const Launch &, const SgsOps<double> &, const double *,
                                       double *, const DevState *);
template void launch_sgs_finish<float>(const Launch &, const Ops<float> &, Work<float> &, int,
                                       long long);
template void launch_sgs_finish<double>(const Launch &, const Ops<double> &, Work<double> &, int,
                                        long long);

}  // namespace emin
