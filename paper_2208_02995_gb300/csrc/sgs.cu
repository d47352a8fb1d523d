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
#include <vector>

#include "device_util.cuh"
#include "emin_internal.cuh"

namespace emin {
namespace {

constexpr int kSgsMaxCols = 8;        // columns per group
constexpr int kSgsMaxRows = 65535;    // rows per group (16-bit local indices)

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
        const int e = aent[o];
        const double di = dsq[own[o]], a = Av[e], dl = dsq[Aj[e]];
        if constexpr (sizeof(T) == 4)
            val[o] = (float)di * (float)a * (float)dl;
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
template <class T, int GM, int LPG>
__device__ __forceinline__ void sgs_sweep_levels(T *u, int G, int nl, const unsigned short *lvl,
                                                 const unsigned short *row,
                                                 const unsigned short *optr,
                                                 const unsigned short *idx, const T *val,
                                                 int sub, unsigned mask) {
    for (int lv = 0; lv < nl; ++lv) {
        const int a = lvl[lv], b = lvl[lv + 1];
        for (int x = a + sub; x < b; x += LPG) {
            const int t = row[x];
            T acc[GM];
#pragma unroll
            for (int c = 0; c < GM; ++c) acc[c] = (c < G) ? u[t * G + c] : T(0);
            const int o1 = optr[x + 1];
            for (int o = optr[x]; o < o1; ++o) {
                const int tl = idx[o];
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
template <class T, int GM, int LPG>
__global__ void k_sgs_sweep(int ngroups, const int *__restrict__ hdr, const int *__restrict__ rpos,
                            const uint4 *__restrict__ blob, const T *__restrict__ fval,
                            const T *__restrict__ bval, const T *__restrict__ R,
                            T *__restrict__ Z, const DevState *st, int slot) {
    if (st->stop) return;
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
            u[x] = R[rpos[r0 + t] + c];
        }
        __syncwarp(mask);
        const SgsView v = sgs_view(ib, m, nlf, nlb, nf);
        sgs_sweep_levels<T, GM, LPG>(u, G, nlf, v.flvl, v.frow, v.foptr, v.fidx, fv, sub, mask);
        sgs_sweep_levels<T, GM, LPG>(u, G, nlb, v.blvl, v.brow, v.boptr, v.bidx, bv, sub, mask);
        for (int x = sub; x < m * G; x += LPG) {
            const int t = x / G, c = x - t * G;
            Z[rpos[r0 + t] + c] = u[x];
        }
        __syncwarp(mask);  // the slot is refilled by the next group
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
    std::vector<GroupOut> part(nth);
    std::vector<int> bad(nth, 0);
    auto work = [&](int tid) {
        GroupOut &o = part[tid];
        const int g0 = (int)((long long)ng * tid / nth), g1 = (int)((long long)ng * (tid + 1) / nth);
        std::vector<int> loc(n, -1);
        for (int g = g0; g < g1 && !bad[tid]; ++g) {
            const int j = gcol[g], G = gsize[g], m = colp[j + 1] - colp[j];
            std::vector<int> rows(crow.begin() + colp[j], crow.begin() + colp[j + 1]);
            for (int t = 0; t < m; ++t) loc[rows[t]] = t;
            std::vector<std::vector<int>> lo(m), lo_e(m), up(m), up_e(m);
            long long nf = 0, nb = 0;
            for (int t = 0; t < m; ++t) {
                const int i = rows[t];
                for (int e = Ap[i]; e < Ap[i + 1]; ++e) {
                    const int l = Aj[e];
                    if (l == i || l < 0 || l >= n) continue;
                    const int tl = loc[l];
                    if (tl < 0) continue;
                    if (tl < t) {
                        lo[t].push_back(tl);
                        lo_e[t].push_back(e);
                        ++nf;
                    } else {
                        up[t].push_back(tl);
                        up_e[t].push_back(e);
                        ++nb;
                    }
                }
            }
            for (int t = 0; t < m; ++t) loc[rows[t]] = -1;
            if (nf > 65535 || nb > 65535) {  // 16-bit coupling pointers
                bad[tid] = 1;
                break;
            }
            std::vector<int> fl(m, 0), bl(m, 0);
            for (int t = 0; t < m; ++t)
                for (int tl : lo[t]) fl[t] = std::max(fl[t], fl[tl] + 1);
            for (int t = m - 1; t >= 0; --t)
                for (int tu : up[t]) bl[t] = std::max(bl[t], bl[tu] + 1);
            std::vector<unsigned short> flvl, frow, foptr, fidx, blvl, brow, boptr, bidx;
            const int fo0 = (int)o.fa.size(), bo0 = (int)o.ba.size();
            emit_sweep(fl, lo, lo_e, rows, flvl, frow, foptr, fidx, o.fown, o.fa);
            emit_sweep(bl, up, up_e, rows, blvl, brow, boptr, bidx, o.bown, o.ba);
            const int b0 = (int)o.blob.size();
            for (auto *v : {&flvl, &frow, &foptr, &blvl, &brow, &boptr, &fidx, &bidx})
                o.blob.insert(o.blob.end(), v->begin(), v->end());
            while (o.blob.size() % 8) o.blob.push_back(0);  // 16-byte units
            const int r0 = (int)o.rpos.size();
            for (int t = 0; t < m; ++t) o.rpos.push_back(cpos[colp[j] + t]);
            const int h[kHdr] = {m, G, r0, b0 / 8, (int)(o.blob.size() - b0) / 8, fo0, bo0,
                                 (int)nf, (int)nb, (int)flvl.size() - 1, (int)blvl.size() - 1, j};
            o.hdr.insert(o.hdr.end(), h, h + kHdr);
        }
    };
    if (nth == 1) {
        work(0);
    } else {
        std::vector<std::thread> th;
        for (unsigned t = 0; t < nth; ++t) th.emplace_back(work, (int)t);
        for (auto &t : th) t.join();
    }
    for (unsigned t = 0; t < nth; ++t)
        if (bad[t]) return EMIN_ERR_ARG;
    // concatenate the parts, shifting their row, blob and coupling offsets
    out = SgsHost();
    out.ngroups = ng;
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
            // bytes of u + blob + values (float / double) if staged
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
    kern<<<(int)blocks, threads, smem, L.stream>>>(s.ngroups, s.hdr, s.rpos, s.blob, s.fval,
                                                   s.bval, R, Z, st, (int)slot);
}
}  // namespace

// Every warp owns a slot of at least 4 KB (8 KB for double) and at least the
// largest u; groups that fit their slot whole are staged.  (Two groups per
// warp on 16 lanes each was measured slower: different groups' level and
// coupling counts make the two halves diverge.)
template <class T>
void launch_sgs_sweep(const Launch &L, const SgsOps<T> &s, const T *R, T *Z, const DevState *st) {
    if (s.ngroups <= 0) return;
    const long long ubytes = ((long long)s.cap * sizeof(T) + 15) / 16 * 16;
    const long long slot = std::max(ubytes, (long long)(sizeof(T) == 4 ? 4096 : 8192));
    if (s.gmax <= 1)
        sweep_with<T, 1, 32>(L, s, R, Z, st, slot);
    else
        sweep_with<T, kSgsMaxCols, 32>(L, s, R, Z, st, slot);
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
                                      float *, const DevState *);
template void launch_sgs_sweep<double>(const Launch &, const SgsOps<double> &, const double *,
                                       double *, const DevState *);
template void launch_sgs_finish<float>(const Launch &, const Ops<float> &, Work<float> &, int,
                                       long long);
template void launch_sgs_finish<double>(const Launch &, const Ops<double> &, Work<double> &, int,
                                        long long);

}  // namespace emin
