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
// of row i (= grow[x] for the rows x of the plan, ops optr[x] .. optr[x+1]).
template <class T>
__global__ void k_sgs_values(long long nrows, const int *__restrict__ grow,
                             const int *__restrict__ optr, const int *__restrict__ aent,
                             const int *__restrict__ Aj, const double *__restrict__ Av,
                             const double *__restrict__ dsq, T *__restrict__ val) {
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < nrows;
         x += (long long)gridDim.x * blockDim.x) {
        const double di = dsq[grow[x]];
        for (int o = optr[x]; o < optr[x + 1]; ++o) {
            const int e = aent[o];
            const double a = Av[e], dl = dsq[Aj[e]];
            if constexpr (sizeof(T) == 4)
                val[o] = (float)di * (float)a * (float)dl;
            else
                val[o] = di * a * dl;
        }
    }
}

// One level-ordered unit-diagonal triangular sweep of a group held in u
// (row t, column c at u[t * G + c]): for the rows x of each level,
// u_t -= sum over the row's couplings (t', v) of v u_t'.
template <class T, int GM>
__device__ __forceinline__ void sgs_sweep_levels(T *u, int G, int l0, int nl,
                                                 const int *__restrict__ lvl,
                                                 const unsigned short *__restrict__ row,
                                                 const int *__restrict__ optr,
                                                 const unsigned short *__restrict__ idx,
                                                 const T *__restrict__ val, int lane) {
    for (int lv = 0; lv < nl; ++lv) {
        const int a = lvl[l0 + lv], b = lvl[l0 + lv + 1];
        for (int x = a + lane; x < b; x += 32) {
            const int t = row[x];
            T acc[GM];
#pragma unroll
            for (int c = 0; c < GM; ++c) acc[c] = (c < G) ? u[t * G + c] : T(0);
            for (int o = optr[x]; o < optr[x + 1]; ++o) {
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
        __syncwarp();  // the next level reads this level's rows
    }
}

// z~ = (L^ + I)^{-T} (L^ + I)^{-1} r~, one warp per group (grid-stride),
// `cap` values of shared memory per warp.  Header per group (8 ints):
// rows m, columns G, first plan row r0, forward levels (start, count),
// backward levels (start, count).
template <class T, int GM>
__global__ void k_sgs_sweep(int ngroups, const int *__restrict__ hdr, const int *__restrict__ rpos,
                            const int *__restrict__ flvl, const unsigned short *__restrict__ frow,
                            const int *__restrict__ foptr, const unsigned short *__restrict__ fidx,
                            const T *__restrict__ fval, const int *__restrict__ blvl,
                            const unsigned short *__restrict__ brow,
                            const int *__restrict__ boptr, const unsigned short *__restrict__ bidx,
                            const T *__restrict__ bval, const T *__restrict__ R, T *__restrict__ Z,
                            const DevState *st, int cap) {
    if (st->stop) return;
    extern __shared__ __align__(16) unsigned char sgs_smem[];
    T *u = reinterpret_cast<T *>(sgs_smem) + (size_t)(threadIdx.x >> 5) * cap;
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < ngroups; g += nwarps) {
        const int *h = hdr + 8 * (size_t)g;
        const int m = h[0], G = h[1], r0 = h[2];
        // the block's entries of r~: row t, column c at rpos[r0 + t] + c
        for (int x = lane; x < m * G; x += 32) {
            const int t = x / G, c = x - t * G;
            u[x] = R[rpos[r0 + t] + c];
        }
        __syncwarp();
        sgs_sweep_levels<T, GM>(u, G, h[3], h[4], flvl, frow, foptr, fidx, fval, lane);
        sgs_sweep_levels<T, GM>(u, G, h[5], h[6], blvl, brow, boptr, bidx, bval, lane);
        for (int x = lane; x < m * G; x += 32) {
            const int t = x / G, c = x - t * G;
            Z[rpos[r0 + t] + c] = u[x];
        }
        __syncwarp();  // u is refilled by the warp's next group
    }
}

// ---------------------------------------------------------------------------
// host plan
// ---------------------------------------------------------------------------
struct GroupOut {
    std::vector<int> hdr, rpos, flvl, blvl, foptr, boptr, fa, ba, fgrow, bgrow;
    std::vector<unsigned short> frow, brow, fidx, bidx;
};

// one sweep's part of a group: rows ordered by level, their couplings
void emit_sweep(const std::vector<int> &level, const std::vector<std::vector<int>> &cpl,
                const std::vector<std::vector<int>> &ent, const std::vector<int> &rows, int base_row,
                std::vector<int> &lvl, std::vector<unsigned short> &orow, std::vector<int> &optr,
                std::vector<unsigned short> &idx, std::vector<int> &aent, std::vector<int> &grow,
                int &nlev) {
    const int m = (int)rows.size();
    int maxl = -1;
    for (int t = 0; t < m; ++t) maxl = std::max(maxl, level[t]);
    nlev = maxl + 1;
    std::vector<int> cnt(nlev + 1, 0);
    for (int t = 0; t < m; ++t) cnt[level[t] + 1]++;
    for (int l = 0; l < nlev; ++l) cnt[l + 1] += cnt[l];
    std::vector<int> order(m);
    {
        std::vector<int> fill(cnt.begin(), cnt.end() - 1);
        for (int t = 0; t < m; ++t) order[fill[level[t]]++] = t;  // stable within a level
    }
    for (int l = 0; l <= nlev; ++l) lvl.push_back(base_row + cnt[l]);
    for (int x = 0; x < m; ++x) {
        const int t = order[x];
        orow.push_back((unsigned short)t);
        grow.push_back(rows[t]);
        optr.push_back((int)idx.size());
        for (size_t q = 0; q < cpl[t].size(); ++q) {
            idx.push_back((unsigned short)cpl[t][q]);
            aent.push_back(ent[t][q]);
        }
    }
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
    auto work = [&](int tid) {
        GroupOut &o = part[tid];
        const int g0 = (int)((long long)ng * tid / nth), g1 = (int)((long long)ng * (tid + 1) / nth);
        std::vector<int> loc(n, -1);
        for (int g = g0; g < g1; ++g) {
            const int j = gcol[g], G = gsize[g], m = colp[j + 1] - colp[j];
            std::vector<int> rows(crow.begin() + colp[j], crow.begin() + colp[j + 1]);
            for (int t = 0; t < m; ++t) loc[rows[t]] = t;
            std::vector<std::vector<int>> lo(m), lo_e(m), up(m), up_e(m);
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
                    } else {
                        up[t].push_back(tl);
                        up_e[t].push_back(e);
                    }
                }
            }
            std::vector<int> fl(m, 0), bl(m, 0);
            for (int t = 0; t < m; ++t)
                for (int tl : lo[t]) fl[t] = std::max(fl[t], fl[tl] + 1);
            for (int t = m - 1; t >= 0; --t)
                for (int tu : up[t]) bl[t] = std::max(bl[t], bl[tu] + 1);
            const int r0 = (int)o.rpos.size();
            for (int t = 0; t < m; ++t) o.rpos.push_back(cpos[colp[j] + t]);
            const int lf0 = (int)o.flvl.size(), lb0 = (int)o.blvl.size();
            int nlf = 0, nlb = 0;
            emit_sweep(fl, lo, lo_e, rows, r0, o.flvl, o.frow, o.foptr, o.fidx, o.fa, o.fgrow, nlf);
            emit_sweep(bl, up, up_e, rows, r0, o.blvl, o.brow, o.boptr, o.bidx, o.ba, o.bgrow, nlb);
            const int h[8] = {m, G, r0, lf0, nlf, lb0, nlb, j};
            o.hdr.insert(o.hdr.end(), h, h + 8);
            for (int t = 0; t < m; ++t) loc[rows[t]] = -1;
        }
    };
    if (nth == 1) {
        work(0);
    } else {
        std::vector<std::thread> th;
        for (unsigned t = 0; t < nth; ++t) th.emplace_back(work, (int)t);
        for (auto &t : th) t.join();
    }
    // concatenate the parts, shifting their row, level and op offsets
    out = SgsHost();
    out.ngroups = ng;
    int row_off = 0, lf_off = 0, lb_off = 0, fo_off = 0, bo_off = 0;
    for (unsigned t = 0; t < nth; ++t) {
        GroupOut &o = part[t];
        for (size_t g = 0; g < o.hdr.size(); g += 8) {
            int h[8];
            std::copy(o.hdr.begin() + g, o.hdr.begin() + g + 8, h);
            h[2] += row_off;
            h[3] += lf_off;
            h[5] += lb_off;
            out.cap = std::max(out.cap, h[0] * h[1]);
            out.gmax = std::max(out.gmax, h[1]);
            out.hdr.insert(out.hdr.end(), h, h + 8);
        }
        out.rpos.insert(out.rpos.end(), o.rpos.begin(), o.rpos.end());
        for (int v : o.flvl) out.flvl.push_back(v + row_off);
        for (int v : o.blvl) out.blvl.push_back(v + row_off);
        for (int v : o.foptr) out.foptr.push_back(v + fo_off);
        for (int v : o.boptr) out.boptr.push_back(v + bo_off);
        out.frow.insert(out.frow.end(), o.frow.begin(), o.frow.end());
        out.brow.insert(out.brow.end(), o.brow.begin(), o.brow.end());
        out.fgrow.insert(out.fgrow.end(), o.fgrow.begin(), o.fgrow.end());
        out.bgrow.insert(out.bgrow.end(), o.bgrow.begin(), o.bgrow.end());
        out.fidx.insert(out.fidx.end(), o.fidx.begin(), o.fidx.end());
        out.bidx.insert(out.bidx.end(), o.bidx.begin(), o.bidx.end());
        out.fa.insert(out.fa.end(), o.fa.begin(), o.fa.end());
        out.ba.insert(out.ba.end(), o.ba.begin(), o.ba.end());
        row_off += (int)o.rpos.size();
        lf_off += (int)o.flvl.size();
        lb_off += (int)o.blvl.size();
        fo_off += (int)o.fidx.size();
        bo_off += (int)o.bidx.size();
        GroupOut().hdr.swap(o.hdr);
    }
    out.foptr.push_back((int)out.fidx.size());  // sentinels: the last row's end
    out.boptr.push_back((int)out.bidx.size());
    return EMIN_OK;
}

template <class T>
void launch_sgs_values(const Launch &L, const SgsOps<T> &s, const int *fgrow, const int *bgrow,
                       const int *fa, const int *ba, const int *Aj, const double *Av,
                       const double *dsq, T *fval, T *bval) {
    if (s.nrows <= 0) return;
    const int g = grid_for(s.nrows, L.grid_rows);
    k_sgs_values<T><<<g, kBlock, 0, L.stream>>>(s.nrows, fgrow, s.foptr, fa, Aj, Av, dsq, fval);
    note_launch();
    k_sgs_values<T><<<g, kBlock, 0, L.stream>>>(s.nrows, bgrow, s.boptr, ba, Aj, Av, dsq, bval);
    note_launch();
}

// warps per block for a given shared-memory need per warp
int sgs_warps_per_block(int cap, int vbytes) {
    const long long per = (long long)cap * vbytes;
    if (per <= 0) return 8;
    long long w = (96 * 1024) / per;
    if (w > 8) w = 8;
    if (w < 1) w = 1;
    return (int)w;
}

template <class T>
void launch_sgs_sweep(const Launch &L, const SgsOps<T> &s, const T *R, T *Z, const DevState *st) {
    if (s.ngroups <= 0) return;
    const int wpb = sgs_warps_per_block(s.cap, (int)sizeof(T));
    const int threads = 32 * wpb;
    const size_t smem = (size_t)wpb * s.cap * sizeof(T);
    const bool one = s.gmax <= 1;
    static int attr_set[2] = {0, 0};
    const int ti = sizeof(T) == 4 ? 0 : 1;
    if (!attr_set[ti]) {
        // opt in to more than 48 KB of dynamic shared memory per block
        cudaFuncSetAttribute(k_sgs_sweep<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
        cudaFuncSetAttribute(k_sgs_sweep<T, kSgsMaxCols>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaGetLastError();
        attr_set[ti] = 1;
    }
    int per_sm = 1;
    if ((one ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sgs_sweep<T, 1>, threads,
                                                             smem)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                   &per_sm, k_sgs_sweep<T, kSgsMaxCols>, threads, smem)) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    long long blocks = ((long long)s.ngroups + wpb - 1) / wpb;
    const long long resident = (long long)L.nsm * per_sm;
    if (blocks > resident) blocks = resident;
    if (one)
        k_sgs_sweep<T, 1><<<(int)blocks, threads, smem, L.stream>>>(
            s.ngroups, s.hdr, s.rpos, s.flvl, s.frow, s.foptr, s.fidx, s.fval, s.blvl, s.brow,
            s.boptr, s.bidx, s.bval, R, Z, st, s.cap);
    else
        k_sgs_sweep<T, kSgsMaxCols><<<(int)blocks, threads, smem, L.stream>>>(
            s.ngroups, s.hdr, s.rpos, s.flvl, s.frow, s.foptr, s.fidx, s.fval, s.blvl, s.brow,
            s.boptr, s.bidx, s.bval, R, Z, st, s.cap);
    note_launch();
}

template void launch_sgs_values<float>(const Launch &, const SgsOps<float> &, const int *,
                                       const int *, const int *, const int *, const int *,
                                       const double *, const double *, float *, float *);
template void launch_sgs_values<double>(const Launch &, const SgsOps<double> &, const int *,
                                        const int *, const int *, const int *, const int *,
                                        const double *, const double *, double *, double *);
template void launch_sgs_sweep<float>(const Launch &, const SgsOps<float> &, const float *,
                                      float *, const DevState *);
template void launch_sgs_sweep<double>(const Launch &, const SgsOps<double> &, const double *,
                                       double *, const DevState *);

}  // namespace emin
