// Internal declarations shared by the CUDA translation units of libemin.
//
// Data layout in device memory (all arrays library-owned):
//   A      CSR: rowptr int32[n+1], col int32[nnz(A)], val f64[nnz(A)]
//          (+ f32 copy in mixed precision)
//   P      CSR pattern: rowptr int32[n+1], col int32[nnz(P)]; every vector of
//          the iteration (R, Y, Y_, dW, P0) is a value array on this pattern
//   B      f64[n*k] row-major; Bc f64[nc*k] row-major (+ f32 copy)
//   Ginv   per row, the inverse (or pseudo-inverse) of the Gram matrix
//          G_i = B_i^T B_i, packed lower triangle, f64[n*k(k+1)/2] (+ f32)
//   dinv   1/A(i,i), f64[n] and f32[n]
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include <cstddef>
#include <cstdint>

#include "../../include/emin.h"

namespace emin {

constexpr int kMaxK = 8;           // near-kernel vectors per row
constexpr int kMaxRowP = 1024;     // entries of a row of P (warp kernel staging)
constexpr int kBlock = 256;        // threads per block of every kernel
constexpr int kMaxGrid = 8192;     // blocks of a reducing kernel (partials buffer)
constexpr double kRankTol = 1e-12; // pivot tolerance relative to max diag(G_i)
constexpr double kGammaFloor = 1e-28;

// device-side error flags (bit set) found while validating / setting up
enum : int {
    F_ROWPTR = 1,     // row pointers not monotone or out of range
    F_COL = 2,        // a column index out of range
    F_ORDER = 4,      // columns not strictly ascending in a row
    F_DIAG = 8,       // A(i,i) missing, not positive or not finite
    F_RANK = 16,      // rank-deficient Gram matrix (strict policy)
    F_NONFINITE = 32, // non-finite value in A, B, Bc or P0
    F_ROWLEN = 64,    // a row of P longer than kMaxRowP
};

// Scalars of one restricted PCG run (Algorithm 3), resident on the device.
struct DevState {
    double gamma;        // r^T z of the current residual
    double gamma_old;
    double alpha;        // gamma / y^T y_
    double beta;         // gamma / gamma_old (0 before the first step)
    double ydy;          // y^T y_
    double dE1;          // dE of the first computed iteration
    double dE_last;
    double gamma_floor;  // convergence floor of gamma
    double tau;          // tolerance of Eq. (relRed)
    double aux;          // result of a stand-alone reduction (energy, ...)
    int k;               // iterations computed since (re)start
    int applied;         // steps applied since (re)start
    int stop;            // 0 running, 1 converged, 2 error
    int status;          // emin_status of a device-detected error
    int loop_left;       // iterations left in the current call (graph while-loop)
    unsigned int ticket[4];
};

// reduction targets of the masked-product kernel
// (DOT_START: the start of Algorithm 3 on the packed k = 1 plan, see
// launch_kprod_start)
enum DotMode : int { DOT_NONE = 0, DOT_ALPHA = 1, DOT_AUX = 2, DOT_START = 3 };
// modes of the update kernel: UPD_STEP applies the step and forms gamma =
// <r~, r~> (Jacobi: z = r); UPD_INIT forms gamma_0; UPD_FLOOR sets the
// convergence floor from the residual; with another preconditioner the step
// (UPD_XR, no reduction) and gamma = <r~, z~> (UPD_GZ_INIT / UPD_GZ_STEP,
// after z is formed) are separate passes
enum UpdMode : int {
    UPD_INIT = 0, UPD_STEP = 1, UPD_FLOOR = 2, UPD_XR = 3, UPD_GZ_INIT = 4, UPD_GZ_STEP = 5
};

// One restricted PCG workspace in value type T.
template <class T>
struct Work {
    T *R = nullptr, *Y = nullptr, *Yb = nullptr, *X = nullptr;
    T *Z = nullptr;  // preconditioned residual (SGS only; Jacobi uses z = r)
    DevState *st = nullptr;
    double *partials = nullptr;
    double *hist = nullptr;
    int hist_cap = 0;
    // the captured iteration loop (CUDA graph) for gn iterations
    cudaGraphExec_t gexec = nullptr;
    int gn = -1, gtimed = -1;
    long long gexec_launches = 0;  // kernels in the unrolled graph
    // one iteration as the body of a conditional while node: runs until the
    // call's count is used up or the stop test fires, for any count
    cudaGraphExec_t gwhile = nullptr;
    int gwhile_per_pass = 0;  // kernels in one pass of the while body
};

// The projected block SGS plan on the device (see sgs.cu).
// Level path: per group a header of 12 ints (rows m, columns G, first plan
// row r0, index blob offset and length in 16-byte units, first forward /
// backward coupling, coupling counts, level counts, first column), per plan
// row the position of its first entry, the uint16 index blobs, and the
// coupling values A^ of both sweeps in group order.
// Batched path: classes of structurally identical one-column groups, 32
// groups (lanes) per batch, one CTA per batch; per class a header of 8 ints
// (rows m, couplings nv, forward / backward level counts, word offset of
// its sweep structure, forward / backward row counts, its padded length in
// words), per batch 4 ints (class, first position, first value, 0), the
// positions on P's pattern and the coupling values interleaved by lane.
// Batches are launched in up to two buckets of similar shared-memory size.
struct SgsBucket {
    int b0 = 0, b1 = 0;          // batch range
    int umax = 0, vmax = 0;      // largest m and nv of the bucket's classes
    int wmax = 0;                // largest sweep structure (words) of its classes
    int grid32 = 0, grid64 = 0;  // CTAs (float / double launch)
};
constexpr int kSgsBuckets = 2;
constexpr int kSgsWarps = 8;  // warps of a batched-sweep CTA

template <class T>
struct SgsOps {
    int nbatch = 0, nbucket = 0;
    SgsBucket bucket[kSgsBuckets];
    const int *cls_hdr = nullptr, *bat_hdr = nullptr, *bat_rpos = nullptr;
    const unsigned *cls_blob = nullptr;
    const T *bat_val = nullptr;
    long long nbat_rpos = 0, nbat_val = 0, ncls_blob = 0;
    // gamma formed by the batched sweep and the projection applied in the
    // direction update (k = 1, every group batched)
    bool fused = false;
    int ngroups = 0;
    int cap = 0;                 // largest m * G
    int gmax = 0;                // largest G
    long long stage32 = 0, stage64 = 0;  // largest staged group (bytes, float / double)
    const int *hdr = nullptr, *rpos = nullptr;
    const uint4 *blob = nullptr;
    const T *fval = nullptr, *bval = nullptr;
    int *chk = nullptr;  // bounds checks: the context's check word (null: off)
    long long ny = 0;    // entries of the vectors on P's pattern
    bool active() const { return nbatch > 0 || ngroups > 0; }
};

// The staged node-block product (nbs_kernels.cu): tiles of whole nodes, per
// tile two int4 headers ({blob offset16, blob len16, first run, runs},
// {pairs, nodes, aggregates, Y len16}), the runs of rows of Y to stage
// ({src16, len16, dst16, 0}, in 16-byte units of Y and of the staging area),
// and the fill lists that put the values of A^, Ginv and B_c into the blob
// at every set-up.
struct NbsOps {
    int ntiles = 0, W = 0, stage_cap16 = 0, per_sm = 0;  // largest tile: blob + zero block + Y
    long long blob16 = 0;                                 // 16-byte units of the blob
    const int4 *hdr = nullptr, *runs = nullptr;
    const int4 *fill_pair = nullptr;
    const int2 *fill_node = nullptr, *fill_agg = nullptr;
    long long nfill_pair = 0, nfill_node = 0, nfill_agg = 0;
};

struct NbsHost {
    int W = 4, ntiles = 0, esize = 4, stage_cap16 = 0;
    std::vector<int4> hdr, runs, fill_pair;
    std::vector<int2> fill_node, fill_agg;
    std::vector<uint4> blob;  // static records (values zero)
};

// Everything a masked-product launch needs to know about the problem.
// Av is either A itself (plain products: energy, adjoint right-hand sides)
// or the symmetrically scaled A^ = D^{-1/2} A D^{-1/2} the iteration runs
// on.  qv and the sell_* arrays are the k = 1 plan (null when there is none).
template <class T>
struct Ops {
    int n, nc, k;
    const int *Ap, *Aj;
    const T *Av;
    const int *Pp, *Pj;
    const T *Bc;
    const T *Ginv;
    const T *qv;                  // k = 1: b / |b| per entry of P (the Q of Pi_B = I - q q^T)
    // the k = 1 plan in SELL-32 order (slices of 32 rows, entry j of the 32
    // rows contiguous, rows padded to the slice's longest): sell_ptr[s] is
    // the first position of slice s; sa holds A^ at those positions
    const int *sell_ptr;
    const T *sa;
    const int *soff;
    const unsigned short *smap;
    // packed form of the same plan: per entry one word (o - p0_i) << 12 | map,
    // o the offset of row l of P and p0_i that of the entry's own row (null
    // when some offset difference does not fit 20 bits); for float the value
    // and the word are interleaved (spk), for double they are separate (sa, sw)
    const unsigned int *sw;
    const uint2 *spk;
    // node-block plan (3 dofs per node, k = 6): per stored 3 x 3 block (v,b)
    // the offset and row length of node b's rows of P and the slot map
    const int *boff;
    const unsigned short *blen;
    const unsigned int *bmap;
    // warp tiles of output blocks (node v, slot s) coded v << 3 | s, -1 padding
    const int *tile_map;
    int ntiles;
    int maxrow;                   // longest row of P
    int lanes;                    // lanes per row of the row kernels (1 or 32)
    SgsOps<T> sgs;                // projected block SGS (ngroups 0: Jacobi)
    NbsOps nbs;                   // staged node-block product (ntiles 0: none)
    const T *nbs_blob = nullptr;  // its blob in this precision (null: not formed)
    // bounds checks (emin_opts.checks): the context's check word, null when off;
    // nnz_p bounds every gather of a vector on P's pattern
    int *chk = nullptr;
    long long nnz_p = 0;
};

struct Launch {
    cudaStream_t stream;
    int grid_rows;    // grid of thread-per-row kernels
    int grid_warps;   // grid of warp-per-row kernels
    int grid_staged;  // resident grid of the staged masked product
    int nsm;          // streaming multiprocessors of the device
    int grid_flat32;  // resident grids of the flat vector streams (float, double)
    int grid_flat64;
};

// shared-memory slots per warp for a row of P: the longest row rounded up
// to a multiple of 32 (at least 32, at most kMaxRowP)
inline int staging_cap(int maxrow) {
    int c = ((maxrow + 31) / 32) * 32;
    if (c < 32) c = 32;
    return c > kMaxRowP ? kMaxRowP : c;
}

// process-wide count of kernels launched by the library (instrumentation)
void note_launch();
void note_launches(long long k);  // k may be negative (launches captured, not run)
long long launches_so_far();

// ---- set-up kernels (setup_kernels.cu) ----
void launch_validate_csr(const Launch &L, int nrows, int ncols, const int *rowptr, int nnz,
                         const int *col, int *flags, int *maxrow);
void launch_check_finite(const Launch &L, const double *v, long long count, int *flags);
void launch_diag(const Launch &L, int n, const int *Ap, const int *Aj, const double *Av,
                 double *dinv64, float *dinv32, int *flags);
// rep: consecutive rows sharing their columns of P (3 for node-blocked
// problems, else 1); their Gram matrix is factorised once
void launch_gram(const Launch &L, int n, int k, const int *Pp, const int *Pj, const double *Bc,
                 double *Ginv, float *Ginv32, int policy, int *flags, int *ndef, int rep);
// P = base + f_i * add (add64 or add32, f may be null = 1), then, if
// `correct`, the least-norm constraint correction of every row
void launch_restore(const Launch &L, int n, int k, const int *Pp, const int *Pj,
                    const double *Bc, const double *B, const double *Ginv, const double *base,
                    const double *add64, const float *add32, const double *f, int correct,
                    double *P);
void launch_to_float(const Launch &L, const double *src, float *dst, long long count);
void launch_to_double(const Launch &L, const float *src, double *dst, long long count);

void launch_diag_scales(const Launch &L, int n, const double *dinv, double *dsq, double *dhalf);
// whole k = 1 set-up per row (rows of P with at most 4 entries); see
// setup_kernels.cu.  dsq32 (float path, may be null) receives D^{-1/2} as the
// float it is taken in
template <class Tit>
void launch_setup_k1(const Launch &L, int n, const int *dpos, const double *Av, const int *Pp,
                     const int *Pj, const double *Bc, const double *B, const double *P0_in,
                     int policy, int *flags, int *ndef, double *dsq, double *dhalf, float *dsq32,
                     double *Ginv, Tit *qv, double *P0, Tit *x0);
// P = P0 + D^{-1/2} X (+ least-norm constraint correction), k = 1, rows <= 4
template <class Tx>
void launch_final_k1(const Launch &L, int n, const int *Pp, const int *Pj, const double *Bc,
                     const double *Ginv, const double *P0, const Tx *X, const double *dsq,
                     const double *B, int correct, double *P);
// SELL-32 plan: slice lengths (longest row of A per 32 rows), then the plan
// in slice order once sell_ptr (exclusive scan of 32 * length) is known
void launch_sell_len(const Launch &L, int n, const int *Ap, int *slen);
// slice lengths -> slice starts in place, the entry count into *total (device)
void launch_sell_scan(const Launch &L, int ns, int *sptr, long long *total);
// sw may be null (no packed words); *wide is set when an offset difference
// does not fit the packed word
void launch_sell_plan(const Launch &L, int n, const int *Ap, const int *Aj, const int *Pp,
                      const int *Pj, const int *sell_ptr, int *soff, unsigned short *smap,
                      unsigned int *sw, int *wide, int *dpos, long long nsell, int *chk);
// A^ in plan order into sa, or (float, spk non-null) interleaved with the
// packed words sw into spk; dsq32 (float, may be null): D^{-1/2} as floats
// (when dsq holds float-exact values), read instead of narrowing dsq
template <class T>
void launch_sell_values(const Launch &L, int n, const int *Ap, const int *Aj, const double *Av,
                        const double *dsq, const int *sell_ptr, T *sa,
                        const unsigned int *sw = nullptr, uint2 *spk = nullptr,
                        const float *dsq32 = nullptr);
template <class T>
void launch_scale_a(const Launch &L, int n, const int *Ap, const int *Aj, const double *Av,
                    const double *dsq, T *Ahat);
template <class T>
void launch_qvec_k1(const Launch &L, int n, const int *Pp, const int *Pj, const double *Bc, T *qv);

// ---- iteration kernels (iter_kernels.cu) ----
template <class T>
void launch_kprod(const Launch &L, const Ops<T> &o, const T *Y, T *out, int project,
                  int dot_mode, Work<T> &w, int check_stop);
template <class T>
void launch_project(const Launch &L, const Ops<T> &o, T *x, T scale);
// The start of Algorithm 3 in one launch when the packed k = 1 plan serves
// the product: R = -Pi mask(A^ x0), the convergence floor from the
// unprojected product and (gamma0 != 0, Jacobi) gamma_0 = <R, R>.  Returns
// false (nothing launched) for any other plan.
template <class T>
bool launch_kprod_start(const Launch &L, const Ops<T> &o, const T *x0, T *R, Work<T> &w,
                        int gamma0);
template <class T>
void launch_ydir(const Launch &L, long long count, Work<T> &w);
template <class T>
void launch_update(const Launch &L, long long count, Work<T> &w, int mode);
// out[s] = (Tout)(scale * f[i] * in[s]) for every entry s of row i
template <class Tin, class Tout>
void launch_row_scale(const Launch &L, int n, const int *Pp, int lanes, const double *f,
                      double scale, const Tin *in, Tout *out);
void launch_state_reset(const Launch &L, DevState *st);
void set_iter_attributes();
int staged_blocks_per_sm();
// resident blocks per SM of the packed product's iteration launch; also makes
// every instantiation's occupancy query at create, outside any graph capture
int pk_blocks_per_sm(int double_precision);
int flat_blocks_per_sm(int double_precision);

// projected block SGS (sgs.cu)
struct SgsHost {
    // level path (groups without enough structural twins)
    int ngroups = 0, cap = 0, gmax = 0;
    long long stage32 = 0, stage64 = 0;
    std::vector<int> hdr, rpos, fown, fa, bown, ba;
    std::vector<unsigned short> blob;
    // batched path: classes of identical structure, batches of 32 groups
    int nbatch = 0, nbucket = 0;
    SgsBucket bucket[kSgsBuckets];
    std::vector<int> cls_hdr, bat_hdr, bat_rpos, bat_own, bat_ent;
    std::vector<unsigned> cls_blob;
};
int build_sgs_plan(int n, int nc, const int *Ap, const int *Aj, const int *Pp, const int *Pj,
                   SgsHost &out);
template <class T>
void launch_sgs_values(const Launch &L, const int *fown, const int *fa, long long nf,
                       const int *bown, const int *ba, long long nb, const int *Aj,
                       const double *Av, const double *dsq, T *fval, T *bval);
// with the packed k = 1 plan: the batched couplings' A entries turned into
// plan positions (once), and their values read from A^ in plan order
void launch_sgs_sell_pos(const Launch &L, long long nops, const int *own, int *ent,
                         const int *Ap, const int *sell_ptr);
template <class T>
void launch_sgs_values_sell(const Launch &L, long long nops, const int *own, const int *pos,
                            const T *sa, const uint2 *spk, T *val);
// z~ <- Pi z~ and gamma = <r~, z~> after the sweep (init: gamma_0)
template <class T>
void launch_sgs_finish(const Launch &L, const Ops<T> &o, Work<T> &w, int init, long long nnz_p);
// z~ = (L^ + I)^{-T} (L^ + I)^{-1} r~ over every group; with s.fused the
// batched sweep also forms gamma = |(L^ + I)^{-1} r~|^2 (init: gamma_0)
template <class T>
void launch_sgs_sweep(const Launch &L, const SgsOps<T> &s, const T *R, T *Z, DevState *st,
                      double *partials, int init);
// CTAs per bucket of the batched sweep (once per plan, outside any capture)
int sgs_prepare(int nsm, SgsHost &h);
// y~ = Pi z~ + beta y~ (k = 1), the direction step of the fused SGS path
template <class T>
void launch_ydir_proj_k1(const Launch &L, int n, int maxrow, const int *Pp, const T *qv,
                         const T *Z, T *Y, const DevState *st);
void set_adjoint_attributes();
void launch_state_begin(const Launch &L, DevState *st, double tau, int n_iters);
// the while-loop control of the captured iteration graph (one thread)
void launch_loop_control(const Launch &L, DevState *st, cudaGraphConditionalHandle h);

// ---- node-block kernels (block_kernels.cu) ----
// returns 1 if it launched the structure test (flag in *bad), 0 if the
// problem cannot be node-blocked (k != 6 or n not a multiple of 3)
int launch_detect_blocks(const Launch &L, int n, int k, const int *Ap, const int *Aj,
                         const int *Pp, const int *Pj, int *bad);
void launch_block_plan(const Launch &L, int n, const int *Ap, const int *Aj, const int *Pp,
                       const int *Pj, int *boff, unsigned short *blen, unsigned int *bmap,
                       long long nentries, int *chk);
long long block_plan_entries(long long nnz_a);
void launch_node_slots(const Launch &L, int n, const int *Pp, int *na);
template <class T>
void launch_kprod_blk(const Launch &L, const Ops<T> &o, const T *Y, T *out, int project,
                      int dot_mode, Work<T> &w, int check_stop);

// ---- staged node-block product (nbs_kernels.cu) ----
// tiles of at most W warps and `budget` bytes of blob plus staged rows of Y;
// esize = sizeof(T) of the precision the blob is built for.  EMIN_ERR_ARG if
// the problem does not fit the scheme (then the node-block product serves).
int build_nbs_plan(int n, const int *Ap, const int *Aj, const int *Pp, const int *Pj, int esize,
                   int W, long long budget, NbsHost &h);
long long tile_len16_host(int esize, int W, int npairs, int nnodes, int naggs);
template <class T>
void launch_nbs_fill(const Launch &L, const NbsOps &nb, const int *Ap, const int *Aj,
                     const double *Av, const double *dsq, const double *Ginv, const double *Bc,
                     T *blob);
template <class T>
int nbs_prepare(const NbsOps &nb);
template <class T>
void launch_kprod_nbs(const Launch &L, const NbsOps &nb, const T *blob, const T *Y, T *out,
                      int project, int dot_mode, Work<T> &w, int check_stop, int *chk,
                      long long ny, int gamma0 = 0);

// ---- adjoint kernels (adjoint_kernels.cu) ----
void launch_outer(const Launch &L, int n, const int *Ap, const int *Aj, const int *Pp,
                  const int *Pj, const double *U, const double *V, double scale, double *out,
                  int maxrow);
void launch_lsq(const Launch &L, int n, int k, const int *Pp, const int *Pj, const double *Bc,
                const double *Ginv, const double *x, double *mu);
void launch_axpby(const Launch &L, long long count, double a, const double *x, double b,
                  double *y);
// <x, y> into st->aux
void launch_dot_aux(const Launch &L, long long count, const double *x, const double *y,
                    DevState *st, double *partials);
// out[i] += scale * dsq_i^pw * sum over row i of P of u v
void launch_row_dot_acc(const Launch &L, int n, const int *Pp, const double *u, const double *v,
                        const double *dsq, int pw, double scale, double *out);
// gradient with respect to the stored values of A from the one with
// respect to A^ = D^{-1/2} A D^{-1/2} and the extra diagonal terms dext
void launch_grad_a(const Launch &L, int n, const int *Ap, const int *Aj, const double *Av,
                   const double *dsq, const double *ghat, const double *dext, double *gA);

}  // namespace emin
