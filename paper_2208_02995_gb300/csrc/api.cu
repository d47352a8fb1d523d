// Host side of libemin: the C ABI of include/emin.h.  Owns every device
// buffer, validates inputs, sequences the set-up (Algorithm 2), the
// restricted PCG iterations (Algorithm 3), the final prolongation and the
// implicit adjoint.  All device work runs on the context's stream.
#include <cuda_runtime.h>

#include <cmath>

#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "emin_internal.cuh"

using namespace emin;

struct emin_ctx {
    int n = 0, nc = 0, k = 0;
    long long nnz_a = 0, nnz_p = 0;
    emin_opts opts{};
    cudaStream_t stream = nullptr;
    int device = 0;
    Launch L{};
    int maxrow_p = 0;
    int lanes = 1;
    int ndef = 0;
    int sticky = EMIN_OK;  // device-detected error, reported by every later call
    // inputs (library-owned copies)
    int *Ap = nullptr, *Aj = nullptr, *Pp = nullptr, *Pj = nullptr;
    double *Av = nullptr, *P0_in = nullptr, *P0 = nullptr, *B = nullptr, *Bc = nullptr;
    float *Bc32 = nullptr;
    // set-up products
    double *Ginv = nullptr, *dinv = nullptr, *dsq = nullptr, *dhalf = nullptr, *rn = nullptr;
    bool fast_k1 = false;  // k = 1, rows of P <= 4: fused set-up / final kernels and SELL plan
    float *Ginv32 = nullptr, *dinv32 = nullptr;
    float *dsq32 = nullptr;  // D^{-1/2} as floats (mixed k = 1 fast path)
    // the iteration runs on A^ = D^{-1/2} A D^{-1/2} (float and/or double)
    float *Ah32 = nullptr, *qv32 = nullptr;
    double *Ah64 = nullptr, *qv64 = nullptr;
    bool have64 = false;  // Ah64 / qv64 formed for the current values
    // k = 1 plan of the fixed pattern (built once per context), SELL-32 order
    int *sell_ptr = nullptr, *soff = nullptr, *dpos = nullptr;
    unsigned short *smap = nullptr;
    unsigned int *sw = nullptr;  // packed words (null: some offset difference is too wide)
    uint2 *spk32 = nullptr;      // float values interleaved with the packed words
    float *sa32 = nullptr;
    double *sa64 = nullptr;
    long long nnz_sell = 0;
    // node-block plan (3 dofs per node, k = 6)
    int *boff = nullptr;
    unsigned short *blen = nullptr;
    unsigned int *bmap = nullptr;
    int *tile_map = nullptr;
    int ntiles = 0;
    // staged node-block product (nbs_kernels.cu): plan and the blob of the
    // context's iteration precision (float in EMIN_MIXED, double in EMIN_FP64)
    NbsOps nbs;
    int4 *nbs_hdr = nullptr, *nbs_runs = nullptr, *nbs_fill_pair = nullptr;
    int2 *nbs_fill_node = nullptr, *nbs_fill_agg = nullptr;
    uint4 *nbs_blob = nullptr;
    // projected block SGS plan (EMIN_SGS), built once per context
    int sgs_ngroups = 0, sgs_cap = 0, sgs_gmax = 0;
    long long sgs_nf = 0, sgs_nb = 0, sgs_stage32 = 0, sgs_stage64 = 0;
    int *sgs_hdr = nullptr, *sgs_rpos = nullptr;
    int *sgs_fown = nullptr, *sgs_fa = nullptr, *sgs_bown = nullptr, *sgs_ba = nullptr;
    unsigned short *sgs_blob = nullptr;
    int sgs_nbatch = 0, sgs_nbucket = 0;
    SgsBucket sgs_bucket[kSgsBuckets];
    long long sgs_nbval = 0, sgs_nbrpos = 0, sgs_ncls_blob = 0;
    int *sgs_cls_hdr = nullptr, *sgs_bat_hdr = nullptr, *sgs_bat_rpos = nullptr;
    int *sgs_bat_own = nullptr, *sgs_bat_ent = nullptr;
    unsigned *sgs_cls_blob = nullptr;
    float *sgs_batval32 = nullptr;
    double *sgs_batval64 = nullptr;
    bool sgs_sellpos = false;  // bat_ent holds plan positions (values read from A^ in plan order)
    float *sgs_fval32 = nullptr, *sgs_bval32 = nullptr;
    double *sgs_fval64 = nullptr, *sgs_bval64 = nullptr;
    double *Pstar = nullptr, *t64c = nullptr;
    // restricted PCG workspaces
    Work<double> w64;   // forward, EMIN_FP64
    Work<float> w32;    // forward, EMIN_MIXED
    Work<double> adj;   // adjoint (always double), allocated on first use
    Work<double> aux;   // stand-alone reductions (energy)
    // scratch
    double *t64a = nullptr, *t64b = nullptr, *tA = nullptr, *tmu = nullptr;
    // unrolled adjoint: vectors on P's pattern (checkpoints, segment, work)
    std::vector<double *> unr;
    double *unr_ghat = nullptr, *unr_dext = nullptr, *unr_gA = nullptr;
    float *t32a = nullptr, *t32b = nullptr;
    int *dint = nullptr;       // [0] flags, [1] longest row of P, [2] rank-deficient rows
    int *chkw = nullptr;       // bounds-check word (emin_opts.checks), never cleared
    DevState *hstate = nullptr;  // pinned mirror
    int *hint = nullptr;         // pinned mirror of dint
    int applied_seen = 0;
    std::vector<void *> dev_allocs;
    cudaMemPool_t pool = nullptr;  // stream-ordered pool of dev_allocs (null: cudaMalloc)
    void *host_dev = nullptr;      // the pinned host block's device mapping (null: none)
    // create from host arrays: the value arrays are copied on a second
    // stream while the context's stream validates the pattern and builds
    // the plan
    cudaStream_t side = nullptr;
    cudaEvent_t side_ev = nullptr;
    void *host_blk = nullptr;      // pinned block holding hstate and hint
    // instrumentation
    int timing = 0;  // 0 off, else time the masked product of every timing-th iteration
    std::vector<cudaEvent_t> events;  // start/stop pairs, one per timed launch
    double tms[3] = {0, 0, 0};
    long long tlaunch[3] = {0, 0, 0};
    long long launches_at_create = 0;
};

namespace emin {
static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace emin

namespace {

thread_local char g_last_error[256] = "";

int with_checks(emin_ctx *c, int st);  // below: the bounds-check word after a call

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Device memory of every context comes from one stream-ordered pool per
// device that keeps what is freed (release threshold: unlimited): a context
// created after another of similar size maps no new pages, and a destroyed
// context returns its memory without a device-wide synchronisation.
// emin_trim_memory() gives the cached memory back to the driver.
constexpr int kMaxDevices = 64;
std::mutex g_pool_mutex;
cudaMemPool_t g_pools[kMaxDevices] = {};
std::vector<void *> g_host_blocks;  // recycled pinned blocks (kHostBlock bytes)
constexpr size_t kHostBlock = 256;
constexpr size_t kHintOffset = 128;
constexpr int kHintChk = 8;  // the mirror of the check word: hint[kHintChk]
constexpr int kHintTotal = 10;  // a 64-bit count read back at creation: hint[10..11]
static_assert(sizeof(DevState) <= kHintOffset, "state mirror overlaps the flag mirror");

cudaMemPool_t device_pool(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mutex);
    if (!g_pools[dev]) {
        int supported = 0;
        if (cudaDeviceGetAttribute(&supported, cudaDevAttrMemoryPoolsSupported, dev) !=
                cudaSuccess ||
            !supported) {
            cudaGetLastError();
            return nullptr;
        }
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        unsigned long long keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pools[dev] = pool;
    }
    return g_pools[dev];
}

void *host_block_get() {
    {
        std::lock_guard<std::mutex> lk(g_pool_mutex);
        if (!g_host_blocks.empty()) {
            void *b = g_host_blocks.back();
            g_host_blocks.pop_back();
            return b;
        }
    }
    void *b = nullptr;
    if (cudaMallocHost(&b, kHostBlock) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return b;
}

void host_block_put(void *b) {
    if (!b) return;
    std::lock_guard<std::mutex> lk(g_pool_mutex);
    g_host_blocks.push_back(b);
}

void release_dev(emin_ctx *c, void *p) {
    if (c->pool) cudaFreeAsync(p, c->stream);
    else cudaFree(p);
}

template <class T>
int dalloc(emin_ctx *c, T **p, long long count) {
    size_t bytes = (size_t)(count > 0 ? count : 1) * sizeof(T);
    bytes = (bytes + 255) & ~(size_t)255;
    void *q = nullptr;
    const cudaError_t e =
        c->pool ? cudaMallocFromPoolAsync(&q, bytes, c->pool, c->stream) : cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        std::snprintf(g_last_error, sizeof(g_last_error), "device allocation of %zu bytes: %s",
                      bytes, cudaGetErrorName(e));
        cudaGetLastError();
        return EMIN_ERR_NOMEM;
    }
    c->dev_allocs.push_back(q);
    *p = static_cast<T *>(q);
    return EMIN_OK;
}

// releases one allocation made by dalloc before the context is destroyed
template <class T>
void dfree(emin_ctx *c, T *&p) {
    if (!p) return;
    for (size_t i = 0; i < c->dev_allocs.size(); ++i)
        if (c->dev_allocs[i] == static_cast<void *>(p)) {
            release_dev(c, c->dev_allocs[i]);
            c->dev_allocs.erase(c->dev_allocs.begin() + (long)i);
            break;
        }
    p = nullptr;
}

int cuda_status_at(cudaError_t e, const char *where) {
    if (e == cudaSuccess) return EMIN_OK;
    std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", where, cudaGetErrorName(e),
                  cudaGetErrorString(e));
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? EMIN_ERR_NOMEM : EMIN_ERR_CUDA;
}

#define cuda_status(e) cuda_status_at((e), __func__)

int check_launch_at(const char *where) { return cuda_status_at(cudaGetLastError(), where); }
#define check_launch() check_launch_at(__func__)

#define EMIN_TRY(expr)                   \
    do {                                 \
        int _s = (expr);                 \
        if (_s != EMIN_OK) return _s;    \
    } while (0)

int copy_in(emin_ctx *c, void *dst, const void *src, size_t bytes, int on_device) {
    if (bytes == 0) return EMIN_OK;
    if (!src) return EMIN_ERR_ARG;
    return cuda_status(cudaMemcpyAsync(dst, src, bytes,
                                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                       c->stream));
}

int copy_out(emin_ctx *c, void *dst, const void *src, size_t bytes, int on_device) {
    if (bytes == 0) return EMIN_OK;
    if (!dst) return EMIN_ERR_ARG;
    return cuda_status(cudaMemcpyAsync(dst, src, bytes,
                                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                       c->stream));
}

int sync(emin_ctx *c) { return cuda_status(cudaStreamSynchronize(c->stream)); }

__global__ void k_fetch_words(const unsigned *__restrict__ src, unsigned *dst, int nwords) {
    for (int i = threadIdx.x; i < nwords; i += blockDim.x) dst[i] = src[i];
}

// A few words of device memory into the context's pinned host block: stored
// by a one-warp kernel through the block's device mapping when there is one
// (no copy engine, so the read does not wait behind bulk host-to-device
// copies in flight on another stream), else by cudaMemcpyAsync.  Complete
// after the next sync.
int fetch_words(emin_ctx *c, void *hdst, const void *dsrc, size_t bytes) {
    const size_t off = (size_t)(static_cast<char *>(hdst) - static_cast<char *>(c->host_blk));
    if (c->host_dev && bytes % 4 == 0 && off + bytes <= kHostBlock &&
        reinterpret_cast<uintptr_t>(dsrc) % 4 == 0) {
        unsigned *d = reinterpret_cast<unsigned *>(static_cast<char *>(c->host_dev) + off);
        k_fetch_words<<<1, 32, 0, c->stream>>>(static_cast<const unsigned *>(dsrc), d,
                                               (int)(bytes / 4));
        note_launch();
        return check_launch();
    }
    return cuda_status(cudaMemcpyAsync(hdst, dsrc, bytes, cudaMemcpyDeviceToHost, c->stream));
}

// masked products on the unscaled A (energy, adjoint right-hand sides)
// bounds checks of the kernels (emin_opts.checks)
template <class T>
void set_checks(const emin_ctx *c, Ops<T> &o) {
    o.nnz_p = c->nnz_p;
    o.sgs.ny = c->nnz_p;
    if (c->opts.checks && c->chkw) {
        o.chk = c->chkw;
        o.sgs.chk = c->chkw;
    }
}

Ops<double> plain_ops64(const emin_ctx *c) {
    Ops<double> o{c->n, c->nc, c->k, c->Ap, c->Aj, c->Av, c->Pp, c->Pj, c->Bc, c->Ginv,
                  nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, c->boff, c->blen, c->bmap, c->tile_map, c->ntiles,
                  c->maxrow_p, c->lanes};
    set_checks(c, o);
    return o;
}

// the SGS plan with the values of one precision (an empty plan: Jacobi);
// qv (k = 1) lets a fully batched plan take the fused path
template <class T>
SgsOps<T> sgs_ops(const emin_ctx *c, const T *fval, const T *bval, const T *batval,
                  const T *qv) {
    SgsOps<T> s;
    if (c->opts.precond != EMIN_SGS || (c->sgs_ngroups <= 0 && c->sgs_nbatch <= 0)) return s;
    s.nbatch = c->sgs_nbatch;
    s.nbucket = c->sgs_nbucket;
    for (int b = 0; b < kSgsBuckets; ++b) s.bucket[b] = c->sgs_bucket[b];
    s.cls_hdr = c->sgs_cls_hdr;
    s.bat_hdr = c->sgs_bat_hdr;
    s.bat_rpos = c->sgs_bat_rpos;
    s.cls_blob = c->sgs_cls_blob;
    s.bat_val = batval;
    s.nbat_rpos = c->sgs_nbrpos;
    s.nbat_val = c->sgs_nbval;
    s.ncls_blob = c->sgs_ncls_blob;
    s.ngroups = c->sgs_ngroups;
    s.cap = c->sgs_cap;
    s.gmax = c->sgs_gmax;
    s.stage32 = c->sgs_stage32;
    s.stage64 = c->sgs_stage64;
    s.hdr = c->sgs_hdr;
    s.rpos = c->sgs_rpos;
    s.blob = reinterpret_cast<const uint4 *>(c->sgs_blob);
    s.fval = fval;
    s.bval = bval;
    s.fused = c->k == 1 && qv != nullptr && c->sgs_ngroups == 0 && c->sgs_nbatch > 0;
    return s;
}

// the iteration's operator A^ with its plan
Ops<double> iter_ops64(const emin_ctx *c) {
    Ops<double> o{c->n, c->nc, c->k, c->Ap, c->Aj, c->Ah64, c->Pp, c->Pj, c->Bc, c->Ginv,
                       c->qv64, c->sell_ptr, c->sa64, c->soff, c->smap, c->sw, nullptr, c->boff, c->blen, c->bmap, c->tile_map, c->ntiles,
                       c->maxrow_p, c->lanes};
    o.sgs = sgs_ops<double>(c, c->sgs_fval64, c->sgs_bval64, c->sgs_batval64, c->qv64);
    if (c->nbs_blob && c->opts.precision == EMIN_FP64) {
        o.nbs = c->nbs;
        o.nbs_blob = reinterpret_cast<const double *>(c->nbs_blob);
    }
    set_checks(c, o);
    return o;
}

Ops<float> iter_ops32(const emin_ctx *c) {
    // (A^ in CSR order is not formed when the staged product serves: null)
    Ops<float> o{c->n, c->nc, c->k, c->Ap, c->Aj, c->nbs_blob ? nullptr : c->Ah32, c->Pp, c->Pj, c->Bc32, c->Ginv32,
                      c->qv32, c->sell_ptr, c->sa32, c->soff, c->smap, c->sw, c->spk32, c->boff, c->blen, c->bmap, c->tile_map, c->ntiles,
                      c->maxrow_p, c->lanes};
    o.sgs = sgs_ops<float>(c, c->sgs_fval32, c->sgs_bval32, c->sgs_batval32, c->qv32);
    if (c->nbs_blob && c->opts.precision == EMIN_MIXED) {
        o.nbs = c->nbs;
        o.nbs_blob = reinterpret_cast<const float *>(c->nbs_blob);
    }
    set_checks(c, o);
    return o;
}

template <class T>
int upload(emin_ctx *c, T **dst, const std::vector<T> &src);

// values of the staged product's blob (A^, Ginv, B_c) for the current set-up
void fill_nbs(emin_ctx *c) {
    if (!c->nbs_blob) return;
    if (c->opts.precision == EMIN_MIXED)
        launch_nbs_fill<float>(c->L, c->nbs, c->Ap, c->Aj, c->Av, c->dsq, c->Ginv, c->Bc,
                               reinterpret_cast<float *>(c->nbs_blob));
    else
        launch_nbs_fill<double>(c->L, c->nbs, c->Ap, c->Aj, c->Av, c->dsq, c->Ginv, c->Bc,
                                reinterpret_cast<double *>(c->nbs_blob));
}

// The staged node-block plan from host copies of both patterns (host code,
// once per context); the problem keeps the node-block product if it does not
// fit the scheme or the staged kernel cannot launch
int build_nbs(emin_ctx *c, const int *hAp, const int *hAj, const int *hPp, const int *hPj) {
    // float (EMIN_MIXED) only: the FP64 product is bound by the FP64 pipe, and
    // the node-block kernel, which skips a neighbour that does not hold the
    // lane's aggregate, issues fewer FP64 instructions than the staged one
    if (c->opts.precision != EMIN_MIXED) return EMIN_OK;
    const int esize = 4;
    NbsHost h;
    // 4 warps and about 100 KB of blob and staged rows per tile (two CTAs per SM)
    const long long budget = 100 * 1024;
    if (build_nbs_plan(c->n, hAp, hAj, hPp, hPj, esize, 4, budget, h) != EMIN_OK) return EMIN_OK;
    NbsOps nb;
    nb.ntiles = h.ntiles;
    nb.W = h.W;
    nb.stage_cap16 = h.stage_cap16;
    nb.blob16 = (long long)h.blob.size();
    nb.per_sm = esize == 4 ? nbs_prepare<float>(nb) : nbs_prepare<double>(nb);
    if (nb.per_sm <= 0) return EMIN_OK;
    EMIN_TRY(upload(c, &c->nbs_hdr, h.hdr));
    EMIN_TRY(upload(c, &c->nbs_runs, h.runs));
    EMIN_TRY(upload(c, &c->nbs_fill_pair, h.fill_pair));
    EMIN_TRY(upload(c, &c->nbs_fill_node, h.fill_node));
    EMIN_TRY(upload(c, &c->nbs_fill_agg, h.fill_agg));
    EMIN_TRY(upload(c, &c->nbs_blob, h.blob));
    nb.hdr = c->nbs_hdr;
    nb.runs = c->nbs_runs;
    nb.fill_pair = c->nbs_fill_pair;
    nb.fill_node = c->nbs_fill_node;
    nb.fill_agg = c->nbs_fill_agg;
    nb.nfill_pair = (long long)h.fill_pair.size();
    nb.nfill_node = (long long)h.fill_node.size();
    nb.nfill_agg = (long long)h.fill_agg.size();
    c->nbs = nb;
    return sync(c);  // the host vectors must outlive the transfers
}

template <class T>
int alloc_work(emin_ctx *c, Work<T> &w, bool vectors) {
    if (vectors) {
        EMIN_TRY(dalloc(c, &w.R, c->nnz_p));
        EMIN_TRY(dalloc(c, &w.Y, c->nnz_p));
        EMIN_TRY(dalloc(c, &w.Yb, c->nnz_p));
        EMIN_TRY(dalloc(c, &w.X, c->nnz_p));
        if (c->opts.precond == EMIN_SGS) EMIN_TRY(dalloc(c, &w.Z, c->nnz_p));
    }
    EMIN_TRY(dalloc(c, &w.st, 1));
    EMIN_TRY(dalloc(c, &w.partials, kMaxGrid));
    w.hist_cap = 4096;
    EMIN_TRY(dalloc(c, &w.hist, w.hist_cap));
    EMIN_TRY(cuda_status(cudaMemsetAsync(w.st, 0, sizeof(DevState), c->stream)));
    return EMIN_OK;
}

// Start of Algorithm 3 in the scaled variables: r~ = -Pi_B A^ x0~ with
// x0~ = D^{1/2} p0 (so r~ = D^{-1/2} r), the convergence floor from the
// unprojected residual, and gamma_0 = <r~, r~>.  For the adjoint x0 is null
// and the caller has put the scaled right-hand side in R.
template <class T>
int start_pcg(emin_ctx *c, const Ops<T> &o, Work<T> &w, const T *x0) {
    launch_state_reset(c->L, w.st);
    if (c->nnz_p > 0) {
        EMIN_TRY(cuda_status(cudaMemsetAsync(w.Y, 0, sizeof(T) * c->nnz_p, c->stream)));
        EMIN_TRY(cuda_status(cudaMemsetAsync(w.X, 0, sizeof(T) * c->nnz_p, c->stream)));
    }
    // on the packed k = 1 plan one launch forms r~, the floor and (Jacobi)
    // gamma_0; otherwise the product, the floor, the projection and gamma_0
    // are separate passes
    const bool sgs = o.sgs.active();
    const bool fused = x0 && launch_kprod_start<T>(c->L, o, x0, w.R, w, sgs ? 0 : 1);
    if (!fused) {
        if (x0) launch_kprod<T>(c->L, o, x0, w.R, 0, DOT_NONE, w, 0);
        launch_update<T>(c->L, c->nnz_p, w, UPD_FLOOR);
        launch_project<T>(c->L, o, w.R, x0 ? T(-1) : T(1));
    }
    if (sgs) {
        // z~_0 = Pi (L^ + I)^{-T} (L^ + I)^{-1} r~_0, gamma_0 = <r~, z~> (fused:
        // gamma_0 from the sweep, Pi in the first direction update)
        launch_sgs_sweep<T>(c->L, o.sgs, w.R, w.Z, w.st, w.partials, 1);
        if (!o.sgs.fused) launch_sgs_finish<T>(c->L, o, w, 1, c->nnz_p);
    } else if (!fused) {
        launch_update<T>(c->L, c->nnz_p, w, UPD_INIT);
    }
    return check_launch();
}

template <class T>
int dalloc_once(emin_ctx *c, T **p, long long count) {
    if (*p) return EMIN_OK;
    return dalloc(c, p, count);
}

template <class T>
int upload(emin_ctx *c, T **dst, const std::vector<T> &src) {
    EMIN_TRY(dalloc(c, dst, (long long)src.size()));
    if (!src.empty())
        EMIN_TRY(cuda_status(cudaMemcpyAsync(*dst, src.data(), sizeof(T) * src.size(),
                                             cudaMemcpyHostToDevice, c->stream)));
    return EMIN_OK;
}

// The projected block SGS plan from host copies of both patterns (the plan
// builder is host code, run once per context), uploaded to the device.
int build_sgs(emin_ctx *c) {
    const int n = c->n;
    std::vector<int> Ap(n + 1), Aj(c->nnz_a), Pp(n + 1), Pj(c->nnz_p);
    EMIN_TRY(cuda_status(cudaMemcpyAsync(Ap.data(), c->Ap, sizeof(int) * (n + 1),
                                         cudaMemcpyDeviceToHost, c->stream)));
    EMIN_TRY(cuda_status(cudaMemcpyAsync(Aj.data(), c->Aj, sizeof(int) * c->nnz_a,
                                         cudaMemcpyDeviceToHost, c->stream)));
    EMIN_TRY(cuda_status(cudaMemcpyAsync(Pp.data(), c->Pp, sizeof(int) * (n + 1),
                                         cudaMemcpyDeviceToHost, c->stream)));
    EMIN_TRY(cuda_status(cudaMemcpyAsync(Pj.data(), c->Pj, sizeof(int) * c->nnz_p,
                                         cudaMemcpyDeviceToHost, c->stream)));
    EMIN_TRY(sync(c));
    SgsHost h;
    const int st = build_sgs_plan(n, c->nc, Ap.data(), Aj.data(), Pp.data(), Pj.data(), h);
    if (st != EMIN_OK) {
        std::snprintf(g_last_error, sizeof(g_last_error),
                      "SGS plan: a column of P with more than 65535 rows or couplings");
        return st;
    }
    // one group's block must fit the shared memory of one block of one warp
    if (((long long)h.cap * (long long)sizeof(double) + 15) / 16 * 16 > 96LL * 1024) {
        std::snprintf(g_last_error, sizeof(g_last_error),
                      "SGS plan: a column group of %d values exceeds shared memory", h.cap);
        return EMIN_ERR_ARG;
    }
    c->sgs_ngroups = h.ngroups;
    c->sgs_cap = h.cap;
    c->sgs_gmax = h.gmax;
    c->sgs_stage32 = h.stage32;
    c->sgs_stage64 = h.stage64;
    EMIN_TRY(upload(c, &c->sgs_hdr, h.hdr));
    EMIN_TRY(upload(c, &c->sgs_rpos, h.rpos));
    EMIN_TRY(upload(c, &c->sgs_blob, h.blob));
    EMIN_TRY(upload(c, &c->sgs_fown, h.fown));
    EMIN_TRY(upload(c, &c->sgs_fa, h.fa));
    EMIN_TRY(upload(c, &c->sgs_bown, h.bown));
    EMIN_TRY(upload(c, &c->sgs_ba, h.ba));
    if (const int ps = sgs_prepare(c->L.nsm, h)) {
        std::snprintf(g_last_error, sizeof(g_last_error),
                      "SGS plan: the batched sweep's shared memory could not be set up");
        return ps;
    }
    c->sgs_nbatch = h.nbatch;
    c->sgs_nbucket = h.nbucket;
    for (int b = 0; b < kSgsBuckets; ++b) c->sgs_bucket[b] = h.bucket[b];
    EMIN_TRY(upload(c, &c->sgs_cls_hdr, h.cls_hdr));
    EMIN_TRY(upload(c, &c->sgs_bat_hdr, h.bat_hdr));
    EMIN_TRY(upload(c, &c->sgs_bat_rpos, h.bat_rpos));
    EMIN_TRY(upload(c, &c->sgs_bat_own, h.bat_own));
    EMIN_TRY(upload(c, &c->sgs_bat_ent, h.bat_ent));
    EMIN_TRY(upload(c, &c->sgs_cls_blob, h.cls_blob));
    c->sgs_nbval = (long long)h.bat_ent.size();
    if (c->sell_ptr && c->sgs_nbval > 0) {
        launch_sgs_sell_pos(c->L, c->sgs_nbval, c->sgs_bat_own, c->sgs_bat_ent, c->Ap,
                            c->sell_ptr);
        c->sgs_sellpos = true;
    }
    c->sgs_nbrpos = (long long)h.bat_rpos.size();
    c->sgs_ncls_blob = (long long)h.cls_blob.size();
    const long long nf = (long long)h.fa.size(), nb = (long long)h.ba.size();
    if (c->opts.precision == EMIN_MIXED) {
        EMIN_TRY(dalloc(c, &c->sgs_fval32, nf));
        EMIN_TRY(dalloc(c, &c->sgs_bval32, nb));
        EMIN_TRY(dalloc(c, &c->sgs_batval32, c->sgs_nbval));
    } else {
        EMIN_TRY(dalloc(c, &c->sgs_fval64, nf));
        EMIN_TRY(dalloc(c, &c->sgs_bval64, nb));
        EMIN_TRY(dalloc(c, &c->sgs_batval64, c->sgs_nbval));
    }
    c->sgs_nf = nf;
    c->sgs_nb = nb;
    return sync(c);  // the host vectors must outlive the transfers
}

// the SGS values A^ at the plan's couplings (level and batched paths), in
// the precision of T
template <class T>
void form_sgs_values(emin_ctx *c, T *fval, T *bval, T *batval) {
    if (c->opts.precond != EMIN_SGS) return;
    launch_sgs_values<T>(c->L, c->sgs_fown, c->sgs_fa, c->sgs_nf, c->sgs_bown, c->sgs_ba,
                         c->sgs_nb, c->Aj, c->Av, c->dsq, fval, bval);
    if (c->sgs_sellpos) {  // A^ in plan order was formed just before, in this precision
        if constexpr (sizeof(T) == 4)
            launch_sgs_values_sell<float>(c->L, c->sgs_nbval, c->sgs_bat_own, c->sgs_bat_ent,
                                          c->sa32, c->spk32, batval);
        else
            launch_sgs_values_sell<double>(c->L, c->sgs_nbval, c->sgs_bat_own, c->sgs_bat_ent,
                                           c->sa64, nullptr, batval);
    } else {
        launch_sgs_values<T>(c->L, c->sgs_bat_own, c->sgs_bat_ent, c->sgs_nbval, nullptr, nullptr,
                             0, c->Aj, c->Av, c->dsq, batval, nullptr);
    }
}

// A^ and q in double (the FP64 path, or the adjoint of a mixed context)
void form_scaled64(emin_ctx *c) {
    if (c->sell_ptr)
        launch_sell_values<double>(c->L, c->n, c->Ap, c->Aj, c->Av, c->dsq, c->sell_ptr, c->sa64);
    else
        launch_scale_a<double>(c->L, c->n, c->Ap, c->Aj, c->Av, c->dsq, c->Ah64);
    if (c->k == 1) launch_qvec_k1<double>(c->L, c->n, c->Pp, c->Pj, c->Bc, c->qv64);
    if (c->sgs_fval64) form_sgs_values<double>(c, c->sgs_fval64, c->sgs_bval64, c->sgs_batval64);
    c->have64 = true;
}

// Algorithm 2 plus the start of Algorithm 3 from the stored inputs.
int run_setup(emin_ctx *c) {
    const Launch &L = c->L;
    EMIN_TRY(cuda_status(cudaMemsetAsync(c->dint, 0, 3 * sizeof(int), c->stream)));
    c->have64 = false;
    if (c->fast_k1) {
        const bool mixed = c->opts.precision == EMIN_MIXED;
        if (mixed) {
            launch_setup_k1<float>(L, c->n, c->dpos, c->Av, c->Pp, c->Pj, c->Bc, c->B, c->P0_in,
                                   c->opts.rank_policy, c->dint, c->dint + 2, c->dsq, c->dhalf,
                                   c->dsq32, c->Ginv, c->qv32, c->P0, c->t32a);
            launch_to_float(L, c->Bc, c->Bc32, (long long)c->nc * c->k);
            launch_sell_values<float>(L, c->n, c->Ap, c->Aj, c->Av, c->dsq, c->sell_ptr, c->sa32,
                                      c->sw, c->spk32, c->dsq32);
            form_sgs_values<float>(c, c->sgs_fval32, c->sgs_bval32, c->sgs_batval32);
            EMIN_TRY(start_pcg<float>(c, iter_ops32(c), c->w32, c->t32a));
        } else {
            launch_setup_k1<double>(L, c->n, c->dpos, c->Av, c->Pp, c->Pj, c->Bc, c->B, c->P0_in,
                                    c->opts.rank_policy, c->dint, c->dint + 2, c->dsq, c->dhalf,
                                    nullptr, c->Ginv, c->qv64, c->P0, c->t64c);
            launch_sell_values<double>(L, c->n, c->Ap, c->Aj, c->Av, c->dsq, c->sell_ptr, c->sa64);
            form_sgs_values<double>(c, c->sgs_fval64, c->sgs_bval64, c->sgs_batval64);
            c->have64 = true;
            EMIN_TRY(start_pcg<double>(c, iter_ops64(c), c->w64, c->t64c));
        }
        c->applied_seen = 0;
        return check_launch();
    }
    launch_diag(L, c->n, c->Ap, c->Aj, c->Av, c->dinv, c->dinv32, c->dint);
    launch_diag_scales(L, c->n, c->dinv, c->dsq, c->dhalf);
    launch_gram(L, c->n, c->k, c->Pp, c->Pj, c->Bc, c->Ginv, c->Ginv32, c->opts.rank_policy,
                c->dint, c->dint + 2, c->boff ? 3 : 1);
    fill_nbs(c);
    launch_restore(L, c->n, c->k, c->Pp, c->Pj, c->Bc, c->B, c->Ginv, c->P0_in, nullptr, nullptr,
                   nullptr, 1, c->P0);
    c->have64 = false;
    if (c->opts.precision == EMIN_MIXED) {
        launch_to_float(L, c->Bc, c->Bc32, (long long)c->nc * c->k);
        if (c->sell_ptr)
            launch_sell_values<float>(L, c->n, c->Ap, c->Aj, c->Av, c->dsq, c->sell_ptr, c->sa32,
                                      c->sw, c->spk32);
        else if (!c->nbs_blob)  // the staged product reads A^ from its own blob
            launch_scale_a<float>(L, c->n, c->Ap, c->Aj, c->Av, c->dsq, c->Ah32);
        if (c->k == 1) launch_qvec_k1<float>(L, c->n, c->Pp, c->Pj, c->Bc, c->qv32);
        form_sgs_values<float>(c, c->sgs_fval32, c->sgs_bval32, c->sgs_batval32);
        launch_row_scale<double, float>(L, c->n, c->Pp, c->lanes, c->dhalf, 1.0, c->P0, c->t32a);
        EMIN_TRY(start_pcg<float>(c, iter_ops32(c), c->w32, c->t32a));
    } else {
        form_scaled64(c);
        launch_row_scale<double, double>(L, c->n, c->Pp, c->lanes, c->dhalf, 1.0, c->P0, c->t64c);
        EMIN_TRY(start_pcg<double>(c, iter_ops64(c), c->w64, c->t64c));
    }
    c->applied_seen = 0;
    return check_launch();
}

int read_flags(emin_ctx *c) {
    EMIN_TRY(fetch_words(c, c->hint, c->dint, 3 * sizeof(int)));
    EMIN_TRY(sync(c));
    const int f = c->hint[0];
    c->ndef = c->hint[2];
    if (f & (F_ROWPTR | F_COL | F_ORDER)) return EMIN_ERR_PATTERN;
    if (f & F_NONFINITE) return EMIN_ERR_ARG;
    if (f & F_DIAG) return EMIN_ERR_DIAG;
    if (f & F_RANK) return EMIN_ERR_RANK;
    return EMIN_OK;
}

int read_state(emin_ctx *c, const DevState *st) {
    EMIN_TRY(cuda_status(
        cudaMemcpyAsync(c->hstate, st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream)));
    return sync(c);
}

// current P = P0 + D^{-1/2} dW~ on P's pattern, in double, into dst (device);
// every row is then corrected onto its constraint in double (in FP64 the
// correction is at rounding level: it removes the drift that the
// per-iteration projections accumulate when G_i is ill-conditioned)
int form_p(emin_ctx *c, double *dst) {
    if (c->fast_k1) {
        if (c->opts.precision == EMIN_MIXED)
            launch_final_k1<float>(c->L, c->n, c->Pp, c->Pj, c->Bc, c->Ginv, c->P0, c->w32.X,
                                   c->dsq, c->B, 1, dst);
        else
            launch_final_k1<double>(c->L, c->n, c->Pp, c->Pj, c->Bc, c->Ginv, c->P0, c->w64.X,
                                    c->dsq, c->B, 1, dst);
        return check_launch();
    }
    if (c->opts.precision == EMIN_MIXED)
        launch_restore(c->L, c->n, c->k, c->Pp, c->Pj, c->Bc, c->B, c->Ginv, c->P0, nullptr,
                       c->w32.X, c->dsq, 1, dst);
    else
        launch_restore(c->L, c->n, c->k, c->Pp, c->Pj, c->Bc, c->B, c->Ginv, c->P0, c->w64.X,
                       nullptr, c->dsq, 1, dst);
    return check_launch();
}

int create_impl(emin_ctx *c, const int *A_rowptr, const int *A_col, const double *A_val,
                const int *P_rowptr, const int *P_col, const double *P0_val, const double *B,
                const double *Bc, int on_dev) {
    const int n = c->n;
    // sizes from the row pointers
    int ends[4] = {0, 0, 0, 0};
    if (on_dev) {
        EMIN_TRY(cuda_status(cudaMemcpy(&ends[0], A_rowptr, sizeof(int), cudaMemcpyDeviceToHost)));
        EMIN_TRY(cuda_status(cudaMemcpy(&ends[1], A_rowptr + n, sizeof(int), cudaMemcpyDeviceToHost)));
        EMIN_TRY(cuda_status(cudaMemcpy(&ends[2], P_rowptr, sizeof(int), cudaMemcpyDeviceToHost)));
        EMIN_TRY(cuda_status(cudaMemcpy(&ends[3], P_rowptr + n, sizeof(int), cudaMemcpyDeviceToHost)));
    } else {
        ends[0] = A_rowptr[0];
        ends[1] = A_rowptr[n];
        ends[2] = P_rowptr[0];
        ends[3] = P_rowptr[n];
    }
    if (ends[0] != 0 || ends[2] != 0 || ends[1] < 0 || ends[3] < 0) return EMIN_ERR_PATTERN;
    c->nnz_a = ends[1];
    c->nnz_p = ends[3];
    const long long nk = (long long)n * c->k, nck = (long long)c->nc * c->k;
    const long long kk = (long long)n * (c->k * (c->k + 1) / 2);
    const bool k1 = (c->k == 1);

    EMIN_TRY(dalloc(c, &c->Ap, n + 1));
    EMIN_TRY(dalloc(c, &c->Aj, c->nnz_a));
    EMIN_TRY(dalloc(c, &c->Av, c->nnz_a));
    EMIN_TRY(dalloc(c, &c->Pp, n + 1));
    EMIN_TRY(dalloc(c, &c->Pj, c->nnz_p));
    EMIN_TRY(dalloc(c, &c->P0_in, c->nnz_p));
    EMIN_TRY(dalloc(c, &c->P0, c->nnz_p));
    EMIN_TRY(dalloc(c, &c->B, nk));
    EMIN_TRY(dalloc(c, &c->Bc, nck));
    EMIN_TRY(dalloc(c, &c->Ginv, kk));
    EMIN_TRY(dalloc(c, &c->Ginv32, kk));
    EMIN_TRY(dalloc(c, &c->dinv, n));
    EMIN_TRY(dalloc(c, &c->dinv32, n));
    EMIN_TRY(dalloc(c, &c->dsq, n));
    EMIN_TRY(dalloc(c, &c->dhalf, n));
    EMIN_TRY(dalloc(c, &c->rn, n));
    EMIN_TRY(dalloc(c, &c->dint, 4));
    if (c->opts.checks) {
        EMIN_TRY(dalloc(c, &c->chkw, 1));
        EMIN_TRY(cuda_status(cudaMemsetAsync(c->chkw, 0, sizeof(int), c->stream)));
    }
    EMIN_TRY(dalloc(c, &c->t64a, c->nnz_p));
    EMIN_TRY(dalloc(c, &c->t64b, c->nnz_p));
    EMIN_TRY(dalloc(c, &c->t64c, c->nnz_p));
    if (c->opts.precision == EMIN_MIXED) {
        EMIN_TRY(dalloc(c, &c->Ah32, c->nnz_a));
        if (k1) EMIN_TRY(dalloc(c, &c->qv32, c->nnz_p));
        if (k1) EMIN_TRY(dalloc(c, &c->qv64, c->nnz_p));
        EMIN_TRY(dalloc(c, &c->Bc32, nck));
        EMIN_TRY(dalloc(c, &c->t32a, c->nnz_p));
        EMIN_TRY(dalloc(c, &c->t32b, c->nnz_p));
        EMIN_TRY(alloc_work(c, c->w32, true));
    } else {
        EMIN_TRY(dalloc(c, &c->Ah64, c->nnz_a));
        if (k1) EMIN_TRY(dalloc(c, &c->qv64, c->nnz_p));
        EMIN_TRY(alloc_work(c, c->w64, true));
    }
    EMIN_TRY(alloc_work(c, c->aux, false));
    c->host_blk = host_block_get();
    if (!c->host_blk) return EMIN_ERR_NOMEM;
    c->hstate = static_cast<DevState *>(c->host_blk);
    c->hint = reinterpret_cast<int *>(static_cast<char *>(c->host_blk) + kHintOffset);
    if (cudaHostGetDevicePointer(&c->host_dev, c->host_blk, 0) != cudaSuccess) {
        cudaGetLastError();
        c->host_dev = nullptr;
    }

    // the patterns first, on the context's stream
    EMIN_TRY(copy_in(c, c->Ap, A_rowptr, sizeof(int) * (n + 1), on_dev));
    EMIN_TRY(copy_in(c, c->Aj, A_col, sizeof(int) * c->nnz_a, on_dev));
    EMIN_TRY(copy_in(c, c->Pp, P_rowptr, sizeof(int) * (n + 1), on_dev));
    EMIN_TRY(copy_in(c, c->Pj, P_col, sizeof(int) * c->nnz_p, on_dev));
    // the values: from host arrays on the second stream, ordered after the
    // pattern copies (and the allocations, which are stream-ordered on the
    // context's stream) so that the patterns, which the plan build needs
    // first, have the host link to themselves; the values then cross it
    // while the pattern is validated and the plan is built, and the value
    // checks and the set-up wait for them
    const bool split = !on_dev && (c->nnz_a > 0 || c->nnz_p > 0);
    cudaStream_t cs = c->stream;
    if (split) {
        if (!c->side) {
            EMIN_TRY(cuda_status(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking)));
            EMIN_TRY(cuda_status(cudaEventCreateWithFlags(&c->side_ev, cudaEventDisableTiming)));
        }
        EMIN_TRY(cuda_status(cudaEventRecord(c->side_ev, c->stream)));
        EMIN_TRY(cuda_status(cudaStreamWaitEvent(c->side, c->side_ev, 0)));
        cs = c->side;
    }
    auto copy_values = [&](void *dst, const void *src, size_t bytes) -> int {
        if (bytes == 0) return EMIN_OK;
        if (!src) return EMIN_ERR_ARG;
        return cuda_status(cudaMemcpyAsync(
            dst, src, bytes, on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, cs));
    };
    // The value arrays cross the link while the patterns are checked and
    // planned: P0, B and B_c right behind the patterns, A's values (the
    // largest) once the plan's arrays are allocated.  An allocation or free
    // from the pool blocks the host while a transfer is in flight, so every
    // allocation of the plan is made while only the small arrays travel and
    // the unused ones are freed after the set-up (`late`).
    EMIN_TRY(copy_values(c->P0_in, P0_val, sizeof(double) * c->nnz_p));
    EMIN_TRY(copy_values(c->B, B, sizeof(double) * nk));
    EMIN_TRY(copy_values(c->Bc, Bc, sizeof(double) * nck));
    bool av_issued = false;
    auto issue_av = [&]() -> int {
        if (av_issued) return EMIN_OK;
        av_issued = true;
        EMIN_TRY(copy_values(c->Av, A_val, sizeof(double) * c->nnz_a));
        if (split) EMIN_TRY(cuda_status(cudaEventRecord(c->side_ev, c->side)));
        return EMIN_OK;
    };
    void *late[2] = {nullptr, nullptr};

    // validate the patterns on the device before any kernel indexes through
    // them (the values are checked once they have arrived, below; their
    // flag is read with the set-up's)
    EMIN_TRY(cuda_status(cudaMemsetAsync(c->dint, 0, 4 * sizeof(int), c->stream)));
    launch_validate_csr(c->L, n, n, c->Ap, (int)c->nnz_a, c->Aj, c->dint, c->dint + 3);
    launch_validate_csr(c->L, n, c->nc, c->Pp, (int)c->nnz_p, c->Pj, c->dint, c->dint + 1);
    EMIN_TRY(check_launch());
    EMIN_TRY(fetch_words(c, c->hint, c->dint, 4 * sizeof(int)));
    EMIN_TRY(sync(c));
    const int f = c->hint[0];
    if (f & (F_ROWPTR | F_COL | F_ORDER)) return EMIN_ERR_PATTERN;
    c->maxrow_p = c->hint[1];
    if (c->maxrow_p > kMaxRowP) return EMIN_ERR_ARG;
    c->lanes = (c->maxrow_p <= 8) ? 1 : 32;
    c->fast_k1 = (c->k == 1 && c->maxrow_p <= 4 && n > 0);
    if (c->fast_k1 && n > 0) {
        // the plan of the fixed pattern in SELL-32 order: built once, reused by
        // every product of every iteration
        const int ns = (n + 31) / 32;
        EMIN_TRY(dalloc(c, &c->sell_ptr, ns + 1));
        launch_sell_len(c->L, n, c->Ap, c->sell_ptr);
        // slice starts by a scan on the device; only the entry count comes
        // back (no upload that would queue behind the value copies)
        long long *dtotal = nullptr;
        EMIN_TRY(dalloc(c, &dtotal, 1));
        launch_sell_scan(c->L, ns, c->sell_ptr, dtotal);
        long long *htotal = reinterpret_cast<long long *>(c->hint + kHintTotal);
        EMIN_TRY(fetch_words(c, htotal, dtotal, sizeof(long long)));
        EMIN_TRY(sync(c));
        const long long acc = *htotal;
        dfree(c, dtotal);
        if (acc > 0x7fffffffLL) return EMIN_ERR_ARG;
        c->nnz_sell = acc;
        EMIN_TRY(dalloc(c, &c->soff, acc));
        EMIN_TRY(dalloc(c, &c->smap, acc));
        EMIN_TRY(dalloc(c, &c->sw, acc));
        EMIN_TRY(dalloc(c, &c->dpos, n));
        // A^ in plan order: packed records (float) or values (double); a float
        // plan that turns out plain takes its values in a smaller array below
        if (c->opts.precision == EMIN_MIXED) {
            EMIN_TRY(dalloc(c, &c->dsq32, n));
            EMIN_TRY(dalloc(c, &c->spk32, acc));
        } else {
            EMIN_TRY(dalloc(c, &c->sa64, acc));
        }
        EMIN_TRY(issue_av());
        EMIN_TRY(cuda_status(cudaMemsetAsync(c->dint + 3, 0, sizeof(int), c->stream)));
        launch_sell_plan(c->L, n, c->Ap, c->Aj, c->Pp, c->Pj, c->sell_ptr, c->soff, c->smap,
                         c->sw, c->dint + 3, c->dpos, acc, c->opts.checks ? c->chkw : nullptr);
        EMIN_TRY(fetch_words(c, c->hint + 3, c->dint + 3, sizeof(int)));
        EMIN_TRY(sync(c));  // the plan's verdict (do the offsets fit the packed word?)
        // the packed plan when every offset difference fits its word, else the
        // plain one; the arrays of the other are freed after the set-up
        if (c->hint[3] == 0) {
            late[0] = c->soff;
            late[1] = c->smap;
            c->soff = nullptr;
            c->smap = nullptr;
        } else {
            late[0] = c->sw;
            c->sw = nullptr;
            if (c->opts.precision == EMIN_MIXED) {
                late[1] = c->spk32;
                c->spk32 = nullptr;
                EMIN_TRY(dalloc(c, &c->sa32, acc));
            }
        }
    }
    EMIN_TRY(issue_av());

    if (!c->fast_k1) {
        // node-blocked problems (elasticity): plan of 3 x 3 / 3 x 6 blocks
        EMIN_TRY(cuda_status(cudaMemsetAsync(c->dint + 3, 0, sizeof(int), c->stream)));
        if (launch_detect_blocks(c->L, n, c->k, c->Ap, c->Aj, c->Pp, c->Pj, c->dint + 3)) {
            EMIN_TRY(fetch_words(c, c->hint + 3, c->dint + 3, sizeof(int)));
            EMIN_TRY(sync(c));
            if (c->hint[3] == 0) {
                const long long ne = block_plan_entries(c->nnz_a);
                EMIN_TRY(dalloc(c, &c->boff, ne));
                EMIN_TRY(dalloc(c, &c->blen, ne));
                EMIN_TRY(dalloc(c, &c->bmap, ne));
                launch_block_plan(c->L, n, c->Ap, c->Aj, c->Pp, c->Pj, c->boff, c->blen, c->bmap,
                                  ne, c->opts.checks ? c->chkw : nullptr);
                // warp tiles of output blocks: whole nodes per warp, packed greedily
                const int nn = n / 3;
                int *dna = nullptr;
                EMIN_TRY(dalloc(c, &dna, nn));
                launch_node_slots(c->L, n, c->Pp, dna);
                std::vector<int> na(nn);
                EMIN_TRY(cuda_status(cudaMemcpyAsync(na.data(), dna, sizeof(int) * nn,
                                                     cudaMemcpyDeviceToHost, c->stream)));
                EMIN_TRY(sync(c));
                std::vector<int> tm;
                tm.reserve((size_t)nn * 6);
                int fill = 0;
                for (int v = 0; v < nn; ++v) {
                    if (fill + na[v] > 32) {
                        while (fill < 32) { tm.push_back(-1); ++fill; }
                        fill = 0;
                    }
                    for (int s2 = 0; s2 < na[v]; ++s2) tm.push_back((v << 3) | s2);
                    fill += na[v];
                }
                while (fill % 32) { tm.push_back(-1); ++fill; }
                c->ntiles = (int)(tm.size() / 32);
                if (c->ntiles > 0) {
                    EMIN_TRY(dalloc(c, &c->tile_map, (long long)tm.size()));
                    EMIN_TRY(cuda_status(cudaMemcpyAsync(c->tile_map, tm.data(),
                                                         sizeof(int) * tm.size(),
                                                         cudaMemcpyHostToDevice, c->stream)));
                    EMIN_TRY(sync(c));
                }
                // the staged product, from host copies of both patterns
                std::vector<int> hAp, hAj, hPp, hPj;
                const int *pAp = A_rowptr, *pAj = A_col, *pPp = P_rowptr, *pPj = P_col;
                if (on_dev) {
                    hAp.resize(n + 1);
                    hAj.resize(c->nnz_a);
                    hPp.resize(n + 1);
                    hPj.resize(c->nnz_p);
                    EMIN_TRY(cuda_status(cudaMemcpyAsync(hAp.data(), c->Ap, sizeof(int) * (n + 1),
                                                         cudaMemcpyDeviceToHost, c->stream)));
                    EMIN_TRY(cuda_status(cudaMemcpyAsync(hAj.data(), c->Aj, sizeof(int) * c->nnz_a,
                                                         cudaMemcpyDeviceToHost, c->stream)));
                    EMIN_TRY(cuda_status(cudaMemcpyAsync(hPp.data(), c->Pp, sizeof(int) * (n + 1),
                                                         cudaMemcpyDeviceToHost, c->stream)));
                    EMIN_TRY(cuda_status(cudaMemcpyAsync(hPj.data(), c->Pj, sizeof(int) * c->nnz_p,
                                                         cudaMemcpyDeviceToHost, c->stream)));
                    EMIN_TRY(sync(c));
                    pAp = hAp.data();
                    pAj = hAj.data();
                    pPp = hPp.data();
                    pPj = hPj.data();
                }
                EMIN_TRY(build_nbs(c, pAp, pAj, pPp, pPj));
            }
        }
    }

    if (c->opts.precond == EMIN_SGS && n > 0) EMIN_TRY(build_sgs(c));

    if (split) EMIN_TRY(cuda_status(cudaStreamWaitEvent(c->stream, c->side_ev, 0)));
    EMIN_TRY(run_setup(c));
    // the value checks after the set-up (which clears the flags first): a
    // non-finite value only makes the set-up's arithmetic non-finite, no
    // index depends on it, and read_flags reports it before any flag the
    // set-up raised
    launch_check_finite(c->L, c->Av, c->nnz_a, c->dint);
    launch_check_finite(c->L, c->P0_in, c->nnz_p, c->dint);
    launch_check_finite(c->L, c->B, nk, c->dint);
    launch_check_finite(c->L, c->Bc, nck, c->dint);
    EMIN_TRY(check_launch());
    EMIN_TRY(read_flags(c));
    for (void *p : late) dfree(c, p);
    return with_checks(c, EMIN_OK);
}

// The launches of n_iters iterations of Algorithm 3 (scaled variables):
// y~ = r~ + beta y~; y_~ = Pi A^ y~ with y~^T y_~ -> alpha; dW~, r~ updates
// with gamma -> beta.  With `timed`, the masked product of every iteration
// is bracketed by CUDA events on the context's stream.
template <class T>
int launch_iterations(emin_ctx *c, const Ops<T> &o, Work<T> &w, int n_iters, bool timed) {
    for (int it = 0; it < n_iters; ++it) {
        if (o.sgs.fused)
            launch_ydir_proj_k1<T>(c->L, o.n, o.maxrow, o.Pp, o.qv, w.Z, w.Y, w.st);
        else
            launch_ydir<T>(c->L, c->nnz_p, w);
        // external records, so that the events also time the launches when
        // the loop is captured into a graph; every c->timing-th iteration
        const bool t = timed && (it % c->timing) == 0;
        if (t) cudaEventRecordWithFlags(c->events[(size_t)it * 2], c->stream, cudaEventRecordExternal);
        launch_kprod<T>(c->L, o, w.Y, w.Yb, 1, DOT_ALPHA, w, 1);
        if (t) cudaEventRecordWithFlags(c->events[(size_t)it * 2 + 1], c->stream, cudaEventRecordExternal);
        if (o.sgs.active()) {
            // projected SGS: the step, then z~ = Pi M^-1 r~ and gamma = <r~, z~>
            // (fused: gamma from the sweep, Pi in the next direction update)
            launch_update<T>(c->L, c->nnz_p, w, UPD_XR);
            launch_sgs_sweep<T>(c->L, o.sgs, w.R, w.Z, w.st, w.partials, 0);
            if (!o.sgs.fused) launch_sgs_finish<T>(c->L, o, w, 0, c->nnz_p);
        } else {
            launch_update<T>(c->L, c->nnz_p, w, UPD_STEP);
        }
    }
    return check_launch();
}

bool capturable(cudaStream_t s) {
    return s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
}

// One iteration as the body of a conditional while node (captured once per
// workspace): the loop control at the end of the body keeps it running while
// iterations of the call are left and the stop test of Eq. (relRed) has not
// fired, so a call stops launching work as soon as the energy criterion is met.
template <class T>
void build_while_graph(emin_ctx *c, const Ops<T> &o, Work<T> &w) {
    cudaGraph_t graph = nullptr;
    if (cudaGraphCreate(&graph, 0) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaGraphConditionalHandle h;
    bool ok = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) ==
              cudaSuccess;
    cudaGraphNodeParams p = {};
    if (ok) {
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = h;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t node;
        ok = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &p) == cudaSuccess;
    }
    if (ok) {
        cudaGraph_t body = p.conditional.phGraph_out[0];
        const long long before = launches_so_far();
        ok = cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            launch_iterations<T>(c, o, w, 1, false);
            launch_loop_control(c->L, w.st, h);
            cudaGraph_t captured = nullptr;
            ok = cudaStreamEndCapture(c->stream, &captured) == cudaSuccess;
        }
        w.gwhile_per_pass = (int)(launches_so_far() - before);
        note_launches(before - launches_so_far());  // captured, not run
    }
    if (ok && cudaGraphInstantiate(&w.gwhile, graph, 0) != cudaSuccess) w.gwhile = nullptr;
    cudaGraphDestroy(graph);
    cudaGetLastError();
}

template <class T>
int iterate_impl(emin_ctx *c, const Ops<T> &o, Work<T> &w, int n_iters, double tol,
                 bool timed = false) {
    launch_state_begin(c->L, w.st, tol, n_iters);
    timed = timed && c->timing > 0 && o.n > 0;
    if (timed) {
        const size_t need = (size_t)n_iters * 2;
        while (c->events.size() < need) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return cuda_status(cudaGetLastError());
            c->events.push_back(e);
        }
    }
    bool launched = false, looped = false;
    if (n_iters > 0 && o.n > 0 && capturable(c->stream) && !timed) {
        if (!w.gwhile) build_while_graph<T>(c, o, w);
        if (w.gwhile && cudaGraphLaunch(w.gwhile, c->stream) == cudaSuccess) launched = looped = true;
        cudaGetLastError();
    }
    if (!launched && n_iters > 0 && o.n > 0 && capturable(c->stream)) {
        // the whole loop unrolled into one CUDA graph, captured once per
        // (count, timing): the timed runs bracket single launches with events
        const int tkey = timed ? c->timing : 0;
        if (!(w.gexec && w.gn == n_iters && w.gtimed == tkey)) {
            if (w.gexec) {
                cudaGraphExecDestroy(w.gexec);
                w.gexec = nullptr;
            }
            const long long before = launches_so_far();
            cudaGraph_t graph = nullptr;
            if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                launch_iterations<T>(c, o, w, n_iters, timed);
                if (cudaStreamEndCapture(c->stream, &graph) == cudaSuccess && graph) {
                    if (cudaGraphInstantiate(&w.gexec, graph, 0) != cudaSuccess) w.gexec = nullptr;
                    cudaGraphDestroy(graph);
                }
            }
            cudaGetLastError();
            w.gexec_launches = launches_so_far() - before;
            note_launches(before - launches_so_far());  // captured, not run
            w.gn = n_iters;
            w.gtimed = tkey;
        }
        if (w.gexec && cudaGraphLaunch(w.gexec, c->stream) == cudaSuccess) {
            note_launches(w.gexec_launches);
            launched = true;
        }
        cudaGetLastError();
    }
    if (!launched) EMIN_TRY(launch_iterations<T>(c, o, w, n_iters, timed));
    EMIN_TRY(check_launch());
    EMIN_TRY(read_state(c, w.st));
    if (looped) note_launches((long long)w.gwhile_per_pass * (n_iters - c->hstate->loop_left));
    if (timed) {
        for (int it = 0; it < n_iters; it += c->timing) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, c->events[(size_t)it * 2], c->events[(size_t)it * 2 + 1]) ==
                cudaSuccess) {
                c->tms[0] += ms;
                c->tlaunch[0] += 1;
            }
        }
        cudaGetLastError();
    }
    return EMIN_OK;
}

}  // namespace

extern "C" {

void emin_default_opts(emin_opts *opts) {
    if (!opts) return;
    opts->precision = EMIN_FP64;
    opts->precond = EMIN_JACOBI;
    opts->rank_policy = EMIN_RANK_STRICT;
    opts->checks = 0;
    opts->stream = nullptr;
}

const char *emin_last_error(void) { return g_last_error; }

int emin_trim_memory(void) {
    std::lock_guard<std::mutex> lk(g_pool_mutex);
    for (cudaMemPool_t pool : g_pools)
        if (pool && cudaMemPoolTrimTo(pool, 0) != cudaSuccess) return cuda_status(cudaGetLastError());
    return EMIN_OK;
}

const char *emin_strerror(int status) {
    switch (status) {
        case EMIN_OK: return "ok";
        case EMIN_ERR_ARG: return "invalid argument or unsupported size";
        case EMIN_ERR_PATTERN: return "invalid CSR pattern (row pointers, range, order or duplicates)";
        case EMIN_ERR_RANK: return "rank-deficient row constraint (m_i < k or Gram matrix not SPD)";
        case EMIN_ERR_DIAG: return "diagonal entry of A missing or not positive";
        case EMIN_ERR_BREAKDOWN: return "conjugate gradient breakdown (y^T K y <= 0 or non-finite)";
        case EMIN_ERR_CUDA: return "CUDA runtime error";
        case EMIN_ERR_NOMEM: return "out of device or pinned host memory";
        case EMIN_ERR_TIMEOUT: return "bounded device wait expired";
        case EMIN_ERR_STATE: return "call not valid in the current state";
        default: return "unknown status";
    }
}

void emin_destroy(emin_ctx *c) {
    if (!c) return;
    {
        DeviceGuard g(c->device);
        if (c->side) cudaStreamSynchronize(c->side);
        cudaStreamSynchronize(c->stream);
        for (cudaGraphExec_t g : {c->w64.gexec, c->adj.gexec, c->aux.gexec})
            if (g) cudaGraphExecDestroy(g);
        if (c->w32.gexec) cudaGraphExecDestroy(c->w32.gexec);
        for (cudaGraphExec_t g : {c->w64.gwhile, c->adj.gwhile, c->aux.gwhile, c->w32.gwhile})
            if (g) cudaGraphExecDestroy(g);
        for (void *p : c->dev_allocs) release_dev(c, p);
        for (cudaEvent_t e : c->events) cudaEventDestroy(e);
        host_block_put(c->host_blk);
        if (c->side_ev) cudaEventDestroy(c->side_ev);
        if (c->side) cudaStreamDestroy(c->side);
        cudaGetLastError();
    }
    delete c;
}

int emin_create(emin_ctx **out, int n, int nc, int k, const int *A_rowptr, const int *A_col,
                const double *A_val, const int *P_rowptr, const int *P_col, const double *P0_val,
                const double *B, const double *Bc, const emin_opts *opts, int inputs_on_device) {
    if (!out) return EMIN_ERR_ARG;
    *out = nullptr;
    if (n < 0 || nc < 0 || k < 1 || k > kMaxK || !A_rowptr || !P_rowptr) return EMIN_ERR_ARG;
    emin_opts o;
    emin_default_opts(&o);
    if (opts) o = *opts;
    if ((o.precision != EMIN_FP64 && o.precision != EMIN_MIXED) ||
        (o.precond != EMIN_JACOBI && o.precond != EMIN_SGS) ||
        (o.rank_policy != EMIN_RANK_STRICT && o.rank_policy != EMIN_RANK_PINV) ||
        (o.checks != 0 && o.checks != 1))
        return EMIN_ERR_ARG;
    emin_ctx *c = new (std::nothrow) emin_ctx();
    if (!c) return EMIN_ERR_NOMEM;
    c->n = n;
    c->nc = nc;
    c->k = k;
    c->opts = o;
    c->stream = static_cast<cudaStream_t>(o.stream);
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return EMIN_ERR_CUDA;
    }
    int nsm = 0, occ_rows = 0, occ_warps = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    if (nsm <= 0) nsm = 1;
    occ_rows = 8;   // 2048 resident threads per SM at 256 threads per block
    occ_warps = 8;
    c->pool = device_pool(c->device);
    c->L.stream = c->stream;
    c->L.nsm = nsm;
    c->L.grid_rows = nsm * occ_rows;
    c->L.grid_warps = nsm * occ_warps;
    if (c->L.grid_rows > kMaxGrid) c->L.grid_rows = kMaxGrid;
    c->L.grid_staged = nsm * staged_blocks_per_sm();
    if (c->L.grid_staged > kMaxGrid) c->L.grid_staged = kMaxGrid;
    pk_blocks_per_sm(0);  // occupancy of every packed-product instantiation, queried now
    pk_blocks_per_sm(1);
    c->L.grid_flat32 = nsm * flat_blocks_per_sm(0);
    if (c->L.grid_flat32 > kMaxGrid) c->L.grid_flat32 = kMaxGrid;
    c->L.grid_flat64 = nsm * flat_blocks_per_sm(1);
    if (c->L.grid_flat64 > kMaxGrid) c->L.grid_flat64 = kMaxGrid;
    if (c->L.grid_warps > kMaxGrid) c->L.grid_warps = kMaxGrid;
    set_iter_attributes();
    set_adjoint_attributes();
    c->launches_at_create = launches_so_far();
    int st = create_impl(c, A_rowptr, A_col, A_val, P_rowptr, P_col, P0_val, B, Bc,
                         inputs_on_device);
    if (st != EMIN_OK) {
        emin_destroy(c);
        return st;
    }
    *out = c;
    return EMIN_OK;
}

static int call_reset(emin_ctx *c) {
    if (!c) return EMIN_ERR_ARG;
    DeviceGuard g(c->device);
    if (c->sticky == EMIN_ERR_CUDA) return c->sticky;
    c->sticky = EMIN_OK;
    return run_setup(c);
}

static int call_set_values(emin_ctx *c, const double *A_val, const double *B, const double *P0_val,
                    int on_device) {
    if (!c) return EMIN_ERR_ARG;
    DeviceGuard g(c->device);
    if (A_val) EMIN_TRY(copy_in(c, c->Av, A_val, sizeof(double) * c->nnz_a, on_device));
    if (B) EMIN_TRY(copy_in(c, c->B, B, sizeof(double) * c->n * c->k, on_device));
    if (P0_val) EMIN_TRY(copy_in(c, c->P0_in, P0_val, sizeof(double) * c->nnz_p, on_device));
    EMIN_TRY(cuda_status(cudaMemsetAsync(c->dint, 0, 4 * sizeof(int), c->stream)));
    launch_check_finite(c->L, c->Av, c->nnz_a, c->dint);
    launch_check_finite(c->L, c->P0_in, c->nnz_p, c->dint);
    launch_check_finite(c->L, c->B, (long long)c->n * c->k, c->dint);
    EMIN_TRY(cuda_status(cudaMemcpyAsync(c->hint, c->dint, sizeof(int), cudaMemcpyDeviceToHost,
                                         c->stream)));
    EMIN_TRY(sync(c));
    if (c->hint[0] & F_NONFINITE) return EMIN_ERR_ARG;
    c->sticky = EMIN_OK;
    EMIN_TRY(run_setup(c));
    return read_flags(c);
}

static int call_iterate(emin_ctx *c, int n_iters, double tol, int *iters_done, double *rel_dE_last) {
    if (!c || n_iters < 0 || !(tol >= 0)) return EMIN_ERR_ARG;
    DeviceGuard g(c->device);
    if (iters_done) *iters_done = 0;
    if (c->sticky != EMIN_OK) return c->sticky;
    int s;
    const DevState *hs = c->hstate;
    if (c->opts.precision == EMIN_MIXED)
        s = iterate_impl<float>(c, iter_ops32(c), c->w32, n_iters, tol, true);
    else
        s = iterate_impl<double>(c, iter_ops64(c), c->w64, n_iters, tol, true);
    if (s != EMIN_OK) {
        c->sticky = s;
        return s;
    }
    if (iters_done) *iters_done = hs->applied - c->applied_seen;
    c->applied_seen = hs->applied;
    if (rel_dE_last) *rel_dE_last = (hs->k > 0 && hs->dE1 != 0.0) ? hs->dE_last / hs->dE1 : 0.0;
    if (hs->status != EMIN_OK) {
        c->sticky = hs->status;
        return hs->status;
    }
    return EMIN_OK;
}

static int call_get_p(emin_ctx *c, double *P_out, int out_on_device) {
    if (!c) return EMIN_ERR_ARG;
    DeviceGuard g(c->device);
    if (c->sticky != EMIN_OK) return c->sticky;
    EMIN_TRY(form_p(c, c->t64a));
    EMIN_TRY(copy_out(c, P_out, c->t64a, sizeof(double) * c->nnz_p, out_on_device));
    return sync(c);
}

static int call_energy(emin_ctx *c, double *E) {
    if (!c || !E) return EMIN_ERR_ARG;
    DeviceGuard g(c->device);
    if (c->sticky != EMIN_OK) return c->sticky;
    EMIN_TRY(form_p(c, c->t64a));
    launch_state_reset(c->L, c->aux.st);
    launch_kprod<double>(c->L, plain_ops64(c), c->t64a, c->t64b, 0, DOT_AUX, c->aux, 0);
    EMIN_TRY(check_launch());
    EMIN_TRY(read_state(c, c->aux.st));
    *E = c->hstate->aux;
    return EMIN_OK;
}

static int call_kprod(emin_ctx *c, const double *X, double *out, int project, int on_device) {
    if (!c) return EMIN_ERR_ARG;
    DeviceGuard g(c->device);
    // the iteration's kernel on x~ = D^{1/2} X, scaled back: y = D^{1/2} y~
    EMIN_TRY(copy_in(c, c->t64a, X, sizeof(double) * c->nnz_p, on_device));
    if (c->opts.precision == EMIN_MIXED) {
        launch_row_scale<double, float>(c->L, c->n, c->Pp, c->lanes, c->dhalf, 1.0, c->t64a, c->t32a);
        launch_kprod<float>(c->L, iter_ops32(c), c->t32a, c->t32b, project ? 1 : 0, DOT_NONE, c->w32, 0);
        launch_row_scale<float, double>(c->L, c->n, c->Pp, c->lanes, c->dhalf, 1.0, c->t32b, c->t64b);
    } else {
        launch_row_scale<double, double>(c->L, c->n, c->Pp, c->lanes, c->dhalf, 1.0, c->t64a, c->t64c);
        launch_kprod<double>(c->L, iter_ops64(c), c->t64c, c->t64a, project ? 1 : 0, DOT_NONE, c->aux, 0);
        launch_row_scale<double, double>(c->L, c->n, c->Pp, c->lanes, c->dhalf, 1.0, c->t64a, c->t64b);
    }
    EMIN_TRY(check_launch());
    EMIN_TRY(copy_out(c, out, c->t64b, sizeof(double) * c->nnz_p, on_device));
    return sync(c);
}

static int call_outer(emin_ctx *c, const double *U, const double *V, double *out, int on_device) {
    if (!c) return EMIN_ERR_ARG;
    DeviceGuard g(c->device);
    if (!c->tA) EMIN_TRY(dalloc(c, &c->tA, c->nnz_a));
    EMIN_TRY(copy_in(c, c->t64a, U, sizeof(double) * c->nnz_p, on_device));
    EMIN_TRY(copy_in(c, c->t64b, V, sizeof(double) * c->nnz_p, on_device));
    launch_outer(c->L, c->n, c->Ap, c->Aj, c->Pp, c->Pj, c->t64a, c->t64b, 1.0, c->tA, c->maxrow_p);
    EMIN_TRY(check_launch());
    EMIN_TRY(copy_out(c, out, c->tA, sizeof(double) * c->nnz_a, on_device));
    return sync(c);
}

static int call_energy_grad(emin_ctx *c, const double *X, double scale, double *E, double *dE_dX,
                     double *dE_dAval, int on_device) {
    if (!c || !X) return EMIN_ERR_ARG;
    DeviceGuard g(c->device);
    if (c->sticky == EMIN_ERR_CUDA) return c->sticky;
    EMIN_TRY(copy_in(c, c->t64a, X, sizeof(double) * c->nnz_p, on_device));
    if (E || dE_dX) {
        // mask_P(A X) on the unscaled A in double, with <X, mask_P(A X)>
        launch_state_reset(c->L, c->aux.st);
        launch_kprod<double>(c->L, plain_ops64(c), c->t64a, c->t64b, 0, E ? DOT_AUX : DOT_NONE,
                             c->aux, 0);
    }
    if (dE_dX) {
        launch_axpby(c->L, c->nnz_p, 2.0 * scale, c->t64b, 0.0, c->t64b);
        EMIN_TRY(check_launch());
        EMIN_TRY(copy_out(c, dE_dX, c->t64b, sizeof(double) * c->nnz_p, on_device));
    }
    if (dE_dAval) {
        if (!c->tA) EMIN_TRY(dalloc(c, &c->tA, c->nnz_a));
        launch_outer(c->L, c->n, c->Ap, c->Aj, c->Pp, c->Pj, c->t64a, c->t64a, scale, c->tA,
                     c->maxrow_p);
        EMIN_TRY(check_launch());
        EMIN_TRY(copy_out(c, dE_dAval, c->tA, sizeof(double) * c->nnz_a, on_device));
    }
    EMIN_TRY(check_launch());
    if (E) {
        EMIN_TRY(read_state(c, c->aux.st));
        *E = c->hstate->aux;
        return EMIN_OK;
    }
    return sync(c);
}

}  // extern "C"

namespace {

// the idx-th vector on P's pattern of the unrolled adjoint (allocated once)
int unr_vec(emin_ctx *c, size_t idx, double **out) {
    while (c->unr.size() <= idx) {
        double *p = nullptr;
        EMIN_TRY(dalloc(c, &p, c->nnz_p));
        c->unr.push_back(p);
    }
    *out = c->unr[idx];
    return EMIN_OK;
}

int read_aux(emin_ctx *c, const Work<double> &w, double *v) {
    EMIN_TRY(cuda_status(cudaMemcpyAsync(v, &w.st->aux, sizeof(double), cudaMemcpyDeviceToHost,
                                         c->stream)));
    return sync(c);
}

// The gradient of exactly n_iters steps of Algorithm 3 (Jacobi, FP64) from
// the set-up's P0, by reverse accumulation through the steps in the scaled
// variables (r~ = D^{-1/2} r, y~ = D^{1/2} y, x~ = D^{1/2} dW on
// A^ = D^{-1/2} A D^{-1/2}):
//   gamma_k = <r~,r~>, beta_k = gamma_k/gamma_{k-1}, y~_k = r~_k + beta_k y~_{k-1},
//   w~_k = Pi K^ y~_k, delta_k = <y~_k, w~_k>, alpha_k = gamma_k/delta_k,
//   x~ += alpha_k y~_k, r~ -= alpha_k w~_k;  P = p0 + D^{-1/2} x~_n,
// r~_0 = -Pi K^ D^{1/2} p0.  The adjoint of each step, from k = n-1 down:
//   abar = <xbar, y~_k> - <rbar, w~_k>, dbar = -abar alpha_k / delta_k,
//   wbar = -alpha_k rbar + dbar y~_k,
//   ybar_k = (carry) + alpha_k xbar + dbar w~_k + K^ Pi wbar,
//   ghat += mask_A((Pi wbar) y~_k^T),  betabar = <ybar_k, y~_{k-1}>,
//   gammabar_k = (carry) + abar/delta_k + betabar/gamma_{k-1},
//   rbar += ybar_k + 2 gammabar_k r~_k,  carries: beta_k ybar_k and
//   -betabar gamma_k / gamma_{k-1}^2,
// with xbar = D^{-1/2} dL/dP.  The iterates are checkpointed every
// s = ceil(sqrt(n)) steps (r~_k and y~_{k-1}) and each segment is run forward
// again before its steps are reversed: O(sqrt(n)) stored vectors.
int unrolled_backward(emin_ctx *c, const double *dLdP, int n_iters, double *gA, double *gB) {
    const Ops<double> o = iter_ops64(c);
    Work<double> &w = c->adj;
    const Launch &L = c->L;
    const long long np = c->nnz_p, na = c->nnz_a;
    const int n = c->n;
    const int sgl = (int)std::ceil(std::sqrt((double)n_iters));
    const int ncp = (n_iters + sgl - 1) / sgl;
    // vectors: checkpoints r, y; segment r, y; pt0, xbar, rbar, ybar, wt, wb, pw, tmp, zero
    size_t q = 0;
    std::vector<double *> cpr(ncp), cpy(ncp), sr(sgl), sy(sgl);
    for (int i = 0; i < ncp; ++i) EMIN_TRY(unr_vec(c, q++, &cpr[i]));
    for (int i = 0; i < ncp; ++i) EMIN_TRY(unr_vec(c, q++, &cpy[i]));
    for (int i = 0; i < sgl; ++i) EMIN_TRY(unr_vec(c, q++, &sr[i]));
    for (int i = 0; i < sgl; ++i) EMIN_TRY(unr_vec(c, q++, &sy[i]));
    double *pt0, *xbar, *rbar, *ybar, *wt, *wb, *pw, *tmp, *zero;
    for (double **v : {&pt0, &xbar, &rbar, &ybar, &wt, &wb, &pw, &tmp, &zero})
        EMIN_TRY(unr_vec(c, q++, v));
    if (!c->unr_ghat) EMIN_TRY(dalloc(c, &c->unr_ghat, na));
    if (!c->unr_dext) EMIN_TRY(dalloc(c, &c->unr_dext, n));
    double *R = w.R, *Y = w.Y, *Yb = w.Yb, *X = w.X;
    const size_t vb = sizeof(double) * np;
    auto dcopy = [&](double *dst, const double *src) {
        return cuda_status(cudaMemcpyAsync(dst, src, vb, cudaMemcpyDeviceToDevice, c->stream));
    };
    auto dot = [&](const double *x, const double *y, double *v) {
        launch_dot_aux(L, np, x, y, w.st, w.partials);
        return read_aux(c, w, v);
    };
    std::vector<double> gam(n_iters), bet(n_iters), del(n_iters), alp(n_iters);
    // forward, keeping the scalars and the checkpoints
    launch_row_scale<double, double>(L, n, c->Pp, c->lanes, c->dhalf, 1.0, c->P0, pt0);
    launch_kprod<double>(L, o, pt0, R, 1, DOT_NONE, w, 0);
    launch_axpby(L, np, 0.0, R, -1.0, R);
    EMIN_TRY(cuda_status(cudaMemsetAsync(X, 0, vb, c->stream)));
    EMIN_TRY(cuda_status(cudaMemsetAsync(Y, 0, vb, c->stream)));
    EMIN_TRY(cuda_status(cudaMemsetAsync(zero, 0, vb, c->stream)));
    for (int k = 0; k < n_iters; ++k) {
        if (k % sgl == 0) {
            EMIN_TRY(dcopy(cpr[k / sgl], R));
            EMIN_TRY(dcopy(cpy[k / sgl], Y));
        }
        EMIN_TRY(dot(R, R, &gam[k]));
        bet[k] = k ? gam[k] / gam[k - 1] : 0.0;
        launch_axpby(L, np, 1.0, R, bet[k], Y);
        launch_kprod<double>(L, o, Y, Yb, 1, DOT_AUX, w, 0);
        EMIN_TRY(read_aux(c, w, &del[k]));
        if (!(del[k] > 0.0) || !std::isfinite(del[k]) || !std::isfinite(gam[k]))
            return EMIN_ERR_BREAKDOWN;
        alp[k] = gam[k] / del[k];
        launch_axpby(L, np, alp[k], Y, 1.0, X);
        launch_axpby(L, np, -alp[k], Yb, 1.0, R);
    }
    // reverse: xbar = D^{-1/2} dL/dP; the output's dependence on d
    launch_row_scale<double, double>(L, n, c->Pp, c->lanes, c->dsq, 1.0, dLdP, xbar);
    EMIN_TRY(cuda_status(cudaMemsetAsync(c->unr_dext, 0, sizeof(double) * n, c->stream)));
    launch_row_dot_acc(L, n, c->Pp, dLdP, X, c->dsq, 3, -0.5, c->unr_dext);
    EMIN_TRY(cuda_status(cudaMemsetAsync(rbar, 0, vb, c->stream)));
    EMIN_TRY(cuda_status(cudaMemsetAsync(ybar, 0, vb, c->stream)));
    EMIN_TRY(cuda_status(cudaMemsetAsync(c->unr_ghat, 0, sizeof(double) * na, c->stream)));
    double gcarry = 0.0;
    for (int seg = ncp - 1; seg >= 0; --seg) {
        const int k0 = seg * sgl, k1 = std::min(k0 + sgl, n_iters);
        EMIN_TRY(dcopy(R, cpr[seg]));
        EMIN_TRY(dcopy(Y, cpy[seg]));
        for (int k = k0; k < k1; ++k) {  // the segment again, from its checkpoint
            EMIN_TRY(dcopy(sr[k - k0], R));
            launch_axpby(L, np, 1.0, R, bet[k], Y);
            EMIN_TRY(dcopy(sy[k - k0], Y));
            launch_kprod<double>(L, o, Y, Yb, 1, DOT_NONE, w, 0);
            launch_axpby(L, np, -alp[k], Yb, 1.0, R);
        }
        for (int k = k1 - 1; k >= k0; --k) {
            const double *yk = sy[k - k0], *rk = sr[k - k0];
            const double *ykm1 = k == 0 ? zero : (k > k0 ? sy[k - k0 - 1] : cpy[seg]);
            launch_kprod<double>(L, o, yk, wt, 1, DOT_NONE, w, 0);
            double a1, a2;
            EMIN_TRY(dot(xbar, yk, &a1));
            EMIN_TRY(dot(rbar, wt, &a2));
            const double abar = a1 - a2;
            const double dbar = -abar * alp[k] / del[k];
            EMIN_TRY(dcopy(wb, rbar));
            launch_axpby(L, np, dbar, yk, -alp[k], wb);
            EMIN_TRY(dcopy(pw, wb));
            launch_project<double>(L, o, pw, 1.0);
            launch_kprod<double>(L, o, pw, tmp, 0, DOT_NONE, w, 0);
            launch_axpby(L, np, alp[k], xbar, 1.0, ybar);
            launch_axpby(L, np, dbar, wt, 1.0, ybar);
            launch_axpby(L, np, 1.0, tmp, 1.0, ybar);
            launch_outer(L, n, c->Ap, c->Aj, c->Pp, c->Pj, pw, yk, 1.0, c->tA, c->maxrow_p);
            launch_axpby(L, na, 1.0, c->tA, 1.0, c->unr_ghat);
            double bbar = 0.0;
            if (k > 0) EMIN_TRY(dot(ybar, ykm1, &bbar));
            const double gbar = gcarry + abar / del[k] + (k > 0 ? bbar / gam[k - 1] : 0.0);
            launch_axpby(L, np, 1.0, ybar, 1.0, rbar);
            launch_axpby(L, np, 2.0 * gbar, rk, 1.0, rbar);
            gcarry = k > 0 ? -bbar * gam[k] / (gam[k - 1] * gam[k - 1]) : 0.0;
            launch_axpby(L, np, 0.0, ybar, bet[k], ybar);
        }
    }
    // r~_0 = -Pi K^ p~0: p~0bar = -K^ Pi rbar, ghat += mask_A(-(Pi rbar) p~0^T)
    EMIN_TRY(dcopy(pw, rbar));
    launch_project<double>(L, o, pw, 1.0);
    launch_kprod<double>(L, o, pw, tmp, 0, DOT_NONE, w, 0);  // tmp = -p~0bar
    launch_outer(L, n, c->Ap, c->Aj, c->Pp, c->Pj, pw, pt0, -1.0, c->tA, c->maxrow_p);
    launch_axpby(L, na, 1.0, c->tA, 1.0, c->unr_ghat);
    // p0bar = dL/dP + D^{1/2} p~0bar;  p~0 = D^{1/2} p0 puts 1/2 d^{-1/2} <p~0bar, p0> on d
    launch_row_scale<double, double>(L, n, c->Pp, c->lanes, c->dhalf, -1.0, tmp, pw);
    launch_axpby(L, np, 1.0, dLdP, 1.0, pw);
    launch_row_dot_acc(L, n, c->Pp, tmp, c->P0, c->dsq, 1, -0.5, c->unr_dext);
    launch_grad_a(L, n, c->Ap, c->Aj, c->Av, c->dsq, c->unr_ghat, c->unr_dext, gA);
    // the corrected P0 moves with B: dL/dB(i,:) = G_i^{-1} B_i^T p0bar_i
    launch_lsq(L, n, c->k, c->Pp, c->Pj, c->Bc, c->Ginv, pw, gB);
    return check_launch();
}

}  // namespace

extern "C" {

static int call_backward_unrolled(emin_ctx *c, const double *dL_dP, int n_iters, double *dL_dAval,
                           double *dL_dB, int on_device) {
    if (!c || !dL_dP || n_iters < 1) return EMIN_ERR_ARG;
    DeviceGuard g(c->device);
    if (c->sticky != EMIN_OK) return c->sticky;
    if (c->opts.precond != EMIN_JACOBI || c->opts.precision != EMIN_FP64) {
        std::snprintf(g_last_error, sizeof(g_last_error),
                      "unrolled adjoint: needs an FP64 context with the Jacobi preconditioner");
        return EMIN_ERR_ARG;
    }
    if (!c->adj.R) {
        EMIN_TRY(alloc_work(c, c->adj, true));
        if (!c->tA) EMIN_TRY(dalloc(c, &c->tA, c->nnz_a));
        EMIN_TRY(dalloc(c, &c->tmu, (long long)c->n * c->k));
        EMIN_TRY(dalloc(c, &c->Pstar, c->nnz_p));
        if (!c->Ah64) EMIN_TRY(dalloc(c, &c->Ah64, c->nnz_a));
        if (c->sell_ptr && !c->sa64) EMIN_TRY(dalloc(c, &c->sa64, c->nnz_sell));
        if (c->k == 1 && !c->qv64) EMIN_TRY(dalloc(c, &c->qv64, c->nnz_p));
    }
    if (!c->have64) form_scaled64(c);
    if (c->n == 0) return EMIN_OK;
    EMIN_TRY(copy_in(c, c->t64b, dL_dP, sizeof(double) * c->nnz_p, on_device));
    double *gA = nullptr;
    if (!c->unr_ghat) EMIN_TRY(dalloc(c, &c->unr_ghat, c->nnz_a));
    EMIN_TRY(dalloc_once(c, &c->unr_gA, c->nnz_a));
    gA = c->unr_gA;
    EMIN_TRY(unrolled_backward(c, c->t64b, n_iters, gA, c->tmu));
    if (dL_dAval) EMIN_TRY(copy_out(c, dL_dAval, gA, sizeof(double) * c->nnz_a, on_device));
    if (dL_dB)
        EMIN_TRY(copy_out(c, dL_dB, c->tmu, sizeof(double) * (size_t)c->n * c->k, on_device));
    return sync(c);
}

static int call_backward(emin_ctx *c, const double *dL_dP, double *dL_dAval, double *dL_dB,
                  int max_adj_iters, double adj_tol, int on_device, int *adj_iters) {
    if (!c || !dL_dP || max_adj_iters < 0 || !(adj_tol >= 0)) return EMIN_ERR_ARG;
    DeviceGuard g(c->device);
    if (c->sticky != EMIN_OK) return c->sticky;
    if (!c->adj.R) {
        EMIN_TRY(alloc_work(c, c->adj, true));
        if (!c->tA) EMIN_TRY(dalloc(c, &c->tA, c->nnz_a));
        EMIN_TRY(dalloc(c, &c->tmu, (long long)c->n * c->k));
        EMIN_TRY(dalloc(c, &c->Pstar, c->nnz_p));
        if (!c->Ah64) EMIN_TRY(dalloc(c, &c->Ah64, c->nnz_a));
        if (c->sell_ptr && !c->sa64) EMIN_TRY(dalloc(c, &c->sa64, c->nnz_sell));
        if (c->k == 1 && !c->qv64) EMIN_TRY(dalloc(c, &c->qv64, c->nnz_p));
        if (c->opts.precond == EMIN_SGS && !c->sgs_fval64) {
            EMIN_TRY(dalloc(c, &c->sgs_fval64, c->sgs_nf));
            EMIN_TRY(dalloc(c, &c->sgs_bval64, c->sgs_nb));
            EMIN_TRY(dalloc(c, &c->sgs_batval64, c->sgs_nbval));
            c->have64 = false;
        }
    }
    if (!c->have64) form_scaled64(c);
    const Ops<double> o = iter_ops64(c);
    Work<double> &w = c->adj;
    // P* (kept from the forward) and dL/dP
    EMIN_TRY(form_p(c, c->Pstar));
    EMIN_TRY(copy_in(c, c->t64b, dL_dP, sizeof(double) * c->nnz_p, on_device));
    // Pi K Pi u = 1/2 Pi dL/dP from u = 0, in the scaled variables
    // (right-hand side D^{-1/2} dL/dP / 2, solution u = D^{-1/2} u~)
    launch_row_scale<double, double>(c->L, c->n, c->Pp, c->lanes, c->dsq, 0.5, c->t64b, w.R);
    EMIN_TRY(start_pcg<double>(c, o, w, nullptr));
    EMIN_TRY(iterate_impl<double>(c, o, w, max_adj_iters, adj_tol));
    if (c->hstate->status != EMIN_OK) return c->hstate->status;
    if (adj_iters) *adj_iters = c->hstate->applied;
    launch_row_scale<double, double>(c->L, c->n, c->Pp, c->lanes, c->dsq, 1.0, w.X, c->t64c);
    // S = mask(A U);  x = dL/dP - 2 S;  mu = G^{-1} B_i^T x
    launch_kprod<double>(c->L, plain_ops64(c), c->t64c, w.Yb, 0, DOT_NONE, w, 0);
    launch_axpby(c->L, c->nnz_p, 1.0, c->t64b, -2.0, w.Yb);
    if (dL_dB) {
        launch_lsq(c->L, c->n, c->k, c->Pp, c->Pj, c->Bc, c->Ginv, w.Yb, c->tmu);
        EMIN_TRY(check_launch());
        EMIN_TRY(copy_out(c, dL_dB, c->tmu, sizeof(double) * c->n * c->k, on_device));
    }
    if (dL_dAval) {
        launch_outer(c->L, c->n, c->Ap, c->Aj, c->Pp, c->Pj, c->t64c, c->Pstar, -2.0, c->tA,
                     c->maxrow_p);
        EMIN_TRY(check_launch());
        EMIN_TRY(copy_out(c, dL_dAval, c->tA, sizeof(double) * c->nnz_a, on_device));
    }
    return sync(c);
}

int emin_stats(emin_ctx *c, double *dE_hist, int cap, int *n_hist, int *n_rank_deficient,
               int *n_applied) {
    if (!c) return EMIN_ERR_ARG;
    DeviceGuard g(c->device);
    const Work<double> *w64 = &c->w64;
    const DevState *st = (c->opts.precision == EMIN_MIXED) ? c->w32.st : w64->st;
    const double *hist = (c->opts.precision == EMIN_MIXED) ? c->w32.hist : w64->hist;
    const int hcap = (c->opts.precision == EMIN_MIXED) ? c->w32.hist_cap : w64->hist_cap;
    EMIN_TRY(read_state(c, st));
    const int k = c->hstate->k;
    if (n_hist) *n_hist = k;
    if (n_applied) *n_applied = c->hstate->applied;
    if (n_rank_deficient) *n_rank_deficient = c->ndef;
    if (dE_hist && cap > 0) {
        int m = k < cap ? k : cap;
        if (m > hcap) m = hcap;
        if (m > 0) {
            EMIN_TRY(cuda_status(cudaMemcpyAsync(dE_hist, hist, sizeof(double) * m,
                                                 cudaMemcpyDeviceToHost, c->stream)));
            EMIN_TRY(sync(c));
        }
    }
    return EMIN_OK;
}

int emin_set_timing(emin_ctx *c, int enable) {
    if (!c) return EMIN_ERR_ARG;
    c->timing = enable > 0 ? enable : 0;
    for (int j = 0; j < 3; ++j) {
        c->tms[j] = 0.0;
        c->tlaunch[j] = 0;
    }
    return EMIN_OK;
}

int emin_timing(emin_ctx *c, double *ms, long long *launches, long long *total_launches) {
    if (!c) return EMIN_ERR_ARG;
    for (int j = 0; j < 3; ++j) {
        if (ms) ms[j] = c->tms[j];
        if (launches) launches[j] = c->tlaunch[j];
    }
    if (total_launches) *total_launches = launches_so_far() - c->launches_at_create;
    return EMIN_OK;
}

int emin_sizes(emin_ctx *c, long long *nnz_a, long long *nnz_p) {
    if (!c) return EMIN_ERR_ARG;
    if (nnz_a) *nnz_a = c->nnz_a;
    if (nnz_p) *nnz_p = c->nnz_p;
    return EMIN_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// With emin_opts.checks the gather kernels bound-check their indices and OR a
// fault into the context's check word; every call below reads the word after
// its work and reports a fault as EMIN_ERR_PATTERN (sticky: the context's
// later calls report it too).
// ---------------------------------------------------------------------------
namespace {
int with_checks(emin_ctx *c, int st) {
    if (!c || st != EMIN_OK || !c->opts.checks || !c->chkw) return st;
    int *hw = c->hint + kHintChk;
    EMIN_TRY(cuda_status(cudaMemcpyAsync(hw, c->chkw, sizeof(int), cudaMemcpyDeviceToHost,
                                         c->stream)));
    EMIN_TRY(sync(c));
    if (*hw != 0) {
        std::snprintf(g_last_error, sizeof(g_last_error),
                      "bounds check: a kernel index fell outside its array (plan or input fault)");
        c->sticky = EMIN_ERR_PATTERN;
        return EMIN_ERR_PATTERN;
    }
    return EMIN_OK;
}
}  // namespace

extern "C" {

int emin_reset(emin_ctx *c) { return with_checks(c, call_reset(c)); }
int emin_set_values(emin_ctx *c, const double *A_val, const double *B, const double *P0_val,
                    int on_device) {
    return with_checks(c, call_set_values(c, A_val, B, P0_val, on_device));
}
int emin_iterate(emin_ctx *c, int n_iters, double tol, int *iters_done, double *rel_dE_last) {
    return with_checks(c, call_iterate(c, n_iters, tol, iters_done, rel_dE_last));
}
int emin_get_p(emin_ctx *c, double *P_out, int out_on_device) {
    return with_checks(c, call_get_p(c, P_out, out_on_device));
}
int emin_energy(emin_ctx *c, double *E) { return with_checks(c, call_energy(c, E)); }
int emin_kprod(emin_ctx *c, const double *X, double *out, int project, int on_device) {
    return with_checks(c, call_kprod(c, X, out, project, on_device));
}
int emin_outer(emin_ctx *c, const double *U, const double *V, double *out, int on_device) {
    return with_checks(c, call_outer(c, U, V, out, on_device));
}
int emin_energy_grad(emin_ctx *c, const double *X, double scale, double *E, double *dE_dX,
                     double *dE_dAval, int on_device) {
    return with_checks(c, call_energy_grad(c, X, scale, E, dE_dX, dE_dAval, on_device));
}
int emin_backward_unrolled(emin_ctx *c, const double *dL_dP, int n_iters, double *dL_dAval,
                           double *dL_dB, int on_device) {
    return with_checks(c, call_backward_unrolled(c, dL_dP, n_iters, dL_dAval, dL_dB, on_device));
}
int emin_backward(emin_ctx *c, const double *dL_dP, double *dL_dAval, double *dL_dB,
                  int max_adj_iters, double adj_tol, int on_device, int *adj_iters) {
    return with_checks(c, call_backward(c, dL_dP, dL_dAval, dL_dB, max_adj_iters, adj_tol,
                                        on_device, adj_iters));
}

}  // extern "C"
