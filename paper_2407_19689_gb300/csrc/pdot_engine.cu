// pdot_engine.cu -- host engine and C ABI (include/pdot.h) of the GB300 PDOT
// library: workspaces in HBM, the launch sequence of Algorithm 2 with the
// Sec. 5 controller (one solve = an init check, then chunks of K passes plus
// one check, captured as CUDA graphs), Algorithm 3 rounding, and the
// continuous-batching engine.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <limits>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/pdot.h"
#include "pdot_internal.h"

// NVTX ranges (header-only NVTX v3) name the phases of a solve and of the
// batch engine for profilers (Nsight Systems, ncu --nvtx).  With no tool
// attached a push or pop is one call through a no-op function pointer.
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define PDOT_HAVE_NVTX 1
#endif

using namespace pdot;

namespace pdot {
int launch_round_rowsum(const void* X, int xtype, long long m, long long n, long long ldx, const double* rs,
                        const double* cs, double* rowout, double* colpart, int colparts, void* stream);
int launch_round_write(const void* X, int xtype, long long m, long long n, long long ldx, const double* rs,
                       const double* cs, const double* er, const double* ec, double inv_l1, void* Xout,
                       long long ldo, const void* C, int ctype, long long ldc, const GenSpec* gen,
                       double* objpart, int parts, void* stream);
int launch_colreduce(const double* colpart, int parts, long long n, double* out, void* stream);
int launch_dual_bound(const void* C, int ctype, long long ldc, const GenSpec* gen, const double* p,
                      const double* f, const double* g, long long m, long long n, double* colmin, int parts,
                      double* q, double* out, void* stream);
}  // namespace pdot

namespace {

using Clock = std::chrono::steady_clock;

struct CudaError {
    cudaError_t e;
};

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) throw CudaError{e_};           \
    } while (0)

#define CKL(call)                                             \
    do {                                                      \
        int e_ = (call);                                      \
        if (e_ != 0) throw CudaError{(cudaError_t)e_};        \
    } while (0)

struct ArgError {
    const char* what;
};

// A host-thread NVTX range for the lifetime of the object.
struct Range {
    explicit Range(const char* name) {
#ifdef PDOT_HAVE_NVTX
        nvtxRangePushA(name);
#else
        (void)name;
#endif
    }
    ~Range() {
#ifdef PDOT_HAVE_NVTX
        nvtxRangePop();
#endif
    }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// The plan kernels read C in 16-byte units (row starts 16-byte aligned): FP32
// and FP64 rows need ldc % 4 == 0, BF16 rows ldc % 8 == 0.
bool c_layout_ok(const void* C, int ctype, long long ldc) {
    const long long q = ctype == PDOT_BF16 ? 8 : 4;
    return ((uintptr_t)C % 16) == 0 && ldc % q == 0;
}
long long padded_ldc(long long n, int ctype) {
    const long long q = ctype == PDOT_BF16 ? 8 : 4;
    return (n + q - 1) / q * q;
}

int ttype_of(int ctype) {
    return ctype == PDOT_F64 ? TT_F64 : ctype == PDOT_BF16 ? TT_BF16 : ctype == PDOT_POINTS ? TT_GEN : TT_F32;
}
// Bytes per stored cost entry (a generated cost stores none).
size_t csize_of(int ctype) {
    return ctype == PDOT_F64 ? 8 : ctype == PDOT_BF16 ? 2 : ctype == PDOT_POINTS ? 0 : 4;
}

// The generated cost of a PDOT_POINTS descriptor (host memory, checked by
// check_common_args).
GenSpec gen_spec_of(const void* C) {
    const pdot_points_cost* d = static_cast<const pdot_points_cost*>(C);
    GenSpec g;
    g.xs = d->xs;
    g.ys = d->ys;
    g.d = d->d;
    g.kind = (int)d->dist;
    g.div = d->divisor;
    g.inv = 1.0f / d->divisor;
    return g;
}
size_t xsize_of(int xtype) { return xtype == PDOT_F64 ? 8 : 4; }

// One instance's device buffers (a single cudaMalloc carved into pieces).
struct Work {
    long long m = 0, n = 0, ldx = 0;
    int xtype = 0, tile_rows = 0;
    int nstrips = 0, nchunks = 0, ntiles = 0, nvt = 0;
    void* base = nullptr;
    size_t bytes = 0;
    void* X = nullptr;
    double* V = nullptr;
    double* rowpart = nullptr;
    double* colpart = nullptr;
    double* rowpart2 = nullptr;
    double* colpart2 = nullptr;
    double* tpart = nullptr;
    double* vpart = nullptr;
    Ctrl* ctrl = nullptr;
    unsigned* ticket = nullptr;
    // internal copy of C when the caller's layout does not allow 16-byte loads
    void* Cpad = nullptr;
    size_t cpad_bytes = 0;
};

size_t work_bytes(long long m, long long n, int xtype, int tile_rows, Work* w) {
    const long long ldx = (n + 3) / 4 * 4;
    const int nstrips = (int)((n + STRIP - 1) / STRIP);
    const int nchunks = (int)((m + tile_rows - 1) / tile_rows);
    const long long ntiles = (long long)nstrips * nchunks;
    const int nvt = (int)((m + n + VE - 1) / VE);
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = align_up(off + b, 256); return o; };
    const size_t oX = take((size_t)NSLOT * m * ldx * xsize_of(xtype));
    const size_t oV = take((size_t)NSLOT * 2 * (m + n) * sizeof(double));
    const size_t oR = take((size_t)nstrips * m * sizeof(double));
    const size_t oC = take((size_t)nchunks * ldx * sizeof(double));
    const size_t oR2 = take((size_t)nstrips * m * sizeof(double));
    const size_t oC2 = take((size_t)nchunks * ldx * sizeof(double));
    const size_t oT = take((size_t)ntiles * TP * sizeof(double));
    const size_t oP = take((size_t)nvt * VP * sizeof(double));
    const size_t oS = take(sizeof(Ctrl));
    const size_t oK = take(sizeof(unsigned));
    if (w) {
        w->m = m; w->n = n; w->ldx = ldx; w->xtype = xtype; w->tile_rows = tile_rows;
        w->nstrips = nstrips; w->nchunks = nchunks; w->ntiles = (int)ntiles; w->nvt = nvt;
        char* b = (char*)w->base;
        w->X = b + oX;
        w->V = (double*)(b + oV);
        w->rowpart = (double*)(b + oR);
        w->colpart = (double*)(b + oC);
        w->rowpart2 = (double*)(b + oR2);
        w->colpart2 = (double*)(b + oC2);
        w->tpart = (double*)(b + oT);
        w->vpart = (double*)(b + oP);
        w->ctrl = (Ctrl*)(b + oS);
        w->ticket = (unsigned*)(b + oK);
    }
    return off;
}

Inst make_inst(const Work& w, const void* C, int ctype, long long ldc, const double* f, const double* g) {
    Inst I;
    memset(&I, 0, sizeof(I));
    I.m = w.m; I.n = w.n; I.ldc = ldc; I.ldx = w.ldx;
    I.C = C; I.ctype = ctype; I.xtype = w.xtype;
    if (ctype == PDOT_POINTS) {
        I.gen = gen_spec_of(C);
        I.C = nullptr;
        I.ldc = 0;
    }
    I.f = f; I.g = g;
    I.X = w.X; I.xslot = w.m * w.ldx;
    I.V = w.V; I.vslot = 2 * (w.m + w.n);
    I.rowpart = w.rowpart; I.colpart = w.colpart; I.tpart = w.tpart; I.vpart = w.vpart;
    I.rowpart2 = w.rowpart2; I.colpart2 = w.colpart2;
    I.ctrl = w.ctrl; I.ticket = w.ticket;
    I.nstrips = w.nstrips; I.nchunks = w.nchunks; I.tile_rows = w.tile_rows; I.ntiles = w.ntiles; I.nvt = w.nvt;
    I.l2_keep_c = 0;
    return I;
}

struct Graph {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        if (g) cudaGraphDestroy(g);
        exec = nullptr;
        g = nullptr;
        kernels = 0;
    }
};

}  // namespace

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------
struct BatchEngine;

struct pdot_handle {
    pdot_options opt;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sm_count = 0;
    LaunchCfg cfg{};
    LaunchCfg cfg_base{};
    unsigned* wctr = nullptr;
    int64_t launches = 0;
    std::string last_error;

    // single-instance path
    Work ws;
    Inst* d_inst = nullptr;
    TileRef* d_tmap = nullptr;
    TileRef* d_vmap = nullptr;
    size_t tmap_cap = 0, vmap_cap = 0;
    int* d_cnt = nullptr;        // [0] plan tiles, [1] vector tiles of the single-instance path
    int* h_cnt = nullptr;        // pinned staging
    Ctrl* h_ctrl = nullptr;      // pinned
    Inst* h_inst = nullptr;      // pinned
    int* h_status = nullptr;     // pinned [2]
    Graph chunk;                 // K x (pass, dual) + (kkt, checkvec)
    long long chunk_key[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    std::map<long long, std::pair<int, int>> tune_cache;   // (m, n, ttype) -> (pass kernel, tile_rows)
    int autotune = 1;            // time pass-kernel candidates on a shape's first solve
    int batch_min_rows = 16;     // smallest tile height of a batched instance (even)
    int res_clusters = 0;        // resident-kernel clusters the device holds at once (0: not available)
    int* d_res1 = nullptr;       // {0, 1}: the list and count of a single-instance resident launch
    bool res_on = false;         // the current single-instance call runs in the resident kernel
    // host staging for pdot_solve_host
    void* stage = nullptr;
    size_t stage_bytes = 0;
    double* round_scratch = nullptr;
    size_t round_scratch_bytes = 0;
    double* d_sched = nullptr;   // step-size schedule factors (see Ctrl::sched)
    long long sched_len = 0;

    BatchEngine* batch = nullptr;
    int l2_hint = 0;             // L2 eviction-priority hints in the bulk pass (measured slower; opt-in)
    int coop = 0;                // 1: single FP32-plan solves run one cooperative launch per chunk (opt-in: measured slower)
    GridBar* d_gb = nullptr;
    long long l2_bytes = 0;
    void* d_tp = nullptr;        // pdot_time_pass: a second instance view and controller
};

namespace {

void free_work(Work& w) {
    if (w.base) cudaFree(w.base);
    if (w.Cpad) cudaFree(w.Cpad);
    w = Work();
}

void ensure_work(pdot_handle* h, long long m, long long n, int xtype, int tile_rows) {
    Work& w = h->ws;
    if (w.base && w.m == m && w.n == n && w.xtype == xtype && w.tile_rows == tile_rows) return;
    h->chunk.reset();
    void* cpad = w.Cpad;
    size_t cpb = w.cpad_bytes;
    w.Cpad = nullptr;
    if (w.base) cudaFree(w.base);
    w = Work();
    w.Cpad = cpad;
    w.cpad_bytes = cpb;
    const size_t bytes = work_bytes(m, n, xtype, tile_rows, nullptr);
    void* base = nullptr;
    cudaError_t e = cudaMalloc(&base, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw CudaError{cudaErrorMemoryAllocation};
    }
    w.base = base;
    w.bytes = bytes;
    work_bytes(m, n, xtype, tile_rows, &w);
    CK(cudaMemsetAsync(w.ticket, 0, sizeof(unsigned), h->stream));
}

void ensure_maps(pdot_handle* h) {
    const Work& w = h->ws;
    if ((size_t)w.ntiles > h->tmap_cap) {
        if (h->d_tmap) cudaFree(h->d_tmap);
        h->d_tmap = nullptr;
        CK(cudaMalloc(&h->d_tmap, sizeof(TileRef) * (size_t)w.ntiles));
        h->tmap_cap = (size_t)w.ntiles;
    }
    if ((size_t)w.nvt > h->vmap_cap) {
        if (h->d_vmap) cudaFree(h->d_vmap);
        h->d_vmap = nullptr;
        CK(cudaMalloc(&h->d_vmap, sizeof(TileRef) * (size_t)w.nvt));
        h->vmap_cap = (size_t)w.nvt;
    }
    std::vector<TileRef> tm((size_t)w.ntiles), vm((size_t)w.nvt);
    for (int t = 0; t < w.ntiles; ++t) tm[(size_t)t] = TileRef{0, t};
    for (int t = 0; t < w.nvt; ++t) vm[(size_t)t] = TileRef{0, t};
    CK(cudaMemcpyAsync(h->d_tmap, tm.data(), sizeof(TileRef) * tm.size(), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->d_vmap, vm.data(), sizeof(TileRef) * vm.size(), cudaMemcpyHostToDevice, h->stream));
    h->h_cnt[0] = w.ntiles;
    h->h_cnt[1] = w.nvt;
    CK(cudaMemcpyAsync(h->d_cnt, h->h_cnt, 2 * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));   // vectors above are pageable and go out of scope
}

void validate_marginals(pdot_handle* h, long long m, long long n, const double* f, const double* g, bool host,
                        double* norm_b) {
    std::vector<double> hf((size_t)m), hg((size_t)n);
    if (host) {
        memcpy(hf.data(), f, sizeof(double) * (size_t)m);
        memcpy(hg.data(), g, sizeof(double) * (size_t)n);
    } else {
        CK(cudaMemcpyAsync(hf.data(), f, sizeof(double) * (size_t)m, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(hg.data(), g, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    double sf = 0.0, sg = 0.0, nb = 0.0;
    for (double v : hf) {
        if (!(v >= 0.0) || !std::isfinite(v)) throw ArgError{"f has a negative or non-finite entry"};
        sf += v;
        nb += v * v;
    }
    for (double v : hg) {
        if (!(v >= 0.0) || !std::isfinite(v)) throw ArgError{"g has a negative or non-finite entry"};
        sg += v;
        nb += v * v;
    }
    if (std::fabs(sf - sg) > 1e-9 * std::max(sf, 1.0)) throw ArgError{"sum(f) != sum(g)"};
    *norm_b = std::sqrt(nb);
}

// Rows per plan tile.  `kernel`: the FP32-plan pass kernel the tiles are for
// (0 register, 1 bulk per row, 2 bulk per 4-row group).
// split: for the grouped kernel too, one tile per resident warp instead of
// 32-row tiles through the queue.
int tile_rows_for(pdot_handle* h, long long m, long long n, int ttype, int kernel, bool batch, bool split = false) {
    if (h->opt.tile_rows > 0) return h->opt.tile_rows;
    const long long nstrips = (n + STRIP - 1) / STRIP;
    if (ttype == TT_F64) kernel = 0;
    if (batch) {
        // A batched instance's tiles depend on its own shape only, so its
        // result is the same alone or in any mix: the split a single solve
        // takes (one tile per resident warp, for a large instance running
        // nearly alone at the end of a batch or in a sparse stream), but no
        // fewer than batch_min_rows rows (in a crowded batch, per-tile costs
        // stay small) and no more than 64.
        long long tr = tile_rows_for(h, m, n, ttype, ttype == TT_F64 ? 0 : h->cfg_base.pass_bulk, false, true);
        tr = std::max<long long>(tr, h->batch_min_rows);
        tr = std::min<long long>(tr, 64);
        return (int)tr;
    }
    if (kernel == 2 && !split) return 32;   // grouped kernel: short tiles through the dynamic queue
    // Otherwise split the instance evenly over the resident warps, one tile
    // each (the last wave of a dynamic queue would leave a tail), as tall as
    // that allows (fewer column partials).
    const long long blocks = ttype == TT_F64 ? h->cfg.tile_blocks_f64
                             : kernel == 1   ? (h->coop && h->cfg.coop_blocks > 0 ? h->cfg.coop_blocks
                                                                                  : h->cfg.bulk_blocks)
                             : kernel == 2   ? h->cfg.group_blocks
                                             : h->cfg.tile_blocks;
    const long long warps = blocks * TWARPS;
    long long nch = warps / nstrips;
    if (nch < 1) nch = 1;
    long long tr = (m + nch - 1) / nch;
    tr = (tr + 1) / 2 * 2;
    if (tr < 2) tr = 2;
    if (tr > 4096) tr = 4096;
    return (int)tr;
}

// Autotuner cache key: shape, cost type and (generated costs) coordinate count.
long long tune_key(long long m, long long n, int ttype, int gen_d) {
    return ((m * 1000003LL + n) * 4 + ttype) * 16 + gen_d;
}
int gen_dims_of(const void* C, int ctype) {
    return ctype == PDOT_POINTS ? (int)static_cast<const pdot_points_cost*>(C)->d : 0;
}

int pick_tile_rows(pdot_handle* h, long long m, long long n, int ttype, bool batch = false, int gen_d = 0) {
    if (!batch && h->opt.tile_rows <= 0) {
        const long long key = tune_key(m, n, ttype, gen_d);
        auto it = h->tune_cache.find(key);
        if (it != h->tune_cache.end() && it->second.first == h->cfg.pass_bulk) return it->second.second;
    }
    return tile_rows_for(h, m, n, ttype, h->cfg.pass_bulk, batch);
}

const void* prepare_C(pdot_handle* h, long long m, long long n, const void* C, int ctype, long long ldc,
                      long long* ldc_used) {
    const size_t cs = csize_of(ctype);
    if (ctype == PDOT_POINTS) {   // nothing stored: the descriptor travels in the instance
        *ldc_used = 0;
        return C;
    }
    if (c_layout_ok(C, ctype, ldc)) {
        *ldc_used = ldc;
        return C;
    }
    // Copy into a padded buffer whose rows start on 16-byte boundaries.
    Work& w = h->ws;
    const long long ldp = padded_ldc(n, ctype);
    const size_t bytes = (size_t)m * ldp * cs;
    if (w.cpad_bytes < bytes) {
        if (w.Cpad) cudaFree(w.Cpad);
        w.Cpad = nullptr;
        w.cpad_bytes = 0;
        CK(cudaMalloc(&w.Cpad, bytes));
        w.cpad_bytes = bytes;
    }
    CK(cudaMemcpy2DAsync(w.Cpad, ldp * cs, C, ldc * cs, n * cs, m, cudaMemcpyDeviceToDevice, h->stream));
    *ldc_used = ldp;
    return w.Cpad;
}

void init_ctrl(pdot_handle* h, Ctrl* S, long long m, long long n, double tol, double norm_b, double norm_C,
               bool fixed, double eta_fixed, double omega_fixed) {
    const pdot_options& o = h->opt;
    memset(S, 0, sizeof(Ctrl));
    S->adaptive_step = fixed ? 0 : o.adaptive_step;
    S->adaptive_restart = o.adaptive_restart;
    S->pw_update = o.primal_weight_update;
    double eta = o.eta0;
    if (!(eta > 0.0)) eta = S->adaptive_step ? 1.0 / std::sqrt((double)(m + n)) : 0.5 / std::sqrt((double)(m + n));
    double omega = o.omega0 > 0.0 ? o.omega0 : 1.0;
    if (fixed) {
        eta = eta_fixed;
        omega = omega_fixed;
    }
    S->eta = eta;
    S->omega = omega;
    S->wavg = 1.0;
    S->tau = eta / omega;
    S->sigma = eta * omega;
    S->tol = tol;
    S->beta = o.beta;
    S->beta_suff = o.beta_suff;
    S->beta_nec = o.beta_nec;
    S->beta_art = o.beta_art;
    S->theta = o.theta;
    S->R = o.R;
    S->eps_zero = o.eps_zero;
    S->rel_mode = o.rel_mode;
    S->max_passes = o.max_iter > 0 ? o.max_iter : std::numeric_limits<long long>::max() / 4;
    S->norm_b = norm_b;
    S->norm_C = norm_C;
    S->sched = h->d_sched;
    S->sched_len = h->sched_len;
    S->cur = 0; S->anc = 0; S->bar = 1; S->nxt = 2; S->barn = 3;
    S->status = ST_RUNNING;
    S->res_slot = S->res_xslot = 0;
}

void launch_count(pdot_handle* h, int k) { h->launches += k; }

// Keep C resident in L2 when it takes at most half of it (it is re-read every
// pass; the plan streams get evict-first so they do not push it out).
bool keep_c_in_l2(pdot_handle* h, const Inst& I) {
    if (!h->l2_hint || h->l2_bytes <= 0 || I.ctype == PDOT_POINTS) return false;
    const double cbytes = (double)I.m * (double)I.ldc * (double)csize_of(I.ctype);
    return cbytes <= 0.5 * (double)h->l2_bytes;
}

// Upload the instance descriptor and reset the work counters.
void stage_instance(pdot_handle* h, const Inst& I) {
    *h->h_inst = I;
    h->h_inst->l2_keep_c = keep_c_in_l2(h, I) ? 1 : 0;
    h->cfg.gen_dims = I.ctype == PDOT_POINTS ? I.gen.d : 0;
    CK(cudaMemcpyAsync(h->d_inst, h->h_inst, sizeof(Inst), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemsetAsync(h->wctr, 0, sizeof(unsigned) * WC_N, h->stream));
}

void run_check(pdot_handle* h, int ttype, int mode) {
    const Work& w = h->ws;
    CKL(launch_kkt(ttype, h->d_inst, h->d_tmap, h->d_cnt, h->wctr, mode, h->cfg, h->stream));
    CKL(launch_checkvec(h->d_inst, h->d_vmap, h->d_cnt + 1, w.nvt, h->wctr, mode, h->cfg, h->stream));
    launch_count(h, 2);
}

void run_step(pdot_handle* h, int ttype) {
    const Work& w = h->ws;
    CKL(launch_pass(ttype, h->d_inst, h->d_tmap, h->d_cnt, h->wctr, h->cfg, h->stream));
    CKL(launch_dual(h->d_inst, h->d_vmap, h->d_cnt + 1, w.nvt, h->wctr, h->cfg, h->stream, true));
    launch_count(h, 2);
}

// After a check: form the average plan it picked, if it picked one.
void run_avgfix(pdot_handle* h, int ttype) {
    CKL(launch_avgfix(ttype, h->d_inst, h->d_tmap, h->d_cnt, h->cfg, h->stream));
    launch_count(h, 1);
}

void issue_chunk_kernels(pdot_handle* h, int ttype, int K) {
    for (int s = 0; s < K; ++s) run_step(h, ttype);
    run_check(h, ttype, MODE_CHECK);
    run_avgfix(h, ttype);
}

// An instance runs in the resident kernel when the option allows it, the
// device can hold its clusters, it has an FP32 plan and a stored FP32 / BF16
// cost, and its plan and average fit a cluster's shared memory.
bool resident_for(pdot_handle* h, long long m, long long n, int ttype) {
    return h->opt.resident == 1 && h->opt.tile_rows == 0 && h->res_clusters > 0 && h->opt.x_dtype == PDOT_F32 &&
           (ttype == TT_F32 || ttype == TT_BF16) && resident_fits(m, n);
}

bool use_coop(pdot_handle* h, int ttype) {
    return h->coop && h->cfg.coop_blocks > 0 && ttype != TT_F64 && ttype != TT_GEN && h->cfg.pass_bulk == 1;
}

void launch_chunk(pdot_handle* h, int ttype, int K) {
    const Work& w = h->ws;
    if (h->res_on) {
        // the whole check period (K passes and the check) in one resident launch
        CKL(launch_resident(ttype, h->d_inst, h->d_res1, h->d_res1 + 1, 1, K, K, 0, h->cfg, h->stream));
        launch_count(h, 1);
        return;
    }
    if (use_coop(h, ttype)) {
        CK(cudaMemsetAsync(h->wctr, 0, sizeof(unsigned) * WC_N, h->stream));
        CK(cudaMemsetAsync(h->d_gb, 0, sizeof(GridBar), h->stream));
        CKL(launch_chunk_coop(ttype, h->d_inst, h->d_tmap, h->d_cnt, h->d_vmap, h->d_cnt + 1, h->wctr, h->d_gb, K,
                              h->cfg, h->stream));
        launch_count(h, 1);
        run_avgfix(h, ttype);
        return;
    }
    const long long key[8] = {(long long)(uintptr_t)w.base,
                              (long long)(uintptr_t)h->d_tmap ^ ((long long)(uintptr_t)h->d_vmap << 1),
                              w.m * 4 + ttype,
                              w.n,
                              K,
                              (long long)h->cfg.comp * 1000 + (long long)h->cfg.pdl * 100 +
                                  (long long)h->cfg.pass_bulk * 10 + (long long)h->cfg.pass_u,
                              w.tile_rows,
                              h->cfg.gen_dims};
    if (!h->opt.use_graph) {
        issue_chunk_kernels(h, ttype, K);
        return;
    }
    if (!h->chunk.exec || memcmp(key, h->chunk_key, sizeof(key)) != 0) {
        h->chunk.reset();
        const int64_t before = h->launches;
        CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        try {
            issue_chunk_kernels(h, ttype, K);
        } catch (...) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(h->stream, &g);
            if (g) cudaGraphDestroy(g);
            h->launches = before;
            throw;
        }
        CK(cudaStreamEndCapture(h->stream, &h->chunk.g));
        CK(cudaGraphInstantiate(&h->chunk.exec, h->chunk.g, 0));
        h->chunk.kernels = (int)(h->launches - before);
        h->launches = before;
        memcpy(h->chunk_key, key, sizeof(key));
    }
    CK(cudaGraphLaunch(h->chunk.exec, h->stream));
    launch_count(h, h->chunk.kernels);
}

void fill_result(const Ctrl& S, pdot_result* r, pdot_status st) {
    r->status = st;
    r->primal_obj = S.r_cx;
    r->dual_obj = S.r_dual;
    r->gap = S.r_gap;
    r->kkt = S.r_kkt;
    r->rel_kkt = S.r_rel;
    r->rel_primal = S.r_rel_p;
    r->rel_dual = S.r_rel_d;
    r->rel_gap = S.r_rel_gap;
    r->iters = S.total;
    r->passes = S.passes;
    r->restarts = S.restarts;
    r->rejected_steps = S.rejected;
    r->eta = S.eta;
    r->omega = S.omega;
    r->returned_average = S.res_avg;
    r->tile_rows = 0;   // set by the caller, which knows the workspace
}

pdot_status map_status(int st) {
    switch (st) {
        case ST_OK: return PDOT_OK;
        case ST_ARG: return PDOT_ERR_ARG;
        case ST_DEVICE: return PDOT_ERR_CUDA;   // a bounded device wait gave up
        case ST_NUMERIC: return PDOT_ERR_NUMERIC;
        case ST_MAX_ITER: return PDOT_MAX_ITER;
        case ST_TIMEOUT: return PDOT_TIMEOUT;
        case ST_CANCELLED: return PDOT_CANCELLED;
        default: return PDOT_ERR_CUDA;
    }
}

// Copy the plan of a slot (m x ldx) out as dense m x n.
void copy_plan_out(pdot_handle* h, int slot, void* X_out, cudaMemcpyKind kind) {
    const Work& w = h->ws;
    const size_t xs = xsize_of(w.xtype);
    const char* src = (const char*)w.X + (size_t)slot * w.m * w.ldx * xs;
    CK(cudaMemcpy2DAsync(X_out, (size_t)w.n * xs, src, (size_t)w.ldx * xs, (size_t)w.n * xs, (size_t)w.m, kind,
                         h->stream));
}

void copy_duals_out(pdot_handle* h, int slot, double* p_out, double* q_out, cudaMemcpyKind kind) {
    const Work& w = h->ws;
    const double* V = w.V + (size_t)slot * 2 * (w.m + w.n);
    if (p_out) CK(cudaMemcpyAsync(p_out, V, sizeof(double) * (size_t)w.m, kind, h->stream));
    if (q_out) CK(cudaMemcpyAsync(q_out, V + w.m, sizeof(double) * (size_t)w.n, kind, h->stream));
}

// Upload a dense m x n plan and its duals into slot 0.
void upload_state(pdot_handle* h, const void* X, const double* p, const double* q) {
    const Work& w = h->ws;
    const size_t xs = xsize_of(w.xtype);
    CK(cudaMemsetAsync(w.X, 0, (size_t)w.m * w.ldx * xs, h->stream));
    CK(cudaMemcpy2DAsync(w.X, (size_t)w.ldx * xs, X, (size_t)w.n * xs, (size_t)w.n * xs, (size_t)w.m,
                         cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemsetAsync(w.V, 0, sizeof(double) * 2 * (size_t)(w.m + w.n), h->stream));
    CK(cudaMemcpyAsync(w.V, p, sizeof(double) * (size_t)w.m, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(w.V + w.m, q, sizeof(double) * (size_t)w.n, cudaMemcpyDeviceToDevice, h->stream));
}

void check_common_args(pdot_handle* h, long long m, long long n, const void* C, int ctype, long long ldc,
                       const double* f, const double* g) {
    if (!h) throw ArgError{"null handle"};
    if (m < 1 || n < 1) throw ArgError{"m and n must be >= 1"};
    if (!C || !f || !g) throw ArgError{"null C, f or g"};
    if (ctype != PDOT_F32 && ctype != PDOT_BF16 && ctype != PDOT_F64 && ctype != PDOT_POINTS)
        throw ArgError{"unknown c_dtype"};
    const int xt = h->opt.x_dtype;
    if (xt != PDOT_F32 && xt != PDOT_F64) throw ArgError{"x_dtype must be F32 or F64"};
    if (ctype == PDOT_POINTS) {
        const pdot_points_cost* d = static_cast<const pdot_points_cost*>(C);
        if (d->d < 1 || d->d > GEN_DMAX) throw ArgError{"points cost: d must be in 1..8"};
        if ((int)d->dist < 0 || (int)d->dist > 3) throw ArgError{"points cost: unknown dist"};
        if (!d->xs || !d->ys) throw ArgError{"points cost: null coordinates"};
        if (!(std::isfinite(d->divisor) && d->divisor > 0.f)) throw ArgError{"points cost: divisor must be finite and > 0"};
        if (xt != PDOT_F32) throw ArgError{"generated costs need F32 plans"};
    } else if (ldc < n) {
        throw ArgError{"ldc < n"};
    }
    if ((xt == PDOT_F64) != (ctype == PDOT_F64))
        throw ArgError{"F64 plans need F64 costs and F32 plans need F32/BF16 costs"};
    if (m > (1LL << 31) / 2 || n > (1LL << 31) / 2) throw ArgError{"dimension too large"};
}

// Algorithm 3 on the plan of `slot` (or an external device plan), writing
// X_out (dense m x n).  Returns <C, X_feas> when C is given.
double round_plan_dev(pdot_handle* h, long long m, long long n, int xtype, const void* Xsrc, long long ldx,
                      const double* f, const double* g, void* X_out, const void* C, int ctype, long long ldc,
                      const GenSpec* gen);

// Compensated reduced cost (option compensated_cost; reading C9): 2 = on
// where a pass is latency-bound (fewer than 4M plan entries, the autotuner's
// threshold too), where it costs nothing, and off above, where it costs about
// 6 % per pass at 4096^2.  The batch engine (many small instances) takes it
// unless it is switched off.
bool compensation_for(pdot_handle* h, long long m, long long n) {
    const int c = h->opt.compensated_cost;
    return c == 1 || (c == 2 && m * n < (1LL << 22));
}

// Autotuner: on the first single-instance solve of a shape (m, n, dtype),
// time whole PDHG steps (fused pass + dual update, constant step) for each
// candidate (pass kernel, tile height) on this device with CUDA events --
// after three untimed steps, so the running average is read -- and keep the
// fastest.  Small shapes are launch-bound: they take the default untimed.
void autotune_pass(pdot_handle* h, long long m, long long n, const void* C, int ctype, long long ldc,
                   const double* f, const double* g) {
    const int ttype = ttype_of(ctype);
    const int gen_d = gen_dims_of(C, ctype);
    h->cfg.comp = compensation_for(h, m, n) ? 1 : 0;
    if (h->opt.pass_kernel > 0) {
        // An explicit kernel choice: no timing, no cache entry.
        int v = h->opt.pass_kernel - 1;
        if (ttype == TT_GEN && gen_d > 4 && v == 2) v = 1;   // no grouped kernel beyond 4 coordinates
        h->cfg.pass_bulk = v;
        return;
    }
    if (ttype == TT_GEN && gen_d > 4) {
        // More than 4 coordinates: the per-row kernel is the only bulk one.
        h->cfg.pass_bulk = h->cfg_base.pass_bulk ? 1 : 0;
        return;
    }
    if (ttype == TT_F64 || h->opt.tile_rows > 0 || !h->cfg_base.pass_bulk) return;
    const long long key = tune_key(m, n, ttype, gen_d);
    auto it = h->tune_cache.find(key);
    if (it != h->tune_cache.end()) {
        h->cfg.pass_bulk = it->second.first;
        return;
    }
    if (!h->autotune || m * n < (1LL << 22)) {
        const int kern = h->autotune ? 1 : h->cfg_base.pass_bulk;
        h->tune_cache[key] = {kern, tile_rows_for(h, m, n, ttype, kern, false)};
        h->cfg.pass_bulk = kern;
        return;
    }
    // Each candidate is timed on whole PDHG steps (pass + dual update): tile
    // height also sets how many partial sums the dual update has to read.
    // Tile height 0: one tile per resident warp.  The first candidate (the
    // grouped kernel with one tile per warp, the fastest at 4096^2 in every
    // measurement) is the default the others must beat by 5 %.
    const int cands[5][2] = {{2, 0}, {1, 0}, {2, 32}, {2, 64}, {2, 128}};
    float best = 1e30f;
    int best_k = 2, best_tr = tile_rows_for(h, m, n, ttype, 2, false, true);
    const int reps = m * n >= (1LL << 26) ? 6 : 20;
    for (const auto& c : cands) {
        const int kern = c[0];
        const int tr = c[1] ? c[1] : tile_rows_for(h, m, n, ttype, kern, false, true);
        h->cfg.pass_bulk = kern;
        ensure_work(h, m, n, h->opt.x_dtype, tr);
        ensure_maps(h);
        Work& w = h->ws;
        long long ldc_used = ldc;
        const void* Cd = prepare_C(h, m, n, C, ctype, ldc, &ldc_used);
        stage_instance(h, make_inst(w, Cd, ctype, ldc_used, f, g));
        Ctrl* S = h->h_ctrl;
        init_ctrl(h, S, m, n, -1.0, 1.0, 1.0, true, 0.5 / std::sqrt((double)(m + n)), 1.0);
        CK(cudaMemcpyAsync(w.ctrl, S, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemsetAsync(w.ticket, 0, sizeof(unsigned), h->stream));
        CK(cudaMemsetAsync(w.X, 0, (size_t)w.m * w.ldx * xsize_of(w.xtype), h->stream));
        CK(cudaMemsetAsync(w.V, 0, sizeof(double) * 2 * (size_t)(w.m + w.n), h->stream));
        run_check(h, ttype, MODE_INIT);
        for (int s2 = 0; s2 < 3; ++s2) run_step(h, ttype);
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        CK(cudaEventRecord(e0, h->stream));
        for (int r = 0; r < reps; ++r) run_step(h, ttype);
        CK(cudaEventRecord(e1, h->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        launch_count(h, 3);
        // The first candidate is the default; another one must beat the best
        // so far by 5 % to be taken, so near-ties (which would change the
        // FP32 summation order, and with it the trajectory, from run to run)
        // keep the default.
        if (best > 1e29f || ms < 0.95f * best) {
            best = ms;
            best_k = kern;
            best_tr = tr;
        }
    }
    h->tune_cache[key] = {best_k, best_tr};
    h->cfg.pass_bulk = best_k;
}

// ---------------------------------------------------------------------------
// Solver-state blob of pdot_solve_from (checkpoint / resume): a header with
// the controller, then the plans of the current, average and anchor slots
// (m x ldx each) and their vector sets ([p | q | r | c]).
// ---------------------------------------------------------------------------
constexpr uint64_t STATE_MAGIC = 0x3230455441545350ull;   // "PSTATE02" (average stored as its deviation)
constexpr size_t STATE_HEAD = 1024;
struct StateHead {
    uint64_t magic;
    long long m, n;
    int xtype;
    int replay;   // 1: the last check stopped at the pass budget before its restart logic ran
    Ctrl ctrl;
};
static_assert(sizeof(StateHead) <= STATE_HEAD, "state header too large");

struct StateLayout {
    size_t plan, vec, total;
    size_t plan_off(int k) const { return STATE_HEAD + (size_t)k * plan; }
    size_t vec_off(int k) const { return STATE_HEAD + 3 * plan + (size_t)k * vec; }
};
StateLayout state_layout(long long m, long long n, int xtype) {
    const long long ldx = (n + 3) / 4 * 4;
    StateLayout L;
    L.plan = align_up((size_t)m * (size_t)ldx * xsize_of(xtype), 256);
    L.vec = align_up(sizeof(double) * 2 * (size_t)(m + n), 256);
    L.total = STATE_HEAD + 3 * L.plan + 3 * L.vec;
    return L;
}

// Write the state of the handle's workspace (controller S, as read back from
// the device after the last chunk) into the device blob `out`.
void export_state(pdot_handle* h, const Ctrl& S, void* out) {
    const Work& w = h->ws;
    const StateLayout L = state_layout(w.m, w.n, w.xtype);
    StateHead hd;
    memset(&hd, 0, sizeof(hd));
    hd.magic = STATE_MAGIC;
    hd.m = w.m;
    hd.n = w.n;
    hd.xtype = w.xtype;
    hd.replay = S.status == ST_MAX_ITER ? 1 : 0;
    hd.ctrl = S;
    char* o = static_cast<char*>(out);
    CK(cudaMemcpyAsync(o, &hd, sizeof(hd), cudaMemcpyHostToDevice, h->stream));
    const int role[3] = {S.cur, S.bar, S.anc};
    const size_t pb = (size_t)w.m * (size_t)w.ldx * xsize_of(w.xtype), vb = sizeof(double) * 2 * (size_t)(w.m + w.n);
    for (int k = 0; k < 3; ++k) {
        CK(cudaMemcpyAsync(o + L.plan_off(k), (const char*)w.X + (size_t)role[k] * pb, pb, cudaMemcpyDeviceToDevice,
                           h->stream));
        CK(cudaMemcpyAsync(o + L.vec_off(k), w.V + (size_t)role[k] * 2 * (size_t)(w.m + w.n), vb,
                           cudaMemcpyDeviceToDevice, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));   // hd lives on this stack frame
}

// Load a blob into the workspace (slots 0, 1, 2 = current, average, anchor)
// and build the controller to upload: the blob's iteration state with the
// handle's options (S holds a freshly initialised controller on entry).
// Returns true when the stopped check must run again (its restart logic).
bool import_state(pdot_handle* h, const void* in, Ctrl* S) {
    const Work& w = h->ws;
    StateHead hd;
    CK(cudaMemcpyAsync(&hd, in, sizeof(hd), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (hd.magic != STATE_MAGIC || hd.m != w.m || hd.n != w.n || hd.xtype != w.xtype)
        throw ArgError{"state_in is not a state blob of this shape and plan type"};
    const StateLayout L = state_layout(w.m, w.n, w.xtype);
    const char* b = static_cast<const char*>(in);
    const size_t pb = (size_t)w.m * (size_t)w.ldx * xsize_of(w.xtype), vb = sizeof(double) * 2 * (size_t)(w.m + w.n);
    for (int k = 0; k < 3; ++k) {
        CK(cudaMemcpyAsync((char*)w.X + (size_t)k * pb, b + L.plan_off(k), pb, cudaMemcpyDeviceToDevice, h->stream));
        CK(cudaMemcpyAsync(w.V + (size_t)k * 2 * (size_t)(w.m + w.n), b + L.vec_off(k), vb, cudaMemcpyDeviceToDevice,
                           h->stream));
    }
    const Ctrl& B = hd.ctrl;
    S->eta = B.eta; S->omega = B.omega; S->tau = B.tau; S->sigma = B.sigma; S->wavg = B.wavg;
    S->kkt0 = B.kkt0; S->kkt_prev = B.kkt_prev;
    S->k = B.k; S->total = B.total; S->passes = B.passes; S->restarts = B.restarts; S->rejected = B.rejected;
    S->checks = B.checks - (hd.replay ? 1 : 0);   // the stopped check runs again
    S->norm_b = B.norm_b; S->norm_C = B.norm_C;
    S->r_rp2 = B.r_rp2; S->r_rd2 = B.r_rd2; S->r_cx = B.r_cx; S->r_dual = B.r_dual; S->r_gap = B.r_gap;
    S->r_kkt = B.r_kkt; S->r_rel_p = B.r_rel_p; S->r_rel_d = B.r_rel_d; S->r_rel_gap = B.r_rel_gap; S->r_rel = B.r_rel;
    S->cur = 0; S->bar = 1; S->anc = 2; S->nxt = 3; S->barn = 4;
    S->status = ST_RUNNING;
    S->res_slot = S->res_xslot = 0;
    S->res_avg = 0;
    return hd.replay != 0;
}

// Initial point of pdot_solve_from in slot 0 (a null part is 0).
void upload_start(pdot_handle* h, const pdot_start* st) {
    const Work& w = h->ws;
    const size_t xs = xsize_of(w.xtype);
    CK(cudaMemsetAsync(w.X, 0, (size_t)w.m * w.ldx * xs, h->stream));
    CK(cudaMemsetAsync(w.V, 0, sizeof(double) * 2 * (size_t)(w.m + w.n), h->stream));
    if (st && st->X0)
        CK(cudaMemcpy2DAsync(w.X, (size_t)w.ldx * xs, st->X0, (size_t)w.n * xs, (size_t)w.n * xs, (size_t)w.m,
                             cudaMemcpyDeviceToDevice, h->stream));
    if (st && st->p0) CK(cudaMemcpyAsync(w.V, st->p0, sizeof(double) * (size_t)w.m, cudaMemcpyDeviceToDevice, h->stream));
    if (st && st->q0)
        CK(cudaMemcpyAsync(w.V + w.m, st->q0, sizeof(double) * (size_t)w.n, cudaMemcpyDeviceToDevice, h->stream));
}

pdot_status solve_impl(pdot_handle* h, long long m, long long n, const void* C, int ctype, long long ldc,
                       const double* f, const double* g, double tol, void* X_out, double* p_out, double* q_out,
                       pdot_result* res, const pdot_start* start = nullptr) {
    const auto t_start = Clock::now();
    if (!res) throw ArgError{"null result"};
    check_common_args(h, m, n, C, ctype, ldc, f, g);
    if (!(tol > 0.0)) throw ArgError{"tol must be > 0"};
    double norm_b = 0.0;
    validate_marginals(h, m, n, f, g, false, &norm_b);
    const int ttype = ttype_of(ctype);
    {
        const Range r_("autotune");
        autotune_pass(h, m, n, C, ctype, ldc, f, g);
    }
    h->res_on = h->opt.pass_kernel == 0 && resident_for(h, m, n, ttype);
    const int tr = pick_tile_rows(h, m, n, ttype, false, gen_dims_of(C, ctype));
    ensure_work(h, m, n, h->opt.x_dtype, tr);
    ensure_maps(h);
    Work& w = h->ws;
    long long ldc_used = ldc;
    const void* Cd = prepare_C(h, m, n, C, ctype, ldc, &ldc_used);
    const Inst I = make_inst(w, Cd, ctype, ldc_used, f, g);
    stage_instance(h, I);

    Ctrl* S = h->h_ctrl;
    init_ctrl(h, S, m, n, tol, norm_b, 0.0, false, 0.0, 0.0);   // norms: computed by the init check
    CK(cudaMemsetAsync(w.ticket, 0, sizeof(unsigned), h->stream));
    {
        const Range r_("start");   // the init check, or the replayed check of a resumed solve
        if (start && start->state_in) {
            // Resume: the saved state, the handle's options; the check the saved
            // solve stopped at runs again with its restart logic.
            const bool replay = import_state(h, start->state_in, S);
            CK(cudaMemcpyAsync(w.ctrl, S, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream));
            if (replay && h->res_on) {
                // the stopped check again, in the kernel that will run the solve
                CKL(launch_resident(ttype, h->d_inst, h->d_res1, h->d_res1 + 1, 1, 0,
                                    std::max(1, h->opt.restart_check_every), 1, h->cfg, h->stream));
                launch_count(h, 1);
            } else if (replay) {
                run_check(h, ttype, MODE_CHECK);
                run_avgfix(h, ttype);
            }
        } else {
            CK(cudaMemcpyAsync(w.ctrl, S, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream));
            upload_start(h, start);   // X = 0, p = q = 0 (C1) unless a starting point is given
            run_check(h, ttype, MODE_INIT);
        }
    }

    const int K = std::max(1, h->opt.restart_check_every);
    const double tlim = h->opt.time_limit_s;
    int status = ST_RUNNING;
    bool timed_out = false;
    cudaEvent_t ev[2];
    CK(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
    try {
        const Range r_("chunks");
        // Keep two chunks in flight: the host reads chunk i's status while
        // chunk i+1 runs (a chunk issued after termination is a no-op).
        long long i = 0;
        launch_chunk(h, ttype, K);
        CK(cudaMemcpyAsync(&h->h_status[0], &w.ctrl->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaEventRecord(ev[0], h->stream));
        for (;;) {
            launch_chunk(h, ttype, K);
            const int nb = (int)((i + 1) & 1);
            CK(cudaMemcpyAsync(&h->h_status[nb], &w.ctrl->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
            CK(cudaEventRecord(ev[nb], h->stream));
            CK(cudaEventSynchronize(ev[i & 1]));
            status = h->h_status[i & 1];
            if (status != ST_RUNNING) break;
            if (tlim > 0.0 && std::chrono::duration<double>(Clock::now() - t_start).count() > tlim) {
                timed_out = true;
                break;
            }
            ++i;
        }
        CK(cudaStreamSynchronize(h->stream));
    } catch (...) {
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        throw;
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    CK(cudaMemcpyAsync(S, w.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const Range r_result("result");
    if (start && start->state_out) export_state(h, *S, start->state_out);
    if (timed_out && S->status == ST_RUNNING) {
        // Evaluate the current iterate and report it.
        run_check(h, ttype, MODE_INIT);
        CK(cudaMemcpyAsync(S, w.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        if (S->status == ST_RUNNING) {
            S->status = ST_TIMEOUT;
            S->res_slot = S->res_xslot = S->cur;
            S->res_avg = 0;
        }
    }
    const pdot_status st = map_status(S->status);
    fill_result(*S, res, st);
    res->tile_rows = h->res_on ? 0 : w.tile_rows;
    const double mn = (double)m * (double)n;
    const double bc = (double)csize_of(ctype), bx = (double)xsize_of(w.xtype);
    res->hbm_bytes = (double)S->passes * mn * (bc + 4.0 * bx) + (double)S->checks * mn * (bc + 3.0 * bx);
    res->rounded_obj = std::numeric_limits<double>::quiet_NaN();
    const int slot = S->res_slot, xslot = S->res_xslot;   // vector set / plan of the reported point
    const char* Xslot = (const char*)w.X + (size_t)xslot * (size_t)(w.m * w.ldx) * xsize_of(w.xtype);
    if (h->opt.round_plan) {
        res->rounded_obj =
            round_plan_dev(h, w.m, w.n, w.xtype, Xslot, w.ldx, f, g, X_out, I.C, ctype, ldc_used, &I.gen);
    } else if (X_out) {
        copy_plan_out(h, xslot, X_out, cudaMemcpyDeviceToDevice);
    }
    copy_duals_out(h, slot, p_out, q_out, cudaMemcpyDeviceToDevice);
    CK(cudaStreamSynchronize(h->stream));
    res->seconds = std::chrono::duration<double>(Clock::now() - t_start).count();
    return st;
}

template <typename F>
pdot_status guarded(pdot_handle* h, F&& fn) {
    try {
        return fn();
    } catch (const ArgError& e) {
        if (h) h->last_error = e.what;
        return PDOT_ERR_ARG;
    } catch (const CudaError& e) {
        if (h) h->last_error = cudaGetErrorString(e.e);
        if (e.e == cudaErrorMemoryAllocation) return PDOT_ERR_OOM;
        return PDOT_ERR_CUDA;
    } catch (const std::bad_alloc&) {
        if (h) h->last_error = "host allocation failed";
        return PDOT_ERR_OOM;
    } catch (...) {
        if (h) h->last_error = "unexpected exception";
        return PDOT_ERR_CUDA;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Algorithm 3 (rounding)
// ---------------------------------------------------------------------------
namespace {
double round_plan_dev(pdot_handle* h, long long m, long long n, int xtype, const void* Xsrc, long long ldx,
                      const double* f, const double* g, void* X_out, const void* C, int ctype, long long ldc,
                      const GenSpec* gen) {
    const int parts = 64;   // column-partial rows (fixed order)
    const size_t need = sizeof(double) * (size_t)(4 * m + 4 * n + (size_t)parts * n + parts + 8);
    if (h->round_scratch_bytes < need) {
        if (h->round_scratch) cudaFree(h->round_scratch);
        h->round_scratch = nullptr;
        h->round_scratch_bytes = 0;
        CK(cudaMalloc(&h->round_scratch, need));
        h->round_scratch_bytes = need;
    }
    double* xs = h->round_scratch;      // row scales (m)
    double* ys = xs + m;                // column scales (n)
    double* rsum = ys + n;              // row sums (m)
    double* csum = rsum + m;            // column sums (n)
    double* er = csum + n;              // err_r (m)
    double* ec = er + m;                // err_c (n)
    double* colpart = ec + n;           // parts x n
    double* objpart = colpart + (size_t)parts * n;
    void* out = X_out;
    void* tmp = nullptr;
    if (!out) {
        CK(cudaMalloc(&tmp, (size_t)m * n * xsize_of(xtype)));
        out = tmp;
    }
    // 1) r = X1 -> x_i = min(f_i / r_i, 1)
    CKL(launch_round_rowsum(Xsrc, xtype, m, n, ldx, nullptr, nullptr, rsum, colpart, parts, h->stream));
    // 2) column sums of diag(x) X -> y_j = min(g_j / c_j, 1)
    // 3) row and column sums of diag(x) X diag(y) -> err_r, err_c
    // The host drives the scalar glue with tiny vector kernels inside the launcher file.
    CKL(launch_colreduce(colpart, parts, n, csum, h->stream));
    launch_count(h, 2);
    // Scales are computed on the host from the sums (O(m+n), once per solve).
    std::vector<double> hr((size_t)m), hc((size_t)n), hf((size_t)m), hg((size_t)n), hx((size_t)m), hy((size_t)n);
    CK(cudaMemcpyAsync(hr.data(), rsum, sizeof(double) * m, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(hf.data(), f, sizeof(double) * m, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(hg.data(), g, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (long long i = 0; i < m; ++i) hx[(size_t)i] = hr[(size_t)i] > 0.0 ? std::min(hf[(size_t)i] / hr[(size_t)i], 1.0) : 1.0;
    CK(cudaMemcpyAsync(xs, hx.data(), sizeof(double) * m, cudaMemcpyHostToDevice, h->stream));
    CKL(launch_round_rowsum(Xsrc, xtype, m, n, ldx, xs, nullptr, rsum, colpart, parts, h->stream));
    CKL(launch_colreduce(colpart, parts, n, csum, h->stream));
    launch_count(h, 2);
    CK(cudaMemcpyAsync(hc.data(), csum, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (long long j = 0; j < n; ++j) hy[(size_t)j] = hc[(size_t)j] > 0.0 ? std::min(hg[(size_t)j] / hc[(size_t)j], 1.0) : 1.0;
    CK(cudaMemcpyAsync(ys, hy.data(), sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    CKL(launch_round_rowsum(Xsrc, xtype, m, n, ldx, xs, ys, rsum, colpart, parts, h->stream));
    CKL(launch_colreduce(colpart, parts, n, csum, h->stream));
    launch_count(h, 2);
    CK(cudaMemcpyAsync(hr.data(), rsum, sizeof(double) * m, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(hc.data(), csum, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    double l1 = 0.0;
    for (long long i = 0; i < m; ++i) { hr[(size_t)i] = hf[(size_t)i] - hr[(size_t)i]; l1 += std::fabs(hr[(size_t)i]); }
    for (long long j = 0; j < n; ++j) hc[(size_t)j] = hg[(size_t)j] - hc[(size_t)j];
    CK(cudaMemcpyAsync(er, hr.data(), sizeof(double) * m, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(ec, hc.data(), sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    const double inv_l1 = l1 > 0.0 ? 1.0 / l1 : 0.0;
    // 4) X_feas = diag(x) X diag(y) + err_r err_c^T / ||err_r||_1, and <C, X_feas>
    CKL(launch_round_write(Xsrc, xtype, m, n, ldx, xs, ys, er, ec, inv_l1, out, n, C, ctype, ldc, gen, objpart,
                           parts, h->stream));
    launch_count(h, 1);
    std::vector<double> ho((size_t)parts);
    CK(cudaMemcpyAsync(ho.data(), objpart, sizeof(double) * parts, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (tmp) cudaFree(tmp);
    double obj = 0.0;
    for (int k = 0; k < parts; ++k) obj += ho[(size_t)k];
    return obj;
}
}  // namespace

// ---------------------------------------------------------------------------
// Continuous-batching engine.
//
// Every resident instance owns a workspace (cudaMallocAsync, stream ordered)
// and a controller; all of them advance together through the same
// multi-instance kernels: one chunk = chunk_checks x (K x (pass, dual) +
// (kkt, checkvec)) plus a controller snapshot copied to pinned host memory,
// captured once as a CUDA graph (tile maps and counts live in device memory,
// so a new batch composition only rewrites those buffers).  Between chunks
// pdot_poll retires finished instances (stream-ordered output copies and
// frees), admits queued requests while the HBM budget and slot count allow,
// runs their init checks, and launches the next chunk, which then overlaps
// with the host's bookkeeping.  Instances join at chunk boundaries, so every
// instance's checks fall after multiples of K of its own passes.
// ---------------------------------------------------------------------------
namespace {

struct BSlot {
    uint64_t id = 0;
    pdot_request req{};
    pdot_points_cost pts{};   // copy of a PDOT_POINTS descriptor (req.C points here)
    int ttype = 0;
    Work w;
    size_t bytes = 0;
    Clock::time_point t_submit;
    bool cancel = false;
    bool timed_out = false;   // past its time limit: a stop request goes out before the next chunk
    bool stop_sent = false;   // that request has been issued
    bool fresh = true;        // admitted, init check not run yet
    bool resident = false;    // runs in the resident kernel (its init check in the tile kernels)
    Ctrl last{};              // last snapshot of its controller
};

template <typename T>
struct DevArr {
    T* d = nullptr;
    T* h = nullptr;   // pinned staging
    size_t cap = 0;
    void ensure(size_t n) {
        if (n <= cap) return;
        size_t c = cap ? cap : 64;
        while (c < n) c *= 2;
        if (d) cudaFree(d);
        if (h) cudaFreeHost(h);
        d = nullptr;
        h = nullptr;
        cap = 0;
        CK(cudaMalloc(&d, sizeof(T) * c));
        CK(cudaMallocHost(&h, sizeof(T) * c));
        cap = c;
    }
    void release() {
        if (d) cudaFree(d);
        if (h) cudaFreeHost(h);
        d = nullptr;
        h = nullptr;
        cap = 0;
    }
};

}  // namespace

// Device count words of the batch engine: plan tiles per type, vector tiles,
// instances, init-check plan tiles per type, init-check vector tiles, and two
// pinned source words for status writes (cancel, time limit).
constexpr int CNT_VEC = NTT, CNT_INST = NTT + 1, CNT_INIT = NTT + 2, CNT_INIT_VEC = 2 * NTT + 2,
              CNT_RES = 2 * NTT + 3, CNT_WORDS = 2 * NTT + 5, CNT_TIMEOUT = 14, CNT_CANCEL = 15;
static_assert(CNT_WORDS <= CNT_TIMEOUT, "count words overlap");

struct BatchEngine {
    std::deque<BSlot*> queue;
    std::vector<BSlot*> live;
    std::vector<std::pair<uint64_t, pdot_result>> done;
    uint64_t next_id = 1;
    size_t budget = 0, used = 0;
    DevArr<Inst> insts;
    DevArr<TileRef> tmap[NTT];
    DevArr<TileRef> vmap;
    DevArr<TileRef> tmap_init[NTT];
    DevArr<TileRef> vmap_init;
    DevArr<int> rlist[2];     // resident instances with FP32 / BF16 costs (indices into insts)
    int res_grid[2] = {0, 0}; // cluster-count bound of each resident launch (bucketed)
    DevArr<Ctrl> snap[2];     // controller snapshots of the two chunks that can be in flight
    DevArr<Ctrl> ctrl_stage;
    DevArr<int> cnt;          // counts, laid out as the CNT_* indices below
    Graph graph;
    int gen_dims = 0;         // largest d of the active generated costs
    int types = 0;            // plan-kernel types of the active instances (bit mask)
    long long graph_key[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // Chunks in flight (oldest first, at most two): each one's snapshot buffer
    // and the instance ids in the order its snapshot lists them.
    struct Flight {
        int buf = 0;
        std::vector<uint64_t> ids;
    };
    std::deque<Flight> flights;
    cudaEvent_t ev_chunk[2] = {nullptr, nullptr};
    int next_buf = 0;
    // Pinned staging (instance table, maps, counts, controllers) is rewritten
    // only after the copies that read it last have run.
    cudaEvent_t ev_staged = nullptr;
    bool staged_pending = false;
    // Results whose output copies are queued behind a chunk still in flight.
    struct Pending {
        cudaEvent_t ev = nullptr;
        std::vector<std::pair<uint64_t, pdot_result>> results;
    };
    std::deque<Pending> pending_done;
    int nv_live = 0;
    int nv_grid = 32;          // vector-kernel grid: live vector tiles rounded up to a power of two
    int64_t chunks = 0;
};

namespace {

size_t slot_bytes(pdot_handle* h, const pdot_request& r, int tile_rows) {
    size_t b = work_bytes(r.m, r.n, h->opt.x_dtype, tile_rows, nullptr);
    if (r.c_dtype != PDOT_POINTS && !c_layout_ok(r.C, r.c_dtype, r.ldc))
        b += align_up((size_t)r.m * padded_ldc(r.n, r.c_dtype) * csize_of(r.c_dtype), 256);
    return b;
}

BatchEngine* batch_of(pdot_handle* h) {
    if (!h->batch) {
        BatchEngine* B = new BatchEngine();
        h->batch = B;
        CK(cudaEventCreateWithFlags(&B->ev_chunk[0], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&B->ev_chunk[1], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&B->ev_staged, cudaEventDisableTiming));
        if (h->opt.hbm_budget_bytes > 0) {
            B->budget = (size_t)h->opt.hbm_budget_bytes;
        } else {
            size_t fr = 0, tot = 0;
            CK(cudaMemGetInfo(&fr, &tot));
            B->budget = (size_t)(0.9 * (double)fr);
        }
        B->cnt.ensure(16);
    }
    return h->batch;
}

void batch_free_slot(pdot_handle* h, BSlot* s) {
    if (s->w.base) CK(cudaFreeAsync(s->w.base, h->stream));
    s->w.base = nullptr;
    h->batch->used -= s->bytes;
}

// Rebuild the device-side composition: instance table, tile maps per type,
// vector-tile map, and the init maps of freshly admitted instances.
void batch_compose(pdot_handle* h) {
    BatchEngine* B = h->batch;
    const int L = (int)B->live.size();
    B->insts.ensure((size_t)std::max(L, 1));
    // The instances the next chunk advances: all, or the oldest and then
    // younger ones (admission order) whose per-pass plan bytes fit the
    // active budget.  A paused instance keeps its state; its trajectory only
    // depends on its own passes, which always come in whole check periods.
    std::vector<char> active((size_t)L, 1);
    if (h->opt.batch_active_bytes > 0) {
        const double cap = (double)h->opt.batch_active_bytes;
        double used = 0.0;
        for (int i = 0; i < L; ++i) {
            const BSlot* s = B->live[(size_t)i];
            const double b = (double)s->req.m * (double)s->req.n *
                             ((double)csize_of(s->req.c_dtype) + 4.0 * (double)xsize_of(h->opt.x_dtype));
            active[(size_t)i] = (i == 0 || used + b <= cap) ? 1 : 0;
            if (active[(size_t)i]) used += b;
        }
    }
    size_t nt[NTT] = {}, nti[NTT] = {}, nv = 0, nvi = 0, nr[2] = {0, 0};
    int gd = 0;
    B->types = 0;
    for (int i = 0; i < L; ++i) {
        BSlot* s = B->live[(size_t)i];
        if (active[(size_t)i] && s->resident) {
            nr[s->ttype == TT_BF16 ? 1 : 0] += 1;
        } else if (active[(size_t)i]) {
            B->types |= 1 << s->ttype;
            if (s->req.c_dtype == PDOT_POINTS) gd = std::max(gd, (int)s->pts.d);
            nt[s->ttype] += (size_t)s->w.ntiles;
            nv += (size_t)s->w.nvt;
        }
        if (s->fresh) {
            nti[s->ttype] += (size_t)s->w.ntiles;
            nvi += (size_t)s->w.nvt;
        }
    }
    for (int t = 0; t < NTT; ++t) {
        B->tmap[t].ensure(std::max<size_t>(nt[t], 1));
        B->tmap_init[t].ensure(std::max<size_t>(nti[t], 1));
    }
    B->vmap.ensure(std::max<size_t>(nv, 1));
    B->vmap_init.ensure(std::max<size_t>(nvi, 1));
    for (int r = 0; r < 2; ++r) B->rlist[r].ensure(std::max<size_t>(nr[r], 1));
    size_t orr[2] = {0, 0};
    B->gen_dims = gd;
    size_t ot[NTT] = {}, oti[NTT] = {}, ov = 0, ovi = 0;
    for (int i = 0; i < L; ++i) {
        BSlot* s = B->live[(size_t)i];
        long long ldc = s->req.ldc;
        const void* Cd = s->req.C;
        if (s->w.Cpad) {
            Cd = s->w.Cpad;
            ldc = padded_ldc(s->req.n, s->req.c_dtype);
        }
        B->insts.h[i] = make_inst(s->w, Cd, s->req.c_dtype, ldc, s->req.f, s->req.g);
        const int tt = s->ttype;
        const bool act = active[(size_t)i] != 0 && !s->resident;
        if (active[(size_t)i] && s->resident) B->rlist[tt == TT_BF16 ? 1 : 0].h[orr[tt == TT_BF16 ? 1 : 0]++] = i;
        for (int t = 0; t < s->w.ntiles; ++t) {
            if (act) B->tmap[tt].h[ot[tt]++] = TileRef{i, t};
            if (s->fresh) B->tmap_init[tt].h[oti[tt]++] = TileRef{i, t};
        }
        for (int t = 0; t < s->w.nvt; ++t) {
            if (act) B->vmap.h[ov++] = TileRef{i, t};
            if (s->fresh) B->vmap_init.h[ovi++] = TileRef{i, t};
        }
    }
    const cudaStream_t st = h->stream;
    if (L > 0) CK(cudaMemcpyAsync(B->insts.d, B->insts.h, sizeof(Inst) * (size_t)L, cudaMemcpyHostToDevice, st));
    for (int t = 0; t < NTT; ++t) {
        if (ot[t]) CK(cudaMemcpyAsync(B->tmap[t].d, B->tmap[t].h, sizeof(TileRef) * ot[t], cudaMemcpyHostToDevice, st));
        if (oti[t])
            CK(cudaMemcpyAsync(B->tmap_init[t].d, B->tmap_init[t].h, sizeof(TileRef) * oti[t], cudaMemcpyHostToDevice, st));
        B->cnt.h[t] = (int)ot[t];
        B->cnt.h[CNT_INIT + t] = (int)oti[t];
    }
    if (ov) CK(cudaMemcpyAsync(B->vmap.d, B->vmap.h, sizeof(TileRef) * ov, cudaMemcpyHostToDevice, st));
    if (ovi) CK(cudaMemcpyAsync(B->vmap_init.d, B->vmap_init.h, sizeof(TileRef) * ovi, cudaMemcpyHostToDevice, st));
    for (int r = 0; r < 2; ++r) {
        if (orr[r]) CK(cudaMemcpyAsync(B->rlist[r].d, B->rlist[r].h, sizeof(int) * orr[r], cudaMemcpyHostToDevice, st));
        B->cnt.h[CNT_RES + r] = (int)orr[r];
        // grid bound, bucketed so the chunk graph is re-captured only when the bucket changes
        int gb = 0;
        if (orr[r]) {
            gb = 4;
            while (gb < (int)orr[r]) gb *= 2;
        }
        B->res_grid[r] = gb;
    }
    B->cnt.h[CNT_VEC] = (int)ov;
    B->cnt.h[CNT_INST] = L;
    B->cnt.h[CNT_INIT_VEC] = (int)ovi;
    CK(cudaMemcpyAsync(B->cnt.d, B->cnt.h, sizeof(int) * CNT_WORDS, cudaMemcpyHostToDevice, st));
    B->nv_live = (int)ov;
    {
        // One CTA per vector tile: size the grid by the live count (bucketed,
        // so the chunk graph is re-captured only when the bucket changes).
        int g = 32;
        while (g < (int)ov) g *= 2;
        B->nv_grid = g;
    }
    // Init checks of the fresh instances (X = 0, p = q = 0; norms; marginal checks).
    if (nvi > 0) {
        CK(cudaMemsetAsync(h->wctr, 0, sizeof(unsigned) * WC_N, st));
        for (int t = 0; t < NTT; ++t) {
            if (!oti[t]) continue;
            CKL(launch_kkt(t, B->insts.d, B->tmap_init[t].d, B->cnt.d + CNT_INIT + t, h->wctr, MODE_INIT, h->cfg,
                           st));
            launch_count(h, 1);
        }
        CKL(launch_checkvec(B->insts.d, B->vmap_init.d, B->cnt.d + CNT_INIT_VEC, (int)nvi, h->wctr, MODE_INIT,
                            h->cfg, st));
        launch_count(h, 1);
        for (BSlot* s : B->live) s->fresh = false;
    }
}

void batch_issue_chunk(pdot_handle* h, int types) {
    BatchEngine* B = h->batch;
    const int K = std::max(1, h->opt.restart_check_every);
    const int checks = std::max(1, h->opt.chunk_checks);
    const cudaStream_t st = h->stream;
    const int nvh = std::max(1, B->nv_live);
    for (int r = 0; r < 2; ++r) {
        if (!B->res_grid[r]) continue;
        // the resident instances' whole chunk (its check periods) in one launch
        CKL(launch_resident(r ? TT_BF16 : TT_F32, B->insts.d, B->rlist[r].d, B->cnt.d + CNT_RES + r, B->res_grid[r],
                            K * checks, K, 0, h->cfg, st));
        launch_count(h, 1);
    }
    for (int c = 0; c < checks; ++c) {
        for (int s = 0; s < K; ++s) {
            for (int t = 0; t < NTT; ++t) {
                if (!(types & (1 << t))) continue;
                CKL(launch_pass(t, B->insts.d, B->tmap[t].d, B->cnt.d + t, h->wctr, h->cfg, st));
                launch_count(h, 1);
            }
            CKL(launch_dual(B->insts.d, B->vmap.d, B->cnt.d + CNT_VEC, B->nv_grid, h->wctr, h->cfg, st));
            launch_count(h, 1);
        }
        for (int t = 0; t < NTT; ++t) {
            if (!(types & (1 << t))) continue;
            CKL(launch_kkt(t, B->insts.d, B->tmap[t].d, B->cnt.d + t, h->wctr, MODE_CHECK, h->cfg, st));
            launch_count(h, 1);
        }
        CKL(launch_checkvec(B->insts.d, B->vmap.d, B->cnt.d + CNT_VEC, B->nv_grid, h->wctr, MODE_CHECK, h->cfg,
                            st));
        launch_count(h, 1);
        for (int t = 0; t < NTT; ++t) {
            if (!(types & (1 << t))) continue;
            CKL(launch_avgfix(t, B->insts.d, B->tmap[t].d, B->cnt.d + t, h->cfg, st));
            launch_count(h, 1);
        }
    }
    (void)nvh;
}

void batch_launch_chunk(pdot_handle* h) {
    BatchEngine* B = h->batch;
    const int types = B->types;
    h->cfg.gen_dims = B->gen_dims;
    h->cfg.comp = h->opt.compensated_cost != 0 ? 1 : 0;
    h->cfg.pass_bulk = h->cfg_base.pass_bulk;   // the batch engine's pass kernel (its tiles were sized for it)
    long long tmaps = 0;
    for (int t = 0; t < NTT; ++t) tmaps ^= (long long)(uintptr_t)B->tmap[t].d << t;
    const long long key[8] = {(long long)(uintptr_t)B->insts.d, (long long)(uintptr_t)B->cnt.d,
                              (long long)(uintptr_t)B->vmap.d, tmaps,
                              types | ((long long)B->gen_dims << 8) | ((long long)B->res_grid[0] << 16) |
                                  ((long long)B->res_grid[1] << 40),
                              h->opt.restart_check_every, h->opt.chunk_checks,
                              h->cfg.comp | ((long long)B->nv_grid << 8)};
    if (!h->opt.use_graph) {
        batch_issue_chunk(h, types);
    } else {
        if (!B->graph.exec || memcmp(key, B->graph_key, sizeof(key)) != 0) {
            B->graph.reset();
            const int64_t before = h->launches;
            CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
            try {
                batch_issue_chunk(h, types);
            } catch (...) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(h->stream, &g);
                if (g) cudaGraphDestroy(g);
                h->launches = before;
                throw;
            }
            CK(cudaStreamEndCapture(h->stream, &B->graph.g));
            CK(cudaGraphInstantiate(&B->graph.exec, B->graph.g, 0));
            B->graph.kernels = (int)(h->launches - before);
            h->launches = before;
            memcpy(B->graph_key, key, sizeof(key));
        }
        CK(cudaGraphLaunch(B->graph.exec, h->stream));
        launch_count(h, B->graph.kernels);
    }
    // Controller snapshot of this chunk into its own buffer (the other one may
    // still belong to the chunk before it).
    BatchEngine::Flight f;
    f.buf = B->next_buf;
    B->next_buf ^= 1;
    DevArr<Ctrl>& snap = B->snap[f.buf];
    snap.ensure(B->insts.cap);
    const int L = (int)B->live.size();
    CKL(launch_snapshot(B->insts.d, B->cnt.d + CNT_INST, L, snap.d, h->stream));
    launch_count(h, 1);
    CK(cudaMemcpyAsync(snap.h, snap.d, sizeof(Ctrl) * (size_t)L, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaEventRecord(B->ev_chunk[f.buf], h->stream));
    f.ids.reserve((size_t)L);
    for (BSlot* sl : B->live) f.ids.push_back(sl->id);
    B->flights.push_back(std::move(f));
    B->chunks += 1;
}

pdot_result batch_result(pdot_handle* h, const BSlot* s, int status) {
    pdot_result r;
    memset(&r, 0, sizeof(r));
    fill_result(s->last, &r, map_status(status));
    r.tile_rows = s->resident ? 0 : s->w.tile_rows;
    const double mn = (double)s->req.m * (double)s->req.n;
    const double bc = (double)csize_of(s->req.c_dtype), bx = (double)xsize_of(h->opt.x_dtype);
    r.hbm_bytes = (double)s->last.passes * mn * (bc + 4.0 * bx) + (double)s->last.checks * mn * (bc + 3.0 * bx);
    r.rounded_obj = std::numeric_limits<double>::quiet_NaN();
    r.seconds = std::chrono::duration<double>(Clock::now() - s->t_submit).count();
    return r;
}

// Retire the instances that finished (or were cancelled / timed out) by the
// end of chunk `f`, whose snapshot lists them in f.ids order; their output
// copies are queued behind every chunk still in flight and their results are
// reported once those copies have run.  True if any instance left.
bool batch_retire(pdot_handle* h, const BatchEngine::Flight& f) {
    BatchEngine* B = h->batch;
    bool changed = false;
    std::map<uint64_t, size_t> pos;
    for (size_t i = 0; i < f.ids.size(); ++i) pos[f.ids[i]] = i;
    std::vector<BSlot*> keep;
    keep.reserve(B->live.size());
    std::vector<std::pair<uint64_t, pdot_result>> res;
    const double tlim = h->opt.time_limit_s;
    for (size_t i = 0; i < B->live.size(); ++i) {
        BSlot* s = B->live[i];
        const auto it = pos.find(s->id);
        if (it == pos.end()) {   // admitted after chunk f was launched
            keep.push_back(s);
            continue;
        }
        s->last = B->snap[f.buf].h[it->second];
        int stt = s->last.status;
        if (s->cancel) stt = ST_CANCELLED;
        else if (stt == ST_RUNNING && tlim > 0.0 &&
                 std::chrono::duration<double>(Clock::now() - s->t_submit).count() > tlim) {
            // The chunk already in flight still advances this instance, so its
            // buffers are read only from the first snapshot after the device
            // has stopped it: batch_apply_cancels sends a stop request before
            // the next chunk, whose first check ends the solve (ST_TIMEOUT).
            s->timed_out = true;
        }
        if (stt == ST_RUNNING) {
            keep.push_back(s);
            continue;
        }
        if (stt != ST_CANCELLED && stt != ST_ARG) {
            const size_t xs = xsize_of(s->w.xtype);
            const int slot = s->last.res_slot;
            if (s->req.X_out) {
                const char* src = (const char*)s->w.X + (size_t)s->last.res_xslot * (size_t)(s->w.m * s->w.ldx) * xs;
                CK(cudaMemcpy2DAsync(s->req.X_out, (size_t)s->w.n * xs, src, (size_t)s->w.ldx * xs,
                                     (size_t)s->w.n * xs, (size_t)s->w.m, cudaMemcpyDeviceToDevice, h->stream));
            }
            const double* V = s->w.V + (size_t)slot * 2 * (size_t)(s->w.m + s->w.n);
            if (s->req.p_out)
                CK(cudaMemcpyAsync(s->req.p_out, V, sizeof(double) * (size_t)s->w.m, cudaMemcpyDeviceToDevice, h->stream));
            if (s->req.q_out)
                CK(cudaMemcpyAsync(s->req.q_out, V + s->w.m, sizeof(double) * (size_t)s->w.n, cudaMemcpyDeviceToDevice,
                                   h->stream));
        }
        batch_free_slot(h, s);
        res.emplace_back(s->id, batch_result(h, s, stt));
        delete s;
        changed = true;
    }
    B->live.swap(keep);
    if (!res.empty()) {
        BatchEngine::Pending p;
        CK(cudaEventCreateWithFlags(&p.ev, cudaEventDisableTiming));
        CK(cudaEventRecord(p.ev, h->stream));
        p.results = std::move(res);
        B->pending_done.push_back(std::move(p));
    }
    return changed;
}

bool batch_admit(pdot_handle* h) {
    BatchEngine* B = h->batch;
    bool changed = false;
    const int max_slots = std::max(1, h->opt.max_batch_slots);
    // Size the pinned controller staging once: async uploads from it are in
    // flight until the next chunk has run.
    B->ctrl_stage.ensure(std::max<size_t>((size_t)max_slots, B->live.size()) + 1);
    while (!B->queue.empty() && (int)B->live.size() < max_slots) {
        BSlot* s = B->queue.front();
        if (s->cancel) {
            B->queue.pop_front();
            pdot_result r;
            memset(&r, 0, sizeof(r));
            r.status = PDOT_CANCELLED;
            r.rounded_obj = std::numeric_limits<double>::quiet_NaN();
            B->done.emplace_back(s->id, r);
            delete s;
            continue;
        }
        if (B->used + s->bytes > B->budget) break;   // FIFO: wait for memory to free up
        B->queue.pop_front();
        const pdot_request& r = s->req;
        const int tr = pick_tile_rows(h, r.m, r.n, s->ttype, true);
        const size_t wb = work_bytes(r.m, r.n, h->opt.x_dtype, tr, nullptr);
        void* base = nullptr;
        CK(cudaMallocAsync(&base, s->bytes, h->stream));
        s->w.base = base;
        s->w.bytes = wb;
        work_bytes(r.m, r.n, h->opt.x_dtype, tr, &s->w);
        if (s->bytes > wb) {
            const long long ldp = padded_ldc(r.n, r.c_dtype);
            const size_t cs = csize_of(r.c_dtype);
            s->w.Cpad = (char*)base + wb;
            CK(cudaMemcpy2DAsync(s->w.Cpad, ldp * cs, r.C, (size_t)r.ldc * cs, (size_t)r.n * cs, (size_t)r.m,
                                 cudaMemcpyDeviceToDevice, h->stream));
        }
        B->used += s->bytes;
        // controller
        Ctrl* S = &B->ctrl_stage.h[B->live.size()];
        init_ctrl(h, S, r.m, r.n, r.tol > 0.0 ? r.tol : h->opt.tol, 0.0, 0.0, false, 0.0, 0.0);
        CK(cudaMemcpyAsync(s->w.ctrl, S, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemsetAsync(s->w.ticket, 0, sizeof(unsigned), h->stream));
        CK(cudaMemsetAsync(s->w.X, 0, (size_t)s->w.m * s->w.ldx * xsize_of(s->w.xtype), h->stream));
        CK(cudaMemsetAsync(s->w.V, 0, sizeof(double) * 2 * (size_t)(s->w.m + s->w.n), h->stream));
        s->fresh = true;
        B->live.push_back(s);
        changed = true;
    }
    return changed;
}

void batch_apply_cancels(pdot_handle* h) {
    // Stop cancelled / timed-out resident instances on the device before the next chunk.
    BatchEngine* B = h->batch;
    B->cnt.h[CNT_CANCEL] = ST_CANCELLED;   // pinned source words of the control writes
    B->cnt.h[CNT_TIMEOUT] = 1;
    for (size_t i = 0; i < B->live.size(); ++i) {
        BSlot* s = B->live[i];
        if (s->cancel) {
            CK(cudaMemcpyAsync(&s->w.ctrl->status, &B->cnt.h[CNT_CANCEL], sizeof(int), cudaMemcpyHostToDevice,
                               h->stream));
        } else if (s->timed_out && !s->stop_sent) {
            // Stop request: the instance's next check reports its current
            // iterate with that iterate's own measures (ST_TIMEOUT).  A solve
            // that finishes first is reported as finished.
            CK(cudaMemcpyAsync(&s->w.ctrl->stop_req, &B->cnt.h[CNT_TIMEOUT], sizeof(int), cudaMemcpyHostToDevice,
                               h->stream));
            s->stop_sent = true;
        }
    }
}

void batch_retire_front(pdot_handle* h, bool& changed) {
    BatchEngine* B = h->batch;
    const BatchEngine::Flight& f = B->flights.front();
    CK(cudaEventSynchronize(B->ev_chunk[f.buf]));
    changed |= batch_retire(h, f);
    B->flights.pop_front();
}

// Move results whose output copies have run to `done` (all of them, waiting,
// when `wait`).
void batch_collect(pdot_handle* h, bool wait) {
    BatchEngine* B = h->batch;
    while (!B->pending_done.empty()) {
        BatchEngine::Pending& p = B->pending_done.front();
        if (wait) {
            CK(cudaEventSynchronize(p.ev));
        } else {
            const cudaError_t q = cudaEventQuery(p.ev);
            if (q == cudaErrorNotReady) break;
            if (q != cudaSuccess) throw CudaError{q};
        }
        cudaEventDestroy(p.ev);
        for (auto& r : p.results) B->done.push_back(r);
        B->pending_done.pop_front();
    }
}

// One poll: retire what finished, admit, and keep up to two chunks in flight
// (the device runs chunk i+1 while the host retires chunk i and prepares
// chunk i+2).
pdot_status batch_poll(pdot_handle* h, uint64_t* ids, pdot_result* results, int cap, int* n_done) {
    BatchEngine* B = batch_of(h);
    bool changed = false;
    {
        const Range r_("retire");
        if (B->flights.size() >= 2) batch_retire_front(h, changed);
        while (!B->flights.empty()) {
            const cudaError_t q = cudaEventQuery(B->ev_chunk[B->flights.front().buf]);
            if (q == cudaErrorNotReady) break;
            if (q != cudaSuccess) throw CudaError{q};
            batch_retire_front(h, changed);
        }
    }
    // The pinned staging buffers are rewritten below: the copies that read
    // them for the previous chunk must have run.
    if (B->staged_pending) {
        CK(cudaEventSynchronize(B->ev_staged));
        B->staged_pending = false;
    }
    batch_apply_cancels(h);
    {
        const Range r_("admit");
        changed |= batch_admit(h);
        // With an active-bytes budget the advancing set can change every chunk.
        if (changed || B->chunks == 0 || h->opt.batch_active_bytes > 0) batch_compose(h);
    }
    CK(cudaEventRecord(B->ev_staged, h->stream));
    B->staged_pending = true;
    if (!B->live.empty()) {
        const Range r_("launch chunk");
        batch_launch_chunk(h);
    } else {
        while (!B->flights.empty()) batch_retire_front(h, changed);
    }
    batch_collect(h, B->live.empty() && B->flights.empty());
    int k = 0;
    const int take = std::min<int>(cap, (int)B->done.size());
    for (; k < take; ++k) {
        if (ids) ids[k] = B->done[(size_t)k].first;
        if (results) results[k] = B->done[(size_t)k].second;
    }
    B->done.erase(B->done.begin(), B->done.begin() + take);
    *n_done = k;
    return PDOT_OK;
}

void batch_destroy(pdot_handle* h) {
    BatchEngine* B = h->batch;
    if (!B) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (BSlot* s : B->live) {
        if (s->w.base) cudaFreeAsync(s->w.base, h->stream);
        delete s;
    }
    for (BSlot* s : B->queue) delete s;
    if (h->stream) cudaStreamSynchronize(h->stream);
    B->graph.reset();
    for (auto& p : B->pending_done) cudaEventDestroy(p.ev);
    B->pending_done.clear();
    B->insts.release();
    for (int t = 0; t < NTT; ++t) {
        B->tmap[t].release();
        B->tmap_init[t].release();
    }
    B->vmap.release();
    B->vmap_init.release();
    B->rlist[0].release();
    B->rlist[1].release();
    B->snap[0].release();
    B->snap[1].release();
    B->ctrl_stage.release();
    B->cnt.release();
    for (int k = 0; k < 2; ++k)
        if (B->ev_chunk[k]) cudaEventDestroy(B->ev_chunk[k]);
    if (B->ev_staged) cudaEventDestroy(B->ev_staged);
    delete B;
    h->batch = nullptr;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void pdot_default_options(pdot_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->tol = 1e-4;
    o->max_iter = 0;
    o->time_limit_s = 0.0;
    o->restart_check_every = 64;
    o->adaptive_step = 1;
    o->adaptive_restart = 1;
    o->primal_weight_update = 1;
    o->beta = 0.2;
    o->beta_suff = 0.1;
    o->beta_nec = 0.9;
    o->beta_art = 0.36;
    o->theta = 0.5;
    o->eta0 = 0.0;
    o->omega0 = 1.0;
    o->R = 1.0;
    o->eps_zero = 1e-10;
    o->rel_mode = 0;
    o->x_dtype = PDOT_F32;
    o->round_plan = 0;
    o->use_graph = 1;
    o->tile_rows = 0;
    o->hbm_budget_bytes = 0;
    o->max_batch_slots = 4096;
    o->chunk_checks = 4;
    o->batch_active_bytes = 0;
    o->pass_kernel = 0;
    o->compensated_cost = 2;
    o->resident = 0;
}

const char* pdot_status_str(pdot_status s) {
    switch (s) {
        case PDOT_OK: return "PDOT_OK";
        case PDOT_ERR_ARG: return "PDOT_ERR_ARG";
        case PDOT_ERR_OOM: return "PDOT_ERR_OOM";
        case PDOT_ERR_CUDA: return "PDOT_ERR_CUDA";
        case PDOT_ERR_NUMERIC: return "PDOT_ERR_NUMERIC";
        case PDOT_MAX_ITER: return "PDOT_MAX_ITER";
        case PDOT_TIMEOUT: return "PDOT_TIMEOUT";
        case PDOT_BUSY: return "PDOT_BUSY";
        case PDOT_PENDING: return "PDOT_PENDING";
        case PDOT_CANCELLED: return "PDOT_CANCELLED";
    }
    return "PDOT_UNKNOWN";
}

const char* pdot_last_error(pdot_handle* h) { return h ? h->last_error.c_str() : "null handle"; }

pdot_status pdot_create(const pdot_options* opt, int device, void* cuda_stream, pdot_handle** out) {
    if (!out) return PDOT_ERR_ARG;
    *out = nullptr;
    pdot_handle* h = new (std::nothrow) pdot_handle();
    if (!h) return PDOT_ERR_OOM;
    if (opt) h->opt = *opt;
    else pdot_default_options(&h->opt);
    pdot_status st = guarded(h, [&]() -> pdot_status {
        if (h->opt.restart_check_every < 1) throw ArgError{"restart_check_every < 1"};
        if (h->opt.tile_rows < 0 || h->opt.tile_rows > 4096 || h->opt.tile_rows % 2 != 0) {
            throw ArgError{"tile_rows must be 0 or an even number in [2, 4096]"};
        }
        if (h->opt.pass_kernel < 0 || h->opt.pass_kernel > 3) throw ArgError{"pass_kernel must be in 0..3"};
        if (h->opt.compensated_cost < 0 || h->opt.compensated_cost > 2) throw ArgError{"compensated_cost must be in 0..2"};
        if (h->opt.resident < 0 || h->opt.resident > 1) throw ArgError{"resident must be 0 or 1"};
        int ndev = 0;
        CK(cudaGetDeviceCount(&ndev));
        if (device < 0 || device >= ndev) throw ArgError{"no such CUDA device"};
        h->device = device;
        CK(cudaSetDevice(device));
        CK(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, device));
        if (cuda_stream) {
            h->stream = (cudaStream_t)cuda_stream;
        } else {
            // A blocking stream: ordered with the legacy default stream, and capturable.
            CK(cudaStreamCreate(&h->stream));
            h->own_stream = true;
        }
        h->cfg.tile_blocks = h->sm_count * occupancy_tile_blocks_per_sm(TT_F32);
        h->cfg.tile_blocks_f64 = h->sm_count * occupancy_tile_blocks_per_sm(TT_F64);
        h->cfg.vec_blocks = h->sm_count * occupancy_vec_blocks_per_sm();
        h->cfg.pass_u = 2;
        const char* pu = getenv("PDOT_PASS_U");
        if (pu && atoi(pu) == 4) h->cfg.pass_u = 4;
        const int bulk = setup_bulk_pass();
        if (bulk > 0) throw CudaError{(cudaError_t)bulk};
        h->cfg.bulk_blocks = h->sm_count * (-bulk);
        const int grp = setup_group_pass();
        if (grp > 0) throw CudaError{(cudaError_t)grp};
        h->cfg.group_blocks = h->sm_count * (-grp);
        const int rc = setup_resident();
        if (rc > 0) throw CudaError{(cudaError_t)rc};
        h->res_clusters = -rc;
        {
            const int one[2] = {0, 1};   // instance list [0] and count 1 of a single-instance resident launch
            CK(cudaMalloc(&h->d_res1, sizeof(one)));
            CK(cudaMemcpy(h->d_res1, one, sizeof(one), cudaMemcpyHostToDevice));
        }
        const int kb = setup_kkt_bulk();
        if (kb > 0) throw CudaError{(cudaError_t)kb};
        h->cfg.kkt_blocks = h->sm_count * (-kb);
        const char* kk = getenv("PDOT_KKT_BULK");
        if (kk && atoi(kk) == 0) h->cfg.kkt_blocks = 0;   // the register KKT pass (comparison)
        const int coop = setup_coop_chunk();
        if (coop > 0) throw CudaError{(cudaError_t)coop};
        int coop_ok = 0;
        CK(cudaDeviceGetAttribute(&coop_ok, cudaDevAttrCooperativeLaunch, device));
        h->cfg.coop_blocks = coop_ok ? h->sm_count * (-coop) : 0;
        const char* cp = getenv("PDOT_COOP");
        if (cp && atoi(cp) == 1) h->coop = 1;
        h->cfg.pass_bulk = 1;
        const char* pb = getenv("PDOT_PASS_BULK");
        if (pb) {
            const int v = atoi(pb);
            if (v >= 0 && v <= 2) {
                h->cfg.pass_bulk = v;
                h->autotune = 0;   // an explicit kernel choice disables the tuner
            }
        }
        const char* bm = getenv("PDOT_BATCH_MIN_ROWS");   // comparison runs only
        if (bm && atoi(bm) >= 2 && atoi(bm) <= 64 && atoi(bm) % 2 == 0) h->batch_min_rows = atoi(bm);
        const char* at = getenv("PDOT_AUTOTUNE");
        if (at && atoi(at) == 0) h->autotune = 0;
        int l2 = 0;
        CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device));
        h->l2_bytes = l2;
        const char* lh = getenv("PDOT_L2HINT");
        if (lh && atoi(lh) == 1) h->l2_hint = 1;
        // Programmatic dependent launch: on (PDOT_PDL=0 turns it off).
        const char* pp = getenv("PDOT_PDL");
        h->cfg.pdl = (pp && atoi(pp) == 0) ? 0 : 1;
        h->cfg.comp = h->opt.compensated_cost == 1 ? 1 : 0;   // set per call (compensation_for)
        h->cfg_base = h->cfg;
        CK(cudaMalloc(&h->wctr, sizeof(unsigned) * WC_N));
        CK(cudaMemset(h->wctr, 0, sizeof(unsigned) * WC_N));
        {
            // t^-0.3 and t^-0.6 for t = 2 .. SCHED + 1, by the C library's pow
            // (the same function the FP64 reference of the rule calls).
            constexpr long long SCHED = 1LL << 19;
            std::vector<double> tab((size_t)(2 * SCHED));
            for (long long i = 0; i < SCHED; ++i) {
                const double t1 = (double)(i + 2);
                tab[(size_t)(2 * i)] = std::pow(t1, -0.3);
                tab[(size_t)(2 * i + 1)] = std::pow(t1, -0.6);
            }
            CK(cudaMalloc(&h->d_sched, sizeof(double) * tab.size()));
            CK(cudaMemcpy(h->d_sched, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice));
            h->sched_len = SCHED;
        }
        CK(cudaMalloc(&h->d_inst, sizeof(Inst)));
        CK(cudaMallocHost(&h->h_ctrl, sizeof(Ctrl)));
        CK(cudaMallocHost(&h->h_inst, sizeof(Inst)));
        CK(cudaMallocHost(&h->h_status, 2 * sizeof(int)));
        CK(cudaMalloc(&h->d_cnt, 4 * sizeof(int)));
        CK(cudaMalloc(&h->d_gb, sizeof(GridBar)));
        CK(cudaMemset(h->d_gb, 0, sizeof(GridBar)));
        CK(cudaMallocHost(&h->h_cnt, 4 * sizeof(int)));
        return PDOT_OK;
    });
    if (st != PDOT_OK) {
        pdot_destroy(h);
        return st;
    }
    *out = h;
    return PDOT_OK;
}

pdot_status pdot_destroy(pdot_handle* h) {
    if (!h) return PDOT_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    batch_destroy(h);
    h->chunk.reset();
    free_work(h->ws);
    if (h->d_tmap) cudaFree(h->d_tmap);
    if (h->d_vmap) cudaFree(h->d_vmap);
    if (h->d_inst) cudaFree(h->d_inst);
    if (h->wctr) cudaFree(h->wctr);
    if (h->round_scratch) cudaFree(h->round_scratch);
    if (h->d_sched) cudaFree(h->d_sched);
    if (h->stage) cudaFree(h->stage);
    if (h->h_ctrl) cudaFreeHost(h->h_ctrl);
    if (h->h_inst) cudaFreeHost(h->h_inst);
    if (h->h_status) cudaFreeHost(h->h_status);
    if (h->d_cnt) cudaFree(h->d_cnt);
    if (h->d_gb) cudaFree(h->d_gb);
    if (h->d_tp) cudaFree(h->d_tp);
    if (h->d_res1) cudaFree(h->d_res1);
    if (h->h_cnt) cudaFreeHost(h->h_cnt);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return PDOT_OK;
}

pdot_status pdot_solve(pdot_handle* h, int64_t m, int64_t n, const void* C, pdot_dtype c_dtype, int64_t ldc,
                       const double* f, const double* g, double tol, void* X_out, double* p_out, double* q_out,
                       pdot_result* res) {
    if (!h) return PDOT_ERR_ARG;
    const Range r_("pdot_solve");
    return guarded(h, [&]() -> pdot_status {
        CK(cudaSetDevice(h->device));
        return solve_impl(h, m, n, C, c_dtype, ldc, f, g, tol, X_out, p_out, q_out, res);
    });
}

int64_t pdot_state_bytes(int64_t m, int64_t n, pdot_dtype x_dtype) {
    if (m < 1 || n < 1 || m > (1LL << 31) / 2 || n > (1LL << 31) / 2) return 0;
    if (x_dtype != PDOT_F32 && x_dtype != PDOT_F64) return 0;
    return (int64_t)state_layout(m, n, x_dtype).total;
}

int32_t pdot_resident_fits(int64_t m, int64_t n) {
    if (m < 1 || n < 1 || m > (1LL << 31) / 2 || n > (1LL << 31) / 2) return 0;
    return resident_fits(m, n) ? 1 : 0;
}

pdot_status pdot_solve_from(pdot_handle* h, int64_t m, int64_t n, const void* C, pdot_dtype c_dtype, int64_t ldc,
                            const double* f, const double* g, double tol, const pdot_start* start, void* X_out,
                            double* p_out, double* q_out, pdot_result* res) {
    if (!h) return PDOT_ERR_ARG;
    const Range r_("pdot_solve_from");
    return guarded(h, [&]() -> pdot_status {
        CK(cudaSetDevice(h->device));
        return solve_impl(h, m, n, C, c_dtype, ldc, f, g, tol, X_out, p_out, q_out, res, start);
    });
}

pdot_status pdot_solve_host(pdot_handle* h, int64_t m, int64_t n, const void* C, pdot_dtype c_dtype, int64_t ldc,
                            const double* f, const double* g, double tol, void* X_out, double* p_out, double* q_out,
                            pdot_result* res) {
    if (!h) return PDOT_ERR_ARG;
    const Range r_("pdot_solve_host");
    return guarded(h, [&]() -> pdot_status {
        CK(cudaSetDevice(h->device));
        const bool pts = c_dtype == PDOT_POINTS;
        if (m < 1 || n < 1 || (!pts && ldc < n) || !C || !f || !g) throw ArgError{"bad arguments"};
        pdot_points_cost dpc{};   // the descriptor with device coordinates
        size_t bxs = 0, bys = 0;
        if (pts) {
            check_common_args(h, m, n, C, c_dtype, ldc, f, g);
            dpc = *static_cast<const pdot_points_cost*>(C);
            bxs = align_up(sizeof(float) * (size_t)m * (size_t)dpc.d, 256);
            bys = align_up(sizeof(float) * (size_t)n * (size_t)dpc.d, 256);
        }
        const size_t cs = csize_of(c_dtype);
        const size_t xs = xsize_of(h->opt.x_dtype);
        const long long ldp = pts ? 0 : padded_ldc(n, c_dtype);
        const size_t bC = pts ? bxs + bys : align_up((size_t)m * ldp * cs, 256);
        const size_t bf = align_up(sizeof(double) * (size_t)m, 256), bg = align_up(sizeof(double) * (size_t)n, 256);
        const size_t bX = X_out ? align_up((size_t)m * n * xs, 256) : 0;
        const size_t bp = p_out ? bf : 0, bq = q_out ? bg : 0;
        const size_t need = bC + bf + bg + bX + bp + bq;
        if (h->stage_bytes < need) {
            if (h->stage) cudaFree(h->stage);
            h->stage = nullptr;
            h->stage_bytes = 0;
            CK(cudaMalloc(&h->stage, need));
            h->stage_bytes = need;
        }
        char* b = (char*)h->stage;
        void* dC = b;
        double* df = (double*)(b + bC);
        double* dg = (double*)(b + bC + bf);
        void* dX = X_out ? (void*)(b + bC + bf + bg) : nullptr;
        double* dp = p_out ? (double*)(b + bC + bf + bg + bX) : nullptr;
        double* dq = q_out ? (double*)(b + bC + bf + bg + bX + bp) : nullptr;
        const void* Cs = dC;
        if (pts) {
            const pdot_points_cost& hc = *static_cast<const pdot_points_cost*>(C);
            CK(cudaMemcpyAsync(b, hc.xs, sizeof(float) * (size_t)m * (size_t)hc.d, cudaMemcpyHostToDevice, h->stream));
            CK(cudaMemcpyAsync(b + bxs, hc.ys, sizeof(float) * (size_t)n * (size_t)hc.d, cudaMemcpyHostToDevice,
                               h->stream));
            dpc.xs = (const float*)b;
            dpc.ys = (const float*)(b + bxs);
            Cs = &dpc;
        } else {
            CK(cudaMemcpy2DAsync(dC, ldp * cs, C, (size_t)ldc * cs, (size_t)n * cs, (size_t)m, cudaMemcpyHostToDevice,
                                 h->stream));
        }
        CK(cudaMemcpyAsync(df, f, sizeof(double) * (size_t)m, cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(dg, g, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, h->stream));
        pdot_status st = solve_impl(h, m, n, Cs, c_dtype, ldp, df, dg, tol, dX, dp, dq, res);
        const auto t0 = Clock::now();
        if (X_out) CK(cudaMemcpyAsync(X_out, dX, (size_t)m * n * xs, cudaMemcpyDeviceToHost, h->stream));
        if (p_out) CK(cudaMemcpyAsync(p_out, dp, sizeof(double) * (size_t)m, cudaMemcpyDeviceToHost, h->stream));
        if (q_out) CK(cudaMemcpyAsync(q_out, dq, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        res->seconds += std::chrono::duration<double>(Clock::now() - t0).count();
        return st;
    });
}

pdot_status pdot_pdhg_steps(pdot_handle* h, int64_t m, int64_t n, const void* C, pdot_dtype c_dtype, int64_t ldc,
                            const double* f, const double* g, int64_t k, double eta, double omega, void* X, double* p,
                            double* q, void* Xbar_out, double* pbar_out, double* qbar_out) {
    if (!h) return PDOT_ERR_ARG;
    const Range r_("pdot_pdhg_steps");
    return guarded(h, [&]() -> pdot_status {
        CK(cudaSetDevice(h->device));
        check_common_args(h, m, n, C, c_dtype, ldc, f, g);
        if (k < 0 || !(eta > 0.0) || !(omega > 0.0) || !X || !p || !q) throw ArgError{"bad k, eta, omega or state"};
        const int ttype = ttype_of(c_dtype);
        autotune_pass(h, m, n, C, c_dtype, ldc, f, g);   // the pass kernel a solve of this shape runs
        const int tr = pick_tile_rows(h, m, n, ttype, false, gen_dims_of(C, c_dtype));
        ensure_work(h, m, n, h->opt.x_dtype, tr);
        ensure_maps(h);
        Work& w = h->ws;
        long long ldc_used = ldc;
        const void* Cd = prepare_C(h, m, n, C, c_dtype, ldc, &ldc_used);
        stage_instance(h, make_inst(w, Cd, c_dtype, ldc_used, f, g));
        Ctrl* S = h->h_ctrl;
        init_ctrl(h, S, m, n, -1.0, 1.0, 1.0, true, eta, omega);
        S->adaptive_restart = 0;
        S->pw_update = 0;
        CK(cudaMemcpyAsync(w.ctrl, S, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemsetAsync(w.ticket, 0, sizeof(unsigned), h->stream));
        upload_state(h, X, p, q);
        run_check(h, ttype, MODE_INIT);   // row/column sums of the starting plan
        if (h->opt.pass_kernel == 0 && resident_for(h, m, n, ttype)) {
            if (k > 0) {   // k steps in one resident launch, no check
                CKL(launch_resident(ttype, h->d_inst, h->d_res1, h->d_res1 + 1, 1, (int)k, 0, 0, h->cfg, h->stream));
                launch_count(h, 1);
            }
        } else {
            for (int64_t s = 0; s < k; ++s) run_step(h, ttype);
        }
        CK(cudaMemcpyAsync(S, w.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        if (S->status == ST_ARG) throw ArgError{"invalid marginals"};
        if (S->status == ST_NUMERIC) return PDOT_ERR_NUMERIC;
        const int cur = S->cur, bar = k > 0 ? S->bar : S->cur;
        copy_plan_out(h, cur, X, cudaMemcpyDeviceToDevice);
        copy_duals_out(h, cur, p, q, cudaMemcpyDeviceToDevice);
        if (Xbar_out) {
            // The average slot holds its deviation from the current plan:
            // form X + D in the free next slot, then copy it out.
            int src = cur;
            if (k > 0) {
                const size_t pe = (size_t)w.m * (size_t)w.ldx, xs = xsize_of(w.xtype);
                const char* base = (const char*)w.X;
                CKL(launch_combine(w.xtype, base + (size_t)cur * pe * xs, base + (size_t)bar * pe * xs,
                                   (char*)w.X + (size_t)S->nxt * pe * xs, (long long)pe, h->stream));
                launch_count(h, 1);
                src = S->nxt;
            }
            copy_plan_out(h, src, Xbar_out, cudaMemcpyDeviceToDevice);
        }
        copy_duals_out(h, bar, pbar_out, qbar_out, cudaMemcpyDeviceToDevice);
        CK(cudaStreamSynchronize(h->stream));
        return PDOT_OK;
    });
}

pdot_status pdot_kkt(pdot_handle* h, int64_t m, int64_t n, const void* C, pdot_dtype c_dtype, int64_t ldc,
                     const double* f, const double* g, const void* X, const double* p, const double* q,
                     pdot_kkt_parts* out) {
    if (!h) return PDOT_ERR_ARG;
    const Range r_("pdot_kkt");
    return guarded(h, [&]() -> pdot_status {
        CK(cudaSetDevice(h->device));
        check_common_args(h, m, n, C, c_dtype, ldc, f, g);
        if (!X || !p || !q || !out) throw ArgError{"null X, p, q or out"};
        double norm_b = 0.0;
        validate_marginals(h, m, n, f, g, false, &norm_b);
        const int ttype = ttype_of(c_dtype);
        const int tr = pick_tile_rows(h, m, n, ttype, false, gen_dims_of(C, c_dtype));
        ensure_work(h, m, n, h->opt.x_dtype, tr);
        ensure_maps(h);
        Work& w = h->ws;
        long long ldc_used = ldc;
        const void* Cd = prepare_C(h, m, n, C, c_dtype, ldc, &ldc_used);
        stage_instance(h, make_inst(w, Cd, c_dtype, ldc_used, f, g));
        Ctrl* S = h->h_ctrl;
        init_ctrl(h, S, m, n, -1.0, norm_b, 0.0, false, 0.0, 0.0);
        CK(cudaMemcpyAsync(w.ctrl, S, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemsetAsync(w.ticket, 0, sizeof(unsigned), h->stream));
        upload_state(h, X, p, q);
        run_check(h, ttype, MODE_INIT);
        CK(cudaMemcpyAsync(S, w.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        if (S->status == ST_ARG) throw ArgError{"invalid marginals"};
        out->rp2 = S->r_rp2; out->rd2 = S->r_rd2; out->cx = S->r_cx; out->dual = S->r_dual; out->gap = S->r_gap;
        out->kkt = S->r_kkt; out->rel_p = S->r_rel_p; out->rel_d = S->r_rel_d; out->rel_gap = S->r_rel_gap;
        out->rel_kkt = S->r_rel;
        return PDOT_OK;
    });
}

pdot_status pdot_round(pdot_handle* h, int64_t m, int64_t n, const void* X, const double* f, const double* g,
                       void* X_out) {
    if (!h) return PDOT_ERR_ARG;
    const Range r_("pdot_round");
    return guarded(h, [&]() -> pdot_status {
        CK(cudaSetDevice(h->device));
        if (m < 1 || n < 1 || !X || !f || !g || !X_out) throw ArgError{"bad arguments"};
        const int xt = h->opt.x_dtype;
        if (xt != PDOT_F32 && xt != PDOT_F64) throw ArgError{"x_dtype must be F32 or F64"};
        round_plan_dev(h, m, n, xt, X, n, f, g, X_out, nullptr, 0, 0, nullptr);
        CK(cudaStreamSynchronize(h->stream));
        return PDOT_OK;
    });
}

int64_t pdot_launch_count(pdot_handle* h) { return h ? h->launches : 0; }

pdot_status pdot_dual_bound(pdot_handle* h, int64_t m, int64_t n, const void* C, pdot_dtype c_dtype, int64_t ldc,
                            const double* f, const double* g, const double* p, double* q_out, double* lower) {
    if (!h) return PDOT_ERR_ARG;
    const Range r_("pdot_dual_bound");
    return guarded(h, [&]() -> pdot_status {
        CK(cudaSetDevice(h->device));
        check_common_args(h, m, n, C, c_dtype, ldc, f, g);
        if (!p || !lower) throw ArgError{"null p or lower"};
        const int parts = (int)std::min<long long>(64, m);   // row groups of the column minima
        const size_t need = sizeof(double) * ((size_t)parts * (size_t)n + (size_t)n + 8);
        if (h->round_scratch_bytes < need) {
            if (h->round_scratch) cudaFree(h->round_scratch);
            h->round_scratch = nullptr;
            h->round_scratch_bytes = 0;
            CK(cudaMalloc(&h->round_scratch, need));
            h->round_scratch_bytes = need;
        }
        double* colmin = h->round_scratch;
        double* q = colmin + (size_t)parts * (size_t)n;
        double* val = q + n;
        GenSpec gs{};
        if (c_dtype == PDOT_POINTS) gs = gen_spec_of(C);
        CKL(launch_dual_bound(C, (int)c_dtype, ldc, &gs, p, f, g, m, n, colmin, parts, q, val, h->stream));
        launch_count(h, 3);
        if (q_out) CK(cudaMemcpyAsync(q_out, q, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, h->stream));
        CK(cudaMemcpyAsync(lower, val, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        return PDOT_OK;
    });
}

pdot_status pdot_batch_submit(pdot_handle* h, const pdot_request* reqs, int count, uint64_t* ticket_ids) {
    if (!h) return PDOT_ERR_ARG;
    const Range r_("pdot_batch_submit");
    return guarded(h, [&]() -> pdot_status {
        CK(cudaSetDevice(h->device));
        if (count < 0 || (count > 0 && (!reqs || !ticket_ids))) throw ArgError{"bad request array"};
        BatchEngine* B = batch_of(h);
        std::vector<BSlot*> slots;
        try {
            for (int i = 0; i < count; ++i) {
                const pdot_request& r = reqs[i];
                check_common_args(h, r.m, r.n, r.C, r.c_dtype, r.ldc, r.f, r.g);
                BSlot* s = new BSlot();
                slots.push_back(s);
                s->req = r;
                if (r.c_dtype == PDOT_POINTS) {
                    s->pts = *static_cast<const pdot_points_cost*>(r.C);
                    s->req.C = &s->pts;
                    s->req.ldc = 0;
                }
                s->ttype = ttype_of(r.c_dtype);
                s->resident = resident_for(h, r.m, r.n, s->ttype);
                s->bytes = slot_bytes(h, r, pick_tile_rows(h, r.m, r.n, s->ttype, true));
                if (s->bytes > B->budget) {
                    for (BSlot* x : slots) delete x;
                    h->last_error = "request exceeds the HBM budget";
                    return PDOT_BUSY;
                }
            }
        } catch (...) {
            for (BSlot* x : slots) delete x;
            throw;
        }
        const auto now = Clock::now();
        for (int i = 0; i < count; ++i) {
            slots[(size_t)i]->id = B->next_id++;
            slots[(size_t)i]->t_submit = now;
            ticket_ids[i] = slots[(size_t)i]->id;
            B->queue.push_back(slots[(size_t)i]);
        }
        return PDOT_OK;
    });
}

pdot_status pdot_poll(pdot_handle* h, uint64_t* done_ids, pdot_result* done_results, int cap, int* n_done) {
    if (!h || !n_done || cap < 0) return PDOT_ERR_ARG;
    const Range r_("pdot_poll");
    *n_done = 0;
    return guarded(h, [&]() -> pdot_status {
        CK(cudaSetDevice(h->device));
        return batch_poll(h, done_ids, done_results, cap, n_done);
    });
}

pdot_status pdot_cancel(pdot_handle* h, uint64_t ticket) {
    if (!h) return PDOT_ERR_ARG;
    const Range r_("pdot_cancel");
    BatchEngine* B = h->batch;
    if (!B) return PDOT_ERR_ARG;
    for (BSlot* s : B->queue)
        if (s->id == ticket) { s->cancel = true; return PDOT_OK; }
    for (BSlot* s : B->live)
        if (s->id == ticket) { s->cancel = true; return PDOT_OK; }
    return PDOT_ERR_ARG;
}

pdot_status pdot_watchdog_selftest(int device, int64_t polls, int32_t* device_status) {
    if (!device_status || polls < 1 || polls > (1LL << 24)) return PDOT_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return PDOT_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return PDOT_ERR_CUDA;
    int* d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return PDOT_ERR_CUDA;
    int hs = -1;
    bool ok = cudaMemset(d, 0xff, sizeof(int)) == cudaSuccess && launch_watchdog_selftest(polls, d, nullptr) == 0 &&
              cudaMemcpy(&hs, d, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
    cudaFree(d);
    if (!ok) return PDOT_ERR_CUDA;
    *device_status = hs;
    return PDOT_OK;
}

pdot_status pdot_batch_pending(pdot_handle* h, int* queued, int* running) {
    if (!h) return PDOT_ERR_ARG;
    BatchEngine* B = h->batch;
    size_t waiting = 0;   // finished, results not yet reported
    if (B)
        for (const auto& p : B->pending_done) waiting += p.results.size();
    if (queued) *queued = B ? (int)B->queue.size() : 0;
    if (running) *running = B ? (int)(B->live.size() + waiting) : 0;
    return PDOT_OK;
}

pdot_status pdot_time_pass(pdot_handle* h, int64_t m, int64_t n, const void* C, pdot_dtype c_dtype, int64_t ldc,
                           const double* f, const double* g, int reps, double* ms_per_pass, double* bytes_per_pass,
                           int32_t* kernel_variant) {
    if (!h) return PDOT_ERR_ARG;
    const Range r_("pdot_time_pass");
    return guarded(h, [&]() -> pdot_status {
        CK(cudaSetDevice(h->device));
        check_common_args(h, m, n, C, c_dtype, ldc, f, g);
        if (reps < 1 || !ms_per_pass) throw ArgError{"reps < 1 or null output"};
        const int ttype = ttype_of(c_dtype);
        autotune_pass(h, m, n, C, c_dtype, ldc, f, g);
        const int tr = pick_tile_rows(h, m, n, ttype, false, gen_dims_of(C, c_dtype));
        ensure_work(h, m, n, h->opt.x_dtype, tr);
        ensure_maps(h);
        Work& w = h->ws;
        long long ldc_used = ldc;
        const void* Cd = prepare_C(h, m, n, C, c_dtype, ldc, &ldc_used);
        stage_instance(h, make_inst(w, Cd, c_dtype, ldc_used, f, g));
        Ctrl* S = h->h_ctrl;
        init_ctrl(h, S, m, n, -1.0, 1.0, 1.0, true, 0.5 / std::sqrt((double)(m + n)), 1.0);
        CK(cudaMemcpyAsync(w.ctrl, S, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemsetAsync(w.ticket, 0, sizeof(unsigned), h->stream));
        CK(cudaMemsetAsync(w.X, 0, (size_t)w.m * w.ldx * xsize_of(w.xtype), h->stream));
        CK(cudaMemsetAsync(w.V, 0, sizeof(double) * 2 * (size_t)(w.m + w.n), h->stream));
        run_check(h, ttype, MODE_INIT);
        for (int s = 0; s < 3; ++s) run_step(h, ttype);   // steady state: k > 0, the average is read
        // Two views of the instance whose controllers swap the current and
        // next roles (and the pass parity, so the row order alternates):
        // launches alternate between them, so each pass reads the plans the
        // previous one wrote, as accepted passes of a solve do; the dual
        // update is left out, so every launch moves the same bytes.
        if (!h->d_tp) {
            CK(cudaMalloc(&h->d_tp, sizeof(Inst) + sizeof(Ctrl) + 256));
        }
        Inst* d_inst2 = reinterpret_cast<Inst*>(h->d_tp);
        Ctrl* d_ctrl2 = reinterpret_cast<Ctrl*>(reinterpret_cast<char*>(h->d_tp) + align_up(sizeof(Inst), 256));
        CK(cudaMemcpyAsync(S, w.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        std::swap(S->cur, S->nxt);
        std::swap(S->bar, S->barn);
        S->passes += 1;
        Inst I2 = *h->h_inst;
        I2.ctrl = d_ctrl2;
        CK(cudaMemcpyAsync(d_ctrl2, S, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(d_inst2, &I2, sizeof(Inst), cudaMemcpyHostToDevice, h->stream));
        CK(cudaStreamSynchronize(h->stream));   // I2 lives on this stack frame
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        CK(cudaEventRecord(e0, h->stream));
        // Alternate two work counters too: each launch resets every counter
        // but its own, so the next launch finds its counter at zero.
        for (int r = 0; r < reps; ++r) {
            const int wc = (r & 1) ? wc_index(WC_AUX, ttype) : wc_index(WC_PASS, ttype);
            CKL(launch_pass(ttype, (r & 1) ? d_inst2 : h->d_inst, h->d_tmap, h->d_cnt, h->wctr, h->cfg, h->stream, wc));
        }
        CK(cudaEventRecord(e1, h->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        launch_count(h, reps);
        *ms_per_pass = (double)ms / reps;
        if (bytes_per_pass)
            *bytes_per_pass = (double)m * (double)n * ((double)csize_of(c_dtype) + 4.0 * (double)xsize_of(w.xtype));
        if (kernel_variant) {
            int v = ttype == TT_F64 ? 0 : h->cfg.pass_bulk;
            if (ttype == TT_GEN && v == 2 && h->cfg.gen_dims > 4) v = 1;   // no grouped kernel beyond 4 coordinates
            *kernel_variant = v;
        }
        return PDOT_OK;
    });
}

}  // extern "C"

