// pdot_internal.h -- device-side data structures shared by the sm_103a kernels
// (pdot_kernels.cu) and the host engine (pdot_engine.cu).
//
// Layout in HBM, per instance (m rows, n columns, ldx = n rounded up to 4):
//   X    : NSLOT plan buffers of m * ldx elements (FP32 or FP64).  Roles
//          (current, next, average, next average, restart anchor) are slot
//          indices kept in Ctrl, so accepting a step, rejecting it or
//          restarting swaps indices instead of copying m*n data.  The
//          average's slots hold its deviation from the current plan.
//   V    : NSLOT vector sets of 2(m+n) doubles, one per plan slot:
//          [p (m) | q (n) | r = X1 (m) | c = X^T1 (n)].
//   rowpart[nstrips][m], colpart[nchunks][ldx]: FP64 partial row/column sums
//          written by the plan-tile kernels and reduced in a fixed order (a
//          pass writes sums of X+ - X; the check, sums of the average);
//          rowpart2 / colpart2: the check's sums of the current plan.
//   tpart[ntiles][TP], vpart[nvt][VP]: FP64 per-tile scalar partials
//          (nvt = ceil((m+n)/VE) vector tiles).
//   Ctrl : the scalar state of Algorithm 2 and the Sec. 5 controller.
#pragma once
#include <cmath>
#include <cstdint>

namespace pdot {

constexpr int NSLOT = 5;
constexpr int STRIP = 128;   // plan-tile width: 32 lanes x 4 consecutive columns
constexpr int TWARPS = 8;    // warps per CTA in the plan-tile kernels
constexpr int VT = 256;      // threads per CTA in the vector kernels
constexpr int VE = 32;       // entries per vector tile (one warp wide)
constexpr int VG = VT / 32;  // partial-sum groups per vector tile
constexpr int TP = 6;        // scalars per plan-tile partial
constexpr int VP = 12;       // scalars per vector-tile partial

constexpr int ST_RUNNING = -1;
constexpr int MODE_CHECK = 0;
constexpr int MODE_INIT = 1;

// Status codes (same values as pdot_status in include/pdot.h).
constexpr int ST_OK = 0, ST_ARG = 1, ST_DEVICE = 3, ST_NUMERIC = 4, ST_MAX_ITER = 5, ST_TIMEOUT = 6,
              ST_CANCELLED = 9;

struct Ctrl {
    // iteration state
    double eta, omega, tau, sigma;
    double wavg;         // 1 / (k + 1): the running average's weight of the next accepted iterate
    double kkt0, kkt_prev;
    long long k, total, passes, restarts, rejected, checks;
    int cur, nxt, bar, barn, anc;
    int status;          // ST_RUNNING or a final status
    int res_slot, res_avg;
    int res_xslot;       // plan slot of the reported point (res_slot: its vector set)
    int stop_req;        // host-written: 1 = stop at the next check with the current iterate (time limit)
    // The average plan slot holds D = Xbar - X (X: the current plan), so the
    // average itself is X + D.  A check that picks the average (a restart to
    // it, or the reported point) sets fix: the next k_avgfix writes
    // X[fix_dst] = X[fix_x] + X[fix_d] (in place for a restart); the next
    // pass clears it.
    int fix, fix_x, fix_d, fix_dst;
    // options
    double tol, beta, beta_suff, beta_nec, beta_art, theta, R, eps_zero;
    long long max_passes;
    int adaptive_step, adaptive_restart, pw_update, rel_mode;
    // data norms ||[f;g]||_2 and ||C||_F
    double norm_b, norm_C;
    // parts of the reported point (last init/check candidate)
    double r_rp2, r_rd2, r_cx, r_dual, r_gap, r_kkt, r_rel_p, r_rel_d, r_rel_gap, r_rel;
    // diagnostics of the last pass
    double last_etabar, last_dX2, last_dy2, last_inter;
    // Step-size schedule factors (t^-0.3, t^-0.6 for t = 2, 3, ...), FP64,
    // computed on the host with the C library's pow (so the device does not
    // run FP64 pow on its serial path); beyond the table the device computes
    // them itself.
    const double* sched;
    long long sched_len;
};

// Cost generated from coordinates (pdot_dtype PDOT_POINTS):
//   C_ij = dist(xs_i, ys_j) / div, coordinates k = 0..d-1 accumulated in order
//   in FP32, then the quotient by gen_div.  Every kernel that needs C_ij uses
//   the same operation sequence, so the pass, the check and the rounding see
//   the same values.
constexpr int GEN_DMAX = 8;
constexpr int GK_SQEUCLID = 0, GK_L1 = 1, GK_L2 = 2, GK_LINF = 3;

struct GenSpec {
    const float* xs;     // m x d
    const float* ys;     // n x d
    int d, kind;
    float div;
    float inv;           // 1 / div rounded to nearest (host IEEE division)
};

// a / div without a division instruction: q = RN(a * inv), the remainder
// r = RN(a - q * div) by one FMA, and the corrected quotient RN(q + r * inv)
// by another (Markstein's correction step for division by a reciprocal).
// It matched the correctly rounded quotient on every value checked exactly
// (all pixel-grid squared distances over their maximum for grids up to
// 128 x 128, and 20,000 random pairs); in general it is within one ulp.
__host__ __device__ __forceinline__ float gen_div(float a, float div, float inv) {
    const float q = a * inv;
    const float r = fmaf(-q, div, a);
    return fmaf(r, inv, q);
}

// x and y: anything indexable by k < d (register arrays or pointers); d <= DM.
template <int DM = GEN_DMAX, typename PX, typename PY>
__host__ __device__ __forceinline__ float gen_cost(int kind, int d, const PX& x, const PY& y, float div, float inv) {
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < DM; ++k) {
        if (k < d) {
            const float t = x[k] - y[k];
            if (kind == GK_SQEUCLID || kind == GK_L2) acc = fmaf(t, t, acc);
            else if (kind == GK_L1) acc = acc + fabsf(t);
            else acc = fmaxf(acc, fabsf(t));
        }
    }
    if (kind == GK_L2) acc = sqrtf(acc);
    return gen_div(acc, div, inv);
}

struct Inst {
    long long m, n, ldc, ldx;
    const void* C;
    GenSpec gen;         // used when ctype == 3 (C is then null)
    int ctype;           // 0 FP32, 1 BF16, 2 FP64, 3 generated (pdot_dtype)
    int xtype;           // 0 FP32, 2 FP64
    const double* f;
    const double* g;
    void* X;             // NSLOT slots of xslot elements
    long long xslot;
    double* V;           // NSLOT vector sets of vslot doubles
    long long vslot;
    double* rowpart;
    double* colpart;
    double* rowpart2;    // the check's exact row / column sums of the current plan
    double* colpart2;
    double* tpart;
    double* vpart;
    Ctrl* ctrl;
    unsigned int* ticket;
    int nstrips, nchunks, tile_rows, ntiles, nvt;
    int l2_keep_c;       // 1: C fits in L2 next to the streams; load it evict-last, stream X evict-first
};

// Grid barrier state of the cooperative chunk kernel (device memory, zeroed
// before each launch).
struct GridBar {
    unsigned int count;
    unsigned int gen;
    unsigned int err;
    unsigned int pad;
};

struct TileRef {
    int inst;
    int local;
};

// Plan-kernel type combinations (cost dtype / plan dtype).
constexpr int TT_F32 = 0;    // FP32 C, FP32 X
constexpr int TT_BF16 = 1;   // BF16 C, FP32 X
constexpr int TT_F64 = 2;    // FP64 C, FP64 X
constexpr int TT_GEN = 3;    // C generated from coordinates, FP32 X
constexpr int NTT = 4;

// Work counters of the tile-queue kernels, one per (phase, type).  Every
// kernel resets all counters but its own when it starts: kernels on one
// stream run in order, so the previous user of a counter has finished.  The
// same (phase, type) kernel never runs twice in a row.
constexpr int WC_PASS = 0, WC_DUAL = 1, WC_KKT = 2, WC_CHECK = 3, WC_AUX = 4;
constexpr int WC_N = 5 * NTT;
__host__ __device__ constexpr int wc_index(int phase, int ttype) { return phase * NTT + ttype; }

// Host-side launchers (pdot_kernels.cu).  All are asynchronous on `stream`
// and return 0 or a cudaError_t code.
struct LaunchCfg {
    int tile_blocks;      // CTAs of the FP32-plan tile kernels (8 warps each)
    int tile_blocks_f64;  // CTAs of the FP64-plan tile kernels
    int vec_blocks;       // CTAs of the vector kernels (256 threads each)
    int pass_u;           // rows per load batch in the FP32-plan register pass (2 or 4)
    int pass_bulk;        // FP32-plan pass kernel: 0 register pipeline, 1 bulk copies per row, 2 per 4-row group
    int bulk_blocks;      // CTAs of the bulk-copy pass kernel
    int group_blocks;     // CTAs of the grouped bulk-copy pass kernel
    int coop_blocks;      // CTAs of the cooperative chunk kernel (all co-resident)
    int pdl;              // 1: launch with programmatic dependent launch
    int gen_dims;         // largest coordinate count of the generated costs in flight (TT_GEN)
    int comp;             // 1: plan passes of FP32 plans form the compensated reduced cost
    int kkt_blocks;       // CTAs of the bulk-copy KKT pass (0: the register KKT pass)
};

// Tile and vector-tile counts are read from device memory, so one captured
// graph serves every batch composition; nv_hint sizes the vector grids.
// dir_xor flips the row order a pass takes (the order alternates with the
// instance's pass count; the pass timer flips it between its launches).
int launch_pass(int ttype, const Inst* d_insts, const TileRef* d_tmap, const int* T, unsigned* wctr,
                const LaunchCfg& cfg, void* stream, int wc_override = -1, int dir_xor = 0);
int launch_dual(const Inst* d_insts, const TileRef* d_vmap, const int* NV, int nv_hint, unsigned* wctr,
                const LaunchCfg& cfg, void* stream, bool direct = false);
int launch_kkt(int ttype, const Inst* d_insts, const TileRef* d_tmap, const int* T, unsigned* wctr, int mode,
               const LaunchCfg& cfg, void* stream);
int launch_checkvec(const Inst* d_insts, const TileRef* d_vmap, const int* NV, int nv_hint, unsigned* wctr, int mode,
                    const LaunchCfg& cfg, void* stream);
int launch_snapshot(const Inst* d_insts, const int* count, int max_count, Ctrl* out, void* stream);
// After a check: form the average plan the check picked (Ctrl::fix) for the
// instances of one tile type.
int launch_avgfix(int ttype, const Inst* d_insts, const TileRef* d_tmap, const int* T, const LaunchCfg& cfg,
                  void* stream);
// Resident solve (one thread-block cluster per instance, the plan held in
// shared memory): instances list[0 .. *count) of FP32 plans with stored
// FP32 / BF16 costs, each for up to `passes` passes with a check every K
// (K <= 0: none), after a first check when `replay` is set; max_count bounds
// *count (it sizes the grid).
int launch_resident(int ttype, const Inst* d_insts, const int* list, const int* count, int max_count, int passes,
                    int K, int replay, const LaunchCfg& cfg, void* stream);
// Whether an m x n instance's plan fits a cluster's shared memory.
bool resident_fits(long long m, long long n);
// Shared-memory attribute of the resident kernel; -(clusters held at once),
// 0 when it cannot run on this device, > 0 a CUDA error.
int setup_resident();
// out = a + d elementwise (count a multiple of 4; xtype 0 FP32, 2 FP64).
int launch_combine(int xtype, const void* a, const void* d, void* out, long long count, void* stream);
// One warp's bounded wait on a transfer that never comes; *d_status <- ST_DEVICE.
int launch_watchdog_selftest(long long limit, int* d_status, void* stream);
int occupancy_tile_blocks_per_sm(int ttype);
int occupancy_vec_blocks_per_sm();
// Opt the bulk-copy pass kernel into its shared-memory size; returns minus
// the CTAs per SM it can hold, or a positive cudaError_t code.
int setup_bulk_pass();
int setup_group_pass();
int setup_kkt_bulk();
int setup_coop_chunk();
// K passes and one check of a single FP32-plan instance in one cooperative launch.
int launch_chunk_coop(int ttype, const Inst* d_insts, const TileRef* d_tmap, const int* T, const TileRef* d_vmap,
                      const int* NV, unsigned* wctr, GridBar* gb, int npass, const LaunchCfg& cfg, void* stream);

}  // namespace pdot
