// pdot_resident.cuh -- resident solve: the persistent multi-instance kernel
// (included by pdot_kernels.cu, which defines the helpers it shares with the
// tile kernels: the reduced cost, the deviation-form average, the step-size
// controller and the restart controller).
//
// One thread-block cluster of RCS CTAs per instance.  The instance's plan X
// and the average's deviation D = Xbar - X stay in the cluster's shared
// memory for a whole launch (8 B per plan entry; CTA r holds rows
// [r * rows_cta, (r + 1) * rows_cta)), so a PDHG pass (Algorithm 2) reads
// only C and the O(m + n) vectors from global memory.  Per pass:
//   sweep 1   each CTA: X+ = max(0, X - tau (C - p1^T - 1q^T)) on its rows,
//             the row sums and column partials of d = X+ - X and ||d||^2
//             (nothing is written);
//   cluster barrier;
//   dual      rows: each CTA its own; columns: CTA r a slice, adding the
//             RCS column partials in rank order through distributed shared
//             memory; p+, q+, their averages, ||dy||^2 and dy^T A dx written
//             as the vector kernel writes them;
//   cluster barrier;
//   control   every CTA adds the RCS scalar triples in rank order and runs
//             the step-size controller (finalize_step) on its own copy of
//             the controller: the same inputs, so the same decision;
//   sweep 2   if the step is accepted: the same X+ again (same inputs, same
//             bits), written over X, and D+ = (1 - w)(D - d).
// Every K passes a check (the KKT pass and finalize_check, as the check
// kernels compute them) with its restart: the plan a restart picks is formed
// in shared memory and also written to the anchor slot in global memory; a
// reported average is formed into the result slot.  At the end of a launch
// X and D go back to their slots and CTA 0 writes the controller, so the
// instance's state is the same as after the tile kernels' chunk.
//
// Synchronisation is the cluster's hardware barrier only: no spin-wait, no
// flag in memory.  Every CTA of a cluster runs the same sequence of
// barriers (the loop's exits depend on the replicated controller alone).
#pragma once
#include <cooperative_groups.h>

namespace pdot {
namespace res {

namespace cg = cooperative_groups;

constexpr int RCS = 8;                // CTAs per cluster (the portable maximum)
constexpr int RT = 512;               // threads per CTA
constexpr int RW = RT / 32;           // warps per CTA
constexpr int RFLUSH = 32;            // rows of FP32 column accumulation before an FP64 add
constexpr int RSMEM = 220 * 1024;     // dynamic shared memory per CTA
constexpr int RSCAL = 16;             // scalars a CTA publishes per exchange

// Shared-memory layout of one CTA (offsets in bytes from the dynamic base).
struct Layout {
    long long rows;       // rows per CTA (rows_cta)
    long long ldx;
    int nstrips, nseg;
    long long off_x, off_d, off_colseg, off_cols, off_rows, off_rowt, off_scal, off_ctrl, off_red, off_prow, total;
};

__host__ __device__ inline long long al16(long long b) { return (b + 15) / 16 * 16; }

__host__ __device__ inline Layout layout(long long m, long long n) {
    Layout L;
    L.rows = (m + RCS - 1) / RCS;
    L.ldx = (n + 3) / 4 * 4;
    L.nstrips = (int)((n + STRIP - 1) / STRIP);
    L.nseg = L.nstrips <= RW ? RW / L.nstrips : 1;
    long long o = 0;
    L.off_x = o;      o = al16(o + L.rows * L.ldx * 4);
    L.off_d = o;      o = al16(o + L.rows * L.ldx * 4);
    L.off_colseg = o; o = al16(o + (long long)L.nseg * L.ldx * 8);   // per-segment column partials
    L.off_cols = o;   o = al16(o + L.ldx * 8);                       // the CTA's column sums (read by the cluster)
    L.off_rows = o;   o = al16(o + (long long)L.nstrips * L.rows * 8);   // per-strip row partials
    L.off_rowt = o;   o = al16(o + L.rows * 8);                      // the CTA's row sums
    L.off_scal = o;   o = al16(o + RSCAL * 8);                       // scalars read by the cluster
    L.off_ctrl = o;   o = al16(o + (long long)sizeof(Ctrl));         // this CTA's copy of the controller
    L.off_red = o;    o = al16(o + RW * RSCAL * 8);                  // per-warp scalar partials
    L.off_prow = o;   o = al16(o + L.rows * 8);                      // the rows' duals, staged per sweep
    L.total = o;
    return L;
}

// An instance runs resident when its layout fits one CTA's shared memory.
__host__ __device__ inline bool fits(long long m, long long n) {
    return m >= 1 && n >= 1 && layout(m, n).total <= RSMEM;
}

// Per-warp partials of up to RSCAL scalars -> thread k < nv holds the block
// total of scalar k (warps added in order).  Ends with a block barrier.
__device__ __forceinline__ void block_sums(double* red, const double* v, int nv, double* out) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = 0; k < nv; ++k) {
        const double t = warp_sum(v[k]);
        if (lane == 0) red[w * RSCAL + k] = t;
    }
    __syncthreads();
    if ((int)threadIdx.x < nv) {
        double t = 0.0;
        for (int w2 = 0; w2 < RW; ++w2) t += red[w2 * RSCAL + threadIdx.x];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}

// The scalars every CTA published (scal[0..nv)), added in rank order; the
// same values in every CTA.  Called by all threads: RCS * nv of them fetch
// one remote value each into buf (one round trip), then every thread adds
// them in order into out.  Block barriers on both sides of the fetch.
__device__ __forceinline__ void cluster_scalars(cg::cluster_group& cl, double* scal, int nv, double* buf,
                                                double* out) {
    const int t = threadIdx.x;
    if (t < RCS * nv) buf[t] = cl.map_shared_rank(scal, (unsigned)(t / nv))[t % nv];
    __syncthreads();
    for (int k = 0; k < nv; ++k) {
        double a = 0.0;
        for (int r = 0; r < RCS; ++r) a += buf[r * nv + k];
        out[k] = a;
    }
    __syncthreads();
}

// Pointers and sizes of one CTA's part of an instance.
struct Part {
    const Inst* I;
    long long m, n, ldx, r0, nr;   // global first row and row count of this CTA
    long long c0, c1;              // the CTA's column slice of the dual update
    Layout L;
    float* Xs;
    float* Ds;
    double* colseg;
    double* cols;
    double* rowp;
    double* rowt;
    double* scal;
    double* red;
    float2* prow;                  // per row: (p_hi, p_lo) in a pass, (p, pbar) in a check
};

constexpr int RU = 4;   // rows whose loads a warp issues together

// The duals of the CTA's rows, staged in shared memory for a sweep: (p_hi,
// p_lo) of vector set vs (PAIR), or (p of vs, p of vb).  Block barriers on
// both sides.
__device__ __forceinline__ void stage_rows(const Part& P, const double* vs, const double* vb, bool pair, bool use_b) {
    __syncthreads();
    for (long long li = threadIdx.x; li < P.nr; li += RT) {
        const double y = __ldcg(vs + P.r0 + li);
        float2 v;
        if (pair) {
            split_dual(y, v.x, v.y);
        } else {
            v.x = (float)y;
            v.y = use_b ? (float)__ldcg(vb + P.r0 + li) : 0.f;
        }
        P.prow[li] = v;
    }
    __syncthreads();
}

// The rows [a0, a1) of strip s that warp `unit` sweeps (see sweep_step).
struct Unit {
    int s, g;
    long long a0, a1, j0;
};
__device__ __forceinline__ Unit unit_of(const Part& P, int unit, int lane) {
    const int ns = P.L.nstrips, nseg = P.L.nseg;
    Unit u;
    u.s = unit % ns;
    u.g = ns <= RW ? unit / ns : 0;
    const long long seg_rows = (P.nr + nseg - 1) / nseg;
    u.a0 = ns <= RW ? (long long)u.g * seg_rows : 0;
    u.a1 = ns <= RW ? min(u.a0 + seg_rows, P.nr) : P.nr;
    u.j0 = (long long)u.s * STRIP + lane * 4;
    return u;
}

// One sweep over the CTA's rows with the plan step of Algorithm 2 at the
// duals of vector set `vs` (p_i, q_j as FP32 hi/lo pairs, reading C9):
//   SUMS:  row sums (rowp) and column partials (colseg) of d = X+ - X, and
//          ||d||^2 into *dx2 (per thread; added by the caller);
//   WRITE: X <- X+, D <- (1 - w)(D - d) (D <- 0 on the first iterate).
// Warp w takes strip w % nstrips and row segment w / nstrips (or, with more
// strips than warps, strips w, w + RW, ... over all rows), RU rows at a time.
template <typename TC, bool CP, bool WRITE>
__device__ __forceinline__ void sweep_step(const Part& P, const double* vs, float tau, float w, bool first,
                                           double* dx2) {
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int ns = P.L.nstrips, nseg = P.L.nseg;
    const double* q = vs + P.m;
    stage_rows(P, vs, nullptr, true, false);
    const int nunits = ns <= RW ? ns * nseg : ns;
    for (int unit = wp; unit < nunits; unit += RW) {
        const Unit U = unit_of(P, unit, lane);
        const long long j0 = U.j0;
        const bool on = j0 < P.n;
        float qh[4], ql[4];
        bool valid[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            valid[e] = j0 + e < P.n;
            split_dual(valid[e] ? __ldcg(q + j0 + e) : 0.0, qh[e], ql[e]);
        }
        const CostRow<TC, float> cr(*P.I, j0);
        float csa[4] = {0.f, 0.f, 0.f, 0.f};
        double cs[4] = {0.0, 0.0, 0.0, 0.0};
        float dxa = 0.f;
        int nb = 0;
        for (long long lb = U.a0; lb < U.a1; lb += RU) {
            float c[RU][4], x[RU][4];
#pragma unroll
            for (int u = 0; u < RU; ++u) {
                const long long li = lb + u;
#pragma unroll
                for (int e = 0; e < 4; ++e) { c[u][e] = 0.f; x[u][e] = 0.f; }
                if (on && li < U.a1) {
                    cr.get(P.r0 + li, c[u]);
                    const float4 t = *reinterpret_cast<const float4*>(P.Xs + li * P.ldx + j0);
                    x[u][0] = t.x; x[u][1] = t.y; x[u][2] = t.z; x[u][3] = t.w;
                }
            }
#pragma unroll
            for (int u = 0; u < RU; ++u) {
                const long long li = lb + u;
                if (li >= U.a1) break;
                const float2 pp = P.prow[li];
                float v[4], d[4], rs = 0.f;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float R = reduced_cost(c[u][e], pp.x, pp.y, qh[e], ql[e], CP);
                    // one explicit FMA, so the accepting sweep recomputes the same bits
                    float vv = __fmaf_rn(-tau, R, x[u][e]);
                    vv = vv > 0.f ? vv : 0.f;
                    v[e] = valid[e] ? vv : 0.f;
                    d[e] = v[e] - x[u][e];
                    rs += d[e];
                }
                if (WRITE) {
                    if (on) {
                        float4* dp = reinterpret_cast<float4*>(P.Ds + li * P.ldx + j0);
                        const float4 od = *dp;
                        const float o[4] = {od.x, od.y, od.z, od.w};
                        float nd[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) nd[e] = avg_dev_next(first ? 0.f : o[e], d[e], w, first);
                        *dp = make_float4(nd[0], nd[1], nd[2], nd[3]);
                        *reinterpret_cast<float4*>(P.Xs + li * P.ldx + j0) = make_float4(v[0], v[1], v[2], v[3]);
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        csa[e] += d[e];
                        dxa += d[e] * d[e];
                    }
                    rs = warp_sum(rs);
                    if (lane == 0) P.rowp[(long long)U.s * P.L.rows + li] = (double)rs;
                    if (++nb == RFLUSH) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) { cs[e] += (double)csa[e]; csa[e] = 0.f; }
                        *dx2 += (double)dxa;
                        dxa = 0.f;
                        nb = 0;
                    }
                }
            }
        }
        if (!WRITE) {
#pragma unroll
            for (int e = 0; e < 4; ++e) cs[e] += (double)csa[e];
            *dx2 += (double)dxa;
            if (on) {
#pragma unroll
                for (int e = 0; e < 4; ++e) P.colseg[(long long)U.g * P.ldx + j0 + e] = cs[e];
            }
        }
    }
}

// One sweep over the CTA's rows for a check (the arithmetic of the KKT
// pass): with AVG = false the current plan's <C,X>, ||[p + q - C]^+||^2,
// ||X - Xa||^2 and, where the average exists, the same three for the average
// X + D with its duals (into e6[0..6), per thread), and the row sums / column
// partials of X; with AVG = true only the row sums / column partials of
// X + D.
constexpr int RUC = 2;   // rows per load batch of a check sweep (more registers per row)

template <typename TC, bool AVG>
__device__ __forceinline__ void sweep_check(const Part& P, const double* Vc, const double* Vb, const float* Xa,
                                            bool avg, double* e6) {
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int ns = P.L.nstrips, nseg = P.L.nseg;
    if (!AVG) stage_rows(P, Vc, Vb, false, avg);
    const int nunits = ns <= RW ? ns * nseg : ns;
    for (int unit = wp; unit < nunits; unit += RW) {
        const Unit U = unit_of(P, unit, lane);
        const long long j0 = U.j0;
        const bool on = j0 < P.n;
        float qv[4], qbv[4];
        bool valid[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            valid[e] = j0 + e < P.n;
            qv[e] = (!AVG && valid[e]) ? (float)__ldcg(Vc + P.m + j0 + e) : 0.f;
            qbv[e] = (!AVG && valid[e] && avg) ? (float)__ldcg(Vb + P.m + j0 + e) : 0.f;
        }
        const CostRow<TC, float> cr(*P.I, j0);
        float t[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float csa[4] = {0.f, 0.f, 0.f, 0.f};
        double cs[4] = {0.0, 0.0, 0.0, 0.0};
        int nb = 0;
        for (long long lb = U.a0; lb < U.a1; lb += RUC) {
            float c[RUC][4], x[RUC][4], dd[RUC][4], xa[RUC][4];
#pragma unroll
            for (int u = 0; u < RUC; ++u) {
                const long long li = lb + u;
#pragma unroll
                for (int e = 0; e < 4; ++e) { c[u][e] = 0.f; x[u][e] = 0.f; dd[u][e] = 0.f; xa[u][e] = 0.f; }
                if (on && li < U.a1) {
                    const long long i = P.r0 + li;
                    if (!AVG) cr.get(i, c[u]);
                    const float4 tx = *reinterpret_cast<const float4*>(P.Xs + li * P.ldx + j0);
                    x[u][0] = tx.x; x[u][1] = tx.y; x[u][2] = tx.z; x[u][3] = tx.w;
                    if (AVG || avg) {
                        const float4 td = *reinterpret_cast<const float4*>(P.Ds + li * P.ldx + j0);
                        dd[u][0] = td.x; dd[u][1] = td.y; dd[u][2] = td.z; dd[u][3] = td.w;
                    }
                    if (!AVG) {
                        const float4 ta = __ldcg(reinterpret_cast<const float4*>(Xa + i * P.ldx + j0));
                        xa[u][0] = ta.x; xa[u][1] = ta.y; xa[u][2] = ta.z; xa[u][3] = ta.w;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < RUC; ++u) {
                const long long li = lb + u;
                if (li >= U.a1) break;
                const float2 pp = AVG ? make_float2(0.f, 0.f) : P.prow[li];   // (p, pbar) of the row
                float rs = 0.f;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (!valid[e]) continue;
                    const float xb = x[u][e] + dd[u][e];   // the average: X + D
                    if (AVG) {
                        rs += xb;
                        csa[e] += xb;
                    } else {
                        const float Rc = (c[u][e] - pp.x) - qv[e];
                        t[0] += c[u][e] * x[u][e];
                        t[1] += Rc < 0.f ? Rc * Rc : 0.f;            // [p + q - C]^+ squared
                        const float da = x[u][e] - xa[u][e];
                        t[4] += da * da;
                        if (avg) {
                            const float Rb = (c[u][e] - pp.y) - qbv[e];
                            t[2] += c[u][e] * xb;
                            t[3] += Rb < 0.f ? Rb * Rb : 0.f;
                            const float db = xb - xa[u][e];
                            t[5] += db * db;
                        }
                        rs += x[u][e];
                        csa[e] += x[u][e];
                    }
                }
                rs = warp_sum(rs);
                if (lane == 0) P.rowp[(long long)U.s * P.L.rows + li] = (double)rs;
                if (++nb == RFLUSH) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) { cs[e] += (double)csa[e]; csa[e] = 0.f; }
                    if (!AVG) {
#pragma unroll
                        for (int k = 0; k < 6; ++k) { e6[k] += (double)t[k]; t[k] = 0.f; }
                    }
                    nb = 0;
                }
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) cs[e] += (double)csa[e];
        if (!AVG) {
#pragma unroll
            for (int k = 0; k < 6; ++k) e6[k] += (double)t[k];
        }
        if (on) {
#pragma unroll
            for (int e = 0; e < 4; ++e) P.colseg[(long long)U.g * P.ldx + j0 + e] = cs[e];
        }
    }
}

// The CTA's row sums (rowt) and column sums (cols) from the sweep's partials,
// in a fixed order.  Starts and ends with a block barrier.
__device__ __forceinline__ void combine_sums(const Part& P) {
    __syncthreads();
    for (long long li = threadIdx.x; li < P.nr; li += RT) {
        double t = 0.0;
        for (int s = 0; s < P.L.nstrips; ++s) t += P.rowp[(long long)s * P.L.rows + li];
        P.rowt[li] = t;
    }
    const int nseg = P.L.nstrips <= RW ? P.L.nseg : 1;
    for (long long j = threadIdx.x; j < P.ldx; j += RT) {
        double t = 0.0;
        for (int g = 0; g < nseg; ++g) t += P.colseg[(long long)g * P.ldx + j];
        P.cols[j] = t;
    }
    __syncthreads();
}

// Column j's sum over the cluster: the CTAs' column sums in rank order.
__device__ __forceinline__ double cluster_col(cg::cluster_group& cl, double* cols, long long j) {
    double t = 0.0;
    for (unsigned r = 0; r < (unsigned)RCS; ++r) t += cl.map_shared_rank(cols, r)[j];
    return t;
}

// The dual update of one row or column (the arithmetic of the vector
// kernel): t = its sum of X+ - X; returns dy for the step-size scalars.
__device__ __forceinline__ double dual_entry(const double* Vc, double* Vn, const double* Vb, double* Vbn,
                                             long long yo, long long so, double b, double t, double sigma,
                                             double w, bool first) {
    const double y = __ldcg(Vc + yo), r = __ldcg(Vc + so);
    const double yn = y + sigma * (b - (r + 2.0 * t));
    Vn[yo] = yn;
    Vn[so] = r + t;
    Vbn[yo] = first ? yn : __ldcg(Vb + yo) + w * (yn - __ldcg(Vb + yo));
    return yn - y;
}

// Check vectors of one row or column (the arithmetic of the check kernel):
// writes the exact sum s of the plan into the set's r / c entry and adds the
// residual, dual-objective and anchor-distance terms.
__device__ __forceinline__ void check_entry(double* V, const double* Va, long long yo, long long so, double b,
                                            double s, double& res2, double& dobj, double& dist2) {
    V[so] = s;
    const double y = __ldcg(V + yo), ya = __ldcg(Va + yo);
    res2 += (s - b) * (s - b);
    dobj += b * y;
    dist2 += (y - ya) * (y - ya);
}

// One check of a resident instance (the arithmetic of the KKT pass and the
// check kernel, then finalize_check): its restart forms the picked plan in
// shared memory and writes the new anchor; a reported average is formed
// into its result slot.  Called by every CTA of the cluster alike.
template <typename TC>
__device__ __forceinline__ void resident_check(cg::cluster_group& cl, const Part& P, const Inst& I, Ctrl* S) {
    const int tid = threadIdx.x;
    const long long m = P.m, n = P.n;
    const long long nv4 = P.nr * P.ldx / 4;
    // ---- check (Sec. 3.1 KKT, Sec. 5 restart and termination) ----
    double* Vcur = slot_v(I, S->cur);
    double* Vbar = slot_v(I, S->bar);
    const double* Va = slot_v(I, S->anc);
    const float* Xa = slot_x<float>(I, S->anc);
    const bool avg = S->k > 0;
    double A[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) A[k] = 0.0;
    sweep_check<TC, false>(P, Vcur, Vbar, Xa, avg, A + 6);
    combine_sums(P);
    cl.sync();   // column sums of X
    for (long long li = tid; li < P.nr; li += RT) {
        const long long i = P.r0 + li;
        check_entry(Vcur, Va, i, m + n + i, I.f[i], P.rowt[li], A[0], A[2], A[4]);
    }
    for (long long j = P.c0 + tid; j < P.c1; j += RT)
        check_entry(Vcur, Va, m + j, 2 * m + n + j, I.g[j], cluster_col(cl, P.cols, j), A[0], A[2], A[4]);
    if (avg) {
        cl.sync();   // the cluster has read this CTA's column sums of X
        sweep_check<TC, true>(P, Vcur, Vbar, Xa, true, nullptr);
        combine_sums(P);
        cl.sync();   // column sums of X + D
        for (long long li = tid; li < P.nr; li += RT) {
            const long long i = P.r0 + li;
            check_entry(Vbar, Va, i, m + n + i, I.f[i], P.rowt[li], A[1], A[3], A[5]);
        }
        for (long long j = P.c0 + tid; j < P.c1; j += RT)
            check_entry(Vbar, Va, m + j, 2 * m + n + j, I.g[j], cluster_col(cl, P.cols, j), A[1], A[3], A[5]);
    }
    block_sums(P.red, A, 12, P.scal);
    cl.sync();   // every CTA's check scalars
    const long long restarts0 = S->restarts;
    {
        double B[12];
        cluster_scalars(cl, P.scal, 12, P.red, B);
        if (tid == 0) finalize_check(S, B, MODE_CHECK);
    }
    __syncthreads();
    const bool fix = S->fix != 0, in_place = S->fix_dst == S->fix_d;
    const bool restarted = S->restarts != restarts0;
    if (fix && in_place) {
        // restart to the average: X <- X + D (the checks' rounding)
        for (long long e = tid; e < P.nr * P.ldx; e += RT) P.Xs[e] = P.Xs[e] + P.Ds[e];
    } else if (fix) {
        // the reported average, formed into its result slot
        float* out = slot_x<float>(I, S->fix_dst) + P.r0 * P.ldx;
        for (long long e = tid; e < P.nr * P.ldx; e += RT) out[e] = P.Xs[e] + P.Ds[e];
    }
    __syncthreads();
    if (restarted) {
        // the new restart anchor, read by the next checks
        float* out = slot_x<float>(I, S->anc) + P.r0 * P.ldx;
        for (long long e = tid; e < nv4; e += RT)
            reinterpret_cast<float4*>(out)[e] = reinterpret_cast<const float4*>(P.Xs)[e];
    }
    if (tid == 0) S->fix = 0;
    __syncthreads();
}

}  // namespace res

// Resident solve of the instances list[0 .. *count): cluster c takes
// instance list[c] and runs up to `passes` PDHG passes on it, with a check
// after every K passes of the instance (K <= 0: no checks, for a fixed
// number of steps).  replay: run a check first (a state exported at a check
// whose restart logic had not run).  Grid: RCS x (a bound of *count) CTAs.
template <typename TC, bool CP>
__global__ void __cluster_dims__(res::RCS, 1, 1) __launch_bounds__(res::RT, 1)
k_resident(const Inst* __restrict__ insts, const int* __restrict__ list, const int* __restrict__ count, int passes,
           int K, int replay) {
    using namespace res;
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cl = cg::this_cluster();
    const unsigned rank = cl.block_rank();
    const int ci = (int)(blockIdx.x / RCS);
    if (ci >= *count) return;   // the whole cluster (one count for all its CTAs)
    const Inst& I = insts[list[ci]];
    const long long m = I.m, n = I.n;
    Part P;
    P.I = &I;
    P.m = m;
    P.n = n;
    P.L = layout(m, n);
    P.ldx = P.L.ldx;
    P.r0 = min((long long)rank * P.L.rows, m);
    P.nr = min(P.L.rows, m - P.r0);
    P.c0 = n * (long long)rank / RCS;
    P.c1 = n * (long long)(rank + 1) / RCS;
    P.Xs = reinterpret_cast<float*>(smem + P.L.off_x);
    P.Ds = reinterpret_cast<float*>(smem + P.L.off_d);
    P.colseg = reinterpret_cast<double*>(smem + P.L.off_colseg);
    P.cols = reinterpret_cast<double*>(smem + P.L.off_cols);
    P.rowp = reinterpret_cast<double*>(smem + P.L.off_rows);
    P.rowt = reinterpret_cast<double*>(smem + P.L.off_rowt);
    P.scal = reinterpret_cast<double*>(smem + P.L.off_scal);
    P.red = reinterpret_cast<double*>(smem + P.L.off_red);
    P.prow = reinterpret_cast<float2*>(smem + P.L.off_prow);
    Ctrl* S = reinterpret_cast<Ctrl*>(smem + P.L.off_ctrl);
    const int tid = threadIdx.x;

    // This CTA's copy of the controller; its rows of X and (if the average
    // exists) D.
    {
        const long long* src = reinterpret_cast<const long long*>(I.ctrl);
        long long* dst = reinterpret_cast<long long*>(S);
        for (int k = tid; k < (int)(sizeof(Ctrl) / 8); k += RT) dst[k] = __ldcg(src + k);
    }
    __syncthreads();
    const long long nv4 = P.nr * P.ldx / 4;
    const bool ran = S->status == ST_RUNNING;   // a finished instance is left as it is
    if (ran) {
        const float4* xg = reinterpret_cast<const float4*>(slot_x<float>(I, S->cur) + P.r0 * P.ldx);
        for (long long e = tid; e < nv4; e += RT) reinterpret_cast<float4*>(P.Xs)[e] = __ldcg(xg + e);
        if (S->k > 0) {
            const float4* dg = reinterpret_cast<const float4*>(slot_x<float>(I, S->bar) + P.r0 * P.ldx);
            for (long long e = tid; e < nv4; e += RT) reinterpret_cast<float4*>(P.Ds)[e] = __ldcg(dg + e);
        }
    }
    __syncthreads();
    if (ran && replay) resident_check<TC>(cl, P, I, S);

    for (int it = 0; it < passes && S->status == ST_RUNNING; ++it) {
        // ---- one PDHG step (Algorithm 2) ----
        const double* Vc = slot_v(I, S->cur);
        double* Vn = slot_v(I, S->nxt);
        const double* Vb = slot_v(I, S->bar);
        double* Vbn = slot_v(I, S->barn);
        const float tau = (float)S->tau, wf = (float)S->wavg;
        const double sigma = S->sigma, wavg = S->wavg;
        const long long k0 = S->k;
        const bool first = k0 == 0;
        // the step-size schedule factors, requested now (used after the sweeps)
        SchedFactors fac = {0.0, 0.0};
        if (tid == 0 && S->adaptive_step) fac = sched_factors(S, S->total);
        double dx2 = 0.0;
        sweep_step<TC, CP, false>(P, Vc, tau, wf, first, &dx2);
        combine_sums(P);
        cl.sync();   // every CTA's column sums of X+ - X are complete
        double a0 = 0.0, a1 = 0.0;
        for (long long li = tid; li < P.nr; li += RT) {
            const long long i = P.r0 + li;
            const double t = P.rowt[li];
            const double dy = dual_entry(Vc, Vn, Vb, Vbn, i, m + n + i, I.f[i], t, sigma, wavg, first);
            a0 += dy * dy;
            a1 += dy * t;
        }
        for (long long j = P.c0 + tid; j < P.c1; j += RT) {
            const double t = cluster_col(cl, P.cols, j);
            const double dy = dual_entry(Vc, Vn, Vb, Vbn, m + j, 2 * m + n + j, I.g[j], t, sigma, wavg, first);
            a0 += dy * dy;
            a1 += dy * t;
        }
        {
            const double v3[3] = {a0, a1, dx2};
            block_sums(P.red, v3, 3, P.scal);
        }
        cl.sync();   // every CTA's step scalars (and its p+, q+) are written
        {
            double tot[3];
            cluster_scalars(cl, P.scal, 3, P.red, tot);
            if (tid == 0) finalize_step(S, tot[2], tot[0], tot[1], fac, 1.0 / (double)(k0 + 2));
        }
        __syncthreads();
        if (S->status != ST_RUNNING) break;
        if (S->k != k0) {   // accepted: X <- X+, D <- D+ (the same X+ as sweep 1)
            sweep_step<TC, CP, true>(P, Vc, tau, wf, first, nullptr);
            __syncthreads();
        }
        if (K <= 0 || S->passes % K != 0) continue;

        res::resident_check<TC>(cl, P, I, S);
    }

    // Write back: X and D to their slots (so the state is the tile kernels'
    // one, also for a stopped solve that is exported), the controller (CTA 0).
    __syncthreads();
    if (ran) {
        float4* xg = reinterpret_cast<float4*>(slot_x<float>(I, S->cur) + P.r0 * P.ldx);
        for (long long e = tid; e < nv4; e += RT) xg[e] = reinterpret_cast<const float4*>(P.Xs)[e];
    }
    if (ran && S->k > 0) {
        float4* dg = reinterpret_cast<float4*>(slot_x<float>(I, S->bar) + P.r0 * P.ldx);
        for (long long e = tid; e < nv4; e += RT) dg[e] = reinterpret_cast<const float4*>(P.Ds)[e];
    }
    if (ran && rank == 0) {
        long long* dst = reinterpret_cast<long long*>(I.ctrl);
        const long long* src = reinterpret_cast<const long long*>(S);
        for (int k = tid; k < (int)(sizeof(Ctrl) / 8); k += RT) dst[k] = src[k];
    }
    cl.sync();   // no CTA leaves while the cluster may still read its shared memory
}

}  // namespace pdot
