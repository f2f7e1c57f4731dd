// pdot_kernels.cu -- sm_103a kernels of restarted PDHG for optimal transport
// (arXiv 2407.19689, Algorithm 2 with the Sec. 5 controller).
//
// One iteration = two launches over a multi-instance work queue:
//   k_pass  (plan tiles, HBM-bound): one read of C, X, Xbar and one write of
//           X+, Xbar+ per element.  Computes the projected primal step of
//           Algorithm 2, X+ = max(0, X - tau (C - p 1^T - 1 q^T)), the running
//           average, and in registers the row sums of X+ (warp shuffles), the
//           column sums of X+ (per-lane accumulators) and ||X+ - X||^2.
//   k_dual  (vector tiles, O(m+n)): fixed-order reduction of the partial sums,
//           the dual updates p+ = p + sigma (f - (2 r+ - r)),
//           q+ = q + sigma (g - (2 c+ - c)) (r = X 1, c = X^T 1 of the current
//           plan, so 2X+ - X is never re-read), the average of (p, q), and the
//           step-size reductions.  The last vector tile of each instance
//           (atomic ticket) runs the scalar controller: PDLP step-size test,
//           accept/reject by swapping slot roles.
// Every K passes:
//   k_kkt      (plan tiles): reads C, X, Xbar, anchor once; <C,X>, <C,Xbar>,
//              ||[p1^T+1q^T-C]^+||^2 for the current and the average duals,
//              distances to the restart anchor, and exact row/column sums of
//              the stored average.
//   k_checkvec (vector tiles): primal residuals, dual objectives, dual
//              distances; the last tile per instance runs the restart /
//              termination / primal-weight logic of Sec. 5.
// The path is a streaming stencil plus reductions: no tensor cores.  Plan
// tiles are one warp wide (128 columns, 16-byte loads per lane) and
// `tile_rows` tall, handed out by an atomic queue so uneven batches balance.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <type_traits>

#include "pdot_internal.h"

namespace pdot {

constexpr int KU = 2;
// Rows a plan pass (KKT pass) accumulates in FP32 per lane before adding into
// its FP64 partial sums: FP64 is a narrow pipe on this part, and the FP32
// partial over 32 (64) rows of one column carries a relative error of order
// 1e-7, far below what the FP64 sums it feeds are compared against.
constexpr int FLUSH_ROWS = 32;
constexpr int KKT_FLUSH_ROWS = 64;
constexpr int BULK_ROW_S = 8;   // row stages per warp in the per-row bulk pass   // rows per load batch in the KKT pass

// ---------------------------------------------------------------------------
// loads and stores of 4 consecutive elements
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double (&v)[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

__device__ __forceinline__ float bf16_bits_to_f32(unsigned int h) { return __uint_as_float(h << 16); }

// Cost entries (read-only for the whole solve: non-coherent path).
template <typename A>
__device__ __forceinline__ void ldc4(const float* p, A (&v)[4]) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = (A)t.x; v[1] = (A)t.y; v[2] = (A)t.z; v[3] = (A)t.w;
}
template <typename A>
__device__ __forceinline__ void ldc4(const unsigned short* p, A (&v)[4]) {
    const uint2 t = __ldg(reinterpret_cast<const uint2*>(p));
    v[0] = (A)bf16_bits_to_f32(t.x & 0xffffu);
    v[1] = (A)bf16_bits_to_f32(t.x >> 16);
    v[2] = (A)bf16_bits_to_f32(t.y & 0xffffu);
    v[3] = (A)bf16_bits_to_f32(t.y >> 16);
}
template <typename A>
__device__ __forceinline__ void ldc4(const double* p, A (&v)[4]) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    v[0] = (A)a.x; v[1] = (A)a.y; v[2] = (A)b.x; v[3] = (A)b.y;
}
// Ragged right edge: only the first `cnt` (< 4) entries exist.
template <typename A>
__device__ __forceinline__ void ldc4_tail(const float* p, long long cnt, A (&v)[4]) {
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = e < cnt ? (A)__ldg(p + e) : A(0);
}
template <typename A>
__device__ __forceinline__ void ldc4_tail(const unsigned short* p, long long cnt, A (&v)[4]) {
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = e < cnt ? (A)bf16_bits_to_f32(__ldg(p + e)) : A(0);
}
template <typename A>
__device__ __forceinline__ void ldc4_tail(const double* p, long long cnt, A (&v)[4]) {
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = e < cnt ? (A)__ldg(p + e) : A(0);
}

// Tag type of the generated cost (TT_GEN): C_ij comes from coordinates of at
// most DM dimensions (the pass kernel has a 4-dimension variant that keeps
// fewer coordinates in registers).
template <int DM>
struct GenC {};
template <typename TC>
struct GenDims { static constexpr int value = 0; };
template <int DM>
struct GenDims<GenC<DM>> { static constexpr int value = DM; };
using GenC8 = GenC<GEN_DMAX>;
using GenC4 = GenC<4>;

// One lane's four cost entries C[i][j0..j0+3]: read from the stored matrix,
// or generated from the coordinates (the four columns' coordinates are kept in
// registers; the row's are read per call).
template <typename TC, typename A>
struct CostRow {
    const TC* C;
    long long ldc, cnt;
    bool full;
    __device__ __forceinline__ CostRow(const Inst& I, long long j0)
        : C(reinterpret_cast<const TC*>(I.C) + j0), ldc(I.ldc), cnt(I.n - j0), full(j0 + 4 <= I.n) {}
    __device__ __forceinline__ void get(long long i, A (&c)[4]) const {
        if (full) ldc4<A>(C + i * ldc, c);
        else ldc4_tail<A>(C + i * ldc, cnt, c);
    }
};
template <int DM, typename A>
struct CostRow<GenC<DM>, A> {
    GenSpec g;
    float y[4][DM];
    __device__ __forceinline__ CostRow(const Inst& I, long long j0) : g(I.gen) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
#pragma unroll
            for (int k = 0; k < DM; ++k)
                y[e][k] = (k < g.d && j0 + e < I.n) ? __ldg(g.ys + (j0 + e) * g.d + k) : 0.f;
        }
    }
    __device__ __forceinline__ void get(long long i, A (&c)[4]) const {
        float x[DM];
#pragma unroll
        for (int k = 0; k < DM; ++k) x[k] = k < g.d ? __ldg(g.xs + i * g.d + k) : 0.f;
#pragma unroll
        for (int e = 0; e < 4; ++e) c[e] = (A)gen_cost<DM>(g.kind, g.d, x, y[e], g.div, g.inv);
    }
};

// ---------------------------------------------------------------------------
// Reduced cost C_ij - p_i - q_j of the plan pass (reading C9)
// ---------------------------------------------------------------------------
// FP32 plans take the FP64 duals as FP32 pairs, y = hi + lo with hi = RN(y)
// and lo = RN(y - hi).  With `comp` the reduced cost is then formed so that
// its error is of its own size, not of the size of p and q: the rounding
// error e of s = c - p_hi is recovered exactly (Knuth's TwoSum: c - p_hi =
// s + e), s - q_hi is exact where the reduced cost is small (Sterbenz: s is
// then within a factor 2 of q_hi), and the small terms e, p_lo, q_lo are
// added last.  Without `comp`: (c - p_hi) - q_hi, two FP32 roundings of the
// size of p and q (the plan's fixed point is then only as accurate as that).
// FP64 plans use the FP64 duals directly.
__device__ __forceinline__ void split_dual(double y, float& hi, float& lo) {
    hi = (float)y;
    lo = (float)(y - (double)hi);
}
__device__ __forceinline__ void split_dual(double y, double& hi, double& lo) {
    hi = y;
    lo = 0.0;
}
__device__ __forceinline__ float reduced_cost(float c, float ph, float pl, float qh, float ql, bool comp) {
    if (!comp) return (c - ph) - qh;
    const float s = c - ph;
    const float bv = s - c;
    const float e = (c - (s - bv)) + (-ph - bv);   // c - ph = s + e exactly
    return (s - qh) + (e - (pl + ql));
}
__device__ __forceinline__ double reduced_cost(double c, double ph, double, double qh, double, bool) {
    return (c - ph) - qh;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
    // Butterfly: every lane ends with the same, order-fixed sum.
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename TX>
__device__ __forceinline__ TX* slot_x(const Inst& I, int s) {
    return reinterpret_cast<TX*>(I.X) + (long long)s * I.xslot;
}
__device__ __forceinline__ double* slot_v(const Inst& I, int s) { return I.V + (long long)s * I.vslot; }

// Warp-level work queue.
__device__ __forceinline__ int warp_next(unsigned* ctr) {
    int t = 0;
    if ((threadIdx.x & 31) == 0) t = (int)atomicAdd(ctr, 1u);
    return __shfl_sync(0xffffffffu, t, 0);
}

// Tile queue of the plan kernels: a warp's first tile is its global warp
// index (no atomic on the path to the first load); later tiles come from the
// counter, after all first tiles.  Which warp runs a tile does not change its
// arithmetic, so results do not depend on the assignment.
__device__ __forceinline__ int tile_next(unsigned* ctr, bool& first) {
    const int W = (int)(gridDim.x * (blockDim.x >> 5));
    if (first) {
        first = false;
        return (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
    }
    return W + warp_next(ctr);
}

// Arrival on an instance's ticket: the atomic releases this thread's earlier
// writes and, for the last arrival, acquires the others' (one acquire-release
// atomic instead of two sequentially consistent fences).
__device__ __forceinline__ unsigned ticket_arrive(unsigned* ctr) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(ctr) : "memory");
    return old;
}

// Programmatic dependent launch: wait for the previous grid in the stream
// (completion and memory visibility; a no-op without the launch attribute).
// Every solve-loop kernel calls this before touching any data or work counter.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Let the next grid start launching: called when a CTA has finished its work
// (a CTA that exits without calling it counts as having called it).
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Before the wait of a dependent launch: pull the warp's first tile reference
// and its instance descriptor into L1.  Both are written by the host before
// the launch, never by the preceding kernel, so this may run while that
// kernel finishes.
__device__ __forceinline__ void prefetch_first_tile(const Inst* insts, const TileRef* tmap, int T) {
    const int t = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
    if (t >= T || (threadIdx.x & 31) != 0) return;
    const TileRef tr = tmap[t];
    const char* ip = reinterpret_cast<const char*>(insts + tr.inst);
    asm volatile("prefetch.global.L1 [%0];" ::"l"(ip));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(ip + 128));
}

__device__ __forceinline__ void reset_other_counters(unsigned* wctr, int mine) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int c = 0; c < WC_N; ++c)
            if (c != mine) wctr[c] = 0u;
    }
}

// ---------------------------------------------------------------------------
// Plan pass: Algorithm 2 primal step + running average + partial sums
// ---------------------------------------------------------------------------
// Row order of a plan tile: every other pass walks its tiles bottom-up, so the
// rows a pass reads first are the ones the previous pass touched last, which
// are still in L2 (C read, X+ and Xbar+ just written) when the plan does not
// fit in it.  Which order a pass takes changes only the order of its FP32
// column partial sums; it is a function of the instance's pass count (and of
// `dir_xor`, a launch parameter used by the pass timer), so runs stay
// reproducible and an instance gives the same result alone or in a batch.
__device__ __forceinline__ bool pass_reversed(const Ctrl& S, int dir_xor) {
    return ((S.passes ^ (long long)dir_xor) & 1) != 0;
}

// Uniform running average of Algorithm 2, kept as its deviation from the
// current plan, D = Xbar - X: Xbar+ = Xbar + w (X+ - Xbar) becomes
// D+ = (1 - w)(D - d) with d = X+ - X, and D+ = 0 for the first iterate of an
// epoch (Xbar+ = X+).  Stored this way, the rounding of each update is
// relative to |D| (the spread of the iterates around their mean, which
// shrinks as the solve converges), not to |Xbar|: an FP32 average updated in
// place loses the late iterates' weight w = 1/(k+1) below its last bit.
__device__ __forceinline__ float avg_dev_next(float dbar, float d, float w, bool first) {
    const float s = dbar - d;
    return first ? 0.f : fmaf(-w, s, s);
}
__device__ __forceinline__ double avg_dev_next(double dbar, double d, double w, bool first) {
    const double s = dbar - d;
    return first ? 0.0 : fma(-w, s, s);
}

// CP: compensated reduced cost (a kernel template parameter, so the plain
// path is compiled without the compensated one and costs nothing extra).
template <typename TC, typename TX, int U, bool CP>
__device__ __forceinline__ void pass_tile(const Inst& I, const Ctrl& S, int lt, int lane, bool rev) {
    typedef TX A;
    const long long m = I.m, n = I.n, ldx = I.ldx;
    const int strip = lt % I.nstrips, chunk = lt / I.nstrips;
    const long long j0 = (long long)strip * STRIP + lane * 4;
    const long long i0 = (long long)chunk * I.tile_rows;
    const long long i1 = min(i0 + (long long)I.tile_rows, m);
    const bool on = j0 < n;
    const CostRow<TC, A> cr(I, j0);
    const TX* X = slot_x<TX>(I, S.cur);
    const TX* Xb = slot_x<TX>(I, S.bar);
    TX* Xn = slot_x<TX>(I, S.nxt);
    TX* Xbn = slot_x<TX>(I, S.barn);
    const double* p = slot_v(I, S.cur);
    const double* q = p + m;
    const bool first = S.k == 0;
    const A tau = (A)S.tau;
    const A w = (A)S.wavg;

    A qv[4], ql[4];
    bool valid[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        valid[e] = j0 + e < n;
        split_dual(valid[e] ? q[j0 + e] : 0.0, qv[e], ql[e]);
    }
    double cs[4] = {0.0, 0.0, 0.0, 0.0};
    double dx2 = 0.0;
    double* rowpart = I.rowpart + (long long)strip * m;
    const long long nb = (i1 - i0 + U - 1) / U;   // batches of U rows, walked in either order

    for (long long bi = 0; bi < nb; ++bi) {
        const long long ib = i0 + (rev ? nb - 1 - bi : bi) * U;
        // Row pointers of the batch (lanes past n never dereference).
        const long long xo = ib * ldx + j0;
        const TX* Xr = X + xo;
        const TX* Xbr = Xb + xo;
        TX* Xnr = Xn + xo;
        TX* Xbnr = Xbn + xo;
        A c[U][4], x[U][4], xb[U][4], pv[U], pl[U];
        // Issue every load of the U-row batch before any arithmetic.
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool rv = ib + u < i1;
            split_dual(rv ? p[ib + u] : 0.0, pv[u], pl[u]);
            if (rv && on) {
                cr.get(ib + u, c[u]);
                ld4(Xr + u * ldx, x[u]);
                if (!first) ld4(Xbr + u * ldx, xb[u]);
                else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) xb[u][e] = A(0);
                }
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) { c[u][e] = A(0); x[u][e] = A(0); xb[u][e] = A(0); }
            }
        }
        A csa[4] = {A(0), A(0), A(0), A(0)};
        A dxa = A(0);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool rv = ib + u < i1;
            A xn[4], xbn[4];
            A rs = A(0);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const A R = reduced_cost(c[u][e], pv[u], pl[u], qv[e], ql[e], CP);   // C - p - q
                A v = x[u][e] - tau * R;
                v = v > A(0) ? v : A(0);                         // projection onto X >= 0
                v = (valid[e] && rv) ? v : A(0);                 // padding columns / rows past the tile stay 0
                const A d = v - x[u][e];
                dxa += d * d;
                rs += d;                                          // row / column sums of X+ - X
                csa[e] += d;
                xn[e] = v;
                xbn[e] = avg_dev_next(xb[u][e], d, w, first);
            }
            if (rv && on) {
                st4(Xnr + u * ldx, xn);
                st4(Xbnr + u * ldx, xbn);
            }
            rs = warp_sum(rs);
            if (rv && lane == 0) rowpart[ib + u] = (double)rs;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) cs[e] += (double)csa[e];
        dx2 += (double)dxa;
    }
    if (on) {
        double* cp = I.colpart + (long long)chunk * ldx + j0;
        reinterpret_cast<double2*>(cp)[0] = make_double2(cs[0], cs[1]);
        reinterpret_cast<double2*>(cp)[1] = make_double2(cs[2], cs[3]);
    }
    dx2 = warp_sum(dx2);
    if (lane == 0) I.tpart[(long long)lt * TP + 0] = dx2;
}

template <typename TC, typename TX, int U, bool CP>
__global__ void __launch_bounds__(TWARPS * 32, sizeof(TX) == 4 ? 2 : 1)
k_pass(const Inst* __restrict__ insts, const TileRef* __restrict__ tmap, const int* __restrict__ Tp, unsigned* wctr, int wc,
       int dir_xor) {
    pdl_enter();
    const int T = *Tp;
    reset_other_counters(wctr, wc);
    const int lane = threadIdx.x & 31;
    bool first = true;
    for (;;) {
        const int t = tile_next(&wctr[wc], first);
        if (t >= T) break;
        const TileRef tr = tmap[t];
        const Inst& I = insts[tr.inst];
        const Ctrl& S = *I.ctrl;
        if (S.status != ST_RUNNING) continue;
        pass_tile<TC, TX, U, CP>(I, S, tr.local, lane, pass_reversed(S, dir_xor));
    }
}

// ---------------------------------------------------------------------------
// Plan pass, bulk-copy pipeline (FP32 plans): the same arithmetic as
// pass_tile, but every warp streams its rows through a ring of S shared-memory
// stages filled by the bulk-copy engine (cp.async.bulk, completion counted on
// one mbarrier per stage).  Rows in flight cost no registers, so each SM keeps
// ~S x 1.5 KB per warp of reads outstanding.  The warp's row stream runs
// across tile boundaries: the producer (lane 0) fetches the next tile from the
// queue as soon as it has issued the current one's last row.
// ---------------------------------------------------------------------------
namespace bulk {

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
    asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// Bulk copy with an L2 eviction-priority policy (createpolicy descriptor).
__device__ __forceinline__ void g2s_hint(unsigned dst, const void* src, unsigned bytes, unsigned bar,
                                         unsigned long long pol) {
    asm volatile(
        "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar), "l"(pol)
        : "memory");
}
__device__ __forceinline__ unsigned long long policy_evict_last() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ unsigned long long policy_evict_first() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void st4_hint(float* p, const float (&v)[4], unsigned long long pol) {
    asm volatile("st.global.L1::no_allocate.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v[0]),
                 "f"(v[1]), "f"(v[2]), "f"(v[3]), "l"(pol)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Bounded wait: a copy that never lands must not hang the GPU.
constexpr long long WAIT_LIMIT = 1LL << 24;
__device__ __forceinline__ bool wait_stage(unsigned bar, unsigned parity, long long limit = WAIT_LIMIT) {
    for (long long it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

constexpr int STAGE_BYTES = 3 * STRIP * 4;   // C (<= 512 B), X (512 B), Xbar (512 B)

// Row duals of a tile are staged in shared memory, as FP32 pairs, per window
// of PWIN rows.
constexpr int PWIN = 128;
template <int S>
__host__ __device__ constexpr int warp_smem_bytes() { return S * STAGE_BYTES + S * 8 + S * 8 + PWIN * 8; }

struct RowRef {       // what a stage holds
    int tile;         // global tile index (into tmap), -1 = none
    int row;          // matrix row
};

}  // namespace bulk

namespace bulk {
// A warp's row pipeline: its shared-memory stages and mbarriers, and the
// counts of issued / consumed rows (they set the mbarrier phases, so they
// persist across passes when one kernel runs several).
template <int S>
struct RowPipe {
    unsigned char* wbase;
    RowRef* refs;
    float2* pbuf;
    unsigned wbase_s, bars_s;
    long long issued, consumed;
};

template <int S>
__device__ __forceinline__ void row_pipe_init(RowPipe<S>& P, unsigned char* dsm, int lane, int warp) {
    P.wbase = dsm + warp * warp_smem_bytes<S>();
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(P.wbase + S * STAGE_BYTES);
    P.refs = reinterpret_cast<RowRef*>(P.wbase + S * STAGE_BYTES + S * 8);
    P.pbuf = reinterpret_cast<float2*>(P.wbase + S * STAGE_BYTES + S * 16);   // p_i of the tile's rows
    P.wbase_s = smem_u32(P.wbase);
    P.bars_s = smem_u32(bars);
    P.issued = P.consumed = 0;
    if (lane == 0) {
        for (int s = 0; s < S; ++s) mbar_init(P.bars_s + 8 * s, 1);
        fence_mbar_init();
    }
    __syncwarp();
}
}  // namespace bulk

// One pass over the tiles handed out by the queue counter `qctr`.  Returns
// false when a stage never completed (bounded wait); the instance's status
// is then set to an error.
template <typename TC, int S, bool CP>
__device__ bool pass_row_run(const Inst* __restrict__ insts, const TileRef* __restrict__ tmap, int T, unsigned* qctr,
                             bulk::RowPipe<S>& P, int lane, int dir_xor) {
    using namespace bulk;
    unsigned char* wbase = P.wbase;
    RowRef* refs = P.refs;
    float2* pbuf = P.pbuf;
    const unsigned wbase_s = P.wbase_s;
    const unsigned bars_s = P.bars_s;
    constexpr int DM = GenDims<TC>::value;
    constexpr bool GEN = DM > 0;                            // C generated, not copied
    constexpr int DA = GEN ? DM : 1;                        // coordinate array size
    constexpr long long CQ = sizeof(TC) == 2 ? 8 : 4;      // C elements per 16 bytes

    // ---- producer: the tile being issued, resolved once per tile ----
    int p_tile = T;
    long long p_row = 0, p_stop = 0, p_r0 = 0, p_last_ragged = -1;
    long long p_dir = 1;                // +1: top-down, -1: bottom-up (pass_reversed)
    const char* p_c0 = nullptr;         // C at the tile's first row, column c0
    const char* p_x0 = nullptr;         // X at the tile's first row
    const char* p_xb0 = nullptr;        // Xbar at the tile's first row
    long long p_cstride = 0, p_xstride = 0;
    unsigned p_cbytes = 0, p_xbytes = 0;
    bool p_first = true;
    bool p_hint = false;                // keep this instance's C in L2 (it fits)
    const unsigned long long pol_keep = policy_evict_last();
    const unsigned long long pol_stream = policy_evict_first();
    bool q_first = true;
    auto next_tile = [&]() {
        for (;;) {
            p_tile = tile_next(qctr, q_first);
            if (p_tile >= T) return;
            const TileRef tr = tmap[p_tile];
            const Inst& I = insts[tr.inst];
            const Ctrl& Sc = *I.ctrl;
            if (Sc.status != ST_RUNNING) continue;
            const int strip = tr.local % I.nstrips, chunk = tr.local / I.nstrips;
            const long long c0 = (long long)strip * STRIP;
            const long long ncols = min((long long)STRIP, I.n - c0);
            const long long r0 = (long long)chunk * I.tile_rows;
            const long long r1 = min(r0 + (long long)I.tile_rows, I.m);
            const bool rev = pass_reversed(Sc, dir_xor);
            p_dir = rev ? -1 : 1;
            p_r0 = r0;
            p_row = rev ? r1 - 1 : r0;
            p_stop = rev ? r0 - 1 : r1;
            p_xstride = I.ldx * 4;
            if constexpr (!GEN) {
                p_cstride = I.ldc * (long long)sizeof(TC);
                p_c0 = reinterpret_cast<const char*>(I.C) + r0 * p_cstride + c0 * (long long)sizeof(TC);
            }
            p_x0 = reinterpret_cast<const char*>(reinterpret_cast<const float*>(I.X) + (long long)Sc.cur * I.xslot +
                                                 r0 * I.ldx + c0);
            p_xb0 = reinterpret_cast<const char*>(reinterpret_cast<const float*>(I.X) + (long long)Sc.bar * I.xslot +
                                                  r0 * I.ldx + c0);
            p_xbytes = (unsigned)(((ncols + 3) / 4) * 16);
            if constexpr (!GEN) {
                p_cbytes = (unsigned)(((ncols + CQ - 1) / CQ) * CQ * (long long)sizeof(TC));
                // The rounded-up C copy could run past the caller's allocation on
                // the last matrix row of a ragged strip: lanes load that row.
                p_last_ragged = (ncols % CQ) != 0 ? I.m - 1 : -1;
            }
            p_first = Sc.k == 0;
            p_hint = I.l2_keep_c != 0;
            return;
        }
    };
    long long issued = P.issued, consumed = P.consumed;
    const long long base = issued;   // rows of earlier passes (ring position)
    auto issue = [&]() {
        const int st = (int)(issued % S);
        const long long dr = p_row - p_r0;
        const char* p_c = p_c0 + dr * p_cstride;
        const char* p_x = p_x0 + dr * p_xstride;
        const char* p_xb = p_xb0 + dr * p_xstride;
        if (lane == 0) {
            refs[st].tile = p_tile;
            refs[st].row = (int)p_row;
            const unsigned bar = bars_s + 8 * st;
            const unsigned dst = wbase_s + st * STAGE_BYTES;
            const unsigned cb = p_row == p_last_ragged ? 0u : p_cbytes;
            fence_proxy_async();
            mbar_expect_tx(bar, cb + p_xbytes + (p_first ? 0u : p_xbytes));
            if (p_hint) {
                // C is re-read every pass and fits in L2: keep it; stream the plan.
                if (cb) g2s_hint(dst, p_c, cb, bar, pol_keep);
                g2s_hint(dst + STRIP * 4, p_x, p_xbytes, bar, pol_stream);
                if (!p_first) g2s_hint(dst + 2 * STRIP * 4, p_xb, p_xbytes, bar, pol_stream);
            } else {
                if (cb) g2s(dst, p_c, cb, bar);
                g2s(dst + STRIP * 4, p_x, p_xbytes, bar);
                if (!p_first) g2s(dst + 2 * STRIP * 4, p_xb, p_xbytes, bar);
            }
        }
        ++issued;
        p_row += p_dir;
        if (p_row == p_stop) next_tile();
    };
    next_tile();
    while (issued - base < S && p_tile < T) issue();

    // ---- consumer: the tile being computed, resolved once per tile ----
    int c_tile = -1;
    const Inst* CI = nullptr;
    const TC* c_C = nullptr;
    long long c_ldc = 0, c_ldx = 0, c_i0 = 0, c_n = 0, c_last_ragged = -1, c_chunk = 0;
    float* c_xn = nullptr;      // X+ at row c_i0, column j0
    float* c_xbn = nullptr;     // Xbar+ at row c_i0, column j0
    double* c_rowpart = nullptr;
    long long j0 = 0;
    bool on = false, valid[4] = {false, false, false, false};
    float qv[4] = {0.f, 0.f, 0.f, 0.f}, ql[4] = {0.f, 0.f, 0.f, 0.f};
    float tau = 0.f, w = 0.f;
    bool first = true;
    double cs[4] = {0.0, 0.0, 0.0, 0.0}, dx2 = 0.0;
    float csa[4] = {0.f, 0.f, 0.f, 0.f}, dxa = 0.f;
    int rows_in_batch = 0;
    int c_local = 0;
    const double* c_p = nullptr;   // p of the consumer's instance
    bool c_hint = false;
    long long c_i1 = 0, c_win = -1;
    // Generated cost: the lane's four columns' coordinates, and the
    // coordinates of a window of 32 rows (lane r holds row window*32 + r).
    GenSpec gs = {nullptr, nullptr, 0, 0, 1.f, 1.f};
    float gy[4][DA], growc[DA];
    long long c_cwin = -1;
    auto flush_tile = [&]() {
        if (c_tile < 0) return;
#pragma unroll
        for (int e = 0; e < 4; ++e) cs[e] += (double)csa[e];
        dx2 += (double)dxa;
        if (on) {
            double* cp = CI->colpart + c_chunk * CI->ldx + j0;
            reinterpret_cast<double2*>(cp)[0] = make_double2(cs[0], cs[1]);
            reinterpret_cast<double2*>(cp)[1] = make_double2(cs[2], cs[3]);
        }
        const double d = warp_sum(dx2);
        if (lane == 0) CI->tpart[(long long)c_local * TP + 0] = d;
    };
    auto open_consumer = [&](int t) {
        flush_tile();
        c_tile = t;
        const TileRef tr = tmap[t];
        CI = &insts[tr.inst];
        const Ctrl& Sc = *CI->ctrl;
        c_local = tr.local;
        const int strip = tr.local % CI->nstrips;
        c_chunk = tr.local / CI->nstrips;
        const long long c0 = (long long)strip * STRIP;
        c_n = CI->n;
        c_ldc = CI->ldc;
        c_ldx = CI->ldx;
        c_i0 = c_chunk * CI->tile_rows;
        const long long i1 = min(c_i0 + (long long)CI->tile_rows, CI->m);
        j0 = c0 + lane * 4;
        on = j0 < c_n;
        if constexpr (GEN) {
            gs = CI->gen;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
#pragma unroll
                for (int k = 0; k < DA; ++k)
                    gy[e][k] = (k < gs.d && j0 + e < c_n) ? __ldg(gs.ys + (j0 + e) * gs.d + k) : 0.f;
            }
            c_cwin = -1;
        } else {
            const long long ncols = min((long long)STRIP, c_n - c0);
            c_last_ragged = (ncols % CQ) != 0 ? CI->m - 1 : -1;
            c_C = reinterpret_cast<const TC*>(CI->C) + j0;
        }
        float* Xb = reinterpret_cast<float*>(CI->X);
        c_xn = Xb + (long long)Sc.nxt * CI->xslot + c_i0 * c_ldx + j0;
        c_xbn = Xb + (long long)Sc.barn * CI->xslot + c_i0 * c_ldx + j0;
        c_rowpart = CI->rowpart + (long long)strip * CI->m;
        const double* pv = slot_v(*CI, Sc.cur);
        const double* q = pv + CI->m;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            valid[e] = j0 + e < c_n;
            split_dual(valid[e] ? q[j0 + e] : 0.0, qv[e], ql[e]);
        }
        tau = (float)Sc.tau;
        w = (float)Sc.wavg;
        first = Sc.k == 0;
        c_p = pv;
        c_i1 = i1;
        c_hint = CI->l2_keep_c != 0;
        c_win = -1;
#pragma unroll
        for (int e = 0; e < 4; ++e) { cs[e] = 0.0; csa[e] = 0.f; }
        dx2 = 0.0;
        dxa = 0.f;
        rows_in_batch = 0;
    };

    bool failed = false;
    while (consumed < issued) {
        const int st = (int)(consumed % S);
        if (!wait_stage(bars_s + 8 * st, (unsigned)((consumed / S) & 1))) { failed = true; break; }
        const RowRef ref = refs[st];
        if (ref.tile != c_tile) open_consumer(ref.tile);
        const long long i = ref.row;
        const long long di = i - c_i0;
        const unsigned char* stage = wbase + st * STAGE_BYTES;
        float c[4], x[4], xb[4];
        if constexpr (GEN) {
            // Every lane takes part in the shuffles (lanes past n included).
            const long long cw = di >> 5;
            if (cw != c_cwin) {
                const long long r = c_i0 + cw * 32 + lane;
#pragma unroll
                for (int k = 0; k < DA; ++k)
                    growc[k] = (k < gs.d && r < c_i1) ? __ldg(gs.xs + r * gs.d + k) : 0.f;
                c_cwin = cw;
            }
            // gen_cost with the coordinate loop outermost (one shuffle per
            // coordinate, four accumulators) and the distance kind resolved
            // once per row: the same operations per entry.
            const int src = (int)(di & 31);
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            if (gs.kind == GK_L1) {
#pragma unroll
                for (int k = 0; k < DA; ++k) {
                    if (k < gs.d) {
                        const float xk = __shfl_sync(0xffffffffu, growc[k], src);
#pragma unroll
                        for (int e = 0; e < 4; ++e) acc[e] = acc[e] + fabsf(xk - gy[e][k]);
                    }
                }
            } else if (gs.kind == GK_LINF) {
#pragma unroll
                for (int k = 0; k < DA; ++k) {
                    if (k < gs.d) {
                        const float xk = __shfl_sync(0xffffffffu, growc[k], src);
#pragma unroll
                        for (int e = 0; e < 4; ++e) acc[e] = fmaxf(acc[e], fabsf(xk - gy[e][k]));
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < DA; ++k) {
                    if (k < gs.d) {
                        const float xk = __shfl_sync(0xffffffffu, growc[k], src);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float t = xk - gy[e][k];
                            acc[e] = fmaf(t, t, acc[e]);
                        }
                    }
                }
                if (gs.kind == GK_L2) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[e] = sqrtf(acc[e]);
                }
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) c[e] = gen_div(acc[e], gs.div, gs.inv);
        }
        if (on) {
            if constexpr (GEN) {
            } else if (i != c_last_ragged) {
                if (sizeof(TC) == 4) {
                    const float4 t = *reinterpret_cast<const float4*>(stage + lane * 16);
                    c[0] = t.x; c[1] = t.y; c[2] = t.z; c[3] = t.w;
                } else {
                    const uint2 t = *reinterpret_cast<const uint2*>(stage + lane * 8);
                    c[0] = bf16_bits_to_f32(t.x & 0xffffu);
                    c[1] = bf16_bits_to_f32(t.x >> 16);
                    c[2] = bf16_bits_to_f32(t.y & 0xffffu);
                    c[3] = bf16_bits_to_f32(t.y >> 16);
                }
            } else {
                ldc4_tail<float>(c_C + i * c_ldc, c_n - j0, c);
            }
            const float4 tx = *reinterpret_cast<const float4*>(stage + STRIP * 4 + lane * 16);
            x[0] = tx.x; x[1] = tx.y; x[2] = tx.z; x[3] = tx.w;
            if (!first) {
                const float4 tb = *reinterpret_cast<const float4*>(stage + 2 * STRIP * 4 + lane * 16);
                xb[0] = tb.x; xb[1] = tb.y; xb[2] = tb.z; xb[3] = tb.w;
            } else {
                xb[0] = xb[1] = xb[2] = xb[3] = 0.f;
            }
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) { c[e] = GEN ? c[e] : 0.f; x[e] = 0.f; xb[e] = 0.f; }
        }
        // Row duals are staged in shared memory per window of PWIN rows
        // instead of one dependent global load per row.
        const long long win = di / PWIN;
        if (win != c_win) {
            const long long r0 = c_i0 + win * PWIN;
            const long long r1 = min(r0 + (long long)PWIN, c_i1);
            __syncwarp();
            for (long long r = r0 + lane; r < r1; r += 32) {
                float h, l;
                split_dual(c_p[r], h, l);
                pbuf[r - r0] = make_float2(h, l);
            }
            __syncwarp();
            c_win = win;
        }
        const float2 pv = pbuf[di - win * PWIN];
        // The stage has been read: release it to the producer.
        __syncwarp();
        ++consumed;
        if (p_tile < T) issue();

        float xn[4], xbn[4], rs = 0.f;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float R = reduced_cost(c[e], pv.x, pv.y, qv[e], ql[e], CP);
            float v = x[e] - tau * R;
            v = v > 0.f ? v : 0.f;
            v = valid[e] ? v : 0.f;
            const float d = v - x[e];
            dxa += d * d;
            rs += d;                                              // row / column sums of X+ - X
            csa[e] += d;
            xn[e] = v;
            xbn[e] = avg_dev_next(xb[e], d, w, first);
        }
        if (on) {
            if (c_hint) {
                st4_hint(c_xn + di * c_ldx, xn, pol_stream);
                st4_hint(c_xbn + di * c_ldx, xbn, pol_stream);
            } else {
                st4(c_xn + di * c_ldx, xn);
                st4(c_xbn + di * c_ldx, xbn);
            }
        }
        rs = warp_sum(rs);
        if (lane == 0) c_rowpart[i] = (double)rs;
        if (++rows_in_batch == FLUSH_ROWS) {
#pragma unroll
            for (int e = 0; e < 4; ++e) { cs[e] += (double)csa[e]; csa[e] = 0.f; }
            dx2 += (double)dxa;
            dxa = 0.f;
            rows_in_batch = 0;
        }
    }
    if (!failed) {
        flush_tile();
    } else if (lane == 0) {
        // A stage never completed: report it and stop (bounded, never a trap).
        const int t = refs[(int)(consumed % S)].tile;
        atomicExch(&insts[tmap[t].inst].ctrl->status, ST_DEVICE);
    }
    // Drain: wait (bounded) for every copy still in flight.
    while (consumed < issued) {
        const int st = (int)(consumed % S);
        wait_stage(bars_s + 8 * st, (unsigned)((consumed / S) & 1));
        ++consumed;
    }
    P.issued = issued;
    P.consumed = consumed;
    return !failed;
}

template <typename TC, int S, bool CP>
__global__ void __launch_bounds__(TWARPS * 32, 2)
k_pass_bulk(const Inst* __restrict__ insts, const TileRef* __restrict__ tmap, const int* __restrict__ Tp,
            unsigned* wctr, int wc, int dir_xor) {
    // Setup that does not depend on the preceding kernel (tile count and maps
    // are host-written; shared-memory barriers are local) runs before the wait.
    const int T = *Tp;
    extern __shared__ __align__(128) unsigned char dsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bulk::RowPipe<S> P;
    bulk::row_pipe_init<S>(P, dsm, lane, warp);
    prefetch_first_tile(insts, tmap, T);
    pdl_enter();
    reset_other_counters(wctr, wc);
    pass_row_run<TC, S, CP>(insts, tmap, T, &wctr[wc], P, lane, dir_xor);
    pdl_release();
}

// ---------------------------------------------------------------------------
// Plan pass, grouped bulk-copy pipeline (default for FP32 plans).  Like
// k_pass_bulk, but a stage holds a group of up to R consecutive rows of one
// tile: one mbarrier wait and one bookkeeping step per group, the group's
// 3R row copies issued by 3R lanes at once, and the R row sums reduced by a
// multi-row butterfly (6 shuffles for 4 rows instead of 20).
// ---------------------------------------------------------------------------
namespace bulk {

struct GroupRef {
    int tile;     // global tile index
    int row0;     // first matrix row of the group
    int count;    // rows in the group (1..R)
    int pad;
};

template <int R, int S>
__host__ __device__ constexpr int warp_smem_bytes_g() { return S * R * STAGE_BYTES + S * 8 + S * 16 + PWIN * 8; }

// Sum v[r] over the 32 lanes for R = 4 rows with 6 shuffles.  The total of
// row r ends in lanes 8r .. 8r+7.
__device__ __forceinline__ float rows4_sum(const float (&v)[4], int lane) {
    const bool hi16 = lane & 16;
    const float s0 = __shfl_xor_sync(0xffffffffu, hi16 ? v[0] : v[2], 16);
    const float s1 = __shfl_xor_sync(0xffffffffu, hi16 ? v[1] : v[3], 16);
    const float a0 = (hi16 ? v[2] : v[0]) + s0;   // row 0 (low half) / row 2 (high half)
    const float a1 = (hi16 ? v[3] : v[1]) + s1;   // row 1 / row 3
    const bool hi8 = lane & 8;
    const float t = __shfl_xor_sync(0xffffffffu, hi8 ? a0 : a1, 8);
    float b = (hi8 ? a1 : a0) + t;
    b += __shfl_xor_sync(0xffffffffu, b, 4);
    b += __shfl_xor_sync(0xffffffffu, b, 2);
    b += __shfl_xor_sync(0xffffffffu, b, 1);
    return b;
}

}  // namespace bulk

template <typename TC, int S, bool CP>
__global__ void __launch_bounds__(TWARPS * 32, 2)
k_pass_group(const Inst* __restrict__ insts, const TileRef* __restrict__ tmap, const int* __restrict__ Tp,
             unsigned* wctr, int wc, int dir_xor) {
    using namespace bulk;
    constexpr int R = 4;
    const int T = *Tp;   // host-written: read before the wait (see k_pass_bulk)
    prefetch_first_tile(insts, tmap, T);
    pdl_enter();
    reset_other_counters(wctr, wc);
    extern __shared__ __align__(128) unsigned char dsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char* wbase = dsm + warp * warp_smem_bytes_g<R, S>();
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(wbase + S * R * STAGE_BYTES);
    GroupRef* refs = reinterpret_cast<GroupRef*>(wbase + S * R * STAGE_BYTES + S * 8);
    float2* pbuf = reinterpret_cast<float2*>(wbase + S * R * STAGE_BYTES + S * 24);
    const unsigned wbase_s = smem_u32(wbase);
    const unsigned bars_s = smem_u32(bars);
    if (lane == 0) {
        for (int s = 0; s < S; ++s) mbar_init(bars_s + 8 * s, 1);
        fence_mbar_init();
    }
    __syncwarp();
    constexpr int DM = GenDims<TC>::value;
    constexpr bool GEN = DM > 0;                         // C generated, not copied
    constexpr int DA = GEN ? DM : 1;                     // coordinate array size
    constexpr long long CQ = sizeof(TC) == 2 ? 8 : 4;   // C elements per 16 bytes

    // ---- producer: a tile's R-row groups, walked in either order (pass_reversed) ----
    int p_tile = T;
    long long p_r0 = 0, p_r1 = 0, p_G = 0, p_gi = 0, p_last_ragged = -1;
    bool p_rev = false;
    const char* p_c0 = nullptr;         // C, X, Xbar at the tile's first row
    const char* p_x0 = nullptr;
    const char* p_xb0 = nullptr;
    long long p_cstride = 0, p_xstride = 0;
    unsigned p_cbytes = 0, p_xbytes = 0;
    bool p_first = true;
    bool q_first = true;
    auto next_tile = [&]() {
        for (;;) {
            p_tile = tile_next(&wctr[wc], q_first);
            if (p_tile >= T) return;
            const TileRef tr = tmap[p_tile];
            const Inst& I = insts[tr.inst];
            const Ctrl& Sc = *I.ctrl;
            if (Sc.status != ST_RUNNING) continue;
            const int strip = tr.local % I.nstrips, chunk = tr.local / I.nstrips;
            const long long c0 = (long long)strip * STRIP;
            const long long ncols = min((long long)STRIP, I.n - c0);
            p_r0 = (long long)chunk * I.tile_rows;
            p_r1 = min(p_r0 + (long long)I.tile_rows, I.m);
            p_G = (p_r1 - p_r0 + R - 1) / R;
            p_gi = 0;
            p_rev = pass_reversed(Sc, dir_xor);
            p_xstride = I.ldx * 4;
            if constexpr (!GEN) {
                p_cstride = I.ldc * (long long)sizeof(TC);
                p_c0 = reinterpret_cast<const char*>(I.C) + p_r0 * p_cstride + c0 * (long long)sizeof(TC);
            }
            p_x0 = reinterpret_cast<const char*>(reinterpret_cast<const float*>(I.X) + (long long)Sc.cur * I.xslot +
                                                 p_r0 * I.ldx + c0);
            p_xb0 = reinterpret_cast<const char*>(reinterpret_cast<const float*>(I.X) + (long long)Sc.bar * I.xslot +
                                                  p_r0 * I.ldx + c0);
            p_xbytes = (unsigned)(((ncols + 3) / 4) * 16);
            if constexpr (!GEN) {
                p_cbytes = (unsigned)(((ncols + CQ - 1) / CQ) * CQ * (long long)sizeof(TC));
                p_last_ragged = (ncols % CQ) != 0 ? I.m - 1 : -1;
            }
            p_first = Sc.k == 0;
            return;
        }
    };
    long long issued = 0, consumed = 0;   // in groups
    auto issue = [&]() {
        const int st = (int)(issued % S);
        const long long p_row = p_r0 + R * (p_rev ? p_G - 1 - p_gi : p_gi);   // the group's first row
        const int g = (int)min((long long)R, p_r1 - p_row);
        const long long dr = p_row - p_r0;
        const char* p_c = p_c0 + dr * p_cstride;
        const char* p_x = p_x0 + dr * p_xstride;
        const char* p_xb = p_xb0 + dr * p_xstride;
        const unsigned bar = bars_s + 8 * st;
        const unsigned dst = wbase_s + st * (R * STAGE_BYTES);
        // The C copy of the last matrix row of a ragged strip is skipped (lanes load it).
        const bool skip_c = p_last_ragged >= p_row && p_last_ragged < p_row + g;
        const unsigned bytes = (unsigned)g * (p_cbytes + p_xbytes + (p_first ? 0u : p_xbytes)) - (skip_c ? p_cbytes : 0u);
        if (lane == 0) {
            refs[st].tile = p_tile;
            refs[st].row0 = (int)p_row;
            refs[st].count = g;
            fence_proxy_async();
            mbar_expect_tx(bar, bytes);
        }
        __syncwarp();
        // Lane k copies array (k % 3) of row (k / 3): 3g copies issued at once.
        if (lane < 3 * g) {
            const int r = lane / 3, arr = lane % 3;
            const unsigned d = dst + r * STAGE_BYTES + arr * (STRIP * 4);
            fence_proxy_async();   // this lane's copy follows the warp's generic reads of the stage
            if (arr == 0) {
                if constexpr (!GEN) {
                    if (!(skip_c && p_row + r == p_last_ragged)) g2s(d, p_c + r * p_cstride, p_cbytes, bar);
                }
            } else if (arr == 1) {
                g2s(d, p_x + r * p_xstride, p_xbytes, bar);
            } else if (!p_first) {
                g2s(d, p_xb + r * p_xstride, p_xbytes, bar);
            }
        }
        ++issued;
        if (++p_gi == p_G) next_tile();
    };
    next_tile();
    while (issued < S && p_tile < T) issue();

    // ---- consumer ----
    int c_tile = -1;
    const Inst* CI = nullptr;
    const TC* c_C = nullptr;
    long long c_ldc = 0, c_ldx = 0, c_i0 = 0, c_n = 0, c_last_ragged = -1, c_chunk = 0;
    float* c_xn = nullptr;
    float* c_xbn = nullptr;
    double* c_rowpart = nullptr;
    long long j0 = 0;
    bool on = false, valid[4] = {false, false, false, false};
    float qv[4] = {0.f, 0.f, 0.f, 0.f}, ql[4] = {0.f, 0.f, 0.f, 0.f};
    float tau = 0.f, w = 0.f;
    bool first = true;
    double cs[4] = {0.0, 0.0, 0.0, 0.0}, dx2 = 0.0;
    float csa[4] = {0.f, 0.f, 0.f, 0.f}, dxa = 0.f;
    int rows_in_batch = 0;
    int c_local = 0;
    const double* c_p = nullptr;
    long long c_i1 = 0, c_win = -1;
    // Generated cost: the lane's four columns' coordinates, and a 32-row
    // window of row coordinates (lane r holds row window * 32 + r).
    GenSpec gs = {nullptr, nullptr, 0, 0, 1.f, 1.f};
    float gy[4][DA], growc[DA];
    long long c_cwin = -1;
    auto flush_tile = [&]() {
        if (c_tile < 0) return;
#pragma unroll
        for (int e = 0; e < 4; ++e) cs[e] += (double)csa[e];
        dx2 += (double)dxa;
        if (on) {
            double* cp = CI->colpart + c_chunk * CI->ldx + j0;
            reinterpret_cast<double2*>(cp)[0] = make_double2(cs[0], cs[1]);
            reinterpret_cast<double2*>(cp)[1] = make_double2(cs[2], cs[3]);
        }
        const double d = warp_sum(dx2);
        if (lane == 0) CI->tpart[(long long)c_local * TP + 0] = d;
    };
    auto open_consumer = [&](int t) {
        flush_tile();
        c_tile = t;
        const TileRef tr = tmap[t];
        CI = &insts[tr.inst];
        const Ctrl& Sc = *CI->ctrl;
        c_local = tr.local;
        const int strip = tr.local % CI->nstrips;
        c_chunk = tr.local / CI->nstrips;
        const long long c0 = (long long)strip * STRIP;
        c_n = CI->n;
        c_ldc = CI->ldc;
        c_ldx = CI->ldx;
        c_i0 = c_chunk * CI->tile_rows;
        c_i1 = min(c_i0 + (long long)CI->tile_rows, CI->m);
        j0 = c0 + lane * 4;
        on = j0 < c_n;
        if constexpr (GEN) {
            gs = CI->gen;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
#pragma unroll
                for (int k = 0; k < DA; ++k)
                    gy[e][k] = (k < gs.d && j0 + e < c_n) ? __ldg(gs.ys + (j0 + e) * gs.d + k) : 0.f;
            }
            c_cwin = -1;
        } else {
            const long long ncols = min((long long)STRIP, c_n - c0);
            c_last_ragged = (ncols % CQ) != 0 ? CI->m - 1 : -1;
            c_C = reinterpret_cast<const TC*>(CI->C) + j0;
        }
        float* Xb = reinterpret_cast<float*>(CI->X);
        c_xn = Xb + (long long)Sc.nxt * CI->xslot + c_i0 * c_ldx + j0;
        c_xbn = Xb + (long long)Sc.barn * CI->xslot + c_i0 * c_ldx + j0;
        c_rowpart = CI->rowpart + (long long)strip * CI->m;
        c_p = slot_v(*CI, Sc.cur);
        const double* q = c_p + CI->m;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            valid[e] = j0 + e < c_n;
            split_dual(valid[e] ? q[j0 + e] : 0.0, qv[e], ql[e]);
        }
        tau = (float)Sc.tau;
        w = (float)Sc.wavg;
        first = Sc.k == 0;
        c_win = -1;
#pragma unroll
        for (int e = 0; e < 4; ++e) { cs[e] = 0.0; csa[e] = 0.f; }
        dx2 = 0.0;
        dxa = 0.f;
        rows_in_batch = 0;
    };

    bool failed = false;
    while (consumed < issued) {
        const int st = (int)(consumed % S);
        if (!wait_stage(bars_s + 8 * st, (unsigned)((consumed / S) & 1))) { failed = true; break; }
        const GroupRef ref = refs[st];
        if (ref.tile != c_tile) open_consumer(ref.tile);
        const unsigned char* stage = wbase + st * (R * STAGE_BYTES);
        float rsv[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            rsv[r] = 0.f;
            if (r >= ref.count) continue;
            const long long i = ref.row0 + r;
            const long long di = i - c_i0;
            const unsigned char* rst = stage + r * STAGE_BYTES;
            // Row duals staged per window of PWIN rows.
            const long long win = di / PWIN;
            if (win != c_win) {
                const long long r0 = c_i0 + win * PWIN;
                const long long r1 = min(r0 + (long long)PWIN, c_i1);
                __syncwarp();
                for (long long rr = r0 + lane; rr < r1; rr += 32) {
                    float h, l;
                    split_dual(c_p[rr], h, l);
                    pbuf[rr - r0] = make_float2(h, l);
                }
                __syncwarp();
                c_win = win;
            }
            const float2 pv = pbuf[di - win * PWIN];
            float c[4], x[4], xb[4];
            if constexpr (GEN) {
                // Same operations as gen_cost; every lane takes part in the shuffles.
                const long long cw = di >> 5;
                if (cw != c_cwin) {
                    const long long rr = c_i0 + cw * 32 + lane;
#pragma unroll
                    for (int k = 0; k < DA; ++k)
                        growc[k] = (k < gs.d && rr < c_i1) ? __ldg(gs.xs + rr * gs.d + k) : 0.f;
                    c_cwin = cw;
                }
                const int src = (int)(di & 31);
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
                if (gs.kind == GK_L1) {
#pragma unroll
                    for (int k = 0; k < DA; ++k) {
                        if (k < gs.d) {
                            const float xk = __shfl_sync(0xffffffffu, growc[k], src);
#pragma unroll
                            for (int e = 0; e < 4; ++e) acc[e] = acc[e] + fabsf(xk - gy[e][k]);
                        }
                    }
                } else if (gs.kind == GK_LINF) {
#pragma unroll
                    for (int k = 0; k < DA; ++k) {
                        if (k < gs.d) {
                            const float xk = __shfl_sync(0xffffffffu, growc[k], src);
#pragma unroll
                            for (int e = 0; e < 4; ++e) acc[e] = fmaxf(acc[e], fabsf(xk - gy[e][k]));
                        }
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < DA; ++k) {
                        if (k < gs.d) {
                            const float xk = __shfl_sync(0xffffffffu, growc[k], src);
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const float t = xk - gy[e][k];
                                acc[e] = fmaf(t, t, acc[e]);
                            }
                        }
                    }
                    if (gs.kind == GK_L2) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) acc[e] = sqrtf(acc[e]);
                    }
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) c[e] = gen_div(acc[e], gs.div, gs.inv);
            }
            if (on) {
                if constexpr (GEN) {
                } else if (i != c_last_ragged) {
                    if (sizeof(TC) == 4) {
                        const float4 t = *reinterpret_cast<const float4*>(rst + lane * 16);
                        c[0] = t.x; c[1] = t.y; c[2] = t.z; c[3] = t.w;
                    } else {
                        const uint2 t = *reinterpret_cast<const uint2*>(rst + lane * 8);
                        c[0] = bf16_bits_to_f32(t.x & 0xffffu);
                        c[1] = bf16_bits_to_f32(t.x >> 16);
                        c[2] = bf16_bits_to_f32(t.y & 0xffffu);
                        c[3] = bf16_bits_to_f32(t.y >> 16);
                    }
                } else {
                    ldc4_tail<float>(c_C + i * c_ldc, c_n - j0, c);
                }
                const float4 tx = *reinterpret_cast<const float4*>(rst + STRIP * 4 + lane * 16);
                x[0] = tx.x; x[1] = tx.y; x[2] = tx.z; x[3] = tx.w;
                if (!first) {
                    const float4 tb = *reinterpret_cast<const float4*>(rst + 2 * STRIP * 4 + lane * 16);
                    xb[0] = tb.x; xb[1] = tb.y; xb[2] = tb.z; xb[3] = tb.w;
                } else {
                    xb[0] = xb[1] = xb[2] = xb[3] = 0.f;
                }
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) { c[e] = GEN ? c[e] : 0.f; x[e] = 0.f; xb[e] = 0.f; }
            }
            float xn[4], xbn[4], rs = 0.f;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float Rc = reduced_cost(c[e], pv.x, pv.y, qv[e], ql[e], CP);
                float v = x[e] - tau * Rc;
                v = v > 0.f ? v : 0.f;
                v = valid[e] ? v : 0.f;
                const float d = v - x[e];
                dxa += d * d;
                rs += d;                                          // row / column sums of X+ - X
                csa[e] += d;
                xn[e] = v;
                xbn[e] = avg_dev_next(xb[e], d, w, first);
            }
            if (on) {
                st4(c_xn + di * c_ldx, xn);
                st4(c_xbn + di * c_ldx, xbn);
            }
            rsv[r] = rs;
        }
        // The group's stage has been read: release it and refill it.
        __syncwarp();
        ++consumed;
        if (p_tile < T) issue();
        const float tot = rows4_sum(rsv, lane);
        if ((lane & 7) == 0 && (lane >> 3) < ref.count) c_rowpart[ref.row0 + (lane >> 3)] = (double)tot;
        rows_in_batch += ref.count;
        if (rows_in_batch >= FLUSH_ROWS) {
#pragma unroll
            for (int e = 0; e < 4; ++e) { cs[e] += (double)csa[e]; csa[e] = 0.f; }
            dx2 += (double)dxa;
            dxa = 0.f;
            rows_in_batch = 0;
        }
    }
    pdl_release();
    if (!failed) {
        flush_tile();
    } else if (lane == 0) {
        const int t = refs[(int)(consumed % S)].tile;
        atomicExch(&insts[tmap[t].inst].ctrl->status, ST_DEVICE);
    }
    while (consumed < issued) {
        const int st = (int)(consumed % S);
        wait_stage(bars_s + 8 * st, (unsigned)((consumed / S) & 1));
        ++consumed;
    }
}

// ---------------------------------------------------------------------------
// Slot bookkeeping
// ---------------------------------------------------------------------------
// nxt and barn <- the two lowest slots not in use as cur, bar or anc.
__device__ __forceinline__ void assign_free(Ctrl* S, int cur, int bar, int anc) {
    const int used = (1 << cur) | (1 << bar) | (1 << anc);
    int picks[2] = {0, 0};
    int np = 0;
    for (int s = 0; s < NSLOT && np < 2; ++s)
        if (!(used & (1 << s))) picks[np++] = s;
    S->nxt = picks[0];
    S->barn = picks[1];
}

// ---------------------------------------------------------------------------
// Dual step + PDLP step-size controller
// ---------------------------------------------------------------------------
// The schedule factors of attempted iteration t1 = total + 2 (reading C6).
struct SchedFactors {
    double f3, f6;   // t1^-0.3, t1^-0.6
};
__device__ __forceinline__ SchedFactors sched_factors(const Ctrl* S, long long total) {
    SchedFactors r;
    if (total < S->sched_len) {
        r.f3 = __ldg(S->sched + 2 * total);
        r.f6 = __ldg(S->sched + 2 * total + 1);
    } else {
        const double t1 = (double)(total + 2);
        r.f3 = pow(t1, -0.3);
        r.f6 = pow(t1, -0.6);
    }
    return r;
}

// The controller fields the step decision reads.  Only the decision itself
// writes them during a dual update, so a copy taken when the update starts
// is current when the instance's last tile decides; taking it early keeps
// those reads off the serial path (after the ticket's acquire they would go
// to L2 again).
struct StepPre {
    double eta, omega;
    long long passes, k, total, rejected;
    int cur, nxt, bar, barn, anc, adaptive_step;
};
__device__ __forceinline__ StepPre step_pre(const Ctrl* S) {
    StepPre P;
    P.eta = S->eta;
    P.omega = S->omega;
    P.passes = S->passes;
    P.k = S->k;
    P.total = S->total;
    P.rejected = S->rejected;
    P.cur = S->cur;
    P.nxt = S->nxt;
    P.bar = S->bar;
    P.barn = S->barn;
    P.anc = S->anc;
    P.adaptive_step = S->adaptive_step;
    return P;
}

// w_next: 1 / (k + 2), the averaging weight after an accepted step (computed
// by the caller early, off this serial path).  P: step_pre(S), taken at any
// point after the previous decision.
__device__ void finalize_step(Ctrl* S, const StepPre& P, double dX2, double dy2, double inter, SchedFactors fac,
                              double w_next) {
    S->passes = P.passes + 1;
    S->last_dX2 = dX2;
    S->last_dy2 = dy2;
    S->last_inter = inter;
    bool accept = true;
    double eta = P.eta;
    if (P.adaptive_step) {
        // Sec. 5 step-size rule in the PDLP form (reading C6); the exponent base
        // is the 1-based index of the attempted iteration plus one.
        // The accept/reject decision is discrete: it is taken in FP64 with
        // the same expression as the FP64 reference of the rule, so that
        // both sides decide alike away from exact ties.
        const double om = P.omega;
        const double etabar = inter != 0.0 ? (om * dX2 + dy2 / om) / (2.0 * fabs(inter)) : CUDART_INF;
        const double a = (1.0 - fac.f3) * etabar;
        const double b = (1.0 + fac.f6) * eta;
        const double eta_next = a < b ? a : b;
        accept = eta <= etabar;
        S->last_etabar = etabar;
        eta = eta_next;
    }
    if (!isfinite(dX2) || !isfinite(dy2) || !isfinite(eta) || !(eta > 0.0)) {
        S->status = ST_NUMERIC;
        S->res_slot = S->res_xslot = P.cur;
        S->res_avg = 0;
        return;
    }
    S->fix = 0;   // the plan a restart picked has been formed before this pass
    if (accept) {
        S->cur = P.nxt;
        S->bar = P.barn;
        assign_free(S, P.nxt, P.barn, P.anc);
        S->k = P.k + 1;
        S->wavg = w_next;
        S->total = P.total + 1;
    } else {
        S->rejected = P.rejected + 1;
    }
    S->eta = eta;
    S->tau = eta / P.omega;
    S->sigma = eta * P.omega;
}

__device__ __forceinline__ void finalize_step(Ctrl* S, double dX2, double dy2, double inter, SchedFactors fac,
                                              double w_next) {
    finalize_step(S, step_pre(S), dX2, dy2, inter, fac, w_next);
}

// One vector tile (VE = 32 entries of [p; q]) per CTA.  All warps add the
// FP64 partial sums of the tile's row or column sums (group g: partials g,
// g + VG, ...); warp 0 combines the groups in order, updates the duals and
// the averages, reduces the tile's step-size scalars with shuffles and takes
// the instance's ticket; the last tile of an instance finishes the step.
// Everything that does not depend on the partial sums is requested before
// them, and only one block-wide barrier is on the path (FP64 is a narrow pipe
// on this part: block-wide FP64 reductions cost more than they save).
__device__ void dual_tile(const Inst& I, Ctrl* S, int lvt, double* sgrp) {
    const long long m = I.m, n = I.n;
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const long long e = (long long)lvt * VE + lane;
    const bool row = e < m, col = !row && e < m + n;
    const long long idx = row ? e : e - m;
    const long long yo = row ? idx : m + idx;                   // p_i or q_j
    const long long so = row ? m + n + idx : 2 * m + n + idx;   // r_i or c_j
    int status = ST_RUNNING;
    double sigma = 0.0, b = 0.0, r = 0.0, y = 0.0, ybar = 0.0, wavg = 1.0, w_next = 0.5;
    long long k = 0;
    double* Vn = nullptr;
    double* Vbn = nullptr;
    SchedFactors fac = {0.0, 0.0};
    // The step decision's controller fields, used only by the instance's last
    // tile (lane 0 of warp 0 copies and later reads them: no barrier needed).
    __shared__ StepPre s_pre;
    if (grp == 0) {
        status = S->status;
        if (lane == 0) s_pre = step_pre(S);
        sigma = S->sigma;
        k = S->k;
        wavg = S->wavg;
        w_next = 1.0 / (double)(k + 2);   // used by the instance's last tile, if the step is accepted
        // requested now, used only by the instance's last tile
        if (S->adaptive_step) fac = sched_factors(S, S->total);
        const double* Vc = slot_v(I, S->cur);
        const double* Vb = slot_v(I, S->bar);
        Vn = slot_v(I, S->nxt);
        Vbn = slot_v(I, S->barn);
        if (row || col) {
            b = row ? I.f[idx] : I.g[idx];
            r = Vc[so];
            y = Vc[yo];
            if (k != 0) ybar = Vb[yo];
        }
    }
    double s = 0.0;
    if (row || col) {
        const double* part = row ? I.rowpart : I.colpart;
        const long long stride = row ? m : I.ldx;
        const int count = row ? I.nstrips : I.nchunks;
#pragma unroll 8
        for (int kk = grp; kk < count; kk += VG) s += part[(long long)kk * stride + idx];
    }
    // This tile's slice of the plan tiles' ||X+ - X||^2 partials, requested
    // with the partial sums above (before the barrier, off the serial path).
    double a2 = 0.0;
    if (grp == 0) {
        const long long T = I.ntiles;
        const long long t0 = T * lvt / I.nvt, t1 = T * (lvt + 1) / I.nvt;
        for (long long tt = t0 + lane; tt < t1; tt += 32) a2 += I.tpart[tt * TP + 0];
    }
    sgrp[grp * 32 + lane] = s;
    __syncthreads();
    if (grp == 0 && status == ST_RUNNING) {
        double t = 0.0;
#pragma unroll
        for (int g2 = 0; g2 < VG; ++g2) t += sgrp[g2 * 32 + lane];
        double a0 = 0.0, a1 = 0.0;   // ||dy||^2, dy^T A dx (this tile's slice; a2: ||dX||^2)
        if (row || col) {
            // t: this row's or column's sum of X+ - X (the pass sums the change
            // itself, so the step-size term dy^T A dX below is not a difference
            // of two nearly equal sums); (2X+ - X) 1 = r + 2t, X+ 1 = r + t.
            const double w = wavg;
            const double yn = y + sigma * (b - (r + 2.0 * t));
            Vn[yo] = yn;
            Vn[so] = r + t;
            Vbn[yo] = k == 0 ? yn : ybar + w * (yn - ybar);
            const double dy = yn - y;
            a0 = dy * dy;
            a1 = dy * t;
        }
        a0 = warp_sum(a0);
        a1 = warp_sum(a1);
        a2 = warp_sum(a2);
        unsigned old = 0;
        if (lane == 0) {
            double* vp = I.vpart + (long long)lvt * VP;
            vp[0] = a0; vp[1] = a1; vp[2] = a2;
            old = ticket_arrive(I.ticket);
        }
        old = __shfl_sync(0xffffffffu, old, 0);
        __syncwarp();
        if (old == (unsigned)(I.nvt - 1)) {
            double b0 = 0.0, b1 = 0.0, b2 = 0.0;
            for (int v = lane; v < I.nvt; v += 32) {
                const double* vp = I.vpart + (long long)v * VP;
                b0 += __ldcg(vp + 0);
                b1 += __ldcg(vp + 1);
                b2 += __ldcg(vp + 2);
            }
            b0 = warp_sum(b0);
            b1 = warp_sum(b1);
            b2 = warp_sum(b2);
            if (lane == 0) {
                *I.ticket = 0u;
                finalize_step(S, s_pre, b2, b0, b1, fac, w_next);
            }
        }
    }
    __syncthreads();   // sgrp is reused by the caller's next tile
}

__global__ void __launch_bounds__(VT) k_dual(const Inst* __restrict__ insts, const TileRef* __restrict__ vmap,
                                             const int* __restrict__ NVp, unsigned* wctr, int direct) {
    // One CTA per vector tile (no work queue): the grid covers the tile count.
    // direct: one instance whose vector tiles are exactly the grid (no map or
    // count to read before the work).
    __shared__ double sgrp[VG * 32];
    pdl_enter();
    // The next pass may start launching now: it waits for this grid to
    // complete before it reads anything this grid writes, and its CTAs use
    // the time to set up (a no-op without programmatic dependent launch).
    pdl_release();
    // No work counter of its own, but it still resets the others for the
    // kernels that follow (block 0, before any early exit).
    reset_other_counters(wctr, wc_index(WC_DUAL, 0));
    TileRef tr;
    if (direct) {
        tr.inst = 0;
        tr.local = (int)blockIdx.x;
    } else {
        const int NV = *NVp;
        if ((int)blockIdx.x >= NV) return;
        tr = vmap[blockIdx.x];
    }
    const Inst& I = insts[tr.inst];
    // The instance's status is read inside (warp 0), next to the other
    // controller fields; a finished instance's tile does nothing.
    dual_tile(I, I.ctrl, tr.local, sgrp);
}

// ---------------------------------------------------------------------------
// KKT pass (every K passes, and once at the start)
// ---------------------------------------------------------------------------
template <typename TC, typename TX>
__device__ __forceinline__ void kkt_tile(const Inst& I, const Ctrl& S, int lt, int lane, int mode) {
    typedef TX A;
    const long long m = I.m, n = I.n, ldx = I.ldx;
    const int strip = lt % I.nstrips, chunk = lt / I.nstrips;
    const long long j0 = (long long)strip * STRIP + lane * 4;
    const long long i0 = (long long)chunk * I.tile_rows;
    const long long i1 = min(i0 + (long long)I.tile_rows, m);
    const bool on = j0 < n;
    const CostRow<TC, A> cr(I, j0);
    const bool init = mode == MODE_INIT;
    const bool avg = !init && S.k > 0;      // the running average exists
    const bool sums = init || avg;          // exact row/col sums of X (init) or Xbar (check)
    const TX* X = slot_x<TX>(I, S.cur);
    const TX* Xb = slot_x<TX>(I, S.bar);
    const TX* Xa = slot_x<TX>(I, S.anc);
    const double* p = slot_v(I, S.cur);
    const double* q = p + m;
    const double* pb = slot_v(I, S.bar);
    const double* qb = pb + m;

    // The check's dual residual [p + q - C]^+ takes the plain reduced cost:
    // its FP32 rounding (of the size of p and q) is far below ||C||_F, the
    // scale this term is measured against.
    A qv[4], qbv[4];
    bool valid[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        valid[e] = j0 + e < n;
        qv[e] = valid[e] ? (A)q[j0 + e] : A(0);
        qbv[e] = (valid[e] && avg) ? (A)qb[j0 + e] : A(0);
    }
    double acc[TP] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};   // cxc, rd2c, cxb, rd2b, dXac, dXab
    double cs[4] = {0.0, 0.0, 0.0, 0.0};
    double cs2[4] = {0.0, 0.0, 0.0, 0.0};   // check: exact column sums of the current plan
    double* rowpart = I.rowpart + (long long)strip * m;
    double* rowpart2 = I.rowpart2 + (long long)strip * m;

    // FP32 plans accumulate in FP32 over KKT_FLUSH_ROWS rows before adding
    // into the FP64 partials (an FP64 add per batch of two rows would make
    // this pass bound by the narrow FP64 pipe) -- the same grouping as
    // k_kkt_bulk, so both give the same bits.
    constexpr int KFLUSH = sizeof(A) == 4 ? KKT_FLUSH_ROWS / KU : 1;
    A t[TP] = {A(0), A(0), A(0), A(0), A(0), A(0)};
    A csa[4] = {A(0), A(0), A(0), A(0)}, csa2[4] = {A(0), A(0), A(0), A(0)};
    int nbatch = 0;
    for (long long ib = i0; ib < i1; ib += KU) {
        A c[KU][4], x[KU][4], xb[KU][4], xa[KU][4], pv[KU], pbv[KU];
#pragma unroll
        for (int u = 0; u < KU; ++u) {
            const long long i = ib + u;
            const bool rv = i < i1;
            pv[u] = rv ? (A)p[i] : A(0);
            pbv[u] = (rv && avg) ? (A)pb[i] : A(0);
#pragma unroll
            for (int e = 0; e < 4; ++e) { c[u][e] = A(0); x[u][e] = A(0); xb[u][e] = A(0); xa[u][e] = A(0); }
            if (rv && on) {
                cr.get(i, c[u]);
                ld4(X + i * ldx + j0, x[u]);
                if (avg) {
                    ld4(Xb + i * ldx + j0, xb[u]);
                    ld4(Xa + i * ldx + j0, xa[u]);
#pragma unroll
                    for (int e = 0; e < 4; ++e) xb[u][e] = x[u][e] + xb[u][e];   // the average: X + D
                } else if (!init) {
                    ld4(Xa + i * ldx + j0, xa[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < KU; ++u) {
            const long long i = ib + u;
            const bool rv = i < i1;
            A rs = A(0), rs2 = A(0);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (!valid[e] || !rv) continue;
                const A Rc = (c[u][e] - pv[u]) - qv[e];
                t[0] += c[u][e] * x[u][e];
                t[1] += Rc < A(0) ? Rc * Rc : A(0);             // [p + q - C]^+ squared
                const A da = x[u][e] - xa[u][e];
                t[4] += da * da;
                if (init) t[2] += c[u][e] * c[u][e];             // ||C||_F^2 (once per solve)
                if (avg) {
                    const A Rb = (c[u][e] - pbv[u]) - qbv[e];
                    t[2] += c[u][e] * xb[u][e];
                    t[3] += Rb < A(0) ? Rb * Rb : A(0);
                    const A db = xb[u][e] - xa[u][e];
                    t[5] += db * db;
                }
                const A sv = init ? x[u][e] : xb[u][e];
                rs += sv;
                csa[e] += sv;
                rs2 += x[u][e];
                csa2[e] += x[u][e];
            }
            if (sums) {
                rs = warp_sum(rs);
                if (rv && lane == 0) rowpart[i] = (double)rs;
            }
            if (!init) {
                rs2 = warp_sum(rs2);
                if (rv && lane == 0) rowpart2[i] = (double)rs2;
            }
        }
        if (++nbatch == KFLUSH || ib + KU >= i1) {
#pragma unroll
            for (int k = 0; k < TP; ++k) {
                acc[k] += (double)t[k];
                t[k] = A(0);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                cs[e] += (double)csa[e];
                cs2[e] += (double)csa2[e];
                csa[e] = A(0);
                csa2[e] = A(0);
            }
            nbatch = 0;
        }
    }
    if (sums && on) {
        double* cp = I.colpart + (long long)chunk * ldx + j0;
        reinterpret_cast<double2*>(cp)[0] = make_double2(cs[0], cs[1]);
        reinterpret_cast<double2*>(cp)[1] = make_double2(cs[2], cs[3]);
    }
    if (!init && on) {
        double* cp = I.colpart2 + (long long)chunk * ldx + j0;
        reinterpret_cast<double2*>(cp)[0] = make_double2(cs2[0], cs2[1]);
        reinterpret_cast<double2*>(cp)[1] = make_double2(cs2[2], cs2[3]);
    }
#pragma unroll
    for (int k = 0; k < TP; ++k) acc[k] = warp_sum(acc[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < TP; ++k) I.tpart[(long long)lt * TP + k] = acc[k];
    }
}

template <typename TC, typename TX>
__global__ void __launch_bounds__(TWARPS * 32, sizeof(TX) == 4 ? 2 : 1)
k_kkt(const Inst* __restrict__ insts, const TileRef* __restrict__ tmap, const int* __restrict__ Tp, unsigned* wctr, int wc, int mode) {
    pdl_enter();
    const int T = *Tp;
    reset_other_counters(wctr, wc);
    const int lane = threadIdx.x & 31;
    bool first = true;
    for (;;) {
        const int t = tile_next(&wctr[wc], first);
        if (t >= T) break;
        const TileRef tr = tmap[t];
        const Inst& I = insts[tr.inst];
        const Ctrl& S = *I.ctrl;
        if (S.status != ST_RUNNING) continue;
        kkt_tile<TC, TX>(I, S, tr.local, lane, mode);
    }
}

// ---------------------------------------------------------------------------
// KKT pass, bulk-copy pipeline (FP32 plans with a stored FP32 or BF16 cost):
// the arithmetic of kkt_tile, with each warp streaming its tile's rows of C,
// X, Xbar and the restart anchor through KS shared-memory stages filled by
// cp.async.bulk (completion counted on one mbarrier per stage, bounded wait),
// so a warp keeps KS rows of four arrays in flight without holding them in
// registers.  The FP32 accumulators are added into FP64 every 16 rows.
// ---------------------------------------------------------------------------
constexpr int KS = 4;                     // stages per warp (two CTAs per SM: 64 rows of 4 arrays in flight)
constexpr int KSTAGE = 4 * STRIP * 4;     // C (<= 512 B), X, Xbar, anchor (512 B each)
constexpr int KACC = TP + 8;              // FP64 accumulators per lane kept in shared memory (6 scalars, 2 x 4 columns)
__host__ __device__ constexpr int kkt_warp_smem() {
    return KS * KSTAGE + KS * 8 + KS * 8 + bulk::PWIN * 8 + KACC * 32 * 8;
}
constexpr int kkt_smem() { return TWARPS * kkt_warp_smem(); }

template <typename TC>
__global__ void __launch_bounds__(TWARPS * 32, 2)
k_kkt_bulk(const Inst* __restrict__ insts, const TileRef* __restrict__ tmap, const int* __restrict__ Tp,
           unsigned* wctr, int wc, int mode) {
    using namespace bulk;
    const int T = *Tp;   // host-written: read before the wait
    extern __shared__ __align__(128) unsigned char dsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char* wbase = dsm + warp * kkt_warp_smem();
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(wbase + KS * KSTAGE);
    RowRef* refs = reinterpret_cast<RowRef*>(wbase + KS * KSTAGE + KS * 8);
    float2* pbuf = reinterpret_cast<float2*>(wbase + KS * KSTAGE + KS * 16);   // (p_i, pbar_i) of a row window
    // The lane's FP64 accumulators (kept out of registers): [k * 32 + lane],
    // k < TP the tile scalars, then 4 column sums (average / initial plan), 4
    // column sums (current plan).
    double* sacc = reinterpret_cast<double*>(wbase + KS * KSTAGE + KS * 16 + bulk::PWIN * 8);
    const unsigned wbase_s = smem_u32(wbase);
    const unsigned bars_s = smem_u32(bars);
    if (lane == 0) {
        for (int s = 0; s < KS; ++s) mbar_init(bars_s + 8 * s, 1);
        fence_mbar_init();
    }
    __syncwarp();
    prefetch_first_tile(insts, tmap, T);
    pdl_enter();
    reset_other_counters(wctr, wc);
    const bool init = mode == MODE_INIT;
    constexpr long long CQ = sizeof(TC) == 2 ? 8 : 4;   // C elements per 16 bytes

    // ---- producer ----
    int p_tile = T;
    long long p_row = 0, p_end = 0, p_r0 = 0, p_last_ragged = -1;
    const char* p_c0 = nullptr;     // C, X, Xbar, anchor at the tile's first row
    const char* p_x0 = nullptr;
    const char* p_xb0 = nullptr;
    const char* p_xa0 = nullptr;
    long long p_cstride = 0, p_xstride = 0;
    unsigned p_cbytes = 0, p_xbytes = 0;
    bool p_avg = false;
    bool q_first = true;
    auto next_tile = [&]() {
        for (;;) {
            p_tile = tile_next(&wctr[wc], q_first);
            if (p_tile >= T) return;
            const TileRef tr = tmap[p_tile];
            const Inst& I = insts[tr.inst];
            const Ctrl& Sc = *I.ctrl;
            if (Sc.status != ST_RUNNING) continue;
            const int strip = tr.local % I.nstrips, chunk = tr.local / I.nstrips;
            const long long c0 = (long long)strip * STRIP;
            const long long ncols = min((long long)STRIP, I.n - c0);
            p_r0 = (long long)chunk * I.tile_rows;
            p_row = p_r0;
            p_end = min(p_r0 + (long long)I.tile_rows, I.m);
            p_xstride = I.ldx * 4;
            p_cstride = I.ldc * (long long)sizeof(TC);
            p_c0 = reinterpret_cast<const char*>(I.C) + p_r0 * p_cstride + c0 * (long long)sizeof(TC);
            const float* Xb = reinterpret_cast<const float*>(I.X);
            p_x0 = reinterpret_cast<const char*>(Xb + (long long)Sc.cur * I.xslot + p_r0 * I.ldx + c0);
            p_xb0 = reinterpret_cast<const char*>(Xb + (long long)Sc.bar * I.xslot + p_r0 * I.ldx + c0);
            p_xa0 = reinterpret_cast<const char*>(Xb + (long long)Sc.anc * I.xslot + p_r0 * I.ldx + c0);
            p_xbytes = (unsigned)(((ncols + 3) / 4) * 16);
            p_cbytes = (unsigned)(((ncols + CQ - 1) / CQ) * CQ * (long long)sizeof(TC));
            // The rounded-up C copy could run past the caller's allocation on
            // the last matrix row of a ragged strip: lanes load that row.
            p_last_ragged = (ncols % CQ) != 0 ? I.m - 1 : -1;
            p_avg = !init && Sc.k > 0;
            return;
        }
    };
    long long issued = 0, consumed = 0;
    auto issue = [&]() {
        const int st = (int)(issued % KS);
        const long long dr = p_row - p_r0;
        if (lane == 0) {
            refs[st].tile = p_tile;
            refs[st].row = (int)p_row;
            const unsigned bar = bars_s + 8 * st;
            const unsigned dst = wbase_s + st * KSTAGE;
            const unsigned cb = p_row == p_last_ragged ? 0u : p_cbytes;
            fence_proxy_async();
            mbar_expect_tx(bar, cb + p_xbytes + (p_avg ? p_xbytes : 0u) + (init ? 0u : p_xbytes));
            if (cb) g2s(dst, p_c0 + dr * p_cstride, cb, bar);
            g2s(dst + STRIP * 4, p_x0 + dr * p_xstride, p_xbytes, bar);
            if (p_avg) g2s(dst + 2 * STRIP * 4, p_xb0 + dr * p_xstride, p_xbytes, bar);
            if (!init) g2s(dst + 3 * STRIP * 4, p_xa0 + dr * p_xstride, p_xbytes, bar);
        }
        ++issued;
        if (++p_row >= p_end) next_tile();
    };
    next_tile();
    while (issued < KS && p_tile < T) issue();

    // ---- consumer ----
    int c_tile = -1, c_local = 0;
    const Inst* CI = nullptr;
    const TC* c_C = nullptr;
    long long c_ldc = 0, c_i0 = 0, c_i1 = 0, c_n = 0, c_last_ragged = -1, c_chunk = 0, c_win = -1, j0 = 0;
    bool on = false, c_avg = false, valid[4] = {false, false, false, false};
    float qv[4] = {0.f, 0.f, 0.f, 0.f}, qbv[4] = {0.f, 0.f, 0.f, 0.f};
    const double* c_p = nullptr;
    const double* c_pb = nullptr;
    double* c_rowpart = nullptr;
    double* c_rowpart2 = nullptr;
    float t[TP], csa[4], csa2[4];
    int rows_in_batch = 0;
    auto flush_acc = [&]() {
#pragma unroll
        for (int k = 0; k < TP; ++k) { sacc[k * 32 + lane] += (double)t[k]; t[k] = 0.f; }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            sacc[(TP + e) * 32 + lane] += (double)csa[e];
            sacc[(TP + 4 + e) * 32 + lane] += (double)csa2[e];
            csa[e] = 0.f;
            csa2[e] = 0.f;
        }
        rows_in_batch = 0;
    };
    auto flush_tile = [&]() {
        if (c_tile < 0) return;
        flush_acc();
        const double* cs = sacc + TP * 32;
        if (on && (init || c_avg)) {
            double* cp = CI->colpart + c_chunk * CI->ldx + j0;
            reinterpret_cast<double2*>(cp)[0] = make_double2(cs[0 * 32 + lane], cs[1 * 32 + lane]);
            reinterpret_cast<double2*>(cp)[1] = make_double2(cs[2 * 32 + lane], cs[3 * 32 + lane]);
        }
        if (on && !init) {
            double* cp = CI->colpart2 + c_chunk * CI->ldx + j0;
            reinterpret_cast<double2*>(cp)[0] = make_double2(cs[4 * 32 + lane], cs[5 * 32 + lane]);
            reinterpret_cast<double2*>(cp)[1] = make_double2(cs[6 * 32 + lane], cs[7 * 32 + lane]);
        }
#pragma unroll
        for (int k = 0; k < TP; ++k) {
            const double a = warp_sum(sacc[k * 32 + lane]);
            if (lane == 0) CI->tpart[(long long)c_local * TP + k] = a;
        }
    };
    auto open_consumer = [&](int tt) {
        flush_tile();
        c_tile = tt;
        const TileRef tr = tmap[tt];
        CI = &insts[tr.inst];
        const Ctrl& Sc = *CI->ctrl;
        c_local = tr.local;
        const int strip = tr.local % CI->nstrips;
        c_chunk = tr.local / CI->nstrips;
        const long long c0 = (long long)strip * STRIP;
        c_n = CI->n;
        c_ldc = CI->ldc;
        c_i0 = c_chunk * CI->tile_rows;
        c_i1 = min(c_i0 + (long long)CI->tile_rows, CI->m);
        j0 = c0 + lane * 4;
        on = j0 < c_n;
        const long long ncols = min((long long)STRIP, c_n - c0);
        c_last_ragged = (ncols % CQ) != 0 ? CI->m - 1 : -1;
        c_C = reinterpret_cast<const TC*>(CI->C) + j0;
        c_avg = !init && Sc.k > 0;
        c_p = slot_v(*CI, Sc.cur);
        c_pb = slot_v(*CI, Sc.bar);
        const double* q = c_p + CI->m;
        const double* qb = c_pb + CI->m;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            valid[e] = j0 + e < c_n;
            qv[e] = valid[e] ? (float)q[j0 + e] : 0.f;
            qbv[e] = (valid[e] && c_avg) ? (float)qb[j0 + e] : 0.f;
        }
        c_rowpart = CI->rowpart + (long long)strip * CI->m;
        c_rowpart2 = CI->rowpart2 + (long long)strip * CI->m;
        c_win = -1;
#pragma unroll
        for (int k = 0; k < KACC; ++k) sacc[k * 32 + lane] = 0.0;
#pragma unroll
        for (int k = 0; k < TP; ++k) t[k] = 0.f;
#pragma unroll
        for (int e = 0; e < 4; ++e) { csa[e] = 0.f; csa2[e] = 0.f; }
        rows_in_batch = 0;
    };

    bool failed = false;
    while (consumed < issued) {
        const int st = (int)(consumed % KS);
        if (!wait_stage(bars_s + 8 * st, (unsigned)((consumed / KS) & 1))) { failed = true; break; }
        const RowRef ref = refs[st];
        if (ref.tile != c_tile) open_consumer(ref.tile);
        const long long i = ref.row;
        const long long di = i - c_i0;
        const unsigned char* stage = wbase + st * KSTAGE;
        float c[4], x[4], xb[4], xa[4];
        if (on) {
            if (i != c_last_ragged) {
                if (sizeof(TC) == 4) {
                    const float4 v = *reinterpret_cast<const float4*>(stage + lane * 16);
                    c[0] = v.x; c[1] = v.y; c[2] = v.z; c[3] = v.w;
                } else {
                    const uint2 v = *reinterpret_cast<const uint2*>(stage + lane * 8);
                    c[0] = bf16_bits_to_f32(v.x & 0xffffu);
                    c[1] = bf16_bits_to_f32(v.x >> 16);
                    c[2] = bf16_bits_to_f32(v.y & 0xffffu);
                    c[3] = bf16_bits_to_f32(v.y >> 16);
                }
            } else {
                ldc4_tail<float>(c_C + i * c_ldc, c_n - j0, c);
            }
            const float4 vx = *reinterpret_cast<const float4*>(stage + STRIP * 4 + lane * 16);
            x[0] = vx.x; x[1] = vx.y; x[2] = vx.z; x[3] = vx.w;
            if (c_avg) {
                const float4 vb = *reinterpret_cast<const float4*>(stage + 2 * STRIP * 4 + lane * 16);
                xb[0] = x[0] + vb.x; xb[1] = x[1] + vb.y; xb[2] = x[2] + vb.z; xb[3] = x[3] + vb.w;   // X + D
            } else {
                xb[0] = xb[1] = xb[2] = xb[3] = 0.f;
            }
            if (!init) {
                const float4 va = *reinterpret_cast<const float4*>(stage + 3 * STRIP * 4 + lane * 16);
                xa[0] = va.x; xa[1] = va.y; xa[2] = va.z; xa[3] = va.w;
            } else {
                xa[0] = xa[1] = xa[2] = xa[3] = 0.f;
            }
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) { c[e] = 0.f; x[e] = 0.f; xb[e] = 0.f; xa[e] = 0.f; }
        }
        // Row duals (current and average) staged per window of PWIN rows.
        const long long win = di / PWIN;
        if (win != c_win) {
            const long long r0 = c_i0 + win * PWIN;
            const long long r1 = min(r0 + (long long)PWIN, c_i1);
            __syncwarp();
            for (long long r = r0 + lane; r < r1; r += 32)
                pbuf[r - r0] = make_float2((float)c_p[r], c_avg ? (float)c_pb[r] : 0.f);
            __syncwarp();
            c_win = win;
        }
        const float2 pp = pbuf[di - win * PWIN];
        // The stage has been read: release it to the producer.
        __syncwarp();
        ++consumed;
        if (p_tile < T) issue();

        float rs = 0.f, rs2 = 0.f;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (!valid[e]) continue;
            const float Rc = (c[e] - pp.x) - qv[e];
            t[0] += c[e] * x[e];
            t[1] += Rc < 0.f ? Rc * Rc : 0.f;                  // [p + q - C]^+ squared
            const float da = x[e] - xa[e];
            t[4] += da * da;
            if (init) t[2] += c[e] * c[e];                      // ||C||_F^2 (once per solve)
            if (c_avg) {
                const float Rb = (c[e] - pp.y) - qbv[e];
                t[2] += c[e] * xb[e];
                t[3] += Rb < 0.f ? Rb * Rb : 0.f;
                const float db = xb[e] - xa[e];
                t[5] += db * db;
            }
            const float sv = init ? x[e] : xb[e];
            rs += sv;
            csa[e] += sv;
            rs2 += x[e];
            csa2[e] += x[e];
        }
        if (init || c_avg) {
            rs = warp_sum(rs);
            if (lane == 0) c_rowpart[i] = (double)rs;
        }
        if (!init) {
            rs2 = warp_sum(rs2);
            if (lane == 0) c_rowpart2[i] = (double)rs2;
        }
        if (++rows_in_batch == KKT_FLUSH_ROWS) flush_acc();
    }
    pdl_release();
    if (!failed) {
        flush_tile();
    } else if (lane == 0) {
        const int tt = refs[(int)(consumed % KS)].tile;
        atomicExch(&insts[tmap[tt].inst].ctrl->status, ST_DEVICE);
    }
    while (consumed < issued) {   // drain: wait (bounded) for every copy still in flight
        const int st = (int)(consumed % KS);
        wait_stage(bars_s + 8 * st, (unsigned)((consumed / KS) & 1));
        ++consumed;
    }
}

// ---------------------------------------------------------------------------
// Check: KKT of current and average, restart / termination / primal weight
// ---------------------------------------------------------------------------
struct KP {
    double rp2, rd2, cx, dual, gap, kkt, rel_p, rel_d, rel_gap, rel;
};

__device__ void kkt_parts(const Ctrl* S, double rp2, double rd2, double cx, double dual, KP& o) {
    // KKT error of Sec. 3.1 and the relative measures of reading C5.
    o.rp2 = rp2;
    o.rd2 = rd2;
    o.cx = cx;
    o.dual = dual;
    o.gap = cx - dual;
    const double gr = o.gap / S->R;
    o.kkt = sqrt(rp2 + rd2 + gr * gr);
    double dp = S->norm_b, dd = S->norm_C, dg = fabs(cx) + fabs(dual);
    if (S->rel_mode == 1) { dp += 1.0; dd += 1.0; dg += 1.0; }
    if (!(dp > 0.0)) dp = 1.0;
    if (!(dd > 0.0)) dd = 1.0;
    if (!(dg > 0.0)) dg = 1.0;
    o.rel_p = sqrt(rp2) / dp;
    o.rel_d = sqrt(rd2) / dd;
    o.rel_gap = fabs(o.gap) / dg;
    o.rel = fmax(o.rel_p, fmax(o.rel_d, o.rel_gap));
}

__device__ void report(Ctrl* S, const KP& k) {
    S->r_rp2 = k.rp2; S->r_rd2 = k.rd2; S->r_cx = k.cx; S->r_dual = k.dual; S->r_gap = k.gap;
    S->r_kkt = k.kkt; S->r_rel_p = k.rel_p; S->r_rel_d = k.rel_d; S->r_rel_gap = k.rel_gap; S->r_rel = k.rel;
}

// A: 0 rp2 cur, 1 rp2 avg, 2 dual cur, 3 dual avg, 4 ||dy_anchor||^2 cur, 5 avg,
//    6 <C,X>, 7 rd2 cur, 8 <C,Xbar>, 9 rd2 avg, 10 ||X - Xa||^2, 11 ||Xbar - Xa||^2.
// In MODE_INIT: 1 sum f, 3 sum g, 4 ||[f;g]||^2, 5 invalid marginal entries,
//    8 ||C||_F^2.
__device__ void finalize_check(Ctrl* S, const double* A, int mode) {
    if (mode == MODE_INIT) {
        // Data norms for the relative measures, and the marginal checks of the ABI.
        S->norm_b = sqrt(A[4]);
        S->norm_C = sqrt(A[8]);
        const double sf = A[1], sg = A[3];
        if (A[5] > 0.0 || !(fabs(sf - sg) <= 1e-9 * fmax(sf, 1.0))) {
            S->status = ST_ARG;
            S->res_slot = S->res_xslot = S->cur;
            return;
        }
    }
    KP c;
    kkt_parts(S, A[0], A[7], A[6], A[2], c);
    S->checks += 1;
    if (mode == MODE_CHECK && S->stop_req) {
        // Stopped by the host (time limit): the current iterate, with the
        // measures this check has just computed for it.
        report(S, c);
        S->status = ST_TIMEOUT;
        S->res_slot = S->res_xslot = S->cur;
        S->res_avg = 0;
        return;
    }
    if (mode == MODE_INIT) {
        report(S, c);
        S->kkt0 = c.kkt;
        S->kkt_prev = c.kkt;
        if (!isfinite(c.kkt)) { S->status = ST_NUMERIC; S->res_slot = S->res_xslot = S->cur; S->res_avg = 0; }
        else if (c.rel <= S->tol) { S->status = ST_OK; S->res_slot = S->res_xslot = S->cur; S->res_avg = 0; }
        return;
    }
    if (S->k == 0) {
        // No accepted step since the last restart: only the pass budget is checked.
        if (S->passes >= S->max_passes) {
            report(S, c);
            S->status = ST_MAX_ITER;
            S->res_slot = S->res_xslot = S->cur;
            S->res_avg = 0;
        }
        return;
    }
    KP b;
    kkt_parts(S, A[1], A[9], A[8], A[3], b);
    if (!isfinite(c.kkt) || !isfinite(b.kkt)) {
        report(S, c);
        S->status = ST_NUMERIC;
        S->res_slot = S->res_xslot = S->cur;
        S->res_avg = 0;
        return;
    }
    // Restart candidate (Sec. 5): current iff its KKT is strictly smaller.
    const bool use_avg = S->adaptive_restart ? !(c.kkt < b.kkt) : true;
    const KP& kk = use_avg ? b : c;
    const int cand = use_avg ? S->bar : S->cur;
    report(S, kk);
    if (kk.rel <= S->tol || S->passes >= S->max_passes) {
        S->status = kk.rel <= S->tol ? ST_OK : ST_MAX_ITER;
        S->res_slot = cand;
        S->res_xslot = cand;
        S->res_avg = use_avg ? 1 : 0;
        if (use_avg) {
            // The reported plan X + D is formed into the free next slot, so
            // the current plan, D and the anchor stay as they are (a solve
            // stopped by its pass budget can be resumed from them).
            S->fix = 1;
            S->fix_x = S->cur;
            S->fix_d = S->bar;
            S->fix_dst = S->nxt;
            S->res_xslot = S->nxt;
        }
        return;
    }
    bool restart;
    if (S->adaptive_restart) {
        restart = (kk.kkt <= S->beta_suff * S->kkt0) ||
                  (kk.kkt <= S->beta_nec * S->kkt0 && kk.kkt > S->kkt_prev) ||
                  ((double)S->k >= S->beta_art * (double)S->total);
    } else {
        restart = b.kkt <= S->beta * S->kkt0;   // Eq. (6)
    }
    if (!restart) {
        S->kkt_prev = kk.kkt;
        return;
    }
    if (S->pw_update) {
        // PrimalWeightUpdate of Sec. 5 against the previous restart point.
        const double dX = sqrt(use_avg ? A[11] : A[10]);
        const double dy = sqrt(use_avg ? A[5] : A[4]);
        if (dX > S->eps_zero && dy > S->eps_zero)
            S->omega = exp(S->theta * log(dy / dX) + (1.0 - S->theta) * log(S->omega));
    }
    if (use_avg) {
        // Restart to the average: its slot becomes X + D in place before the
        // next pass (the vector set of that slot already holds the averaged
        // duals and the exact sums of X + D).
        S->fix = 1;
        S->fix_x = S->cur;
        S->fix_d = cand;
        S->fix_dst = cand;
    }
    S->cur = cand;
    S->anc = cand;
    // The average restarts empty: its slot content is not read while k == 0.
    {
        int used = 1 << cand;
        int picks[3] = {0, 0, 0};
        int np = 0;
        for (int s = 0; s < NSLOT && np < 3; ++s)
            if (!(used & (1 << s))) picks[np++] = s;
        S->bar = picks[0];
        S->nxt = picks[1];
        S->barn = picks[2];
    }
    S->k = 0;
    S->wavg = 1.0;
    S->kkt0 = kk.kkt;
    S->kkt_prev = kk.kkt;
    S->restarts += 1;
    S->tau = S->eta / S->omega;
    S->sigma = S->eta * S->omega;
}

// Fixed-order sums of entry `idx` over two partial sets at once (A: the
// average's, or the plan's at the initial check; B: the current plan's):
// group g (warp g) adds partials g, g + VG, ... of each set, then warp 0
// combines the VG group sums in order.  One block barrier; the results are
// valid in warp 0.
__device__ __forceinline__ void group_sum2(const double* pa, const double* pb, long long stride, int count,
                                           long long idx, bool active, bool use_a, bool use_b, double* sgrp,
                                           double& sa, double& sb) {
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    double a = 0.0, b = 0.0;
    if (active) {
#pragma unroll 4
        for (int k = grp; k < count; k += VG) {
            if (use_a) a += pa[(long long)k * stride + idx];
            if (use_b) b += pb[(long long)k * stride + idx];
        }
    }
    sgrp[grp * 32 + lane] = a;
    sgrp[(VG + grp) * 32 + lane] = b;
    __syncthreads();
    sa = 0.0;
    sb = 0.0;
    if (grp == 0) {
#pragma unroll
        for (int g2 = 0; g2 < VG; ++g2) {
            sa += sgrp[g2 * 32 + lane];
            sb += sgrp[(VG + g2) * 32 + lane];
        }
    }
}

// One vector tile of the check: the exact row / column sums (both partial
// sets in one phase), then warp 0 alone forms the residual, dual-objective and
// distance terms, adds the tile partials of the plan pass, reduces the twelve
// scalars with shuffles and takes the instance's ticket; the last tile runs
// the restart / termination logic.  FP64 stays on one warp (a narrow pipe on
// this part) and only one block barrier is on the path.  sgrp: 2 VG x 32
// doubles.
__device__ void checkvec_tile(const Inst& I, Ctrl* S, int lvt, int mode, double* sgrp) {
    const long long m = I.m, n = I.n;
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const long long e = (long long)lvt * VE + lane;
    const bool init = mode == MODE_INIT;
    const bool avg = !init && S->k > 0;
    const bool row = e < m, col = !row && e < m + n;
    const long long idx = row ? e : e - m;          // i or j
    double s = 0.0, s2 = 0.0;
    // A: the plan's sums at the initial check, the average's at a check;
    // B: the current plan's exact sums (the passes carry them forward by sums
    // of changes between checks).
    group_sum2(row ? I.rowpart : I.colpart, row ? I.rowpart2 : I.colpart2, row ? m : I.ldx,
               row ? I.nstrips : I.nchunks, idx, row || col, init || avg, !init, sgrp, s, s2);
    if (grp == 0) {
        double* Vc = slot_v(I, S->cur);
        double* Vb = slot_v(I, S->bar);
        const double* Va = slot_v(I, S->anc);
        double a[VP];
#pragma unroll
        for (int k = 0; k < VP; ++k) a[k] = 0.0;
        if (row || col) {
            const long long yo = row ? idx : m + idx;                   // offset of p_i / q_j in a vector set
            const long long so = row ? m + n + idx : 2 * m + n + idx;   // offset of r_i / c_j
            const double b = row ? I.f[idx] : I.g[idx];
            const double y = Vc[yo];
            if (init) {
                Vc[so] = s;
                a[0] = (s - b) * (s - b);
                a[2] = b * y;
                // marginal statistics: sum f, sum g, ||[f;g]||^2, invalid entries
                if (row) a[1] = b; else a[3] = b;
                a[4] = b * b;
                a[5] = (b >= 0.0 && isfinite(b)) ? 0.0 : 1.0;
            } else {
                Vc[so] = s2;
                a[0] = (s2 - b) * (s2 - b);
                a[2] = b * y;
                const double ya = Va[yo];
                a[4] = (y - ya) * (y - ya);
                if (avg) {
                    Vb[so] = s;
                    const double yb = Vb[yo];
                    a[1] = (s - b) * (s - b);
                    a[3] = b * yb;
                    a[5] = (yb - ya) * (yb - ya);
                }
            }
        }
        const long long T = I.ntiles;
        const long long t0 = T * lvt / I.nvt, t1 = T * (lvt + 1) / I.nvt;
        for (long long t = t0 + lane; t < t1; t += 32) {
#pragma unroll
            for (int k = 0; k < TP; ++k) a[6 + k] += I.tpart[t * TP + k];
        }
#pragma unroll
        for (int k = 0; k < VP; ++k) a[k] = warp_sum(a[k]);
        unsigned old = 0;
        if (lane == 0) {
            double* vp = I.vpart + (long long)lvt * VP;
#pragma unroll
            for (int k = 0; k < VP; ++k) vp[k] = a[k];
            old = ticket_arrive(I.ticket);
        }
        old = __shfl_sync(0xffffffffu, old, 0);
        __syncwarp();
        if (old == (unsigned)(I.nvt - 1)) {
            double b[VP];
#pragma unroll
            for (int k = 0; k < VP; ++k) b[k] = 0.0;
            for (int v = lane; v < I.nvt; v += 32) {
                const double* vp = I.vpart + (long long)v * VP;
#pragma unroll
                for (int k = 0; k < VP; ++k) b[k] += __ldcg(vp + k);
            }
#pragma unroll
            for (int k = 0; k < VP; ++k) b[k] = warp_sum(b[k]);
            if (lane == 0) {
                *I.ticket = 0u;
                finalize_check(S, b, mode);
            }
        }
    }
    __syncthreads();   // sgrp is reused by the caller's next tile
}

__global__ void __launch_bounds__(VT) k_checkvec(const Inst* __restrict__ insts, const TileRef* __restrict__ vmap,
                                                 const int* __restrict__ NVp, unsigned* wctr, int mode) {
    // One CTA per vector tile (no work queue): the grid covers the tile count.
    __shared__ double sgrp[2 * VG * 32];
    pdl_enter();
    // No work counter of its own, but it still resets the others for the
    // kernels that follow (block 0, before any early exit).
    reset_other_counters(wctr, wc_index(WC_CHECK, 0));
    const int NV = *NVp;
    if ((int)blockIdx.x >= NV) return;
    const TileRef tr = vmap[blockIdx.x];
    const Inst& I = insts[tr.inst];
    Ctrl* S = I.ctrl;
    if (S->status != ST_RUNNING) return;
    checkvec_tile(I, S, tr.local, mode, sgrp);
}

// ---------------------------------------------------------------------------
// Cooperative chunk kernel (single instance, FP32 plans): one launch runs K
// passes and the check.  Each pass: the plan pass over all tiles, a grid
// barrier, the dual update (the instance's last vector tile runs the step
// controller), a grid barrier.  Then the KKT pass, a barrier, the check.
// All CTAs are co-resident (cooperative launch).  The barrier is the fence +
// atomic-arrive + fenced-spin pattern, so plain loads after it see every
// other CTA's writes before it; its spin is bounded and sets an error flag.
// ---------------------------------------------------------------------------
constexpr long long BARRIER_SPIN_LIMIT = 1LL << 24;

__device__ bool grid_barrier(GridBar* gb, unsigned nblocks, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* vgen = &gb->gen;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&gb->count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&gb->count, 0u);
            __threadfence();
            atomicAdd(&gb->gen, 1u);
        } else {
            long long it = 0;
            while (*vgen == gen) {
                if (++it > BARRIER_SPIN_LIMIT) {
                    atomicExch(&gb->err, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        if (*(volatile unsigned*)&gb->err) ok = 0;
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

template <typename TC, bool CP>
__global__ void __launch_bounds__(TWARPS * 32, 2)
k_chunk_coop(const Inst* __restrict__ insts, const TileRef* __restrict__ tmap, const int* __restrict__ Tp,
             const TileRef* __restrict__ vmap, const int* __restrict__ NVp, unsigned* wctr, GridBar* gb, int npass,
             int wc_a, int wc_b, int wc_kkt) {
    __shared__ double sgrp[2 * VG * 32];
    __shared__ int s_ok;
    extern __shared__ __align__(128) unsigned char dsm[];
    const int T = *Tp, NV = *NVp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned G = gridDim.x;
    bulk::RowPipe<BULK_ROW_S> P;
    bulk::row_pipe_init<BULK_ROW_S>(P, dsm, lane, warp);
    Ctrl* S0 = insts[0].ctrl;
    bool ok = true;
    for (int s = 0; s < npass && ok; ++s) {
        // Every CTA reads the status after the same barrier: a uniform exit.
        if (*(volatile int*)&S0->status != ST_RUNNING) break;
        const int qc = (s & 1) ? wc_b : wc_a;
        pass_row_run<TC, BULK_ROW_S, CP>(insts, tmap, T, &wctr[qc], P, lane, 0);
        ok = grid_barrier(gb, G, &s_ok);
        if (!ok) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&wctr[qc], 0u);   // ready for pass s + 2
        for (int vt = blockIdx.x; vt < NV; vt += G) {
            const TileRef tr = vmap[vt];
            const Inst& I = insts[tr.inst];
            dual_tile(I, I.ctrl, tr.local, sgrp);
        }
        ok = grid_barrier(gb, G, &s_ok);
    }
    if (ok && *(volatile int*)&S0->status == ST_RUNNING) {
        bool first = true;
        for (;;) {
            const int t = tile_next(&wctr[wc_kkt], first);
            if (t >= T) break;
            const TileRef tr = tmap[t];
            const Inst& I = insts[tr.inst];
            const Ctrl& S = *I.ctrl;
            if (S.status != ST_RUNNING) continue;
            kkt_tile<TC, float>(I, S, tr.local, lane, MODE_CHECK);
        }
        ok = grid_barrier(gb, G, &s_ok);
        if (ok) {
            for (int vt = blockIdx.x; vt < NV; vt += G) {
                const TileRef tr = vmap[vt];
                const Inst& I = insts[tr.inst];
                Ctrl* S = I.ctrl;
                if (S->status != ST_RUNNING) continue;
                checkvec_tile(I, S, tr.local, MODE_CHECK, sgrp);
            }
        }
    }
    if (!ok && blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&S0->status, ST_DEVICE);
}

// ---------------------------------------------------------------------------
// Snapshot of every resident instance's controller (one D2H copy per chunk)
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Average plan forming (after every check): where the check picked the
// running average (a restart to it, or the reported point), write
// X[fix_dst] = X[fix_x] + X[fix_d] -- the current plan plus the stored
// deviation, with the rounding the checks used for the same value.  One warp
// per plan tile; instances without a request cost one controller read.
// ---------------------------------------------------------------------------
template <typename TX>
__global__ void __launch_bounds__(TWARPS * 32)
k_avgfix(const Inst* __restrict__ insts, const TileRef* __restrict__ tmap, const int* __restrict__ Tp) {
    pdl_enter();
    const int T = *Tp;
    const int lane = threadIdx.x & 31;
    const int nw = (int)gridDim.x * TWARPS;
    for (int t = (int)blockIdx.x * TWARPS + (int)(threadIdx.x >> 5); t < T; t += nw) {
        const TileRef tr = tmap[t];
        const Inst& I = insts[tr.inst];
        const Ctrl& S = *I.ctrl;
        if (!S.fix) continue;
        const int strip = tr.local % I.nstrips, chunk = tr.local / I.nstrips;
        const long long j0 = (long long)strip * STRIP + lane * 4;
        if (j0 >= I.n) continue;
        const long long i0 = (long long)chunk * I.tile_rows;
        const long long i1 = min(i0 + (long long)I.tile_rows, I.m);
        const TX* Xa = slot_x<TX>(I, S.fix_x);
        const TX* Xd = slot_x<TX>(I, S.fix_d);
        TX* Xo = slot_x<TX>(I, S.fix_dst);
        for (long long i = i0; i < i1; ++i) {
            TX a[4], d[4];
            ld4(Xa + i * I.ldx + j0, a);
            ld4(Xd + i * I.ldx + j0, d);
#pragma unroll
            for (int e = 0; e < 4; ++e) a[e] = a[e] + d[e];
            st4(Xo + i * I.ldx + j0, a);
        }
    }
}

// out = a + d over `count` elements (a multiple of 4): a plan formed from
// the current plan and the average's deviation, for the host's copies.
template <typename TX>
__global__ void k_combine(const TX* __restrict__ a, const TX* __restrict__ d, TX* out, long long count) {
    const long long stride = (long long)gridDim.x * blockDim.x * 4;
    for (long long e = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4; e < count; e += stride) {
        TX x[4], y[4];
        ld4(a + e, x);
        ld4(d + e, y);
#pragma unroll
        for (int k = 0; k < 4; ++k) x[k] = x[k] + y[k];
        st4(out + e, x);
    }
}

__global__ void k_snapshot(const Inst* __restrict__ insts, const int* __restrict__ count, Ctrl* out) {
    pdl_enter();
    const int n = *count;
    const int words = (int)(sizeof(Ctrl) / sizeof(int));
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * words; t += gridDim.x * blockDim.x) {
        const int i = t / words, w = t % words;
        reinterpret_cast<int*>(out + i)[w] = reinterpret_cast<const int*>(insts[i].ctrl)[w];
    }
}

// ---------------------------------------------------------------------------
// Watchdog self-test: one warp waits, with the pipelines' bounded wait, for a
// 16-byte transfer that is announced on an mbarrier but never issued.  The
// wait gives up after `limit` polls and the kernel reports the status a pass
// would set (ST_DEVICE).  Nothing traps and nothing waits without bound; no
// copy is in flight when the CTA exits.
// ---------------------------------------------------------------------------
__global__ void k_watchdog_selftest(long long limit, int* status) {
    __shared__ __align__(8) unsigned long long bar_mem;
    const unsigned bar = bulk::smem_u32(&bar_mem);
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        bulk::mbar_init(bar, 1);
        bulk::fence_mbar_init();
    }
    __syncwarp();
    if (lane == 0) bulk::mbar_expect_tx(bar, 16u);   // the arrival happens; the bytes never come
    __syncwarp();
    const bool done = bulk::wait_stage(bar, 0u, limit);
    if (lane == 0) *status = done ? ST_OK : ST_DEVICE;
}

}  // namespace pdot

#include "pdot_resident.cuh"

namespace pdot {

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int err(cudaError_t e) { return e == cudaSuccess ? 0 : (int)e; }

// Launch with the programmatic-stream-serialization attribute when enabled.
template <typename... KArgs, typename... Args>
static int launch_k(bool pdl, void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                    Args... args) {
    cudaLaunchConfig_t c = {};
    c.gridDim = dim3(grid);
    c.blockDim = dim3(block);
    c.dynamicSmemBytes = smem;
    c.stream = st;
    cudaLaunchAttribute attr[1];
    if (pdl) {
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        c.attrs = attr;
        c.numAttrs = 1;
    }
    return err(cudaLaunchKernelEx(&c, kern, args...));
}

constexpr int BULK_S = BULK_ROW_S;
constexpr int bulk_smem() { return TWARPS * bulk::warp_smem_bytes<BULK_S>(); }
constexpr int GROUP_S = 2;   // stages of 4 rows: 8 rows in flight per warp
constexpr int group_smem() { return TWARPS * bulk::warp_smem_bytes_g<4, GROUP_S>(); }

template <bool CP>
static int launch_pass_t(int ttype, const Inst* d_insts, const TileRef* d_tmap, const int* T, unsigned* wctr,
                         const LaunchCfg& cfg, void* stream, int wc_override, int dir_xor) {
    const cudaStream_t st = (cudaStream_t)stream;
    const int wc = wc_override >= 0 ? wc_override : wc_index(WC_PASS, ttype);
    const bool pdl = cfg.pdl != 0;
    const unsigned tb = (unsigned)cfg.tile_blocks, th = TWARPS * 32;
    if (ttype == TT_GEN) {
        // Generated cost: the bulk pipelines copy X and Xbar only (the grouped
        // one for up to 4 coordinates), or the register pipeline when the
        // bulk kernels are switched off.
        if (cfg.pass_bulk == 2 && cfg.gen_dims <= 4)
            return launch_k(pdl, k_pass_group<GenC4, GROUP_S, CP>, (unsigned)cfg.group_blocks, th, group_smem(), st,
                            d_insts, d_tmap, T, wctr, wc, dir_xor);
        if (cfg.pass_bulk && cfg.gen_dims <= 4)
            return launch_k(pdl, k_pass_bulk<GenC4, BULK_S, CP>, (unsigned)cfg.bulk_blocks, th, bulk_smem(), st, d_insts,
                            d_tmap, T, wctr, wc, dir_xor);
        if (cfg.pass_bulk)
            return launch_k(pdl, k_pass_bulk<GenC8, BULK_S, CP>, (unsigned)cfg.bulk_blocks, th, bulk_smem(), st, d_insts,
                            d_tmap, T, wctr, wc, dir_xor);
        return launch_k(pdl, k_pass<GenC8, float, 2, CP>, tb, th, 0, st, d_insts, d_tmap, T, wctr, wc, dir_xor);
    }
    if (cfg.pass_bulk == 2 && ttype != TT_F64) {
        if (ttype == TT_BF16)
            return launch_k(pdl, k_pass_group<unsigned short, GROUP_S, CP>, (unsigned)cfg.group_blocks, th, group_smem(), st,
                            d_insts, d_tmap, T, wctr, wc, dir_xor);
        return launch_k(pdl, k_pass_group<float, GROUP_S, CP>, (unsigned)cfg.group_blocks, th, group_smem(), st, d_insts,
                        d_tmap, T, wctr, wc, dir_xor);
    }
    if (cfg.pass_bulk && ttype != TT_F64) {
        if (ttype == TT_BF16)
            return launch_k(pdl, k_pass_bulk<unsigned short, BULK_S, CP>, (unsigned)cfg.bulk_blocks, th, bulk_smem(), st,
                            d_insts, d_tmap, T, wctr, wc, dir_xor);
        return launch_k(pdl, k_pass_bulk<float, BULK_S, CP>, (unsigned)cfg.bulk_blocks, th, bulk_smem(), st, d_insts,
                        d_tmap, T, wctr, wc, dir_xor);
    }
    if (ttype == TT_F64)
        return launch_k(pdl, k_pass<double, double, 2, CP>, (unsigned)cfg.tile_blocks_f64, th, 0, st, d_insts, d_tmap, T,
                        wctr, wc, dir_xor);
    if (ttype == TT_BF16) {
        if (cfg.pass_u == 4)
            return launch_k(pdl, k_pass<unsigned short, float, 4, CP>, tb, th, 0, st, d_insts, d_tmap, T, wctr, wc, dir_xor);
        return launch_k(pdl, k_pass<unsigned short, float, 2, CP>, tb, th, 0, st, d_insts, d_tmap, T, wctr, wc, dir_xor);
    }
    if (cfg.pass_u == 4) return launch_k(pdl, k_pass<float, float, 4, CP>, tb, th, 0, st, d_insts, d_tmap, T, wctr, wc, dir_xor);
    return launch_k(pdl, k_pass<float, float, 2, CP>, tb, th, 0, st, d_insts, d_tmap, T, wctr, wc, dir_xor);
}
int launch_pass(int ttype, const Inst* d_insts, const TileRef* d_tmap, const int* T, unsigned* wctr,
                const LaunchCfg& cfg, void* stream, int wc_override, int dir_xor) {
    if (cfg.comp) return launch_pass_t<true>(ttype, d_insts, d_tmap, T, wctr, cfg, stream, wc_override, dir_xor);
    return launch_pass_t<false>(ttype, d_insts, d_tmap, T, wctr, cfg, stream, wc_override, dir_xor);
}

int launch_dual(const Inst* d_insts, const TileRef* d_vmap, const int* NV, int nv_hint, unsigned* wctr,
                const LaunchCfg& cfg, void* stream, bool direct) {
    // nv_hint: an upper bound of the vector-tile count (one CTA each); with
    // direct, exactly the count of the single instance's vector tiles.
    int blocks = nv_hint;
    if (blocks < 1) blocks = 1;
    return launch_k(cfg.pdl != 0, k_dual, (unsigned)blocks, VT, 0, (cudaStream_t)stream, d_insts, d_vmap, NV, wctr,
                    direct ? 1 : 0);
}
int launch_kkt(int ttype, const Inst* d_insts, const TileRef* d_tmap, const int* T, unsigned* wctr, int mode,
               const LaunchCfg& cfg, void* stream) {
    const cudaStream_t st = (cudaStream_t)stream;
    const int wc = wc_index(WC_KKT, ttype);
    const bool pdl = cfg.pdl != 0;
    const unsigned th = TWARPS * 32;
    if (ttype == TT_F64)
        return launch_k(pdl, k_kkt<double, double>, (unsigned)cfg.tile_blocks_f64, th, 0, st, d_insts, d_tmap, T, wctr,
                        wc, mode);
    if (ttype == TT_GEN)
        return launch_k(pdl, k_kkt<GenC8, float>, (unsigned)cfg.tile_blocks, th, 0, st, d_insts, d_tmap, T, wctr, wc,
                        mode);
    if (cfg.kkt_blocks > 0) {   // bulk-copy pipeline for stored FP32 / BF16 costs
        if (ttype == TT_BF16)
            return launch_k(pdl, k_kkt_bulk<unsigned short>, (unsigned)cfg.kkt_blocks, th, kkt_smem(), st, d_insts,
                            d_tmap, T, wctr, wc, mode);
        return launch_k(pdl, k_kkt_bulk<float>, (unsigned)cfg.kkt_blocks, th, kkt_smem(), st, d_insts, d_tmap, T, wctr,
                        wc, mode);
    }
    if (ttype == TT_BF16)
        return launch_k(pdl, k_kkt<unsigned short, float>, (unsigned)cfg.tile_blocks, th, 0, st, d_insts, d_tmap, T,
                        wctr, wc, mode);
    return launch_k(pdl, k_kkt<float, float>, (unsigned)cfg.tile_blocks, th, 0, st, d_insts, d_tmap, T, wctr, wc,
                    mode);
}
int launch_checkvec(const Inst* d_insts, const TileRef* d_vmap, const int* NV, int nv_hint, unsigned* wctr, int mode,
                    const LaunchCfg& cfg, void* stream) {
    int blocks = nv_hint;
    if (blocks < 1) blocks = 1;
    return launch_k(cfg.pdl != 0, k_checkvec, (unsigned)blocks, VT, 0, (cudaStream_t)stream, d_insts, d_vmap, NV,
                    wctr, mode);
}
int launch_avgfix(int ttype, const Inst* d_insts, const TileRef* d_tmap, const int* T, const LaunchCfg& cfg,
                  void* stream) {
    const cudaStream_t st = (cudaStream_t)stream;
    if (ttype == TT_F64)
        return launch_k(cfg.pdl != 0, k_avgfix<double>, (unsigned)cfg.tile_blocks_f64, TWARPS * 32, 0, st, d_insts,
                        d_tmap, T);
    return launch_k(cfg.pdl != 0, k_avgfix<float>, (unsigned)cfg.tile_blocks, TWARPS * 32, 0, st, d_insts, d_tmap, T);
}
int launch_combine(int xtype, const void* a, const void* d, void* out, long long count, void* stream) {
    if (count <= 0) return 0;
    long long blocks = (count / 4 + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (xtype == 2)
        k_combine<double><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
            static_cast<const double*>(a), static_cast<const double*>(d), static_cast<double*>(out), count);
    else
        k_combine<float><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
            static_cast<const float*>(a), static_cast<const float*>(d), static_cast<float*>(out), count);
    return err(cudaGetLastError());
}
int launch_watchdog_selftest(long long limit, int* d_status, void* stream) {
    k_watchdog_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(limit, d_status);
    return err(cudaGetLastError());
}

int launch_snapshot(const Inst* d_insts, const int* count, int max_count, Ctrl* out, void* stream) {
    const int words = (int)(sizeof(Ctrl) / sizeof(int));
    int blocks = (max_count * words + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 1024) blocks = 1024;
    k_snapshot<<<blocks, 256, 0, (cudaStream_t)stream>>>(d_insts, count, out);
    return err(cudaGetLastError());
}

static int occ(const void* fn, int threads) {
    int a = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, fn, threads, 0);
    return a > 0 ? a : 1;
}
int occupancy_tile_blocks_per_sm(int ttype) {
    if (ttype == TT_F64) {
        const int a = occ((const void*)k_pass<double, double, 2, true>, TWARPS * 32);
        const int b = occ((const void*)k_kkt<double, double>, TWARPS * 32);
        return a < b ? a : b;
    }
    const void* fns[] = {(const void*)k_pass<float, float, 2, true>,          (const void*)k_pass<float, float, 2, false>,
                         (const void*)k_pass<unsigned short, float, 4, true>,  (const void*)k_pass<unsigned short, float, 4, false>,
                         (const void*)k_pass<GenC8, float, 2, true>,           (const void*)k_pass<GenC8, float, 2, false>,
                         (const void*)k_kkt<float, float>,                     (const void*)k_kkt<unsigned short, float>,
                         (const void*)k_kkt<GenC8, float>};
    int r = 1 << 20;
    for (const void* f : fns) {
        const int a = occ(f, TWARPS * 32);
        if (a < r) r = a;
    }
    return r;
}

// Opt every instantiation of a kernel with dynamic shared memory into `bytes`;
// returns minus the fewest CTAs per SM any of them holds, or a positive
// cudaError_t code.
static int setup_dyn(const void* const* fns, int nf, int bytes) {
    int r = 1 << 20;
    for (int i = 0; i < nf; ++i) {
        const cudaError_t e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return (int)e;
        int a = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, fns[i], TWARPS * 32, bytes);
        if (a < r) r = a;
    }
    return -(r > 0 ? r : 1);
}

int setup_coop_chunk() {
    const void* fns[] = {(const void*)k_chunk_coop<float, true>, (const void*)k_chunk_coop<float, false>,
                         (const void*)k_chunk_coop<unsigned short, true>,
                         (const void*)k_chunk_coop<unsigned short, false>};
    return setup_dyn(fns, 4, bulk_smem());
}

int launch_chunk_coop(int ttype, const Inst* d_insts, const TileRef* d_tmap, const int* T, const TileRef* d_vmap,
                      const int* NV, unsigned* wctr, GridBar* gb, int npass, const LaunchCfg& cfg, void* stream) {
    cudaLaunchConfig_t c = {};
    c.gridDim = dim3((unsigned)cfg.coop_blocks);
    c.blockDim = dim3(TWARPS * 32);
    c.dynamicSmemBytes = bulk_smem();
    c.stream = (cudaStream_t)stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    c.attrs = attr;
    c.numAttrs = 1;
    const int wa = wc_index(WC_PASS, ttype), wb = wc_index(WC_AUX, ttype), wk = wc_index(WC_KKT, ttype);
    cudaError_t e;
    if (ttype == TT_BF16)
        e = cfg.comp ? cudaLaunchKernelEx(&c, k_chunk_coop<unsigned short, true>, d_insts, d_tmap, T, d_vmap, NV, wctr,
                                          gb, npass, wa, wb, wk)
                     : cudaLaunchKernelEx(&c, k_chunk_coop<unsigned short, false>, d_insts, d_tmap, T, d_vmap, NV, wctr,
                                          gb, npass, wa, wb, wk);
    else
        e = cfg.comp ? cudaLaunchKernelEx(&c, k_chunk_coop<float, true>, d_insts, d_tmap, T, d_vmap, NV, wctr, gb, npass,
                                          wa, wb, wk)
                     : cudaLaunchKernelEx(&c, k_chunk_coop<float, false>, d_insts, d_tmap, T, d_vmap, NV, wctr, gb,
                                          npass, wa, wb, wk);
    return err(e);
}

int setup_group_pass() {
    const void* fns[] = {(const void*)k_pass_group<float, GROUP_S, true>, (const void*)k_pass_group<float, GROUP_S, false>,
                         (const void*)k_pass_group<unsigned short, GROUP_S, true>,
                         (const void*)k_pass_group<unsigned short, GROUP_S, false>,
                         (const void*)k_pass_group<GenC4, GROUP_S, true>, (const void*)k_pass_group<GenC4, GROUP_S, false>};
    return setup_dyn(fns, 6, group_smem());
}

// Resident kernel: its shared-memory size, and how many of its clusters the
// device holds at once (-count; 0: cannot run, a positive value: an error).
int setup_resident() {
    const void* fns[] = {(const void*)k_resident<float, false>, (const void*)k_resident<float, true>,
                         (const void*)k_resident<unsigned short, false>, (const void*)k_resident<unsigned short, true>};
    int r = 1 << 20;
    for (const void* fn : fns) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, res::RSMEM);
        if (e != cudaSuccess) return (int)e;
        cudaLaunchConfig_t c = {};
        c.gridDim = dim3(res::RCS);
        c.blockDim = dim3(res::RT);
        c.dynamicSmemBytes = res::RSMEM;
        int nc = 0;
        e = cudaOccupancyMaxActiveClusters(&nc, fn, &c);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        if (nc < r) r = nc;
    }
    return -r;
}
bool resident_fits(long long m, long long n) { return res::fits(m, n); }
int launch_resident(int ttype, const Inst* d_insts, const int* list, const int* count, int max_count, int passes,
                    int K, int replay, const LaunchCfg& cfg, void* stream) {
    if (max_count < 1) return 0;
    const cudaStream_t st = (cudaStream_t)stream;
    const dim3 grid((unsigned)(res::RCS * max_count)), block(res::RT);
    if (ttype == TT_BF16) {
        if (cfg.comp)
            k_resident<unsigned short, true><<<grid, block, res::RSMEM, st>>>(d_insts, list, count, passes, K, replay);
        else
            k_resident<unsigned short, false><<<grid, block, res::RSMEM, st>>>(d_insts, list, count, passes, K, replay);
    } else if (ttype == TT_F32) {
        if (cfg.comp)
            k_resident<float, true><<<grid, block, res::RSMEM, st>>>(d_insts, list, count, passes, K, replay);
        else
            k_resident<float, false><<<grid, block, res::RSMEM, st>>>(d_insts, list, count, passes, K, replay);
    } else {
        return (int)cudaErrorInvalidValue;   // FP32 plans with stored FP32 / BF16 costs only
    }
    return err(cudaGetLastError());
}

int setup_kkt_bulk() {
    const void* fns[] = {(const void*)k_kkt_bulk<float>, (const void*)k_kkt_bulk<unsigned short>};
    return setup_dyn(fns, 2, kkt_smem());
}

int setup_bulk_pass() {
    const void* fns[] = {(const void*)k_pass_bulk<float, BULK_S, true>, (const void*)k_pass_bulk<float, BULK_S, false>,
                         (const void*)k_pass_bulk<unsigned short, BULK_S, true>,
                         (const void*)k_pass_bulk<unsigned short, BULK_S, false>,
                         (const void*)k_pass_bulk<GenC4, BULK_S, true>, (const void*)k_pass_bulk<GenC4, BULK_S, false>,
                         (const void*)k_pass_bulk<GenC8, BULK_S, true>, (const void*)k_pass_bulk<GenC8, BULK_S, false>};
    return setup_dyn(fns, 8, bulk_smem());   // negative: blocks per SM
}

int occupancy_vec_blocks_per_sm() {
    const int a = occ((const void*)k_dual, VT);
    const int b = occ((const void*)k_checkvec, VT);
    return a < b ? a : b;
}

}  // namespace pdot
