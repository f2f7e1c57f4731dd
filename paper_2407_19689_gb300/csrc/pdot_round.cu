// pdot_round.cu -- Algorithm 3 of arXiv 2407.19689 (rounding onto the
// transportation polytope, after Altschuler et al.) on the device.
// Runs once per solve, so the kernels are plain and order-deterministic:
// row sums by one warp per row, column sums by fixed row groups, and a final
// write of diag(x) X diag(y) + err_r err_c^T / ||err_r||_1 with <C, X_feas>.
#include <cuda_runtime.h>

#include "pdot_internal.h"

namespace pdot {

namespace {

template <typename TX>
__device__ __forceinline__ double scaled(const TX* X, long long ldx, long long i, long long j, const double* rs,
                                         const double* cs) {
    double v = (double)X[i * ldx + j];
    if (rs) v *= rs[i];
    if (cs) v *= cs[j];
    return v;
}

// rowout[i] = sum_j rs_i X_ij cs_j   (one warp per row)
template <typename TX>
__global__ void k_round_rows(const TX* X, long long m, long long n, long long ldx, const double* rs,
                             const double* cs, double* rowout) {
    const long long row = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= m) return;
    double s = 0.0;
    for (long long j = lane; j < n; j += 32) s += scaled(X, ldx, row, j, rs, cs);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) rowout[row] = s;
}

// colpart[g][j] = sum over rows i of group g of rs_i X_ij cs_j
template <typename TX>
__global__ void k_round_cols(const TX* X, long long m, long long n, long long ldx, const double* rs,
                             const double* cs, double* colpart, int parts) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int grp = blockIdx.y;
    if (j >= n) return;
    const long long r0 = m * grp / parts, r1 = m * (grp + 1) / parts;
    double s = 0.0;
    for (long long i = r0; i < r1; ++i) s += scaled(X, ldx, i, j, rs, cs);
    colpart[(long long)grp * n + j] = s;
}

__global__ void k_colreduce(const double* colpart, int parts, long long n, double* out) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s = 0.0;
    for (int g = 0; g < parts; ++g) s += colpart[(long long)g * n + j];
    out[j] = s;
}

// Cost entry (i, j) for the objective of the rounded plan: a stored matrix
// (null: no objective) or the generated cost.
template <typename TC>
struct StoredCost {
    const TC* C;
    long long ldc;
    __device__ __forceinline__ bool on() const { return C != nullptr; }
    __device__ __forceinline__ double operator()(long long i, long long j) const { return (double)C[i * ldc + j]; }
};
struct PointsCost {
    GenSpec g;
    __device__ __forceinline__ bool on() const { return true; }
    __device__ __forceinline__ double operator()(long long i, long long j) const {
        return (double)gen_cost(g.kind, g.d, g.xs + i * g.d, g.ys + j * g.d, g.div, g.inv);
    }
};

template <typename TX, typename CA>
__global__ void k_round_write(const TX* X, long long m, long long n, long long ldx, const double* rs,
                              const double* cs, const double* er, const double* ec, double inv_l1, TX* out,
                              long long ldo, CA C, double* objpart, int parts) {
    __shared__ double red[32];
    const int grp = blockIdx.x;
    const long long r0 = m * grp / parts, r1 = m * (grp + 1) / parts;
    double obj = 0.0;
    for (long long i = r0; i < r1; ++i) {
        for (long long j = threadIdx.x; j < n; j += blockDim.x) {
            const double v = scaled(X, ldx, i, j, rs, cs) + er[i] * ec[j] * inv_l1;
            const TX vo = (TX)v;
            out[i * ldo + j] = vo;
            if (C.on()) obj += C(i, j) * (double)vo;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) obj += __shfl_xor_sync(0xffffffffu, obj, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = obj;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        objpart[grp] = s;
    }
}

struct Bf16 {
    unsigned short b;
    __device__ operator double() const { return (double)__uint_as_float(((unsigned)b) << 16); }
};

// Weak-duality bound of Eq. (1) from a row dual p (no counterpart in the
// paper; it certifies a result): q_j = min_i (C_ij - p_i) is the largest
// column dual with p_i + q_j <= C_ij for all i, and f^T p + g^T q <= OPT.
// colmin[grp][j] = min over the rows of group grp (one thread per column, so
// a warp reads 32 consecutive entries of a row).  The minimum is exact, so
// the result does not depend on the grouping.
template <typename CA>
__global__ void k_cmin_cols(CA C, const double* p, long long m, long long n, double* colmin, int parts) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int grp = blockIdx.y;
    if (j >= n) return;
    const long long r0 = m * grp / parts, r1 = m * (grp + 1) / parts;
    double v = __longlong_as_double(0x7ff0000000000000LL);   // +inf: an empty group
    for (long long i = r0; i < r1; ++i) {
        const double t = C(i, j) - p[i];
        if (t < v) v = t;
    }
    colmin[(long long)grp * n + j] = v;
}

__global__ void k_cmin_reduce(const double* colmin, int parts, long long n, double* q) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double v = colmin[j];
    for (int g = 1; g < parts; ++g) {
        const double t = colmin[(long long)g * n + j];
        if (t < v) v = t;
    }
    q[j] = v;
}

// out[0] = f^T p + g^T q: one block, fixed-order strided sums, then a tree.
__global__ void k_dual_value(const double* f, const double* p, long long m, const double* g, const double* q,
                             long long n, double* out) {
    __shared__ double red[1024];
    double s = 0.0;
    for (long long i = threadIdx.x; i < m; i += blockDim.x) s += f[i] * p[i];
    for (long long j = threadIdx.x; j < n; j += blockDim.x) s += g[j] * q[j];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

template <typename CA>
void launch_cmin(CA C, const double* p, long long m, long long n, double* colmin, int parts, cudaStream_t st) {
    const dim3 cb((unsigned)((n + 255) / 256), (unsigned)parts);
    k_cmin_cols<CA><<<cb, 256, 0, st>>>(C, p, m, n, colmin, parts);
}

}  // namespace

// The bound above: q (n) and out[0] = f^T p + g^T q.  colmin: parts x n
// scratch, 1 <= parts <= m.  ctype: 0 FP32, 1 BF16, 2 FP64 (row-major with
// leading dimension ldc), 3 generated (gen).
int launch_dual_bound(const void* C, int ctype, long long ldc, const GenSpec* gen, const double* p,
                      const double* f, const double* g, long long m, long long n, double* colmin, int parts,
                      double* q, double* out, void* stream) {
    const cudaStream_t st = (cudaStream_t)stream;
    if (ctype == 3)
        launch_cmin(PointsCost{*gen}, p, m, n, colmin, parts, st);
    else if (ctype == 2)
        launch_cmin(StoredCost<double>{(const double*)C, ldc}, p, m, n, colmin, parts, st);
    else if (ctype == 1)
        launch_cmin(StoredCost<Bf16>{(const Bf16*)C, ldc}, p, m, n, colmin, parts, st);
    else
        launch_cmin(StoredCost<float>{(const float*)C, ldc}, p, m, n, colmin, parts, st);
    k_cmin_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(colmin, parts, n, q);
    k_dual_value<<<1, 1024, 0, st>>>(f, p, m, g, q, n, out);
    return (int)cudaGetLastError();
}

int launch_round_rowsum(const void* X, int xtype, long long m, long long n, long long ldx, const double* rs,
                        const double* cs, double* rowout, double* colpart, int parts, void* stream) {
    const cudaStream_t st = (cudaStream_t)stream;
    const dim3 rb((unsigned)((m + 7) / 8));
    const dim3 cb((unsigned)((n + 255) / 256), (unsigned)parts);
    if (xtype == 2) {
        k_round_rows<double><<<rb, 256, 0, st>>>((const double*)X, m, n, ldx, rs, cs, rowout);
        k_round_cols<double><<<cb, 256, 0, st>>>((const double*)X, m, n, ldx, rs, cs, colpart, parts);
    } else {
        k_round_rows<float><<<rb, 256, 0, st>>>((const float*)X, m, n, ldx, rs, cs, rowout);
        k_round_cols<float><<<cb, 256, 0, st>>>((const float*)X, m, n, ldx, rs, cs, colpart, parts);
    }
    return (int)cudaGetLastError();
}

int launch_colreduce(const double* colpart, int parts, long long n, double* out, void* stream) {
    k_colreduce<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(colpart, parts, n, out);
    return (int)cudaGetLastError();
}

int launch_round_write(const void* X, int xtype, long long m, long long n, long long ldx, const double* rs,
                       const double* cs, const double* er, const double* ec, double inv_l1, void* Xout,
                       long long ldo, const void* C, int ctype, long long ldc, const GenSpec* gen,
                       double* objpart, int parts, void* stream) {
    const cudaStream_t st = (cudaStream_t)stream;
    if (xtype == 2) {
        k_round_write<double><<<parts, 256, 0, st>>>((const double*)X, m, n, ldx, rs, cs, er, ec, inv_l1,
                                                     (double*)Xout, ldo,
                                                     StoredCost<double>{(const double*)C, ldc}, objpart, parts);
    } else if (ctype == 3) {
        k_round_write<float><<<parts, 256, 0, st>>>((const float*)X, m, n, ldx, rs, cs, er, ec, inv_l1,
                                                    (float*)Xout, ldo, PointsCost{*gen}, objpart, parts);
    } else if (ctype == 1) {
        k_round_write<float><<<parts, 256, 0, st>>>((const float*)X, m, n, ldx, rs, cs, er, ec, inv_l1,
                                                    (float*)Xout, ldo, StoredCost<Bf16>{(const Bf16*)C, ldc},
                                                    objpart, parts);
    } else {
        k_round_write<float><<<parts, 256, 0, st>>>((const float*)X, m, n, ldx, rs, cs, er, ec, inv_l1,
                                                    (float*)Xout, ldo, StoredCost<float>{(const float*)C, ldc},
                                                    objpart, parts);
    }
    return (int)cudaGetLastError();
}

}  // namespace pdot
