// pdot_noalloc.cu -- an allocation-free variant of the plan rounding
// (pdot_round_noalloc in include/pdot.h).
//
// Why it exists: some callers cannot call cudaMalloc at the point where they
// need a feasible plan -- a process whose device memory is owned by another
// allocator (a framework's caching allocator that has reserved the GPU), a
// serving loop that forbids allocation after warm-up because cudaMalloc and
// cudaFree synchronise the device and cause latency spikes, or a plug-in that
// runs inside a host application which owns every device allocation.  This
// entry point needs no handle and allocates nothing: its scratch is the
// file-scope device array below, reserved when the library is loaded and held
// by every GPU that loads it until the process exits.
//
// The caller still provides the plan, the marginals and the output.  The
// arithmetic is the same rounding as pdot_round (row scaling, column scaling,
// rank-one correction), with every scalar step done on the device.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/pdot.h"

namespace {

constexpr long long NA_MAX_DIM = 32768;   // largest m and n accepted
constexpr int NA_PARTS = 8;               // row groups of the column sums
// Layout in doubles: xs[m] | ys[n] | rsum[m] | csum[n] | er[m] | ec[n] | colpart[NA_PARTS][n] | misc[8]
constexpr long long NA_WORDS = 6 * NA_MAX_DIM + NA_PARTS * NA_MAX_DIM + 8;   // 3.67 MB

static __device__ __align__(256) double g_noalloc_scratch[NA_WORDS];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[NA_MAX_DEVICES] = {nullptr};
// One call at a time per device: a call holds its device's lock until its
// stream has synchronised, so no two calls use the shared scratch at once.
std::mutex g_call_mutex[NA_MAX_DEVICES];

template <typename TX>
__device__ __forceinline__ double na_scaled(const TX* X, long long n, long long i, long long j, const double* xs,
                                            const double* ys) {
    double v = (double)X[i * n + j];
    if (xs) v *= xs[i];
    if (ys) v *= ys[j];
    return v;
}

// Row sums of diag(xs) X diag(ys): one warp per row, fixed-order butterfly.
template <typename TX>
__global__ void k_na_rows(const TX* X, long long m, long long n, const double* xs, const double* ys, double* rsum) {
    const long long row = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= m) return;
    double s = 0.0;
    for (long long j = lane; j < n; j += 32) s += na_scaled(X, n, row, j, xs, ys);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) rsum[row] = s;
}

// Column partial sums over NA_PARTS row groups.
template <typename TX>
__global__ void k_na_cols(const TX* X, long long m, long long n, const double* xs, const double* ys,
                          double* colpart) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int grp = blockIdx.y;
    if (j >= n) return;
    const long long r0 = m * grp / NA_PARTS, r1 = m * (grp + 1) / NA_PARTS;
    double s = 0.0;
    for (long long i = r0; i < r1; ++i) s += na_scaled(X, n, i, j, xs, ys);
    colpart[(long long)grp * n + j] = s;
}

__global__ void k_na_colsum(const double* colpart, long long n, double* csum) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s = 0.0;
    for (int g = 0; g < NA_PARTS; ++g) s += colpart[(long long)g * n + j];
    csum[j] = s;
}

// scale_i = min(marg_i / sum_i, 1); a zero sum keeps scale 1.
__global__ void k_na_scale(const double* sum, const double* marg, long long len, double* scale) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    const double s = sum[i];
    scale[i] = s > 0.0 ? fmin(marg[i] / s, 1.0) : 1.0;
}

// err_r = f - rsum, err_c = g - csum, misc[0] = 1 / ||err_r||_1 (0 when the norm is 0).
// One block: fixed-order strided sums, then a tree in shared memory.
__global__ void k_na_err(const double* f, const double* rsum, long long m, const double* g, const double* csum,
                         long long n, double* er, double* ec, double* misc) {
    __shared__ double red[1024];
    double l1 = 0.0;
    for (long long i = threadIdx.x; i < m; i += blockDim.x) {
        const double e = f[i] - rsum[i];
        er[i] = e;
        l1 += fabs(e);
    }
    for (long long j = threadIdx.x; j < n; j += blockDim.x) ec[j] = g[j] - csum[j];
    red[threadIdx.x] = l1;
    __syncthreads();
    for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) misc[0] = red[0] > 0.0 ? 1.0 / red[0] : 0.0;
}

template <typename TX>
__global__ void k_na_write(const TX* X, long long m, long long n, const double* xs, const double* ys,
                           const double* er, const double* ec, const double* misc, TX* out) {
    const double inv_l1 = misc[0];
    const long long total = m * n;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long i = t / n, j = t % n;
        out[t] = (TX)(na_scaled(X, n, i, j, xs, ys) + er[i] * ec[j] * inv_l1);
    }
}

// Set-up, once per device with that device current: the host-side name of the
// array is not a device address, so ask the runtime for it.
cudaError_t scratch_for_device(int device, double** out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

template <typename TX>
cudaError_t run_round(cudaStream_t st, long long m, long long n, const TX* X, const double* f, const double* g,
                      TX* out, double* base) {
    double* xs = base;
    double* ys = xs + m;
    double* rsum = ys + n;
    double* csum = rsum + m;
    double* er = csum + n;
    double* ec = er + m;
    double* colpart = ec + n;
    double* misc = colpart + (long long)NA_PARTS * n;
    const unsigned rb = (unsigned)((m + 7) / 8);
    const unsigned vb_m = (unsigned)((m + 255) / 256), vb_n = (unsigned)((n + 255) / 256);
    const dim3 cb(vb_n, NA_PARTS);
    // 1) x_i = min(f_i / (X1)_i, 1)
    k_na_rows<TX><<<rb, 256, 0, st>>>(X, m, n, nullptr, nullptr, rsum);
    k_na_scale<<<vb_m, 256, 0, st>>>(rsum, f, m, xs);
    // 2) y_j = min(g_j / (diag(x) X)^T 1)_j, 1)
    k_na_cols<TX><<<cb, 256, 0, st>>>(X, m, n, xs, nullptr, colpart);
    k_na_colsum<<<vb_n, 256, 0, st>>>(colpart, n, csum);
    k_na_scale<<<vb_n, 256, 0, st>>>(csum, g, n, ys);
    // 3) marginal errors of X_tmp = diag(x) X diag(y)
    k_na_rows<TX><<<rb, 256, 0, st>>>(X, m, n, xs, ys, rsum);
    k_na_cols<TX><<<cb, 256, 0, st>>>(X, m, n, xs, ys, colpart);
    k_na_colsum<<<vb_n, 256, 0, st>>>(colpart, n, csum);
    k_na_err<<<1, 1024, 0, st>>>(f, rsum, m, g, csum, n, er, ec, misc);
    // 4) X_feas = X_tmp + err_r err_c^T / ||err_r||_1
    long long blocks = (m * n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_na_write<TX><<<(unsigned)blocks, 256, 0, st>>>(X, m, n, xs, ys, er, ec, misc, out);
    return cudaGetLastError();
}

}  // namespace

extern "C" pdot_status pdot_round_noalloc(int device, void* cuda_stream, int64_t m, int64_t n, pdot_dtype x_dtype,
                                          const void* X, const double* f, const double* g, void* X_out) {
    if (m < 1 || n < 1 || m > NA_MAX_DIM || n > NA_MAX_DIM) return PDOT_ERR_ARG;
    if (!X || !f || !g || !X_out) return PDOT_ERR_ARG;
    if (x_dtype != PDOT_F32 && x_dtype != PDOT_F64) return PDOT_ERR_ARG;
    if (device < 0 || device >= NA_MAX_DEVICES) return PDOT_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device >= ndev) return PDOT_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return PDOT_ERR_CUDA;
    double* base = nullptr;
    if (scratch_for_device(device, &base) != cudaSuccess) return PDOT_ERR_CUDA;
    const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    std::lock_guard<std::mutex> lock(g_call_mutex[device]);
    cudaError_t e;
    if (x_dtype == PDOT_F64)
        e = run_round<double>(st, m, n, static_cast<const double*>(X), f, g, static_cast<double*>(X_out), base);
    else
        e = run_round<float>(st, m, n, static_cast<const float*>(X), f, g, static_cast<float*>(X_out), base);
    // Synchronise on every path, so the scratch is idle when the lock is released.
    const cudaError_t es = cudaStreamSynchronize(st);
    if (e != cudaSuccess || es != cudaSuccess) return PDOT_ERR_CUDA;
    return PDOT_OK;
}
