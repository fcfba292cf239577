// noalloc.cu -- scaled residual of a CSR system without any device allocation.
//
// Who needs this: code that must not call cudaMalloc at the point where it
// wants the residual.  Typical cases are deployments that hand their whole
// device-memory budget to their own pool allocator when they start (a hidden
// cudaMalloc would fail or break the budget), and loops that cannot afford the
// device-wide synchronization a cudaMalloc/cudaFree pair can cause.  Such
// callers may also be unable to create a kkt_ctx, because kkt_analyze allocates
// the context's workspace.  This entry point needs neither: the caller passes
// the matrix, the vectors and the outputs, and the only scratch is a fixed
// array compiled into the library.
//
// Scratch: one file-scope __device__ array, kNoallocMaxBlocks x 4 doubles
// (4 MiB), holding one partial result per thread block of the residual pass.
// It belongs to the library's device code, so a GPU commits it when that code
// is loaded on it (with CUDA's lazy module loading: at the latest during the
// first call on that device, whose set-up looks the array's address up) and
// holds it until the process exits.  All calls on a device share it and it
// keeps the last call's contents; each call writes every partial it later
// reads, so nothing has to start at zero.  Calls whose execution overlaps on
// the GPU (different streams without ordering) race on the array and must be
// avoided.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "kkt.h"
#include "kernels.cuh"

namespace {

constexpr int kRowsPerBlock = 32;                 // 256 threads, 8 lanes per row
constexpr int kThreads = 256;
constexpr int kNoallocMaxBlocks = 131072;         // 4,194,304 rows at most
constexpr int kMaxDevices = 64;
constexpr unsigned FULL = 0xffffffffu;

// [block][0..3] = max |rho_i|, max |x_i|, max |b_i|, max_i sum_j |a_ij| over the block's rows
static __device__ __align__(256) double g_partials[kNoallocMaxBlocks * 4];

// Host-side copies of the array's device address, one per device, filled the
// first time the entry point runs on that device.
std::mutex g_mu;
double *g_addr[kMaxDevices] = {};

// NaN counts as +infinity in the maxima below: fmax(NaN, y) = y would drop a
// NaN entry from a norm and report a small omega for a broken solution.
__device__ __forceinline__ double abs_nan_inf(double v) { return isnan(v) ? INFINITY : fabs(v); }

// Residual pass: rho = b - A x with 8 lanes per row (the same per-row
// arithmetic as the library's refinement residual), and per-block maxima.
__global__ void __launch_bounds__(kThreads)
k_resid_partials(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                 const double *__restrict__ a, const double *__restrict__ b,
                 const double *__restrict__ x, double *__restrict__ rho,
                 double *__restrict__ partials) {
    __shared__ double red[kThreads / 32][4];
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int sub = threadIdx.x & 7;
    double acc = 0.0, asum = 0.0;
    if (r < n) {
        for (int p = rp[r] + sub; p < rp[r + 1]; p += 8) {
            const double av = a[p];
            acc += av * x[ci[p]];
            asum += fabs(av);
        }
    }
    for (int o = 4; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(FULL, acc, o);
        asum += __shfl_xor_sync(FULL, asum, o);
    }
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (r < n && sub == 0) {
        const double br = b[r];
        const double rv = br - acc;
        rho[r] = rv;
        v[0] = abs_nan_inf(rv);
        v[1] = abs_nan_inf(x[r]);
        v[2] = abs_nan_inf(br);
        v[3] = isnan(asum) ? INFINITY : asum;
    }
    for (int k = 0; k < 4; k++)
        for (int o = 16; o > 0; o >>= 1) v[k] = fmax(v[k], __shfl_xor_sync(FULL, v[k], o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int k = 0; k < 4; k++) red[w][k] = v[k];
    __syncthreads();
    if (threadIdx.x < 4) {
        double m = 0.0;
        for (int q = 0; q < kThreads / 32; q++) m = fmax(m, red[q][threadIdx.x]);
        partials[(size_t)blockIdx.x * 4 + threadIdx.x] = m;
    }
}

// One block folds the partials: out = {omega, ||rho||_inf, ||x||_inf, ||b||_inf, ||A||_inf}.
__global__ void __launch_bounds__(kThreads)
k_resid_finish(int nblocks, const double *__restrict__ partials, double *__restrict__ out) {
    __shared__ double red[kThreads / 32][4];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x)
        for (int k = 0; k < 4; k++) v[k] = fmax(v[k], partials[(size_t)i * 4 + k]);
    for (int k = 0; k < 4; k++)
        for (int o = 16; o > 0; o >>= 1) v[k] = fmax(v[k], __shfl_xor_sync(FULL, v[k], o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int k = 0; k < 4; k++) red[w][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        double m[4] = {0.0, 0.0, 0.0, 0.0};
        for (int q = 0; q < kThreads / 32; q++)
            for (int k = 0; k < 4; k++) m[k] = fmax(m[k], red[q][k]);
        const double den = m[3] * m[1] + m[2];
        const double w = den > 0.0 ? m[0] / den : (m[0] > 0.0 ? INFINITY : 0.0);
        out[0] = isnan(w) ? INFINITY : w;     // inf / inf: a non-finite entry somewhere
        out[1] = m[0];
        out[2] = m[1];
        out[3] = m[2];
        out[4] = m[3];
    }
}

// Device address of g_partials on the current device, looked up once per
// device with that device current.
kkt_status scratch_address(int dev, double **out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess) {
            kkt::set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return KKT_ERR_CUDA;
        }
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return KKT_OK;
}

}  // namespace

kkt_status kkt_scaled_residual_noalloc(int n, const int *row_ptr_dev, const int *col_idx_dev,
                                       const double *values_dev, const double *b_dev,
                                       const double *x_dev, double *rho_dev, double *out_dev,
                                       kkt_stream stream) {
    if (n <= 0 || !row_ptr_dev || !col_idx_dev || !values_dev || !b_dev || !x_dev || !rho_dev ||
        !out_dev)
        return KKT_ERR_ARG;
    const long long nblocks = ((long long)n + kRowsPerBlock - 1) / kRowsPerBlock;
    if (nblocks > kNoallocMaxBlocks) {
        kkt::set_last_error("kkt_scaled_residual_noalloc: n exceeds 4,194,304 rows");
        return KKT_ERR_ARG;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        kkt::set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return KKT_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        kkt::set_last_error("kkt_scaled_residual_noalloc: device ordinal above 63");
        return KKT_ERR_CUDA;
    }
    double *partials = nullptr;
    kkt_status st = scratch_address(dev, &partials);
    if (st != KKT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    k_resid_partials<<<(int)nblocks, kThreads, 0, s>>>(n, row_ptr_dev, col_idx_dev, values_dev, b_dev,
                                                        x_dev, rho_dev, partials);
    if ((e = cudaGetLastError()) != cudaSuccess) {
        kkt::set_last_error(std::string("k_resid_partials launch: ") + cudaGetErrorString(e));
        return KKT_ERR_CUDA;
    }
    k_resid_finish<<<1, kThreads, 0, s>>>((int)nblocks, partials, out_dev);
    if ((e = cudaGetLastError()) != cudaSuccess) {
        kkt::set_last_error(std::string("k_resid_finish launch: ") + cudaGetErrorString(e));
        return KKT_ERR_CUDA;
    }
    return KKT_OK;
}
