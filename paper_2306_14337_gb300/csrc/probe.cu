// probe.cu -- arithmetic-throughput probe for roofline denominators.
//
// The refactorization and the triangular solves are sparse, indexed work; the
// benchmark states how far they are from the device's FMA rate in the factor
// precision.  No vendor figure for the FP64 and FP32 non-tensor FMA rates of
// this GPU is on record here, so this measures them: every thread runs eight
// independent chains of fused multiply-adds (enough independent work to keep
// the pipes full), timed with CUDA events over the whole launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "kkt.h"
#include "kernels.cuh"

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T *out, int iters, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = T(threadIdx.x + k) * T(1e-3);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) x[k] = fma(x[k], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kChains; k++) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

template <typename T> kkt_status run_probe(int blocks, int iters, double *tflops) {
    T *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    kkt_status st = KKT_OK;
    float best = 0.0f;
    if (cudaMalloc(&out, (size_t)blocks * 256 * sizeof(T)) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        kkt::set_last_error("kkt_probe_fma_tflops: allocation failed");
        st = KKT_ERR_CUDA;
    }
    // |a| < 1 keeps the chains finite; the values do not matter for the rate
    for (int rep = 0; st == KKT_OK && rep < 6; rep++) {
        cudaEventRecord(e0);
        k_fma_probe<T><<<blocks, 256>>>(out, iters, T(0.999999), T(1e-7));
        cudaEventRecord(e1);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            kkt::set_last_error(std::string("kkt_probe_fma_tflops: ") + cudaGetErrorString(e));
            st = KKT_ERR_CUDA;
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.0f || ms < best)) best = ms;    // first launch: warm-up
    }
    if (st == KKT_OK) {
        const double flops = 2.0 * kChains * (double)iters * blocks * 256.0;
        *tflops = flops / (best * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    return st;
}

}  // namespace

kkt_status kkt_probe_fma_tflops(int device, int fp64, double *tflops) {
    if (!tflops || device < 0) return KKT_ERR_ARG;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        kkt::set_last_error("kkt_probe_fma_tflops: cannot select the device");
        return KKT_ERR_CUDA;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int blocks = std::max(1, sms) * 8;          // 2,048 threads per SM
    const kkt_status st = fp64 ? run_probe<double>(blocks, 4096, tflops)
                               : run_probe<float>(blocks, 65536, tflops);
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return st;
}
