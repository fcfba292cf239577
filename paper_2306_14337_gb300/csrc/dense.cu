// dense.cu -- the dense root block of the refactorization.
//
// The top of the elimination tree of the ACOPF KKT matrices is a chain of
// separator rows whose trailing block of the combined L+U pattern is nearly
// full (70,000-bus KKT: the last 768 rows completely, the last 1,131 to 80%).
// Eliminated row by row, these rows end the refactorization's critical path:
// each waits for the row above it and then applies a pivot row of up to a
// thousand entries.  Sec. 4 of arXiv 2306.14337 discusses the supernodal
// alternative (dense blocks for groups of columns) and why it fails on the
// small blocks of power-grid matrices; this block is not small.
//
// The analysis makes the trailing block of dense_rows rows a full square
// block (explicit zeros).  The row kernel reduces each of its rows only by the
// pivots below the block -- the Schur complement S = A'_TT - L_TB U_BT -- and
// leaves it in a dense row-major array.  This kernel factors S = L_TT U_TT
// without row exchanges (the fixed pivot sequence, with the row kernel's
// perturbation test) as a left-looking LU by block columns of CW columns:
// CTA j keeps block column j of S in shared memory and, for every block
// column k < j as soon as CTA k has published it,
//   U(k,j) = L_kk^-1 S(k,j)                  (one thread per column)
//   S(i,j) -= L(i,k) U(k,j) for the rows below (one thread per row),
// then factors its own block: the diagonal tile (one warp, a lane per row,
// the pivot tests) and the L part below it (X U_jj = S, a thread per row),
// and publishes the block column (global memory, then a release flag).  The
// CTAs wait on lower-numbered CTAs only, so they are launched cooperatively
// (all resident at once, one per SM).  A chain of block columns is the
// critical path; everything else overlaps it.  Every entry takes its terms
// one at a time in increasing pivot order, a(i,j) <- a(i,j) - l(i,d) u(d,j),
// and a multiplier is the reduced entry times the reciprocal pivot: the row
// kernel's arithmetic, grouped differently.  Finally each CTA writes its block
// column to the combined storage (the tails of the block's rows) and the
// transposed copy.  Waits are bounded by spin_limit polls (KKT_ERR_TIMEOUT,
// results invalid).
#include <cuda_runtime.h>

#include <climits>

#include "kkt.h"
#include "kernels.cuh"

namespace kkt {
namespace {

constexpr unsigned DFULL = 0xffffffffu;
constexpr int DWARPS = 8;
constexpr int DTHREADS = DWARPS * 32;
constexpr int DFLAG = 32;                // ints per published flag (one 128-byte line each)

__device__ __forceinline__ int dn_ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int dn_ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void dn_st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long dn_gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Thread 0 waits until flag *f is set (bounded), then the CTA's barrier.
__device__ __forceinline__ void dn_wait_flag(const RunCfg &rc, const int *f) {
    if (threadIdx.x == 0 && dn_ld_relaxed(f) == 0) {
        long long it = 0;
        unsigned ns = 32;
        for (;;) {
            __nanosleep(ns);
            if (dn_ld_relaxed(f) != 0) break;
            if (ns < 256) ns <<= 1;
            if ((++it & 7) == 0 && dn_ld_relaxed(rc.status + ST_ABORT)) break;
            if (it > rc.spin_limit) {
                atomicExch(rc.status + ST_TIMEOUT, 1);
                atomicExch(rc.status + ST_ABORT, 1);
                break;
            }
        }
    }
    if (threadIdx.x == 0) (void)dn_ld_acquire(f);
    __syncthreads();
}

// The smallest float >= t (t >= 0): for a float p, |p| >= t exactly when
// |p| >= dn_float_up(t), so the FP64 pivot test of an FP32 pivot needs no
// FP64 arithmetic (FP64 instructions are slow on this GPU, and the tests of a
// diagonal tile are sequential).
__device__ __forceinline__ float dn_float_up(double t) { return __double2float_ru(t); }
// !(|p| >= tau): the pivot is too small (or NaN)
template <typename T> __device__ __forceinline__ bool dn_small(T p, double tau, float tau_up);
template <> __device__ __forceinline__ bool dn_small<float>(float p, double, float tau_up) {
    return !(fabsf(p) >= tau_up);
}
template <> __device__ __forceinline__ bool dn_small<double>(double p, double tau, float) {
    return !(fabs(p) >= tau);
}

// 16-byte vectors of T (4 floats or 2 doubles)
template <typename T> struct V16;
template <> struct V16<float> {
    using type = float4;
    static constexpr int N = 4;
    __device__ static float at(const float4 &v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }
};
template <> struct V16<double> {
    using type = double2;
    static constexpr int N = 2;
    __device__ static double at(const double2 &v, int e) { return e == 0 ? v.x : v.y; }
};

// Shared memory of k_dense_lu<T, CW>: the block column col[s][CW + 1] (odd
// pitch: threads on different rows hit different banks), two aligned tiles
// tk / tu [CW][CW + 16 / sizeof(T)] (16-byte rows for broadcast vector reads)
// and the reciprocal pivots.
template <typename T, int CW> struct DnSmem {
    static constexpr int CP = CW + 1;
    static constexpr int TP = CW + 16 / (int)sizeof(T);
    static size_t bytes(int s) {
        const size_t colb = ((size_t)s * CP * sizeof(T) + 15) / 16 * 16;
        return colb + 2 * (size_t)CW * TP * sizeof(T) + (size_t)CW * sizeof(T);
    }
};

template <typename T, int CW>
__global__ void __launch_bounds__(DTHREADS, 1)
k_dense_lu(DevPattern P, RunCfg rc, const double *__restrict__ aval, const double *__restrict__ sp, T *LU,
           T *LUT, T *rcp, double tau_rel) {
    using SM = DnSmem<T, CW>;
    constexpr int CP = SM::CP, TP = SM::TP;
    using VT = typename V16<T>::type;
    constexpr int VN = V16<T>::N;
    extern __shared__ __align__(16) unsigned char dsm[];
    const int lo = rc.dense_lo, s = P.n - lo, ld = rc.dense_ld;
    T *D = reinterpret_cast<T *>(rc.dense);
    int *flag = rc.dense_ctl;
    T(*col)[CP] = reinterpret_cast<T(*)[CP]>(dsm);  // block column j: s rows
    T(*tk)[TP] = reinterpret_cast<T(*)[TP]>(dsm + ((size_t)s * CP * sizeof(T) + 15) / 16 * 16);
    T(*tu)[TP] = tk + CW;                           // U(k,j) rows / unused
    T *srcp = reinterpret_cast<T *>(tu + CW);       // reciprocal pivots of block column j
    const int j = blockIdx.x, c0 = j * CW, nc = min(CW, s - c0);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const double tau = tau_rel * __longlong_as_double((long long)rc.norms[NM_AMAX]);
    const long long tbase = rc.trace_stride * TR_DENSE;
    for (int e = tid; e < s * CW; e += DTHREADS) {
        const int r = e / CW, c = e % CW;
        col[r][c] = c < nc ? __ldcg(D + (size_t)r * ld + c0 + c) : T(0);
    }
    __syncthreads();
    if (rc.trace != nullptr && tid == 0) rc.trace[tbase + 2LL * j] = dn_gtimer();
    // left-looking: block columns k < j, in order
    for (int k = 0; k < j; k++) {
        const int k0 = k * CW;                      // a full block column (k0 + CW <= c0)
        dn_wait_flag(rc, flag + (size_t)k * DFLAG);
        for (int e = tid; e < CW * CW; e += DTHREADS) {
            const int r = e / CW, c = e % CW;
            tk[r][c] = __ldcg(D + (size_t)(k0 + r) * ld + k0 + c);
        }
        __syncthreads();
        if (tid < CW) {                             // U(k,j) = L_kk^-1 S(k,j): a column per thread
            T y[CW];
#pragma unroll
            for (int r = 0; r < CW; r++) y[r] = col[k0 + r][tid];
#pragma unroll
            for (int r = 1; r < CW; r++)
#pragma unroll
                for (int q = 0; q < CW; q++)
                    if (q < r) y[r] = y[r] - tk[r][q] * y[q];
#pragma unroll
            for (int r = 0; r < CW; r++) {
                col[k0 + r][tid] = y[r];
                tu[r][tid] = y[r];                  // columns >= nc stay zero
            }
        }
        __syncthreads();
        // the rows below: S(R, j) -= L(R, k) U(k, j), a row per thread, the
        // row's CW entries in registers, U rows read as broadcast vectors
        for (int R = k0 + CW + tid; R < s; R += DTHREADS) {
            T l[CW], acc[CW];
            const VT *lp = reinterpret_cast<const VT *>(D + (size_t)R * ld + k0);
#pragma unroll
            for (int q = 0; q < CW / VN; q++) {
                const VT v = __ldcg(lp + q);
#pragma unroll
                for (int e = 0; e < VN; e++) l[q * VN + e] = V16<T>::at(v, e);
            }
#pragma unroll
            for (int c = 0; c < CW; c++) acc[c] = col[R][c];
#pragma unroll
            for (int q = 0; q < CW; q++) {
#pragma unroll
                for (int c4 = 0; c4 < CW / VN; c4++) {
                    const VT u = *reinterpret_cast<const VT *>(&tu[q][c4 * VN]);
#pragma unroll
                    for (int e = 0; e < VN; e++) acc[c4 * VN + e] = acc[c4 * VN + e] - l[q] * V16<T>::at(u, e);
                }
            }
#pragma unroll
            for (int c = 0; c < CW; c++) col[R][c] = acc[c];
        }
        __syncthreads();
    }
    // own diagonal tile: warp 0, lane r = row c0 + r
    if (wid == 0) {
        const T tau_t = (T)tau;                     // a perturbed pivot: +-tau rounded to T
        const float tau_up = dn_float_up(tau);
        const bool mine = lane < nc;
        T a[CW];
#pragma unroll
        for (int c = 0; c < CW; c++) a[c] = (mine && c < nc) ? col[c0 + lane][c] : T(0);
        double aii = 0.0;                           // A'_ii: sign of a perturbed pivot
        if (mine) {
            const int i = lo + c0 + lane;
            const int e = P.src[P.diag[i]];
            if (e >= 0) aii = sp[i] * sp[i] * aval[e];
        }
#pragma unroll
        for (int p = 0; p < CW; p++) {
            if (p < nc) {
                T r = T(0);
                if (lane == p) {
                    T pv = a[p];
                    if (dn_small<T>(pv, tau, tau_up) || isinf(pv)) {
                        if (!isfinite(pv)) atomicExch(rc.status + ST_NONFINITE, 1);
                        atomicAdd(rc.status + ST_PERTURBED, 1);
                        atomicAdd(rc.status + ST_PERT_LAST, 1);
                        pv = (aii < 0.0) ? -tau_t : tau_t;
                    }
                    if (pv < T(0)) atomicAdd(rc.status + ST_NEGATIVE, 1);
                    a[p] = pv;
                    r = T(1) / pv;
                    srcp[p] = r;
                    rcp[lo + c0 + p] = r;
                }
                r = __shfl_sync(DFULL, r, p);
                const T l = a[p] * r;               // rows below p: the multiplier
#pragma unroll
                for (int c = 0; c < CW; c++) {
                    if (c > p) {
                        const T u = __shfl_sync(DFULL, a[c], p);
                        if (lane > p) a[c] = a[c] - l * u;
                    }
                }
                if (lane > p) a[p] = l;
            }
        }
        if (lane < CW) {
#pragma unroll
            for (int c = 0; c < CW; c++) {
                if (mine) col[c0 + lane][c] = a[c];
                tk[lane][c] = a[c];                 // U_jj (and L_jj) in the aligned tile
            }
        }
    }
    __syncthreads();
    // L part below the diagonal tile: X U_jj = S, a row per thread
    for (int R = c0 + CW + tid; R < s; R += DTHREADS) {
        T x[CW];
#pragma unroll
        for (int c = 0; c < CW; c++) x[c] = col[R][c];
#pragma unroll
        for (int c = 0; c < CW; c++) {
            x[c] = x[c] * srcp[c];
#pragma unroll
            for (int c4 = 0; c4 < CW / VN; c4++) {
                if ((c4 + 1) * VN - 1 > c) {
                    const VT u = *reinterpret_cast<const VT *>(&tk[c][c4 * VN]);
#pragma unroll
                    for (int e = 0; e < VN; e++)
                        if (c4 * VN + e > c) x[c4 * VN + e] = x[c4 * VN + e] - x[c] * V16<T>::at(u, e);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < CW; c++) col[R][c] = x[c];
    }
    __syncthreads();
    // publish rows >= c0 of the block column (the L part and the diagonal tile)
    for (int e = tid; e < (s - c0) * CW; e += DTHREADS) {
        const int r = c0 + e / CW, c = e % CW;
        if (c < nc) __stcg(D + (size_t)r * ld + c0 + c, col[r][c]);
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        dn_st_release(flag + (size_t)j * DFLAG, 1);
        if (rc.trace != nullptr) rc.trace[tbase + 2LL * j + 1] = dn_gtimer();
    }
    // final values: the combined storage (row tails) and the transposed copy
    for (int e = tid; e < s * CW; e += DTHREADS) {
        const int r = e / CW, c = e % CW;
        if (c < nc) LU[__ldg(P.lu_rp + lo + r + 1) - s + c0 + c] = col[r][c];
    }
    for (int e = tid; e < s * CW; e += DTHREADS) {
        const int c = e / s, r = e % s;
        if (c < nc) LUT[__ldg(P.lu_rp + lo + c0 + c + 1) - s + r] = col[r][c];
    }
}

template <typename T, int CW> size_t dn_smem(int s) { return DnSmem<T, CW>::bytes(s); }

// block-column width of a block of s rows: 32 while a block column fits in
// shared memory, else 16
template <typename T> int dn_width(int s) { return dn_smem<T, 32>(s) <= 200 * 1024 ? 32 : 16; }

}  // namespace

int dense_lu_threads() { return DTHREADS; }

size_t dense_lu_ctl_bytes(int s) { return (size_t)((s + 15) / 16) * DFLAG * sizeof(int); }

int dense_lu_max_rows(int fp32) {
    // the largest block whose 16-column block columns fit in shared memory
    int m = 16;
    while (m < 4096 && (fp32 ? dn_smem<float, 16>(m + 16) : dn_smem<double, 16>(m + 16)) <= 200 * 1024) m += 16;
    return m;
}

// Set the kernel's shared-memory limit for a block of s rows and check that
// all of its CTAs (one per block column) fit on the device at once.
cudaError_t dense_lu_prepare(int fp32, int s, int sms, int *ctas) {
    const void *fn;
    size_t smem;
    int cw;
    if (fp32) {
        cw = dn_width<float>(s);
        fn = cw == 32 ? (const void *)k_dense_lu<float, 32> : (const void *)k_dense_lu<float, 16>;
        smem = cw == 32 ? dn_smem<float, 32>(s) : dn_smem<float, 16>(s);
    } else {
        cw = 16;
        fn = (const void *)k_dense_lu<double, 16>;
        smem = dn_smem<double, 16>(s);
    }
    cudaError_t e = ensure_smem(fn, smem);
    if (e != cudaSuccess) return e;
    int per = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, DTHREADS, smem);
    if (e != cudaSuccess) return e;
    *ctas = (s + cw - 1) / cw;
    if ((long long)per * sms < *ctas) return cudaErrorCooperativeLaunchTooLarge;
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_dense_lu(const DevPattern &P, const RunCfg &rc, const double *aval, const double *sp,
                            T *LU, T *LUT, T *rcp, double tau_rel, cudaStream_t stream) {
    const int s = P.n - rc.dense_lo;
    const int cw = sizeof(T) == 4 ? dn_width<T>(s) : 16;
    cudaError_t e = cudaMemsetAsync(rc.dense_ctl, 0, dense_lu_ctl_bytes(s), stream);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((s + cw - 1) / cw));
    cfg.blockDim = dim3(DTHREADS);
    cfg.dynamicSmemBytes = cw == 32 ? dn_smem<T, 32>(s) : dn_smem<T, 16>(s);   // host arithmetic only
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if constexpr (sizeof(T) == 4) {
        if (cw == 32) return cudaLaunchKernelEx(&cfg, k_dense_lu<T, 32>, P, rc, aval, sp, LU, LUT, rcp, tau_rel);
    }
    return cudaLaunchKernelEx(&cfg, k_dense_lu<T, 16>, P, rc, aval, sp, LU, LUT, rcp, tau_rel);
}

template cudaError_t launch_dense_lu<float>(const DevPattern &, const RunCfg &, const double *, const double *,
                                            float *, float *, float *, double, cudaStream_t);
template cudaError_t launch_dense_lu<double>(const DevPattern &, const RunCfg &, const double *, const double *,
                                             double *, double *, double *, double, cudaStream_t);

}  // namespace kkt
