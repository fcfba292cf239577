// dense.cu -- the dense root block of the refactorization.
//
// The top of the elimination tree of the ACOPF KKT matrices is a chain of
// separator rows whose trailing block of the combined L+U pattern is nearly
// full (70,000-bus KKT: the last 768 rows completely, the last 1,000 to 87%).
// Eliminated row by row, these rows are the end of the refactorization's
// critical path: each waits for the row above it and then applies a pivot row
// of up to a thousand entries.  Sec. 4 of arXiv 2306.14337 discusses the
// supernodal alternative (dense blocks for groups of columns) and why it fails
// on the small blocks of power-grid matrices; this block is not small.
//
// The analysis makes the trailing block of dense_rows rows a full square
// block (explicit zeros).  The row kernel reduces each of its rows only by the
// pivots below the block -- the Schur complement S = A'_TT - L_TB U_BT -- and
// leaves it in a dense row-major array.  This kernel then factors S = L_TT U_TT
// by a right-looking blocked LU without row exchanges (the fixed pivot
// sequence, with the row kernel's FP64 perturbation test), panels of 32:
//   1. every CTA that has panel work factors the 32 x 32 diagonal block
//      itself (one warp, in registers; the arithmetic is identical in every
//      CTA, so all get the same factors; CTA 0 writes them out and counts
//      perturbed and negative pivots), then its warps solve 32-row groups of
//      the L panel (X U_kk = A_ik, one row per lane) and 32-column groups of
//      the U panel (L_kk Y = A_kj, one column per lane);
//   2. grid barrier; the trailing block takes the rank-32 update in 64 x 64
//      tiles (panel pieces staged in shared memory);
//   3. grid barrier; next panel.
// Every entry is reduced by its terms one at a time, in increasing pivot
// order, a(i,j) <- a(i,j) - l(i,d) u(d,j), and a multiplier is the reduced
// entry times the reciprocal pivot -- the row kernel's arithmetic; only the
// grouping of the work differs.  Finally the block is copied into the
// combined storage (its rows' tails) and the transposed copy.  The block
// (at most 2,048^2 words) stays in L2, so every access bypasses L1 (.cg):
// other SMs wrote it since the last barrier.
//
// The CTAs wait on each other at the barriers, so the kernel is launched
// cooperatively (all CTAs resident at once; the launch fails otherwise).
// Each barrier wait is bounded by spin_limit polls; on expiry it raises
// KKT_ERR_TIMEOUT in the status word and the CTA goes on (results invalid).
#include <cuda_runtime.h>

#include <climits>

#include "kkt.h"
#include "kernels.cuh"

namespace kkt {
namespace {

constexpr unsigned DFULL = 0xffffffffu;
constexpr int DNB = 32;                  // panel width
constexpr int DTILE = 64;                // trailing-update tile edge
constexpr int DWARPS = 8;
constexpr int DTHREADS = DWARPS * 32;

__device__ __forceinline__ unsigned dn_ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Barrier over the grid.  The arrival counter only grows during a launch
// (the host zeroes it before each launch): barrier k of a CTA waits until
// k * gridDim.x arrivals, so a CTA whose wait ran out stays in step.
__device__ __forceinline__ void dn_grid_barrier(const RunCfg &rc, unsigned &k) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned target = (++k) * gridDim.x;
        atomicAdd(rc.dense_bar, 1u);
        long long it = 0;
        unsigned ns = 32;
        while (dn_ld_acquire(rc.dense_bar) < target) {
            __nanosleep(ns);
            if (ns < 256) ns <<= 1;
            if (++it > rc.spin_limit) {
                atomicExch(rc.status + ST_TIMEOUT, 1);
                atomicExch(rc.status + ST_ABORT, 1);
                break;
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// Diagonal block [k0, k0 + kb)^2 of S, one warp, lane r = block row r.
// Leaves L (strictly below) and U (on and above the diagonal) in sb and the
// reciprocal pivots in srcp; the writer CTA also stores them to D, rcp and
// the status words.
template <typename T>
__device__ __forceinline__ void dn_factor_diag(const DevPattern &P, const RunCfg &rc,
                                               const double *__restrict__ aval, const double *__restrict__ sp,
                                               T *D, int ld, int lo, int k0, int kb, double tau, T *rcp,
                                               T (*sb)[DNB + 1], T *srcp, bool writer, int lane) {
    T a[DNB];
    const int R = k0 + lane;
    const bool mine = lane < kb;
#pragma unroll
    for (int c = 0; c < DNB; c++) a[c] = (mine && c < kb) ? __ldcg(D + (size_t)R * ld + k0 + c) : T(0);
    double aii = 0.0;                               // A'_ii: sign of a perturbed pivot
    if (mine) {
        const int i = lo + R;
        const int k = P.src[P.diag[i]];
        if (k >= 0) aii = sp[i] * sp[i] * aval[k];
    }
#pragma unroll
    for (int p = 0; p < DNB; p++) {
        if (p < kb) {
            T r = T(0);
            if (lane == p) {                        // pivot test in FP64
                double pv = (double)a[p];
                if (!(fabs(pv) >= tau) || isinf(pv)) {
                    if (writer) {
                        if (!isfinite(pv)) atomicExch(rc.status + ST_NONFINITE, 1);
                        atomicAdd(rc.status + ST_PERTURBED, 1);
                        atomicAdd(rc.status + ST_PERT_LAST, 1);
                    }
                    pv = (aii < 0.0) ? -tau : tau;
                }
                if (writer && pv < 0.0) atomicAdd(rc.status + ST_NEGATIVE, 1);
                a[p] = (T)pv;
                r = T(1) / a[p];
                srcp[p] = r;
                if (writer) rcp[lo + R] = r;
            }
            r = __shfl_sync(DFULL, r, p);
            const T l = a[p] * r;                   // rows below p: the multiplier
#pragma unroll
            for (int c = 0; c < DNB; c++) {
                if (c > p) {
                    const T u = __shfl_sync(DFULL, a[c], p);
                    if (lane > p) a[c] = a[c] - l * u;
                }
            }
            if (lane > p) a[p] = l;
        }
    }
#pragma unroll
    for (int c = 0; c < DNB; c++) sb[lane][c] = a[c];
    if (writer && mine) {
#pragma unroll
        for (int c = 0; c < DNB; c++)
            if (c < kb) __stcg(D + (size_t)R * ld + k0 + c, a[c]);
    }
}

// L panel: rows R = r0 + 32 g + lane, X U_kk = S(R, k0:k0+kb).
template <typename T>
__device__ __forceinline__ void dn_panel_l(T *D, int ld, int s, int k0, int kb, int R,
                                           const T (*sb)[DNB + 1], const T *srcp) {
    T x[DNB];
    const bool ok = R < s;
#pragma unroll
    for (int c = 0; c < DNB; c++) x[c] = (ok && c < kb) ? __ldcg(D + (size_t)R * ld + k0 + c) : T(0);
#pragma unroll
    for (int c = 0; c < DNB; c++) {
        if (c < kb) {
            x[c] = x[c] * srcp[c];
#pragma unroll
            for (int c2 = 0; c2 < DNB; c2++)
                if (c2 > c) x[c2] = x[c2] - x[c] * sb[c][c2];
        }
    }
    if (ok) {
#pragma unroll
        for (int c = 0; c < DNB; c++)
            if (c < kb) __stcg(D + (size_t)R * ld + k0 + c, x[c]);
    }
}

// U panel: columns C = r0 + 32 g + lane, L_kk Y = S(k0:k0+kb, C).
template <typename T>
__device__ __forceinline__ void dn_panel_u(T *D, int ld, int s, int k0, int kb, int C,
                                           const T (*sb)[DNB + 1]) {
    T y[DNB];
    const bool ok = C < s;
#pragma unroll
    for (int r = 0; r < DNB; r++) y[r] = (ok && r < kb) ? __ldcg(D + (size_t)(k0 + r) * ld + C) : T(0);
#pragma unroll
    for (int r = 0; r < DNB; r++) {
        if (r < kb) {
#pragma unroll
            for (int r2 = 0; r2 < DNB; r2++)
                if (r2 > r) y[r2] = y[r2] - sb[r2][r] * y[r];
        }
    }
    if (ok) {
#pragma unroll
        for (int r = 0; r < DNB; r++)
            if (r < kb) __stcg(D + (size_t)(k0 + r) * ld + C, y[r]);
    }
}

// Rank-kb update of one 64 x 64 tile of the trailing block at (R0, C0).
template <typename T>
__device__ __forceinline__ void dn_update_tile(T *D, int ld, int s, int k0, int kb, int R0, int C0,
                                               T (*sl)[DNB + 1], T (*su)[DTILE + 1]) {
    const int tid = threadIdx.x;
    for (int e = tid; e < DTILE * DNB; e += DTHREADS) {
        const int r = e / DNB, k = e % DNB;
        const int R = R0 + r;
        sl[r][k] = (R < s && k < kb) ? __ldcg(D + (size_t)R * ld + k0 + k) : T(0);
    }
    for (int e = tid; e < DNB * DTILE; e += DTHREADS) {
        const int k = e / DTILE, c = e % DTILE;
        const int C = C0 + c;
        su[k][c] = (k < kb && C < s) ? __ldcg(D + (size_t)(k0 + k) * ld + C) : T(0);
    }
    __syncthreads();
    const int ty = tid >> 4, tx = tid & 15;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int R = R0 + ty + 16 * i, C = C0 + tx + 16 * j;
            acc[i][j] = (R < s && C < s) ? __ldcg(D + (size_t)R * ld + C) : T(0);
        }
    for (int k = 0; k < kb; k++) {
        T lv[4], uv[4];
#pragma unroll
        for (int i = 0; i < 4; i++) lv[i] = sl[ty + 16 * i][k];
#pragma unroll
        for (int j = 0; j < 4; j++) uv[j] = su[k][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) acc[i][j] = acc[i][j] - lv[i] * uv[j];
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int R = R0 + ty + 16 * i, C = C0 + tx + 16 * j;
            if (R < s && C < s) __stcg(D + (size_t)R * ld + C, acc[i][j]);
        }
    __syncthreads();                                // the tiles are reused by the next one
}

template <typename T>
__global__ void __launch_bounds__(DTHREADS, 1)
k_dense_lu(DevPattern P, RunCfg rc, const double *__restrict__ aval, const double *__restrict__ sp,
           T *LU, T *LUT, T *rcp, double tau_rel) {
    __shared__ T sb[DNB][DNB + 1];
    __shared__ T srcp[DNB];
    __shared__ T sl[DTILE][DNB + 1];
    __shared__ T su[DNB][DTILE + 1];
    const int lo = rc.dense_lo, s = P.n - lo, ld = rc.dense_ld;
    T *D = reinterpret_cast<T *>(rc.dense);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const double tau = tau_rel * __longlong_as_double((long long)rc.norms[NM_AMAX]);
    const long long ss = (long long)s * s;
    const long long gthreads = (long long)gridDim.x * DTHREADS;
    unsigned bk = 0;
    if (rc.symmetric) {            // LDL^T rows reduced only their upper part: mirror it
        for (long long e = (long long)blockIdx.x * DTHREADS + threadIdx.x; e < ss; e += gthreads) {
            const int r = (int)(e / s), c = (int)(e % s);
            if (r > c) __stcg(D + (size_t)r * ld + c, __ldcg(D + (size_t)c * ld + r));
        }
        dn_grid_barrier(rc, bk);
    }
    for (int k0 = 0; k0 < s; k0 += DNB) {
        const int kb = min(DNB, s - k0);
        const int r0 = k0 + kb, rest = s - r0;
        const int ngrp = (rest + 31) >> 5;
        const int items = 2 * ngrp;                 // L groups, then U groups
        if (blockIdx.x == 0 || (int)blockIdx.x * DWARPS < items) {
            if (wid == 0)
                dn_factor_diag<T>(P, rc, aval, sp, D, ld, lo, k0, kb, tau, rcp, sb, srcp, blockIdx.x == 0, lane);
            __syncthreads();
            const int item = (int)blockIdx.x * DWARPS + wid;
            if (item < ngrp)
                dn_panel_l<T>(D, ld, s, k0, kb, r0 + 32 * item + lane, sb, srcp);
            else if (item < items)
                dn_panel_u<T>(D, ld, s, k0, kb, r0 + 32 * (item - ngrp) + lane, sb);
        }
        dn_grid_barrier(rc, bk);
        if (rest > 0) {
            const int nt = (rest + DTILE - 1) / DTILE;
            for (int t = blockIdx.x; t < nt * nt; t += gridDim.x)
                dn_update_tile<T>(D, ld, s, k0, kb, r0 + (t / nt) * DTILE, r0 + (t % nt) * DTILE, sl, su);
            dn_grid_barrier(rc, bk);
        }
    }
    // the block's rows are the tails of rows lo .. n-1 of the combined storage;
    // entry (r, c) of the block is entry (c, r) of the transposed copy
    for (long long e = (long long)blockIdx.x * DTHREADS + threadIdx.x; e < ss; e += gthreads) {
        const int r = (int)(e / s), c = (int)(e % s);
        const T v = __ldcg(D + (size_t)r * ld + c);
        LU[(long long)P.lu_rp[lo + r + 1] - s + c] = v;
        LUT[(long long)P.lu_rp[lo + c + 1] - s + r] = v;
    }
}

}  // namespace

int dense_lu_threads() { return DTHREADS; }

template <typename T>
cudaError_t launch_dense_lu(const DevPattern &P, const RunCfg &rc, const double *aval, const double *sp,
                            T *LU, T *LUT, T *rcp, double tau_rel, int grid, cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(rc.dense_bar, 0, sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(DTHREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_dense_lu<T>, P, rc, aval, sp, LU, LUT, rcp, tau_rel);
}

template cudaError_t launch_dense_lu<float>(const DevPattern &, const RunCfg &, const double *, const double *,
                                            float *, float *, float *, double, int, cudaStream_t);
template cudaError_t launch_dense_lu<double>(const DevPattern &, const RunCfg &, const double *, const double *,
                                             double *, double *, double *, double, int, cudaStream_t);

// CTAs of k_dense_lu<T> that fit on one SM at once (for the cooperative grid).
cudaError_t dense_lu_per_sm(int fp32, int *per_sm) {
    if (fp32)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_dense_lu<float>, DTHREADS, 0);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_dense_lu<double>, DTHREADS, 0);
}

}  // namespace kkt
