// kkt.cu -- CUDA kernels and C entry points of the fixed-pattern KKT
// refactorization library (see include/kkt.h for the interface).
//
// arXiv 2306.14337 maps onto this file as follows:
//   Sec. 5.2 "fill the values of A into the combined storage for L and U"
//       -> k_scale / k_amax (power-of-two scaling, norms) and the value gather
//          at the start of every row of k_refactor;
//   Sec. 5.2 Algorithm 1 (row-wise, dependency-driven LU)
//       -> k_refactor: one warp per row of the combined L+U (CSR), rows
//          claimed deepest first, the published values themselves as ready
//          signals, the row staged in shared memory, updates placed through
//          precomputed update maps (or a binary search of the row's sorted
//          columns), no atomics;
//   Sec. 5.2 Algorithm 2 (dependency-driven triangular solve)
//       -> k_trisolve<T, BACKWARD, TRANS>: the forward and backward solves
//          and the transposed pair, over longest-path tasks of the
//          elimination tree (long ones on a CTA each), permutation and
//          scaling fused at entry and exit;
//   Sec. 5.1 iterative refinement rho = r - K dx, K delta = rho, dx += delta
//       -> k_resid (FP64 CSR residual fused with the infinity norms) and the
//          refinement loop in kkt_refine (the update is fused into the
//          backward solve); FGMRES with CGS2 through k_spmv, k_mdot, k_vcomb;
//   same-pattern batches and uneven queues
//       -> k_brefactor / k_btrisolve (batch innermost) and k_qrefactor /
//          k_qtrisolve (several patterns in one launch, recorded in a graph).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <numeric>
#include <climits>
#include <string>
#include <vector>
#include <set>
#include <map>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "kkt.h"
#include "analysis.h"
#include "kernels.cuh"

namespace kkt {

constexpr unsigned FULL = 0xffffffffu;
constexpr int WARPS = 8;  // warps per CTA of the persistent kernels

// ---------------------------------------------------------------------------
// synchronisation helpers

__device__ __forceinline__ int ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Optional tracing of work items: claim and completion times (ns).
__device__ __forceinline__ void trace_mark(const RunCfg &rc, long long base, int item, int which, int lane) {
    if (rc.trace != nullptr && lane == 0) rc.trace[base + 2LL * item + which] = gtimer();
}

__device__ __forceinline__ int claim_row(const RunCfg &rc, int lane) {
    int s = 0;
    if (lane == 0) s = atomicAdd(&rc.sched->next, 1);
    return __shfl_sync(FULL, s, 0);
}

// Called by lane 0 of every warp after its failing claim.  The last warp
// resets the queue and publishes the epoch for the next launch.
__device__ __forceinline__ void finish_launch(const RunCfg &rc, int e) {
    const int total = gridDim.x * (blockDim.x >> 5);
    int d = atomicAdd(&rc.sched->done, 1);
    if (d == total - 1) {
        rc.sched->next = 0;
        rc.sched->next_long = 0;
        rc.sched->next_rest = 0;
        rc.sched->done = 0;
        __threadfence();
        rc.sched->epoch = e;
    }
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *p, double v) {
    atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ int floor_half(int e) { return e >= 0 ? e / 2 : -((1 - e) / 2); }

// |v| for a max-reduction that must not lose NaN: fmax(NaN, y) = y would drop
// a NaN entry from an infinity norm, so NaN counts as +infinity.
__device__ __forceinline__ double abs_nan_inf(double v) { return isnan(v) ? INFINITY : fabs(v); }

// ---------------------------------------------------------------------------
// scaling and norms (8 lanes per row)

// s_i = 2^-floor(floor(log2 r_i) / 2), r_i = max_j |a_ij| (1 for a zero or
// non-finite row); sp[new] = s[old]; ||A||_inf; non-finite input flagged.
// Norms over the rows reduce inside the CTA first (warp shuffles, then shared
// memory) and enter the device word with one atomic per CTA: the rows of a
// 490,000-row matrix must not serialize on one address.  The kernels walk the
// rows grid-stride, a warp taking 4 rows at a time (8 lanes per row).
constexpr int RTHREADS = 256;

// max over the CTA of non-negative v (thread 0's return value is valid)
__device__ __forceinline__ double cta_max(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();                                   // red may still be read by a previous call
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 1; k < (int)(blockDim.x >> 5); k++) v = fmax(v, red[k]);
    return v;
}

__global__ void __launch_bounds__(RTHREADS)
k_scale(DevPattern P, const double *__restrict__ aval, double *__restrict__ s_orig,
        double *__restrict__ sp, unsigned long long *norms, int *status, int equil) {
    __shared__ double red[RTHREADS / 32];
    const int sub = threadIdx.x & 7;
    const long long step = (long long)gridDim.x * (blockDim.x >> 3);
    double nmax = 0.0;                                 // ||A||_inf over the finite rows seen
    for (long long r0 = ((long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) >> 3; r0 < P.n; r0 += step) {
        const int r = (int)r0 + ((threadIdx.x & 31) >> 3);
        double rmax = 0.0, rsum = 0.0;
        bool bad = false;
        if (r < P.n) {
            for (int p = P.a_rp[r] + sub; p < P.a_rp[r + 1]; p += 8) {
                double a = fabs(aval[p]);
                if (!isfinite(a)) bad = true;
                rmax = fmax(rmax, a);
                rsum += a;
            }
        }
        for (int o = 4; o > 0; o >>= 1) {
            rmax = fmax(rmax, __shfl_xor_sync(FULL, rmax, o));
            rsum += __shfl_xor_sync(FULL, rsum, o);
            bad |= __shfl_xor_sync(FULL, (int)bad, o);
        }
        if (r < P.n && sub == 0) {
            double s = 1.0;
            if (equil && !bad && rmax > 0.0) s = ldexp(1.0, -floor_half(ilogb(rmax)));
            s_orig[r] = s;
            sp[P.iperm[r]] = s;
            if (bad) atomicExch(status + ST_NONFINITE, 1);
            else nmax = fmax(nmax, rsum);
        }
    }
    nmax = cta_max(nmax, red);
    if (threadIdx.x == 0) atomic_max_nonneg(norms + NM_ANORM, nmax);
}

__global__ void __launch_bounds__(RTHREADS)
k_amax(DevPattern P, const double *__restrict__ aval, const double *__restrict__ s_orig,
       unsigned long long *norms) {
    __shared__ double red[RTHREADS / 32];
    const int sub = threadIdx.x & 7;
    const long long step = (long long)gridDim.x * (blockDim.x >> 3);
    double mmax = 0.0, cmax = 0.0;                     // max|A'|, ||A||_1 over the finite rows seen
    for (long long r0 = ((long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) >> 3; r0 < P.n; r0 += step) {
        const int r = (int)r0 + ((threadIdx.x & 31) >> 3);
        double m = 0.0, csum = 0.0;
        if (r < P.n) {
            const double sr = s_orig[r];
            for (int p = P.a_rp[r] + sub; p < P.a_rp[r + 1]; p += 8) {
                double a = fabs(aval[p]) * sr * s_orig[P.a_ci[p]];
                m = fmax(m, a);
            }
            for (int q = P.at_rp[r] + sub; q < P.at_rp[r + 1]; q += 8) csum += fabs(aval[P.at_src[q]]);
        }
        for (int o = 4; o > 0; o >>= 1) {
            m = fmax(m, __shfl_xor_sync(FULL, m, o));
            csum += __shfl_xor_sync(FULL, csum, o);
        }
        if (r < P.n && sub == 0) {
            if (isfinite(m)) mmax = fmax(mmax, m);
            if (isfinite(csum)) cmax = fmax(cmax, csum);
        }
    }
    mmax = cta_max(mmax, red);
    cmax = cta_max(cmax, red);
    if (threadIdx.x == 0) {
        atomic_max_nonneg(norms + NM_AMAX, mmax);
        atomic_max_nonneg(norms + NM_A1NORM, cmax);
    }
}

// ---------------------------------------------------------------------------
// ready signals carried by the values themselves
//
// A value that is not yet computed holds the all-ones bit pattern (the
// buffers are filled with it before each launch); a producer publishes a
// value with one relaxed store and a consumer polls that word until it
// changes (the idea of Algorithm 2, which waits while x_d is NaN).  One memory
// round trip per dependency, no flag and no fence: aligned 32/64-bit accesses
// are single-copy atomic.  A computed value whose bits equal the marker is
// replaced by a canonical NaN and flagged.

__device__ __forceinline__ double ld_relaxed_v(const double *p) {
    double v;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_relaxed_v(const float *p) {
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_relaxed_v(double *p, double v) {
    asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v));
}
__device__ __forceinline__ void st_relaxed_v(float *p, float v) {
    asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v));
}
__device__ __forceinline__ bool is_marker(double v) { return __double_as_longlong(v) == -1LL; }
__device__ __forceinline__ bool is_marker(float v) { return __float_as_int(v) == -1; }

template <typename T> __device__ __forceinline__ T wait_value(const RunCfg &rc, const T *p) {
    T v = ld_relaxed_v(p);
    if (!is_marker(v)) return v;
    long long it = 0;
    for (;;) {
        __nanosleep(32);
        v = ld_relaxed_v(p);
        if (!is_marker(v)) return v;
        if ((++it & 15) == 0) {
            if (ld_relaxed(rc.status + ST_ABORT)) return T(0);
            if (it > rc.spin_limit) {
                atomicExch(rc.status + ST_TIMEOUT, 1);
                atomicExch(rc.status + ST_ABORT, 1);
                return T(0);
            }
        }
    }
}

// Warp-cooperative wait: every lane with need != 0 loads *p once; while some
// lane still sees the marker, only the lowest such lane polls (exponential
// backoff from 32 ns up to poll_ns_max), then the others reload once.  This keeps the
// polling traffic of thousands of waiting warps off the L2 that the critical
// path needs.  Must be called by all 32 lanes.
template <typename T>
__device__ __forceinline__ T warp_wait_load(const RunCfg &rc, const T *p, bool need, int lane) {
    T v = need ? ld_relaxed_v(p) : T(0);
    unsigned pend = __ballot_sync(FULL, need && is_marker(v));
    while (pend) {
        const int leader = __ffs(pend) - 1;
        int bad = 0;
        if (lane == leader) {
            unsigned ns = 32;
            long long it = 0;
            for (;;) {
                __nanosleep(ns);
                v = ld_relaxed_v(p);
                if (!is_marker(v)) break;
                if (ns < rc.poll_ns_max) ns <<= 1;
                if ((++it & 7) == 0) {
                    if (ld_relaxed(rc.status + ST_ABORT)) { bad = 1; break; }
                    if (it > rc.spin_limit) {
                        atomicExch(rc.status + ST_TIMEOUT, 1);
                        atomicExch(rc.status + ST_ABORT, 1);
                        bad = 1;
                        break;
                    }
                }
            }
        }
        if (__shfl_sync(FULL, bad, leader)) {       // give up: values are invalid
            if (is_marker(v)) v = T(0);
            break;
        }
        if (((pend >> lane) & 1u) && lane != leader) v = ld_relaxed_v(p);
        pend = __ballot_sync(FULL, ((pend >> lane) & 1u) && is_marker(v));
    }
    return v;
}

template <typename T> __device__ __forceinline__ void publish(const RunCfg &rc, T *p, T v) {
    if (is_marker(v)) {
        v = T(NAN);
        atomicExch(rc.status + ST_NONFINITE, 1);
    }
    st_relaxed_v(p, v);
}

// Barrier over the first `threads` threads... of the warps that reach it: a
// named barrier (id 1..15) shared by a subset of the CTA's warps.
__device__ __forceinline__ void named_barrier(int id, int threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// Batch-innermost arrays: entry k of system s at p[k * B + s].  The row and
// task bodies below take either plain pointers (one system) or these (one
// system of a batch), so the batched kernels run the same code per (row or
// task, system) as the single-system ones.
// (Offsets must be summed before they are added: `p + (a + b)`; `p + a`
// already yields a plain pointer into system s's entry a.)
template <typename T> struct Strided {
    T *p;
    int B, s;
    __device__ __forceinline__ T *operator+(long long k) const { return p + k * B + s; }
    __device__ __forceinline__ T &operator[](long long k) const { return p[k * B + s]; }
};

// A row of the dense root block after its pivot steps below the block: its
// multipliers go to their slots (and the transposed copy); its block part,
// the row's last P.n - dense_lo entries, goes to the dense array for
// k_dense_lu.  Nothing is published: only rows of the block read the block.
template <typename T, typename TP>
__device__ __forceinline__ void dense_row_out(const DevPattern &P, const RunCfg &rc, TP LU, TP LUT,
                                              const T *w, int rb, int len, int nst, int i, int lane) {
    T *D = reinterpret_cast<T *>(rc.dense) + (size_t)(i - rc.dense_lo) * rc.dense_ld;
    for (int c = lane; c < len - nst; c += 32) D[c] = w[nst + c];
    for (int t = lane; t < nst; t += 32) {
        LU[rb + t] = w[t];
        LUT[P.tpos[rb + t]] = w[t];
    }
}

// ---------------------------------------------------------------------------
// numeric refactorization: one warp per row of L+U (Algorithm 1's row-wise
// elimination, fixed pivots), rows claimed deepest first (distance to the root).
//
// Row i is gathered (scaled) into shared memory; for every pivot row d < i in
// L(i,:), in increasing d, the multiplier l = w[d] * (1 / U(d,d)) is formed
// and U(d, >d) is subtracted from the row.  Ready signals are the published
// values themselves: the reciprocal pivot rcp[d] and every entry of U(d,:)
// start as the marker, and each lane polls exactly the values it consumes.
// Targets are placed through the update map (relative positions precomputed
// at analysis) or, without a map, by a binary search of the row's sorted
// columns; no atomics.  The metadata of 32 pivot steps is loaded at once
// (one lane per step) and the next step's map segment is prefetched.  The
// finished row is also written to the transposed layout (LUT[tpos[t]]) for
// the transposed solves.
// One row of the refactorization (the warp of lane `lane`); sval / scol are
// the warp's shared-memory row of capacity cap (scol is used only without
// update maps), gw its global warp index (its global scratch row).
template <typename T, typename AV = const double *, typename TP = T *>
__device__ __forceinline__ void refactor_row(const DevPattern &P, const RunCfg &rc, AV aval, AV sp, TP LU,
                                             TP LUT, TP rcp, double tau, int i, T *sval, int *scol,
                                             int cap, int gw, int lane) {
    const bool mapped = P.upd_off != nullptr;
            const int rb = P.lu_rp[i], len = P.lu_rp[i + 1] - rb, dp = P.diag[i] - rb;
            // a row of the dense root block takes only the pivot steps below the block
            const bool dense = i >= rc.dense_lo;
            const int nst = dense ? len - (P.n - rc.dense_lo) : dp;
            // steps t >= tmap (pivots inside the dense root block, when the kernel
            // takes them as sparse steps) have no update map
            const int tmap = i >= P.dense_lo ? len - (P.n - P.dense_lo) : INT_MAX;
            const int *c = P.lu_ci + rb;
            T *w;
            if (len <= cap) {
                w = sval;
                if (!mapped) {
                    for (int t = lane; t < len; t += 32) scol[t] = c[t];
                    c = scol;
                }
            } else {
                w = reinterpret_cast<T *>(rc.scratch) + (size_t)gw * rc.scratch_stride;
            }
            // gather A'(i,:) = s_i a_ij s_j into the row (structural zeros elsewhere)
            const double si = sp[i];
            for (int t = lane; t < len; t += 32) {
                const int k = P.src[rb + t];
                w[t] = (T)((k >= 0) ? si * sp[P.lu_ci[rb + t]] * aval[k] : 0.0);
            }
            __syncwarp();
            // Pivot steps are pipelined: while step t computes, the reciprocal
            // pivot and the first 32 x UJ entries (targets, values) of step t+1 are
            // already in flight; a value still unpublished is polled again.
            constexpr int UJ = sizeof(T) == 4 ? 8 : 4;   // FP32 rows hold twice the entries in flight
            int md = 0, mub = 0, mue = 0;       // metadata of steps t0..t0+31, one per lane
            unsigned mmo = 0;
            auto load_meta = [&](int t0) {
                md = mub = mue = 0;
                mmo = 0;
                if (t0 + lane < nst) {
                    md = P.lu_ci[rb + t0 + lane];
                    mub = P.diag[md];
                    mue = P.lu_rp[md + 1];
                    if (mapped) mmo = P.upd_off[rb + t0 + lane];
                }
            };
            auto target = [&](int t, int ub, unsigned mo, int u) -> int {
                if (mapped && t < tmap) return P.upd_map[mo + (u - ub - 1)];
                const int j = P.lu_ci[u];
                int a_ = t + 1, b_ = len;
                while (a_ < b_) {
                    const int mid = (a_ + b_) >> 1;
                    if (c[mid] < j) a_ = mid + 1; else b_ = mid;
                }
                if (a_ < len && c[a_] == j) return a_;
                atomicExch(rc.status + ST_INTERNAL, 1);       // pattern not closed under fill
                return -1;
            };
            // prefetched state of the next step
            T pr = T(0);
            int plo[UJ];
            T pu[UJ];
            auto prefetch = [&](int t, int d, int ub, int ue, unsigned mo) {
                pr = ld_relaxed_v(rcp + d);
    #pragma unroll
                for (int q = 0; q < UJ; q++) {
                    const int u = ub + 1 + 32 * q + lane;
                    plo[q] = -1;
                    pu[q] = T(0);
                    if (u < ue) {
                        plo[q] = target(t, ub, mo, u);
                        pu[q] = ld_relaxed_v(LU + u);
                    }
                }
            };
            if (nst > 0) {
                load_meta(0);
                prefetch(0, __shfl_sync(FULL, md, 0), __shfl_sync(FULL, mub, 0), __shfl_sync(FULL, mue, 0),
                         __shfl_sync(FULL, mmo, 0));
            }
            for (int t = 0; t < nst; t++) {
                const int k = t & 31;
                const int d = __shfl_sync(FULL, md, k);
                const int ub = __shfl_sync(FULL, mub, k);
                const int ue = __shfl_sync(FULL, mue, k);
                const unsigned mo = __shfl_sync(FULL, mmo, k);
                T r = pr;
                int lo[UJ];
                T uv[UJ];
    #pragma unroll
                for (int q = 0; q < UJ; q++) { lo[q] = plo[q]; uv[q] = pu[q]; }
                // next step's loads go out now
                if (t + 1 < nst) {
                    if (k == 31) load_meta(t + 1);
                    const int k1 = (t + 1) & 31;
                    prefetch(t + 1, __shfl_sync(FULL, md, k1), __shfl_sync(FULL, mub, k1),
                             __shfl_sync(FULL, mue, k1), __shfl_sync(FULL, mmo, k1));
                }
                // this step: reciprocal pivot and first block.  If the prefetch
                // came too early, the reciprocal is reloaded together with the
                // missing values (one round trip) and polled only if still
                // unpublished; the next step's prefetch, just as stale, is then
                // sent again.
                if (__any_sync(FULL, lane == 0 && is_marker(r))) {
                    if (lane == 0) r = ld_relaxed_v(rcp + d);
    #pragma unroll
                    for (int q = 0; q < UJ; q++)
                        if (lo[q] >= 0 && is_marker(uv[q])) uv[q] = ld_relaxed_v(LU + (ub + 1 + 32 * q + lane));
                    if (__any_sync(FULL, lane == 0 && is_marker(r))) {
                        const T w0 = warp_wait_load(rc, rcp + d, lane == 0, lane);
                        if (lane == 0) r = w0;
                    }
                    if (t + 1 < nst && __any_sync(FULL, lane == 0 && is_marker(pr))) {
                        const int k1 = (t + 1) & 31;
                        const int d1 = __shfl_sync(FULL, md, k1), ub1 = __shfl_sync(FULL, mub, k1),
                                  ue1 = __shfl_sync(FULL, mue, k1);
                        pr = ld_relaxed_v(rcp + d1);
    #pragma unroll
                        for (int q = 0; q < UJ; q++) {
                            const int u = ub1 + 1 + 32 * q + lane;
                            if (u < ue1) pu[q] = ld_relaxed_v(LU + u);
                        }
                    }
                }
                const T l = w[t] * __shfl_sync(FULL, r, 0);
                unsigned need = 0;
    #pragma unroll
                for (int q = 0; q < UJ; q++)
                    if (lo[q] >= 0 && is_marker(uv[q])) need |= 1u << q;
                if (__any_sync(FULL, need != 0)) {           // one reload of everything still missing
    #pragma unroll
                    for (int q = 0; q < UJ; q++)
                        if ((need >> q) & 1u) uv[q] = ld_relaxed_v(LU + (ub + 1 + 32 * q + lane));
                    need = 0;
    #pragma unroll
                    for (int q = 0; q < UJ; q++)
                        if (lo[q] >= 0 && is_marker(uv[q])) need |= 1u << q;
                }
                if (__any_sync(FULL, need != 0)) {
    #pragma unroll
                    for (int q = 0; q < UJ; q++) {
                        const bool nq = (need >> q) & 1u;
                        const T v = warp_wait_load(rc, LU + (nq ? ub + 1 + 32 * q + lane : ub), nq, lane);
                        if (nq) uv[q] = v;
                    }
                }
                // rounds past the end of the pivot row are skipped as a whole
                // (an FP64 instruction costs the same with idle lanes)
                // the round's targets are distinct: all loads, then all updates
                {
                    T x[UJ];
    #pragma unroll
                    for (int q = 0; q < UJ; q++) x[q] = (32 * q < ue - ub - 1 && lo[q] >= 0) ? w[lo[q]] : T(0);
    #pragma unroll
                    for (int q = 0; q < UJ; q++)
                        if (32 * q < ue - ub - 1 && lo[q] >= 0) w[lo[q]] = x[q] - l * uv[q];
                }
                // remaining blocks of long pivot rows, double-buffered: the next
                // block's targets and values are in flight while this one updates
                auto load_blk = [&](int u0, int (&bl)[UJ], T (&bv)[UJ]) {
    #pragma unroll
                    for (int q = 0; q < UJ; q++) {
                        const int u = u0 + 32 * q + lane;
                        bl[q] = -1;
                        bv[q] = T(0);
                        if (u < ue) {
                            bl[q] = target(t, ub, mo, u);
                            bv[q] = ld_relaxed_v(LU + u);
                        }
                    }
                };
                if (ub + 1 + 32 * UJ < ue) {
                    int cl[UJ];
                    T cv[UJ];
                    load_blk(ub + 1 + 32 * UJ, cl, cv);
                    for (int u0 = ub + 1 + 32 * UJ; u0 < ue; u0 += 32 * UJ) {
                        int nl[UJ];
                        T nv[UJ];
                        if (u0 + 32 * UJ < ue) load_blk(u0 + 32 * UJ, nl, nv);
                        unsigned bneed = 0;
    #pragma unroll
                        for (int q = 0; q < UJ; q++)
                            if (cl[q] >= 0 && is_marker(cv[q])) bneed |= 1u << q;
                        if (__any_sync(FULL, bneed != 0)) {
    #pragma unroll
                            for (int q = 0; q < UJ; q++) {
                                const bool nq = (bneed >> q) & 1u;
                                const T v = warp_wait_load(rc, LU + (nq ? u0 + 32 * q + lane : ub), nq, lane);
                                if (nq) cv[q] = v;
                            }
                        }
                        T x[UJ];
    #pragma unroll
                        for (int q = 0; q < UJ; q++) x[q] = (u0 + 32 * q < ue && cl[q] >= 0) ? w[cl[q]] : T(0);
    #pragma unroll
                        for (int q = 0; q < UJ; q++)
                            if (u0 + 32 * q < ue && cl[q] >= 0) w[cl[q]] = x[q] - l * cv[q];
    #pragma unroll
                        for (int q = 0; q < UJ; q++) {
                            cl[q] = nl[q];
                            cv[q] = nv[q];
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) w[t] = l;
            }
            if (dense) {
                dense_row_out<T>(P, rc, LU, LUT, w, rb, len, nst, i, lane);
                return;
            }
            // pivot test in FP64 (perturb to sign(a_ii) tau and count)
            if (lane == 0) {
                double pv = (double)w[dp];
                if (!(fabs(pv) >= tau) || isinf(pv)) {
                    const int k = P.src[rb + dp];
                    const double aii = (k >= 0) ? si * si * aval[k] : 0.0;
                    if (!isfinite(pv)) atomicExch(rc.status + ST_NONFINITE, 1);
                    pv = (aii < 0.0) ? -tau : tau;
                    atomicAdd(rc.status + ST_PERTURBED, 1);
                    atomicAdd(rc.status + ST_PERT_LAST, 1);
                }
                if (pv < 0.0) atomicAdd(rc.status + ST_NEGATIVE, 1);
                w[dp] = (T)pv;
            }
            __syncwarp();
            // the reciprocal pivot first (the rows below wait on it, then reload
            // the U part, which is on its way by then), then the U part
            if (lane == 0) {
                LU[rb + dp] = w[dp];
                if (i != rc.unpublished_row) publish(rc, rcp + i, T(1) / w[dp]);
            }
            for (int t = dp + 1 + lane; t < len; t += 32) publish(rc, LU + (rb + t), w[t]);
            for (int t = lane; t < len; t += 32) {
                if (t < dp) LU[rb + t] = w[t];
                LUT[P.tpos[rb + t]] = w[t];
            }
}

// ---------------------------------------------------------------------------
// Staged pivot steps (single-system refactorization with update maps).
//
// A pivot step of row i reads U(d, >d) of its pivot row d and the relative
// positions of those entries in row i (the update map).  Near the top of the
// elimination tree a row takes thousands of pivot steps over pivot rows of
// several hundred entries; loading each step's data when the step starts
// exposes one memory round trip per block of the pivot row (measured: 2.5 us
// per step in FP32, 3.9 us in FP64, on the 70,000-bus KKT).  Here the pivot
// rows are cut into units of SB entries (one SB-entry block of one step), and
// every warp keeps a ring of STAGES units in shared memory that cp.async fills
// STAGES - 1 units ahead of the unit being applied: values and map targets in
// 16-byte chunks (the copy starts at the 16-byte boundary below the block and
// indexes from the remainder), the reciprocal pivot with the first block.
// Values copied before their row was published hold the not-ready marker and
// are reloaded from global memory (marker protocol above); the update maps
// never change.
template <typename T> struct Stage {
    static constexpr int SB = sizeof(T) == 4 ? 256 : 128;       // entries per unit (32 x UJ)
    static constexpr int VE = 16 / (int)sizeof(T);              // values per 16-byte chunk
    static constexpr int STAGES = sizeof(T) == 4 ? 6 : 4;
    static constexpr int VAL_BYTES = ((SB + VE) * (int)sizeof(T) + 15) / 16 * 16;
    static constexpr int MAP_BYTES = ((SB + 8) * 2 + 15) / 16 * 16;
    static constexpr int SLOT = VAL_BYTES + MAP_BYTES + 16 + 32;  // + reciprocal pivot + descriptor
    static constexpr int RING = STAGES * SLOT;
};

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_word(float *dst, const float *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_word(double *dst, const double *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Row i of the refactorization as refactor_row, with the pivot steps fed from
// the warp's staging ring (shared memory, Stage<T>::RING bytes).  Requires the
// update maps.  LU and the update map must be readable 16 bytes past their
// ends (the last chunk of a block is rounded up).
template <typename T>
__device__ __forceinline__ void refactor_row_staged(const DevPattern &P, const RunCfg &rc,
                                                    const double *__restrict__ aval,
                                                    const double *__restrict__ sp, T *LU, T *LUT, T *rcp,
                                                    double tau, int i, T *sval, int cap,
                                                    unsigned char *ring, int gw, int lane) {
    using S = Stage<T>;
    constexpr int UJ = S::SB / 32;
    const int rb = P.lu_rp[i], len = P.lu_rp[i + 1] - rb, dp = P.diag[i] - rb;
    // a row of the dense root block takes only the pivot steps below the block
    const bool dense = i >= rc.dense_lo;
    const int nst = dense ? len - (P.n - rc.dense_lo) : dp;
    T *w = len <= cap ? sval : reinterpret_cast<T *>(rc.scratch) + (size_t)gw * rc.scratch_stride;
    const double si = sp[i];
    for (int t = lane; t < len; t += 32) {
        const int k = P.src[rb + t];
        w[t] = (T)((k >= 0) ? si * sp[P.lu_ci[rb + t]] * aval[k] : 0.0);
    }
    __syncwarp();
    if (nst > 0) {
        // producer: next unit to stage is block pb of step pt; the metadata of
        // steps c0 .. c0 + 31 (lane k: step c0 + k) and of the chunk after it
        int pt = 0, pb = 0, c0 = 0;
        int md = 0, mub = 0, mue = 0, nd = 0, nub = 0, nue = 0;
        unsigned mmo = 0, nmo = 0;
        auto load_meta = [&](int t0, int &d_, int &ub_, int &ue_, unsigned &mo_) {
            d_ = ub_ = ue_ = 0;
            mo_ = 0;
            if (t0 + lane < nst) {
                d_ = P.lu_ci[rb + t0 + lane];
                ub_ = P.diag[d_];
                ue_ = P.lu_rp[d_ + 1];
                mo_ = P.upd_off[rb + t0 + lane];
            }
        };
        load_meta(0, md, mub, mue, mmo);
        load_meta(32, nd, nub, nue, nmo);
        auto issue = [&](int unit) {
            unsigned char *slot = ring + (unit % S::STAGES) * S::SLOT;
            if (pt < nst) {
                if (pt - c0 >= 32) {                    // next metadata chunk
                    c0 += 32;
                    md = nd; mub = nub; mue = nue; mmo = nmo;
                    load_meta(c0 + 32, nd, nub, nue, nmo);
                }
                const int k = pt - c0;
                const int d = __shfl_sync(FULL, md, k), ub = __shfl_sync(FULL, mub, k);
                const int ue = __shfl_sync(FULL, mue, k);
                const unsigned mo = __shfl_sync(FULL, mmo, k);
                const int u0 = ub + 1 + pb * S::SB;
                const int cnt = min(S::SB, ue - u0);
                const int last = (u0 + S::SB >= ue);
                const int vo = u0 & (S::VE - 1);
                const unsigned mstart = mo + (unsigned)(u0 - ub - 1);
                const int mo2 = (int)(mstart & 7u);
                T *sv = reinterpret_cast<T *>(slot);
                unsigned short *sm = reinterpret_cast<unsigned short *>(slot + S::VAL_BYTES);
                T *sr = reinterpret_cast<T *>(slot + S::VAL_BYTES + S::MAP_BYTES);
                int *desc = reinterpret_cast<int *>(slot + S::VAL_BYTES + S::MAP_BYTES + 16);
                const T *vsrc = LU + (u0 - vo);
                const int vch = (vo + cnt + S::VE - 1) / S::VE;
                for (int q = lane; q < vch; q += 32) cp_async16(sv + q * S::VE, vsrc + q * S::VE);
                const unsigned short *msrc = P.upd_map + (mstart - (unsigned)mo2);
                const int mch = (mo2 + cnt + 7) / 8;
                for (int q = lane; q < mch; q += 32) cp_async16(sm + q * 8, msrc + q * 8);
                if (pb == 0 && lane == 0) cp_async_word(sr, rcp + d);
                if (lane == 0) {
                    desc[0] = pt; desc[1] = u0; desc[2] = cnt; desc[3] = vo;
                    desc[4] = mo2; desc[5] = d; desc[6] = (pb == 0) | (last << 1);
                }
                if (last) { pt++; pb = 0; } else { pb++; }
            }
            cp_async_commit();                          // an empty group past the last unit
        };
        for (int q = 0; q < S::STAGES - 1; q++) issue(q);
        T l = T(0);
        for (int unit = 0;; unit++) {
            __syncwarp();                               // the slot issued next was consumed
            issue(unit + S::STAGES - 1);
            cp_async_wait<S::STAGES - 1>();
            __syncwarp();                               // every lane's copies of this unit landed
            unsigned char *slot = ring + (unit % S::STAGES) * S::SLOT;
            const T *sv = reinterpret_cast<const T *>(slot);
            const unsigned short *sm = reinterpret_cast<const unsigned short *>(slot + S::VAL_BYTES);
            const T *sr = reinterpret_cast<const T *>(slot + S::VAL_BYTES + S::MAP_BYTES);
            const int *desc = reinterpret_cast<const int *>(slot + S::VAL_BYTES + S::MAP_BYTES + 16);
            const int t = desc[0], u0 = desc[1], cnt = desc[2], vo = desc[3], mo2 = desc[4], d = desc[5];
            const int flags = desc[6];
            if (flags & 1) {                            // first block: the multiplier
                T r = sr[0];
                if (is_marker(r)) {
                    r = ld_relaxed_v(rcp + d);
                    if (__any_sync(FULL, lane == 0 && is_marker(r))) {
                        const T w0 = warp_wait_load(rc, rcp + d, lane == 0, lane);
                        if (lane == 0) r = w0;
                    }
                    r = __shfl_sync(FULL, r, 0);
                }
                l = w[t] * r;
            }
            int lo[UJ];
            T uv[UJ];
            unsigned need = 0;
#pragma unroll
            for (int q = 0; q < UJ; q++) {
                const int j = 32 * q + lane;
                lo[q] = -1;
                uv[q] = T(0);
                if (j < cnt) {
                    lo[q] = sm[mo2 + j];
                    uv[q] = sv[vo + j];
                    if (is_marker(uv[q])) need |= 1u << q;
                }
            }
            if (__any_sync(FULL, need != 0)) {          // copied before publication: reload once,
#pragma unroll                                          // then wait per entry
                for (int q = 0; q < UJ; q++)
                    if ((need >> q) & 1u) uv[q] = ld_relaxed_v(LU + (u0 + 32 * q + lane));
                need = 0;
#pragma unroll
                for (int q = 0; q < UJ; q++)
                    if (lo[q] >= 0 && is_marker(uv[q])) need |= 1u << q;
                if (__any_sync(FULL, need != 0)) {
#pragma unroll
                    for (int q = 0; q < UJ; q++) {
                        const bool nq = (need >> q) & 1u;
                        const T v = warp_wait_load(rc, LU + (nq ? u0 + 32 * q + lane : u0), nq, lane);
                        if (nq) uv[q] = v;
                    }
                }
            }
            // the block's targets are distinct: all loads, then all updates
            T x[UJ];
#pragma unroll
            for (int q = 0; q < UJ; q++) x[q] = lo[q] >= 0 ? w[lo[q]] : T(0);
#pragma unroll
            for (int q = 0; q < UJ; q++)
                if (lo[q] >= 0) w[lo[q]] = x[q] - l * uv[q];
            if (flags & 2) {                            // last block of step t
                __syncwarp();
                if (lane == 0) w[t] = l;
                if (t + 1 == nst) break;
            }
        }
        cp_async_wait<0>();                             // nothing of this row left in flight
        __syncwarp();
    }
    if (dense) {
        dense_row_out<T>(P, rc, LU, LUT, w, rb, len, nst, i, lane);
        return;
    }
    // pivot test in FP64 (perturb to sign(a_ii) tau and count)
    if (lane == 0) {
        double pv = (double)w[dp];
        if (!(fabs(pv) >= tau) || isinf(pv)) {
            const int k = P.src[rb + dp];
            const double aii = (k >= 0) ? si * si * aval[k] : 0.0;
            if (!isfinite(pv)) atomicExch(rc.status + ST_NONFINITE, 1);
            pv = (aii < 0.0) ? -tau : tau;
            atomicAdd(rc.status + ST_PERTURBED, 1);
            atomicAdd(rc.status + ST_PERT_LAST, 1);
        }
        if (pv < 0.0) atomicAdd(rc.status + ST_NEGATIVE, 1);
        w[dp] = (T)pv;
    }
    __syncwarp();
    if (lane == 0) {
        LU[rb + dp] = w[dp];
        if (i != rc.unpublished_row) publish(rc, rcp + i, T(1) / w[dp]);
    }
    for (int t = dp + 1 + lane; t < len; t += 32) publish(rc, LU + (rb + t), w[t]);
    for (int t = lane; t < len; t += 32) {
        if (t < dp) LU[rb + t] = w[t];
        LUT[P.tpos[rb + t]] = w[t];
    }
}

// ---------------------------------------------------------------------------
// Symmetric values: LDL^T through the same storage (options.symmetric).
//
// For a symmetric A' the Doolittle factors satisfy L = U^T D^-1 with D the
// pivots (A' = L D L^T, the MA57 form of the paper's CPU baseline, Sec. 5.3;
// Sec. 3 on inertia).  Row i then needs no elimination of its own L part:
// its multipliers are l(i,d) = u(d,i) / u(d,d), entries of rows below it that
// are already published, and only its U part is reduced,
//     u(i,j) = a'(i,j) - sum_d l(i,d) u(d,j),   j >= i,
// over the tail U(d, >= i) of each pivot row.  The pivot steps of a row are
// independent of each other (no multiplier waits on an earlier step), each
// touches only the part of U(d,:) at or right of column i, and the flops are
// half those of LU.  L is still written (l(i,d) into row i's L slots), so the
// solves and exports are those of the LU path.  The lower triangle of the
// values is not read: the factorization is that of the symmetric matrix with
// A's upper triangle.  The pivot signs give the inertia (Sylvester's law:
// S P A P^T S is congruent to A).
template <typename T>
__device__ __forceinline__ void refactor_row_sym(const DevPattern &P, const RunCfg &rc,
                                                 const double *__restrict__ aval,
                                                 const double *__restrict__ sp, T *LU, T *LUT, T *rcp,
                                                 double tau, int i, T *sval, int cap,
                                                 unsigned char *ring, int gw, int lane) {
    using S = Stage<T>;
    constexpr int UJ = S::SB / 32;
    const int rb = P.lu_rp[i], len = P.lu_rp[i + 1] - rb, dp = P.diag[i] - rb;
    const int ulen = len - dp;                         // U part, diagonal first
    // a row of the dense root block takes only the pivot steps below the block
    const bool dense = i >= rc.dense_lo;
    const int nst = dense ? len - (P.n - rc.dense_lo) : dp;
    // the row buffer holds the U part only; each multiplier l(i,d) goes to
    // its L slot at once (the address needs no load) and to the transposed
    // factor at the end
    T *w = ulen <= cap ? sval : reinterpret_cast<T *>(rc.scratch) + (size_t)gw * rc.scratch_stride;
    const double si = sp[i];
    for (int t = lane; t < ulen; t += 32) {
        const int k = P.src[rb + dp + t];
        w[t] = (T)((k >= 0) ? si * sp[P.lu_ci[rb + dp + t]] * aval[k] : 0.0);
    }
    __syncwarp();
    if (nst > 0) {
        int pt = 0, pb = 0, c0 = 0;
        int md = 0, mub = 0, mue = 0, mts = 0, nd = 0, nub = 0, nue = 0, nts = 0;
        unsigned mmo = 0, nmo = 0;
        auto load_meta = [&](int t0, int &d_, int &ub_, int &ue_, int &ts_, unsigned &mo_) {
            d_ = ub_ = ue_ = ts_ = 0;
            mo_ = 0;
            if (t0 + lane < nst) {
                d_ = P.lu_ci[rb + t0 + lane];
                ub_ = P.diag[d_];
                ue_ = P.lu_rp[d_ + 1];
                ts_ = P.tpos[rb + t0 + lane];           // slot of u(d,i) in row d
                mo_ = P.upd_off[rb + t0 + lane];
            }
        };
        load_meta(0, md, mub, mue, mts, mmo);
        load_meta(32, nd, nub, nue, nts, nmo);
        auto issue = [&](int unit) {
            unsigned char *slot = ring + (unit % S::STAGES) * S::SLOT;
            if (pt < nst) {
                if (pt - c0 >= 32) {
                    c0 += 32;
                    md = nd; mub = nub; mue = nue; mts = nts; mmo = nmo;
                    load_meta(c0 + 32, nd, nub, nue, nts, nmo);
                }
                const int k = pt - c0;
                const int d = __shfl_sync(FULL, md, k), ub = __shfl_sync(FULL, mub, k);
                const int ue = __shfl_sync(FULL, mue, k), ts = __shfl_sync(FULL, mts, k);
                const unsigned mo = __shfl_sync(FULL, mmo, k);
                const int u0 = ts + pb * S::SB;         // the tail U(d, >= i), u(d,i) first
                const int cnt = min(S::SB, ue - u0);
                const int last = (u0 + S::SB >= ue);
                const int vo = u0 & (S::VE - 1);
                const unsigned mstart = mo + (unsigned)(u0 - ub - 1);
                const int mo2 = (int)(mstart & 7u);
                T *sv = reinterpret_cast<T *>(slot);
                unsigned short *sm = reinterpret_cast<unsigned short *>(slot + S::VAL_BYTES);
                T *sr = reinterpret_cast<T *>(slot + S::VAL_BYTES + S::MAP_BYTES);
                int *desc = reinterpret_cast<int *>(slot + S::VAL_BYTES + S::MAP_BYTES + 16);
                const T *vsrc = LU + (u0 - vo);
                const int vch = (vo + cnt + S::VE - 1) / S::VE;
                for (int q = lane; q < vch; q += 32) cp_async16(sv + q * S::VE, vsrc + q * S::VE);
                const unsigned short *msrc = P.upd_map + (mstart - (unsigned)mo2);
                const int mch = (mo2 + cnt + 7) / 8;
                for (int q = lane; q < mch; q += 32) cp_async16(sm + q * 8, msrc + q * 8);
                if (pb == 0 && lane == 0) cp_async_word(sr, rcp + d);
                if (lane == 0) {
                    desc[0] = pt; desc[1] = u0; desc[2] = cnt; desc[3] = vo;
                    desc[4] = mo2; desc[5] = d; desc[6] = (pb == 0) | (last << 1);
                }
                if (last) { pt++; pb = 0; } else { pb++; }
            }
            cp_async_commit();
        };
        for (int q = 0; q < S::STAGES - 1; q++) issue(q);
        T l = T(0);
        for (int unit = 0;; unit++) {
            __syncwarp();
            issue(unit + S::STAGES - 1);
            cp_async_wait<S::STAGES - 1>();
            __syncwarp();
            unsigned char *slot = ring + (unit % S::STAGES) * S::SLOT;
            const T *sv = reinterpret_cast<const T *>(slot);
            const unsigned short *sm = reinterpret_cast<const unsigned short *>(slot + S::VAL_BYTES);
            const T *sr = reinterpret_cast<const T *>(slot + S::VAL_BYTES + S::MAP_BYTES);
            const int *desc = reinterpret_cast<const int *>(slot + S::VAL_BYTES + S::MAP_BYTES + 16);
            const int t = desc[0], u0 = desc[1], cnt = desc[2], vo = desc[3], mo2 = desc[4], d = desc[5];
            const int flags = desc[6];
            int lo[UJ];
            T uv[UJ];
            unsigned need = 0;
#pragma unroll
            for (int q = 0; q < UJ; q++) {
                const int j = 32 * q + lane;
                lo[q] = -1;
                uv[q] = T(0);
                if (j < cnt) {
                    lo[q] = (int)sm[mo2 + j] - dp;
                    uv[q] = sv[vo + j];
                    if (is_marker(uv[q])) need |= 1u << q;
                }
            }
            if (__any_sync(FULL, need != 0)) {
#pragma unroll
                for (int q = 0; q < UJ; q++)
                    if ((need >> q) & 1u) uv[q] = ld_relaxed_v(LU + (u0 + 32 * q + lane));
                need = 0;
#pragma unroll
                for (int q = 0; q < UJ; q++)
                    if (lo[q] >= 0 && is_marker(uv[q])) need |= 1u << q;
                if (__any_sync(FULL, need != 0)) {
#pragma unroll
                    for (int q = 0; q < UJ; q++) {
                        const bool nq = (need >> q) & 1u;
                        const T v = warp_wait_load(rc, LU + (nq ? u0 + 32 * q + lane : u0), nq, lane);
                        if (nq) uv[q] = v;
                    }
                }
            }
            if (flags & 1) {                            // first block: l(i,d) = u(d,i) / u(d,d)
                T r = sr[0];
                if (is_marker(r)) {
                    r = ld_relaxed_v(rcp + d);
                    if (__any_sync(FULL, lane == 0 && is_marker(r))) {
                        const T w0 = warp_wait_load(rc, rcp + d, lane == 0, lane);
                        if (lane == 0) r = w0;
                    }
                    r = __shfl_sync(FULL, r, 0);
                }
                l = __shfl_sync(FULL, uv[0], 0) * r;     // lane 0, q 0 holds u(d,i)
                if (lane == 0) LU[rb + t] = l;
            }
            T x[UJ];
#pragma unroll
            for (int q = 0; q < UJ; q++) x[q] = lo[q] >= 0 ? w[lo[q]] : T(0);
#pragma unroll
            for (int q = 0; q < UJ; q++)
                if (lo[q] >= 0) w[lo[q]] = x[q] - l * uv[q];
            if ((flags & 2) && t + 1 == nst) break;
        }
        cp_async_wait<0>();
        __syncwarp();
    }
    if (dense) {                       // the block row's upper part, and by symmetry its column
        const int r = i - rc.dense_lo;
        T *D = reinterpret_cast<T *>(rc.dense);
        for (int t = lane; t < ulen; t += 32) {
            D[(size_t)r * rc.dense_ld + r + t] = w[t];
            D[(size_t)(r + t) * rc.dense_ld + r] = w[t];
        }
        for (int t = lane; t < nst; t += 32) LUT[P.tpos[rb + t]] = LU[rb + t];
        return;
    }
    // pivot test in FP64 (perturb to sign(a_ii) tau and count), sign for the inertia
    if (lane == 0) {
        double pv = (double)w[0];
        if (!(fabs(pv) >= tau) || isinf(pv)) {
            const int k = P.src[rb + dp];
            const double aii = (k >= 0) ? si * si * aval[k] : 0.0;
            if (!isfinite(pv)) atomicExch(rc.status + ST_NONFINITE, 1);
            pv = (aii < 0.0) ? -tau : tau;
            atomicAdd(rc.status + ST_PERTURBED, 1);
            atomicAdd(rc.status + ST_PERT_LAST, 1);
        }
        if (pv < 0.0) atomicAdd(rc.status + ST_NEGATIVE, 1);
        w[0] = (T)pv;
    }
    __syncwarp();
    if (lane == 0) {
        LU[rb + dp] = w[0];
        if (i != rc.unpublished_row) publish(rc, rcp + i, T(1) / w[0]);
    }
    for (int t = 1 + lane; t < ulen; t += 32) publish(rc, LU + (rb + dp + t), w[t]);
    for (int t = lane; t < ulen; t += 32) LUT[P.tpos[rb + dp + t]] = w[t];
    for (int t = lane; t < dp; t += 32) LUT[P.tpos[rb + t]] = LU[rb + t];   // lane 0's stores, seen
}                                                                       // after the warp's syncs

// Shared memory of k_refactor: warps 0 .. nbig-1 of every CTA ("big" warps)
// own a row buffer of cap_big entries, the others one of cap entries; the
// rows' columns follow in a second region of the same shape when there are no
// update maps.  Rows longer than cap (the top of the elimination tree, whose
// thousands of pivot steps would otherwise run against global memory) go to
// big warps only.  Three queues, each a subsequence of the deepest-first
// order: "free" rows (no long row below them in the tree, so they wait only
// on free rows), long rows, and the rest.  Every warp drains the free queue
// first (big warps help with the bulk of the tree), then big warps take long
// rows, then everyone takes the rest.  Deadlock-free: take the earliest
// unfinished row r.  Every row before r in r's queue is finished, and each
// warp holds one row at a time; a warp holding a row from a later queue
// entered that queue only after r's queue was fully claimed (free before
// long before rest, and small warps never take long rows), and a warp still
// in an earlier queue finishes its row -- a free row waits only on free rows,
// a long row on rows before it -- so some warp eligible for r's queue
// becomes free and claims r.
template <typename T>
__global__ void __launch_bounds__(WARPS * 32, 2)
k_refactor(DevPattern P, RunCfg rc, const double *__restrict__ aval, const double *__restrict__ sp,
           T *LU, T *LUT, T *rcp, double tau_rel) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // per-warp block: row values [cap], columns [cap] (no update maps), staging ring
    const bool big = wid < rc.nbig;
    const int cap = big ? rc.cap_big : rc.cap;
    unsigned char *mine = smem + (big ? (size_t)wid * rc.warp_bytes_big
                                      : (size_t)rc.nbig * rc.warp_bytes_big +
                                            (size_t)(wid - rc.nbig) * rc.warp_bytes_small);
    T *sval = reinterpret_cast<T *>(mine);
    const size_t vb = ((size_t)cap * sizeof(T) + 15) & ~(size_t)15;
    int *scol = rc.smem_cols ? reinterpret_cast<int *>(mine + vb) : nullptr;
    unsigned char *ring = rc.staged ? mine + vb : nullptr;
    const int e = rc.sched->epoch + 1;
    const int gw = blockIdx.x * nw + wid;
    const double tau = tau_rel * __longlong_as_double((long long)rc.norms[NM_AMAX]);
    auto drain = [&](int *counter, const int *order, int count) {
        for (;;) {
            int slot = 0;
            if (lane == 0) slot = atomicAdd(counter, 1);
            slot = __shfl_sync(FULL, slot, 0);
            if (slot >= count) break;
            const int row = order[slot];
            trace_mark(rc, 0, row, 0, lane);
            if (rc.symmetric)
                refactor_row_sym<T>(P, rc, aval, sp, LU, LUT, rcp, tau, row, sval, cap, ring, gw, lane);
            else if (rc.staged)
                refactor_row_staged<T>(P, rc, aval, sp, LU, LUT, rcp, tau, row, sval, cap, ring, gw, lane);
            else
                refactor_row<T>(P, rc, aval, sp, LU, LUT, rcp, tau, row, sval, scol, cap, gw, lane);
            trace_mark(rc, 0, row, 1, lane);
        }
    };
    drain(&rc.sched->next, P.order_free, P.n_free);
    if (big) drain(&rc.sched->next_long, P.order_long, P.n_long);
    drain(&rc.sched->next_rest, P.order_rest, P.n_rest);
    if (lane == 0) finish_launch(rc, e);
}

// ---------------------------------------------------------------------------
// triangular solves over longest-path tasks (one warp per task).
//
// A task is a path of the elimination tree that follows deepest children, so
// every root-to-leaf path crosses only a few tasks (7 on the 2,000-bus KKT,
// against 597 levels).  The analysis relabels the rows so that each task is a
// contiguous range [lo, hi] and its rows lie back to back in the CSR arrays: a
// warp streams through them, keeps their results in shared memory, reads a
// dependency inside the range from there and polls one outside it in global
// memory (marker protocol above).  The dependency slots of the next row are
// loaded into registers while the current row is computed (32 x SJ slots per
// row; longer rows load their tail directly).
//
// Forward phases (L, U^T) walk a task bottom-up and claim tasks longest-first;
// backward phases (U, L^T) walk top-down and claim them from the root.  Both
// orders are deadlock-free: a task only waits on tasks claimed before it,
// except the few longest (fewer than a quarter of the resident warps), which
// only wait on shorter tasks.
//
//   BACKWARD = false: dependencies in L(i,:) (slots left of the diagonal)
//   BACKWARD = true : dependencies in U(i,:) (slots right of the diagonal)
//   TRANS           : read the transposed factor (A'^T = U^T L^T)
// Forward:  y_i = (rhs'_i - sum dep) [* rcp_i when TRANS], rhs' = s_i rhs[perm[i]]
// Backward: z_i = (y_i - sum dep) [* rcp_i when !TRANS];
//           out[perm[i]] = s_i z_i  (accumulate: +=)
constexpr int SJ = 8;

// Load up to 32 x SJ dependency slots of one row (column, factor value).
template <typename T, typename FP>
__device__ __forceinline__ void load_slots(const DevPattern &P, FP F, int tb, int te,
                                           int lane, int (&col)[SJ], T (&val)[SJ]) {
#pragma unroll
    for (int j = 0; j < SJ; j++) {
        const int t = tb + lane + 32 * j;
        col[j] = -1;
        val[j] = T(0);
        if (t < te) {
            col[j] = P.lu_ci[t];
            val[j] = F[t];
        }
    }
}

// One task of a triangular solve (the warp of lane `lane`); loc is the warp's
// shared-memory buffer of capacity tk.cap.
template <typename T, bool BACKWARD, bool TRANS, typename CF = const T *, typename CD = const double *,
          typename TF = T *, typename DF = double *>
__device__ __forceinline__ void trisolve_task(const DevPattern &P, const RunCfg &rc, const TaskCfg &tk, CF F,
                                              CF rcp, CD rhs, CD sp, CF yin, TF yout, DF out,
                                              int accumulate, int tid, T *loc, int lane) {
    constexpr bool DIV = (TRANS != BACKWARD);
            const int lo = tk.task_lo[tid], hi = tk.task_hi[tid];
            const int m = hi - lo + 1;
            // row of walk step k, and its dependency slot range
            auto row_of = [&](int k) { return BACKWARD ? hi - k : lo + k; };
            auto meta = [&](int k, int &tb, int &te) {
                const int i = row_of(k);
                const int dg = P.diag[i];
                tb = BACKWARD ? dg + 1 : P.lu_rp[i];
                te = BACKWARD ? P.lu_rp[i + 1] : dg;
            };
            // per-lane metadata of the current and the next chunk of 32 steps
            int ctb = 0, cte = 0, ntb = 0, nte = 0;
            if (lane < m) meta(lane, ctb, cte);
            if (32 + lane < m) meta(32 + lane, ntb, nte);
            // owner data of this lane's step in the current chunk
            T obase = T(0), orc = T(1);
            double osp = 0.0, oold = 0.0;
            int oo = 0;
            auto owner = [&](int k) {
                if (k >= m) return;
                const int i = row_of(k);
                if (DIV) orc = rcp[i];
                if (BACKWARD) {
                    obase = yin[i];
                    osp = sp[i];
                    oo = P.perm[i];
                    if (accumulate) oold = out[oo];
                } else {
                    obase = (T)(sp[i] * rhs[P.perm[i]]);
                }
            };
            owner(lane);
            int ncol[SJ];
            T nval[SJ];
            load_slots<T>(P, F, __shfl_sync(FULL, ctb, 0), __shfl_sync(FULL, cte, 0), lane, ncol, nval);
            for (int k = 0; k < m; k++) {
                const int kl = k & 31;
                if (kl == 0 && k > 0) {                      // advance to the next chunk
                    ctb = ntb; cte = nte;
                    ntb = nte = 0;
                    if (k + 32 + lane < m) meta(k + 32 + lane, ntb, nte);
                    owner(k + lane);
                }
                const int i = row_of(k);
                const int tb = __shfl_sync(FULL, ctb, kl), te = __shfl_sync(FULL, cte, kl);
                int col[SJ];
                T val[SJ], v[SJ];
    #pragma unroll
                for (int j = 0; j < SJ; j++) { col[j] = ncol[j]; val[j] = nval[j]; v[j] = T(0); }
                if (k + 1 < m) {                             // next row's slots, in flight meanwhile
                    const int src = (kl == 31) ? 0 : kl + 1;
                    const int nb = (kl == 31) ? __shfl_sync(FULL, ntb, src) : __shfl_sync(FULL, ctb, src);
                    const int ne = (kl == 31) ? __shfl_sync(FULL, nte, src) : __shfl_sync(FULL, cte, src);
                    load_slots<T>(P, F, nb, ne, lane, ncol, nval);
                }
                // dependency values: inside the task from shared memory, else polled
                unsigned needm = 0;
    #pragma unroll
                for (int j = 0; j < SJ; j++) {
                    const int c = col[j];
                    if (c >= 0) {
                        const bool inside = BACKWARD ? (c <= hi) : (c >= lo);
                        if (inside && c - lo < tk.cap) {
                            v[j] = loc[c - lo];
                        } else {
                            v[j] = ld_relaxed_v(yout + c);
                            if (is_marker(v[j])) needm |= 1u << j;
                        }
                    }
                }
                if (__any_sync(FULL, needm != 0)) {
    #pragma unroll
                    for (int j = 0; j < SJ; j++) {
                        const bool nj = (needm >> j) & 1u;
                        const T w = warp_wait_load(rc, yout + (nj ? col[j] : 0), nj, lane);
                        if (nj) v[j] = w;
                    }
                }
                // FP64 instructions cost ~64 cycles each here: only the rounds the row needs
                const int nj = min(SJ, (te - tb + 31) >> 5);
                T acc = 0;
    #pragma unroll
                for (int j = 0; j < SJ; j++)
                    if (j < nj) acc += val[j] * v[j];
                // rows longer than 32 x SJ slots: further blocks of 32 x SJ, every
                // block's loads issued before any of its waits
                for (int t0 = tb + 32 * SJ; t0 < te; t0 += 32 * SJ) {
                    int bc[SJ];
                    T bv[SJ], bx[SJ];
                    load_slots<T>(P, F, t0, te, lane, bc, bv);
                    unsigned bneed = 0;
    #pragma unroll
                    for (int j = 0; j < SJ; j++) {
                        bx[j] = T(0);
                        const int c = bc[j];
                        if (c >= 0) {
                            const bool inside = BACKWARD ? (c <= hi) : (c >= lo);
                            if (inside && c - lo < tk.cap) {
                                bx[j] = loc[c - lo];
                            } else {
                                bx[j] = ld_relaxed_v(yout + c);
                                if (is_marker(bx[j])) bneed |= 1u << j;
                            }
                        }
                    }
                    if (__any_sync(FULL, bneed != 0)) {
    #pragma unroll
                        for (int j = 0; j < SJ; j++) {
                            const bool nq = (bneed >> j) & 1u;
                            const T w = warp_wait_load(rc, yout + (nq ? bc[j] : 0), nq, lane);
                            if (nq) bx[j] = w;
                        }
                    }
                    const int bj = min(SJ, (te - t0 + 31) >> 5);
    #pragma unroll
                    for (int j = 0; j < SJ; j++)
                        if (j < bj) acc += bv[j] * bx[j];
                }
                acc = warp_sum(acc);
                if (lane == kl) {
                    T r = obase - acc;
                    if (DIV) r = r * orc;
                    if (is_marker(r)) {
                        r = T(NAN);
                        atomicExch(rc.status + ST_NONFINITE, 1);
                    }
                    const int p = i - lo;
                    if (p < tk.cap) loc[p] = r;
                    st_relaxed_v(yout + i, r);
                    if (BACKWARD) {
                        const double w = osp * (double)r;
                        out[oo] = accumulate ? oold + w : w;
                    }
                }
                __syncwarp();
            }
}

// ---------------------------------------------------------------------------
// Long tasks: one CTA per task.
//
// The steps of task [lo, hi] (bottom-up for the forward phases, top-down for
// the backward ones) are cut into blocks of CB = 32.  Row i at step k of block
// b = k / 32 splits its dependency slots by where their sources lie:
//   early : other tasks, or steps of this task before block b - 1;
//   late  : steps of block b - 1;
//   diag  : steps of block b (before k).
// Columns grow with the step in the forward phases and shrink in the backward
// ones, so the three groups are contiguous slot ranges; the analysis stores
// their boundaries (cs_late: early | late, cs_diag: late | diag in the forward
// phases; mirrored in the backward ones).
//
// Warp 0 (the walker) solves block b row after row: lane j owns row j of the
// block, the result of lane s is broadcast and every lane applies the diag
// entry of its row to it.  Warp 1 (on another FP64 pipe) applies each result
// as it appears in shared memory to the late entries of block b + 1's rows, so
// the late part of the next block is complete when this block is and a walker
// step is one shuffle and one dependent multiply-add.  The other warps (the
// helpers) meanwhile gather block b + 1: the right-hand side minus
// the early part (a warp per row, external sources polled in global memory)
// and the two 32 x 32 tiles of diag / late entries the walker reads next.
// Where the phase divides by the pivot, the helpers fold the reciprocal pivot
// of each row into its tile rows and right-hand side, so a walker step is one
// shuffle and one multiply-add.  One CTA barrier per block; the per-row
// hand-off is a shuffle instead of a global-memory round trip, and the bulk of
// the dot products runs on the helpers, off the chain of dependent steps.
constexpr int CB = 32;
constexpr int TS = CB + 1;
constexpr int CHAIN_MIN = 24;     // shortest task given a CTA
constexpr int QCHAIN_MAX = 48;    // CTA tasks of a queue's solves
constexpr int ZCAP_MAX = 8192;    // rows of a CTA task cached in shared memory
constexpr size_t CHAIN_SMEM = 200 * 1024;   // shared-memory budget of a CTA task
constexpr int SWARPS = 16;        // warps per CTA of the single-system solves
constexpr int EJ = 4;             // slots per lane of one early-part chunk
constexpr int ER = 3;             // early-part rows a helper works on at once
constexpr int EJ2 = 8;            // slots per lane of the further chunks of a long row

// shared memory of a CTA task, in bytes: tiles, right-hand sides and results
// (T), and per row up to zcap: the right-hand side term, the pivot scale (T)
// and four slot bounds (int)
__host__ __device__ constexpr size_t chain_smem_bytes(int zcap, size_t tsz) {
    return ((size_t)5 * CB * TS + 8 * CB + 3 * (size_t)zcap) * tsz + 5 * sizeof(int) * (size_t)zcap;
}

template <typename T, bool BACKWARD, bool TRANS>
__device__ __forceinline__ void trisolve_chain(const DevPattern &P, const RunCfg &rc, const TaskCfg &tk,
                                               int cidx, int lo, int hi, const T *__restrict__ F,
                                               const T *__restrict__ rcp, const double *__restrict__ rhs,
                                               const double *__restrict__ sp, const T *__restrict__ yin,
                                               T *yout, double *__restrict__ out, int accumulate,
                                               unsigned char *smem) {
    constexpr bool DIV = (TRANS != BACKWARD);
    constexpr bool FOLD = DIV && sizeof(T) == 8;   // pivots folded into the tiles (FP64)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int m = hi - lo + 1, nb = (m + CB - 1) / CB;
    T *td = reinterpret_cast<T *>(smem);       // [2][CB][TS]: diag entries of a block's rows
    T *tl = td + 2 * CB * TS;                  // [2][CB][TS]: late entries of the next block's rows
    T *xb = tl + 2 * CB * TS;                  // [2][CB]: right-hand side minus the early part
    T *red = xb + 2 * CB;                      // [CB][TS]: per-lane partial early sums
    T *sub = red + CB * TS;                    // [4][CB]: partial sums of 8 lanes each
    T *zbuf = sub + 4 * CB;                    // [CB]: the walker's results of the block, marker until written
    T *lateb = zbuf + CB;                      // [CB]: minus the late part of the next block's rows
    T *zs = lateb + CB;                        // [zcap]: results of this task by step
    const int zcap = tk.zcap;
    const T *tiles = reinterpret_cast<const T *>(tk.tiles) + (size_t)tk.chain_blk0[cidx] * 2 * CB * CB;
    T *mb = zs + zcap;                          // [zcap]: right-hand side term by step
    T *ms = mb + zcap;                          // [zcap]: pivot scale (1 without division)
    int4 *mi = reinterpret_cast<int4 *>(ms + zcap);   // [zcap]: slot bounds (see meta)
    int *mo = reinterpret_cast<int *>(mi + zcap);      // [zcap]: 1 if the row's outside sum is an item's
    T *ext = reinterpret_cast<T *>(tk.ext);
    auto row_of = [&](int k) { return BACKWARD ? hi - k : lo + k; };
    auto step_of = [&](int c) { return BACKWARD ? hi - c : c - lo; };
    // Slot bounds of the row at step k: x = first slot of the dependency
    // range, y = cs_late, z = cs_diag, w = end of the range (forward: early
    // [x, y), late [y, z), diag [z, w); backward: diag [x, z), late [z, y),
    // early [y, w)), its right-hand side term and pivot scale; cached in
    // shared memory by the prologue below for steps < zcap.
    // With outside items (ext), the early range covers only the sources
    // inside this task and `out` tells whether an item publishes the rest.
    auto meta_g = [&](int k, int4 &q, T &base, T &scl, int &outside) {
        const int i = row_of(k);
        const int dg = P.diag[i];
        q.x = BACKWARD ? dg + 1 : P.lu_rp[i];
        q.w = BACKWARD ? P.lu_rp[i + 1] : dg;
        outside = 0;
        if (ext) {
            const int ce = tk.cs_ext[i];
            if (BACKWARD) { outside = ce < q.w; q.w = ce; }
            else { outside = ce > q.x; q.x = ce; }
        }
        if (tk.far) {                       // bit 1: far sources summed by a partner
            const int cf = tk.cs_far[i];
            if (BACKWARD) { if (cf < q.w) { outside |= 2; q.w = cf; } }
            else if (cf > q.x) { outside |= 2; q.x = cf; }
        }
        q.y = tk.cs_late[i];
        q.z = tk.cs_diag[i];
        if (BACKWARD) base = yin[i];
        else base = (T)(sp[i] * rhs[P.perm[i]]);
        scl = DIV ? rcp[i] : T(1);
    };
    auto meta = [&](int k, int4 &q, T &base, T &scl) {
        if (k < zcap) {
            q = mi[k];
            base = mb[k];
            scl = ms[k];
        } else {
            int o_;
            meta_g(k, q, base, scl, o_);
        }
    };
    auto outside_of = [&](int k) -> int {
        if (k < zcap) return mo[k];
        int4 q;
        T b_, s_;
        int o_;
        meta_g(k, q, b_, s_, o_);
        return o_;
    };
    {
        const int mm = min(m, zcap);
        constexpr int U = 4;
        for (int k0 = threadIdx.x; k0 < mm; k0 += U * blockDim.x) {
            int4 q[U];
            T bs[U], sc[U];
            int ou[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int k = k0 + u * blockDim.x;
                if (k < mm) meta_g(k, q[u], bs[u], sc[u], ou[u]);
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int k = k0 + u * blockDim.x;
                if (k < mm) {
                    mi[k] = q[u];
                    mb[k] = bs[u];
                    ms[k] = sc[u];
                    mo[k] = ou[u];
                }
            }
        }
        __syncthreads();
    }

    // helpers: prepare block B (x - early, diag tile) and the late tile of block B + 1
    auto prepare = [&](int B) {
        if (wid < 2 || B >= nb) return;
        const int nh = nw - 2, h = wid - 2;
        T *tdb = td + (B & 1) * CB * TS, *tlb = tl + (B & 1) * CB * TS, *xbb = xb + (B & 1) * CB;
        const int k0 = B * CB, cnt = min(CB, m - k0);
        const int cnt1 = (B + 1 < nb) ? min(CB, m - k0 - CB) : 0;
        // the two tiles of block B, packed at refactorization: one coalesced
        // copy (loads first), padded rows in shared memory
        {
            const T *src = tiles + (size_t)B * 2 * CB * CB;
            const int ht = h * 32 + lane, nt = nh * 32;
            constexpr int TQ = (2 * CB * CB + 32 * 8 - 1) / (32 * 8);   // per thread with >= 8 helpers
            T tv[TQ];
#pragma unroll
            for (int q = 0; q < TQ; q++) {
                const int e = ht + q * nt;
                tv[q] = e < 2 * CB * CB ? src[e] : T(0);
            }
#pragma unroll
            for (int q = 0; q < TQ; q++) {
                const int e = ht + q * nt;
                if (e < 2 * CB * CB) {
                    const int tile = e >> 10, j = (e >> 5) & 31, sc_ = e & 31;
                    (tile ? tlb : tdb)[j * TS + sc_] = tv[q];
                }
            }
            for (int e = ht + TQ * nt; e < 2 * CB * CB; e += nt) {      // fewer helpers
                const int tile = e >> 10, j = (e >> 5) & 31, sc_ = e & 31;
                (tile ? tlb : tdb)[j * TS + sc_] = src[e];
            }
        }
        (void)cnt1;
        // early parts: a warp per row, ER rows of a helper at once (their first
        // 32 x EJ slots loaded together, then their sources, then one
        // interleaved reduction); rows with more early slots finish chunk by
        // chunk.
        for (int j0 = h; j0 < cnt; j0 += ER * nh) {
            int eb[ER], ee[ER];
            T base[ER], scl[ER], acc[ER];
            int cc[ER][EJ];
            T fv[ER][EJ];
#pragma unroll
            for (int r = 0; r < ER; r++) {
                const int j = j0 + r * nh;
                eb[r] = ee[r] = 0;
                base[r] = T(0);
                scl[r] = T(1);
                acc[r] = T(0);
                if (j < cnt) {
                    int4 mt;
                    meta(k0 + j, mt, base[r], scl[r]);
                    eb[r] = BACKWARD ? mt.y : mt.x;
                    ee[r] = BACKWARD ? mt.w : mt.y;
                }
            }
            int t0r[ER];
            auto load_chunk = [&](int r, int t0) {
                t0r[r] = t0;
#pragma unroll
                for (int q = 0; q < EJ; q++) {
                    const int t = t0 + 32 * q + lane;
                    cc[r][q] = -1;
                    fv[r][q] = T(0);
                    if (t < ee[r]) {
                        cc[r][q] = P.lu_ci[t];
                        fv[r][q] = F[t];
                    }
                }
            };
            // value of every loaded slot (inside the task from shared memory),
            // then the polls of sources not yet published, then the products
            T v[ER][EJ];
            unsigned need[ER];
            auto gather = [&](int r) {
                need[r] = 0;
#pragma unroll
                for (int q = 0; q < EJ; q++) {
                    const int c = cc[r][q];
                    v[r][q] = T(0);
                    if (c >= 0) {
                        if (c >= lo && c <= hi) {
                            const int st = step_of(c);
                            v[r][q] = st < zcap ? zs[st] : yout[c];
                        } else {
                            v[r][q] = ld_relaxed_v(yout + c);
                        }
                    }
                }
            };
            auto finish = [&](int r) {
#pragma unroll
                for (int q = 0; q < EJ; q++)
                    if (cc[r][q] >= 0 && is_marker(v[r][q])) need[r] |= 1u << q;
                if (__any_sync(FULL, need[r] != 0)) {
#pragma unroll
                    for (int q = 0; q < EJ; q++) {
                        const bool nq = (need[r] >> q) & 1u;
                        const T w = warp_wait_load(rc, yout + (nq ? cc[r][q] : 0), nq, lane);
                        if (nq) v[r][q] = w;
                    }
                }
                // FP64 instructions cost the same with idle lanes: skip the
                // rounds past the end of the row
                const int tq = ee[r] - t0r[r];
#pragma unroll
                for (int q = 0; q < EJ; q++)
                    if (32 * q < tq) acc[r] = fma(fv[r][q], v[r][q], acc[r]);
            };
#pragma unroll
            for (int r = 0; r < ER; r++) load_chunk(r, eb[r]);
#pragma unroll
            for (int r = 0; r < ER; r++) gather(r);
#pragma unroll
            for (int r = 0; r < ER; r++) finish(r);
            // longer rows: the rest in chunks of 32 x E2 slots (E2 = 16 for
            // FP32, 8 for FP64), the next chunk's slots in flight while this
            // one's sources are read
            constexpr int E2 = sizeof(T) == 4 ? 2 * EJ2 : EJ2;
#pragma unroll
            for (int r = 0; r < ER; r++) {
                int t0 = eb[r] + 32 * EJ;
                if (t0 >= ee[r]) continue;
                int c1[E2];
                T f1[E2];
                auto load2 = [&](int tb, int (&c)[E2], T (&f)[E2]) {
#pragma unroll
                    for (int q = 0; q < E2; q++) {
                        const int t = tb + 32 * q + lane;
                        c[q] = -1;
                        f[q] = T(0);
                        if (t < ee[r]) {
                            c[q] = P.lu_ci[t];
                            f[q] = F[t];
                        }
                    }
                };
                load2(t0, c1, f1);
                for (; t0 < ee[r]; t0 += 32 * E2) {
                    int c2[E2];
                    T f2[E2], w2[E2];
                    if (t0 + 32 * E2 < ee[r]) load2(t0 + 32 * E2, c2, f2);
                    unsigned nd = 0;
#pragma unroll
                    for (int q = 0; q < E2; q++) {
                        const int c = c1[q];
                        w2[q] = T(0);
                        if (c >= 0) {
                            if (c >= lo && c <= hi) {
                                const int st = step_of(c);
                                w2[q] = st < zcap ? zs[st] : yout[c];
                            } else {
                                w2[q] = ld_relaxed_v(yout + c);
                                if (is_marker(w2[q])) nd |= 1u << q;
                            }
                        }
                    }
                    if (__any_sync(FULL, nd != 0)) {
#pragma unroll
                        for (int q = 0; q < E2; q++) {
                            const bool nq = (nd >> q) & 1u;
                            const T w = warp_wait_load(rc, yout + (nq ? c1[q] : 0), nq, lane);
                            if (nq) w2[q] = w;
                        }
                    }
                    const int tq = ee[r] - t0;
#pragma unroll
                    for (int q = 0; q < E2; q++)
                        if (32 * q < tq) acc[r] = fma(f1[q], w2[q], acc[r]);
#pragma unroll
                    for (int q = 0; q < E2; q++) {
                        c1[q] = c2[q];
                        f1[q] = f2[q];
                    }
                }
            }
            // per-lane partials to shared memory; summed below across lanes
#pragma unroll
            for (int r = 0; r < ER; r++) {
                const int j = j0 + r * nh;
                if (j < cnt) red[j * TS + lane] = acc[r];
            }
        }
        // transposed reduction (a lane per row instead of a shuffle tree per
        // row: 10 FP64 instructions for the block instead of 5 per row)
        named_barrier(1, nh * 32);
        if (h < 4) {
            T s8 = T(0);
#pragma unroll
            for (int q = 0; q < 8; q++) s8 += red[lane * TS + 8 * h + q];
            sub[h * CB + lane] = s8;
        }
        named_barrier(1, nh * 32);
        if (h == 0) {
            const bool own = lane < cnt;
            int4 mt;
            T base = T(0), scl = T(1);
            int outside = 0;
            if (own) {
                meta(k0 + lane, mt, base, scl);
                outside = (ext || tk.far) ? outside_of(k0 + lane) : 0;
            }
            // the outside sum published by its item and the far sum by a
            // partner (polled; all lanes take part)
            const T xo = warp_wait_load(rc, ext + ((outside & 1) ? row_of(k0 + lane) : 0), (outside & 1) != 0, lane);
            const T *farp = reinterpret_cast<const T *>(tk.far);
            const T xf = warp_wait_load(rc, farp + ((outside & 2) ? row_of(k0 + lane) : 0), (outside & 2) != 0, lane);
            if (own) {
                T e = (sub[lane] + sub[CB + lane]) + (sub[2 * CB + lane] + sub[3 * CB + lane]);
                if (outside & 1) e += xo;
                if (outside & 2) e += xf;
                xbb[lane] = FOLD ? (base - e) * scl : base - e;
            }
        }
    };

    T marker;
    {
        const unsigned long long ones = ~0ull;
        memcpy(&marker, &ones, sizeof(T));
    }
    if (threadIdx.x < CB) {
        zbuf[threadIdx.x] = marker;
        lateb[threadIdx.x] = T(0);
    }
    prepare(0);
    __syncthreads();
    for (int b = 0; b < nb; b++) {
        const int k0 = b * CB, cnt = min(CB, m - k0);
        if (wid == 0) {
            const T *tdb = td + (b & 1) * CB * TS + lane * TS;
            const bool own = lane < cnt;
            T acc = own ? xb[(b & 1) * CB + lane] + lateb[lane] : T(0);
            T orc = T(1);
            if (DIV && !FOLD && own) {
                int4 mt;
                T bs_;
                meta(k0 + lane, mt, bs_, orc);
            }
            T z = T(0);
#pragma unroll
            for (int s = 0; s < CB; s++) {
                if (s < cnt) {
                    const T zl = (DIV && !FOLD) ? acc * orc : acc;
                    const T zb = __shfl_sync(FULL, zl, s);
                    if (lane == s) z = zl;
                    if (lane == 0) *(volatile T *)(zbuf + s) = is_marker(zb) ? T(NAN) : zb;
                    acc = fma(-tdb[s], zb, acc);
                }
            }
            if (own) {
                const int i = row_of(k0 + lane);
                if (is_marker(z)) {
                    z = T(NAN);
                    atomicExch(rc.status + ST_NONFINITE, 1);
                }
                const int k = k0 + lane;
                if (k < zcap) zs[k] = z;
                st_relaxed_v(yout + i, z);
                if (BACKWARD) {
                    const int oo = P.perm[i];
                    const double w = sp[i] * (double)z;
                    out[oo] = accumulate ? out[oo] + w : w;
                }
            }
        } else if (wid == 1) {
            // late part of block b + 1's rows, from the walker's results as they appear
            const T *tlb = tl + (b & 1) * CB * TS + lane * TS;
            T late = T(0);
            bool ok = true;
            for (int s = 0; s < cnt; s++) {
                T zb = *(volatile T *)(zbuf + s);
                long long it = 0;
                while (ok && is_marker(zb)) {           // the walker never waits: a short spin
                    if (++it > rc.spin_limit) {
                        atomicExch(rc.status + ST_TIMEOUT, 1);
                        atomicExch(rc.status + ST_ABORT, 1);
                        ok = false;
                    }
                    zb = *(volatile T *)(zbuf + s);
                }
                late = fma(-tlb[s], ok ? zb : T(0), late);
            }
            __syncwarp();
            lateb[lane] = late;
            zbuf[lane] = marker;                        // for the next block (after the barrier)
        } else {
            prepare(b + 1);
        }
        __syncthreads();
    }
}

// A pack of up to 32 single-row tasks (leaves of the elimination tree), a
// lane per row: forward phases have nothing to wait for (a leaf has no
// descendants), backward phases wait per lane on the row's ancestors.
template <typename T, bool BACKWARD, bool TRANS>
__device__ __forceinline__ void trisolve_pack(const DevPattern &P, const RunCfg &rc, const TaskCfg &tk,
                                              const T *__restrict__ F, const T *__restrict__ rcp,
                                              const double *__restrict__ rhs, const double *__restrict__ sp,
                                              const T *__restrict__ yin, T *yout, double *__restrict__ out,
                                              int accumulate, int pk, int lane) {
    constexpr bool DIV = (TRANS != BACKWARD);
    const int i = tk.pack_rows[32 * pk + lane];
    if (i < 0) return;
    const int dg = P.diag[i];
    const int tb = BACKWARD ? dg + 1 : P.lu_rp[i];
    const int te = BACKWARD ? P.lu_rp[i + 1] : dg;
    const T base = BACKWARD ? yin[i] : (T)(sp[i] * rhs[P.perm[i]]);
    const T sc = DIV ? rcp[i] : T(1);
    T acc = T(0);
    constexpr int U = 8;
    for (int t0 = tb; t0 < te; t0 += U) {
        int c[U];
        T f[U], v[U];
#pragma unroll
        for (int q = 0; q < U; q++) {
            c[q] = -1;
            f[q] = T(0);
            if (t0 + q < te) {
                c[q] = P.lu_ci[t0 + q];
                f[q] = F[t0 + q];
            }
        }
#pragma unroll
        for (int q = 0; q < U; q++) v[q] = c[q] >= 0 ? ld_relaxed_v(yout + c[q]) : T(0);
#pragma unroll
        for (int q = 0; q < U; q++) {
            if (c[q] >= 0 && is_marker(v[q])) v[q] = wait_value(rc, yout + c[q]);
            acc = fma(f[q], v[q], acc);
        }
    }
    T r = (base - acc) * sc;
    if (is_marker(r)) {
        r = T(NAN);
        atomicExch(rc.status + ST_NONFINITE, 1);
    }
    st_relaxed_v(yout + i, r);
    if (BACKWARD) {
        const int oo = P.perm[i];
        const double w = sp[i] * (double)r;
        out[oo] = accumulate ? out[oo] + w : w;
    }
}

// The sum over the slots [tb, te) of one row, F[t] times the published value
// of source lu_ci[t] (a warp per row, loads first, next chunk in flight,
// waiting on sources not yet published); every lane returns the sum.
template <typename T>
__device__ __forceinline__ T trisolve_sum(const DevPattern &P, const RunCfg &rc, const T *__restrict__ F,
                                          const T *yout, int tb, int te, int lane) {
    constexpr int Q = 8;
    auto load = [&](int t0, int (&c)[Q], T (&f)[Q]) {
#pragma unroll
        for (int q = 0; q < Q; q++) {
            const int t = t0 + 32 * q + lane;
            c[q] = -1;
            f[q] = T(0);
            if (t < te) {
                c[q] = P.lu_ci[t];
                f[q] = F[t];
            }
        }
    };
    T acc = T(0);
    int c1[Q];
    T f1[Q];
    load(tb, c1, f1);
    for (int t0 = tb; t0 < te; t0 += 32 * Q) {
        int c2[Q];
        T f2[Q], v[Q];
        if (t0 + 32 * Q < te) load(t0 + 32 * Q, c2, f2);
        unsigned need = 0;
#pragma unroll
        for (int q = 0; q < Q; q++) {
            v[q] = T(0);
            if (c1[q] >= 0) {
                v[q] = ld_relaxed_v(yout + c1[q]);
                if (is_marker(v[q])) need |= 1u << q;
            }
        }
        if (__any_sync(FULL, need != 0)) {
#pragma unroll
            for (int q = 0; q < Q; q++) {
                const bool nq = (need >> q) & 1u;
                const T w = warp_wait_load(rc, yout + (nq ? c1[q] : 0), nq, lane);
                if (nq) v[q] = w;
            }
        }
        const int tq = te - t0;
#pragma unroll
        for (int q = 0; q < Q; q++)
            if (32 * q < tq) acc = fma(f1[q], v[q], acc);
#pragma unroll
        for (int q = 0; q < Q; q++) {
            c1[q] = c2[q];
            f1[q] = f2[q];
        }
    }
    return warp_sum(acc);
}

// The outside part of one row of a CTA task: the sum over its dependencies
// in other tasks, published for the row's CTA.  Runs on warps anywhere on the
// GPU, so the long paths' CTAs only stream their own entries.
template <typename T, bool BACKWARD>
__device__ __forceinline__ void trisolve_ext(const DevPattern &P, const RunCfg &rc, const TaskCfg &tk,
                                             const T *__restrict__ F, T *yout, int i, int lane) {
    const int tb = BACKWARD ? tk.cs_ext[i] : P.lu_rp[i];
    const int te = BACKWARD ? P.lu_rp[i + 1] : tk.cs_ext[i];
    const T acc = trisolve_sum<T>(P, rc, F, yout, tb, te, lane);
    if (lane == 0) publish(rc, reinterpret_cast<T *>(tk.ext) + i, acc);
}

// A partner CTA of a CTA task: its warps sum the far sources of the task's far
// rows (those more than a few blocks back in the task), row after row in step
// order, each waiting in global memory for the rows the task's CTA publishes.
template <typename T, bool BACKWARD>
__device__ __forceinline__ void trisolve_partner(const DevPattern &P, const RunCfg &rc, const TaskCfg &tk,
                                                 const T *__restrict__ F, const T *yout, int p, int wid,
                                                 int nw, int lane) {
    const int4 pt = tk.part[p];
    for (int r = pt.z * nw + wid; r < pt.y; r += pt.w * nw) {
        const int i = tk.far_rows[pt.x + r];
        const int tb = BACKWARD ? tk.cs_far[i] : tk.cs_ext[i];
        const int te = BACKWARD ? tk.cs_ext[i] : tk.cs_far[i];
        const T acc = trisolve_sum<T>(P, rc, F, yout, tb, te, lane);
        if (lane == 0) publish(rc, reinterpret_cast<T *>(tk.far) + i, acc);
    }
}

// Packs, once per refactorization, the tiles the CTA tasks of the four solve
// phases read: for every block b of every CTA task, the diag tile (rows of
// block b, sources in block b) and the late tile (rows of block b + 1, sources
// in block b), 32 x 32 each, reciprocal pivots folded in where the phase
// divides (FP64 only: in FP32 the walker's multiply is cheap and one rounding
// fewer helps refinement).  Phases: 0 forward L (LU), 1 backward U (LU, divides), 2 forward
// U^T (LUT, divides), 3 backward L^T (LUT).  One warp per tile row.
template <typename T>
__global__ void k_pack_tiles(DevPattern P, const int *__restrict__ blk_info, int nblk,
                             const int *__restrict__ cs_fwd, const int *__restrict__ csd_fwd,
                             const int *__restrict__ cs_bwd, const int *__restrict__ csd_bwd,
                             const T *__restrict__ LU, const T *__restrict__ LUT, const T *__restrict__ rcp,
                             T *__restrict__ tiles) {
    const int lane = threadIdx.x & 31;
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= 4LL * nblk * 2 * CB) return;
    const int j = (int)(w & (CB - 1)), which = (int)((w >> 5) & 1);
    const long long pg = w >> 6;                  // phase * nblk + block
    const int ph = (int)(pg / nblk), gb = (int)(pg % nblk);
    const int lo = blk_info[3 * gb], hi = blk_info[3 * gb + 1], b = blk_info[3 * gb + 2];
    const bool bwd = ph & 1, tr = ph >= 2, div = (ph == 1 || ph == 2);
    const T *F = tr ? LUT : LU;
    T *row = tiles + w * CB;
    row[lane] = T(0);
    __syncwarp();
    const int k = CB * (b + which) + j;           // step of the tile row
    if (k >= hi - lo + 1) return;
    const int i = bwd ? hi - k : lo + k;
    const int dg = P.diag[i];
    int sb, se;
    if (!bwd) {
        const int e = cs_fwd[i], d = csd_fwd[i];
        sb = which ? e : d;
        se = which ? d : dg;
    } else {
        const int e = cs_bwd[i], d = csd_bwd[i];
        sb = which ? d : dg + 1;
        se = which ? e : d;
    }
    const T scl = (div && sizeof(T) == 8) ? rcp[i] : T(1);   // FP32 divides in the walker
    const int k0 = CB * b;
    for (int t = sb + lane; t < se; t += 32) {
        const int c = P.lu_ci[t];
        row[(bwd ? hi - c : c - lo) - k0] = F[t] * scl;
    }
}

template <typename T, bool BACKWARD, bool TRANS>
__global__ void __launch_bounds__(SWARPS * 32, 1)
k_trisolve(DevPattern P, RunCfg rc, TaskCfg tk, const T *__restrict__ F, const T *__restrict__ rcp,
           const double *__restrict__ rhs, const double *__restrict__ sp, const T *__restrict__ yin,
           T *yout, double *__restrict__ out, int accumulate) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int e = rc.sched->epoch + 1;
    const long long tbase = (long long)rc.trace_stride * (TRANS ? (BACKWARD ? TR_TBWD : TR_TFWD)
                                                                : (BACKWARD ? TR_BWD : TR_FWD));
    if ((int)blockIdx.x < tk.nchain) {            // a long task on this whole CTA
        const int tid = tk.chain_task[blockIdx.x];
        const int item = tk.ntasks + blockIdx.x;
        if (wid == 0) trace_mark(rc, tbase, item, 0, lane);
        trisolve_chain<T, BACKWARD, TRANS>(P, rc, tk, blockIdx.x, tk.task_lo[tid], tk.task_hi[tid], F, rcp, rhs, sp,
                                           yin, yout, out, accumulate, smem);
        if (wid == 0) trace_mark(rc, tbase, item, 1, lane);
        if (lane == 0) finish_launch(rc, e);
        return;
    }
    if ((int)blockIdx.x < tk.nchain + tk.npart) {  // a partner of a CTA task
        trisolve_partner<T, BACKWARD>(P, rc, tk, F, yout, (int)blockIdx.x - tk.nchain, wid, blockDim.x >> 5, lane);
        if (lane == 0) finish_launch(rc, e);
        return;
    }
    T *loc = reinterpret_cast<T *>(smem) + (size_t)wid * tk.cap;
    const int *order = BACKWARD ? tk.order_b : tk.order_f;
    for (;;) {
        const int slot = claim_row(rc, lane);
        if (slot >= tk.ntasks) break;
        trace_mark(rc, tbase, slot, 0, lane);
        const int tid = order[slot];
        if (tid < 0)
            trisolve_pack<T, BACKWARD, TRANS>(P, rc, tk, F, rcp, rhs, sp, yin, yout, out, accumulate, -1 - tid,
                                              lane);
        else if (tid >= tk.ext_base)
            trisolve_ext<T, BACKWARD>(P, rc, tk, F, yout, tk.ext_rows[tid - tk.ext_base], lane);
        else
            trisolve_task<T, BACKWARD, TRANS>(P, rc, tk, F, rcp, rhs, sp, yin, yout, out, accumulate, tid, loc,
                                              lane);
        trace_mark(rc, tbase, slot, 1, lane);
    }
    if (lane == 0) finish_launch(rc, e);
}

// ---------------------------------------------------------------------------
// FP64 residual rho = b - A x (or b - A^T x), 8 lanes per row, fused with
// ||rho||_inf, ||x||_inf, ||b||_inf.
__global__ void __launch_bounds__(RTHREADS)
k_resid(DevPattern P, const double *__restrict__ aval, const double *__restrict__ b,
        const double *__restrict__ x, double *__restrict__ rho,
        unsigned long long *norms, int transpose) {
    __shared__ double red[RTHREADS / 32];
    const int sub = threadIdx.x & 7;
    const long long step = (long long)gridDim.x * (blockDim.x >> 3);
    double rmax = 0.0, xmax = 0.0, bmax = 0.0;
    for (long long r0 = ((long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) >> 3; r0 < P.n; r0 += step) {
        const int r = (int)r0 + ((threadIdx.x & 31) >> 3);
        double acc = 0.0;
        if (r < P.n) {
            if (!transpose) {
                for (int p = P.a_rp[r] + sub; p < P.a_rp[r + 1]; p += 8) acc += aval[p] * x[P.a_ci[p]];
            } else {
                for (int q = P.at_rp[r] + sub; q < P.at_rp[r + 1]; q += 8) {
                    const int k = P.at_src[q];
                    acc += aval[k] * x[P.a_row[k]];
                }
            }
        }
        for (int o = 4; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
        if (r < P.n && sub == 0) {
            const double br = b[r];
            const double rv = br - acc;
            rho[r] = rv;
            rmax = fmax(rmax, abs_nan_inf(rv));
            xmax = fmax(xmax, abs_nan_inf(x[r]));
            bmax = fmax(bmax, abs_nan_inf(br));
        }
    }
    rmax = cta_max(rmax, red);
    xmax = cta_max(xmax, red);
    bmax = cta_max(bmax, red);
    if (threadIdx.x == 0) {
        atomic_max_nonneg(norms + NM_RMAX, rmax);
        atomic_max_nonneg(norms + NM_XMAX, xmax);
        atomic_max_nonneg(norms + NM_BMAX, bmax);
    }
}

// ---------------------------------------------------------------------------
// FGMRES building blocks (FP64): y = A x or A^T x, multi-dot products,
// vector updates with coefficients held on the device.

__global__ void k_spmv(DevPattern P, const double *__restrict__ aval, const double *__restrict__ x,
                       double *__restrict__ y, int transpose) {
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int sub = threadIdx.x & 7;
    double acc = 0.0;
    if (r < P.n) {
        if (!transpose) {
            for (int p = P.a_rp[r] + sub; p < P.a_rp[r + 1]; p += 8) acc += aval[p] * x[P.a_ci[p]];
        } else {
            for (int q = P.at_rp[r] + sub; q < P.at_rp[r + 1]; q += 8) {
                const int k = P.at_src[q];
                acc += aval[k] * x[P.a_row[k]];
            }
        }
    }
    for (int o = 4; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if (r < P.n && sub == 0) y[r] = acc;
}

// part[b * k + q] = sum over this block's share of i of V[q][i] * w[i]
__global__ void k_mdot(const double *__restrict__ V, long long ld, int k, const double *__restrict__ w,
                       int n, double *__restrict__ part) {
    __shared__ double red[8];
    for (int q = 0; q < k; q++) {
        double acc = 0.0;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x)
            acc += V[q * ld + i] * w[i];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q2 = 0; q2 < (int)(blockDim.x >> 5); q2++) t += red[q2];
            part[(long long)blockIdx.x * k + q] = t;
        }
        __syncthreads();
    }
}

// h[q] (+)= sum_b part[b * k + q]
__global__ void k_mdot_fin(const double *__restrict__ part, int nblk, int k, double *__restrict__ h,
                           int add) {
    const int q = blockIdx.x;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += part[(long long)b * k + q];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q2 = 0; q2 < (int)(blockDim.x >> 5); q2++) t += red[q2];
        h[q] = add ? h[q] + t : t;
    }
}

// w[i] += sgn * sum_q c[q] V[q][i]
__global__ void k_vcomb(double *__restrict__ w, const double *__restrict__ V, long long ld, int k,
                        const double *__restrict__ c, double sgn, int n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = 0.0;
    for (int q = 0; q < k; q++) acc += c[q] * V[q * ld + i];
    w[i] += sgn * acc;
}

// v[i] = w[i] * s  (s = 1 / norm, computed on the host)
__global__ void k_vscale(double *__restrict__ v, const double *__restrict__ w, double s, int n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = w[i] * s;
}

// ---------------------------------------------------------------------------
// Jacobi sweeps for approximate triangular solves (Sec. 6: iterative
// approximation of the triangular solves, after Anzt, Chow and Dongarra 2015).
// One sweep of one factor, 8 lanes per row of the factor storage F (LU, or
// its transposed copy LUT for the transposed system):
//   out[i] = (rhs[i] - sum over the slots on one side of the diagonal of
//             F[t] * in[col t]) * (SCALE ? 1 / pivot_i : 1)
// RIGHT: the slots right of the diagonal (U, or L^T), else left (L, or U^T).
// in == nullptr is the zero vector (the first term of the iteration).  Every
// row is independent: a sweep is one sparse product with no dependency chain.
template <typename T, bool RIGHT, bool SCALE>
__global__ void k_jacobi(DevPattern P, const T *__restrict__ F, const T *__restrict__ rcp,
                         const T *__restrict__ rhs, const T *__restrict__ in, T *__restrict__ out) {
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int sub = threadIdx.x & 7;
    T acc = T(0);
    if (r < P.n && in != nullptr) {
        const int tb = RIGHT ? P.diag[r] + 1 : P.lu_rp[r];
        const int te = RIGHT ? P.lu_rp[r + 1] : P.diag[r];
        for (int t = tb + sub; t < te; t += 8) acc += F[t] * in[P.lu_ci[t]];
    }
    for (int o = 4; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if (r < P.n && sub == 0) {
        T v = rhs[r] - acc;
        if (SCALE) v *= rcp[r];
        out[r] = v;
    }
}

// entry and exit of an approximate solve: c = S P b (factor precision), and
// x[perm[i]] = s_i z_i (or +=, for refinement)
template <typename T>
__global__ void k_perm_in(DevPattern P, const double *__restrict__ sp, const double *__restrict__ b,
                          T *__restrict__ c) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P.n) c[i] = (T)(sp[i] * b[P.perm[i]]);
}
// row permutation Q of a value-aware context: out[k] = in[idx[k]] (gather) and
// out[idx[k]] = in[k] (scatter), for values (nnz) and vectors (n)
__global__ void k_gather(long long m, const int *__restrict__ idx, const double *__restrict__ in,
                         double *__restrict__ out) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < m) out[k] = in[idx[k]];
}
__global__ void k_scatter(long long m, const int *__restrict__ idx, const double *__restrict__ in,
                          double *__restrict__ out) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < m) out[idx[k]] = in[k];
}

template <typename T>
__global__ void k_perm_out(DevPattern P, const double *__restrict__ sp, const T *__restrict__ z,
                           double *__restrict__ x, int accumulate) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P.n) {
        const double v = sp[i] * (double)z[i];
        if (accumulate) x[P.perm[i]] += v; else x[P.perm[i]] = v;
    }
}

// ===========================================================================
// Batched same-pattern systems (batch innermost): value k of system s sits at
// k * B + s, vector entry i of system s at i * B + s.  Work items are (row or
// task, system), claimed in topological order with every system of a row or
// task together; each item runs the single-system body (a warp per row or
// task of one system, the row's columns across the lanes) through Strided
// accessors.  The B systems' independent dependency chains run side by side,
// so the batch fills the GPU that one latency-bound system leaves idle.

// per-(row, system) scaling, ||A||_inf per system
__global__ void k_bscale(DevPattern P, int B, const double *__restrict__ aval, double *__restrict__ s_orig,
                         double *__restrict__ sp, unsigned long long *norms, int *status, int equil) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)P.n * B) return;
    const int r = (int)(gid / B), sy = (int)(gid % B);
    double rmax = 0.0, rsum = 0.0;
    bool bad = false;
    for (int p = P.a_rp[r]; p < P.a_rp[r + 1]; p++) {
        const double a = fabs(aval[(long long)p * B + sy]);
        if (!isfinite(a)) bad = true;
        rmax = fmax(rmax, a);
        rsum += a;
    }
    double s = 1.0;
    if (equil && !bad && rmax > 0.0) s = ldexp(1.0, -floor_half(ilogb(rmax)));
    s_orig[(long long)r * B + sy] = s;
    sp[(long long)P.iperm[r] * B + sy] = s;
    if (bad) atomicExch(status + ST_NONFINITE, 1);
    else atomic_max_nonneg(norms + (long long)NM_ANORM * B + sy, rsum);
}

__global__ void k_bamax(DevPattern P, int B, const double *__restrict__ aval, const double *__restrict__ s_orig,
                        unsigned long long *norms) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)P.n * B) return;
    const int r = (int)(gid / B), sy = (int)(gid % B);
    const double sr = s_orig[(long long)r * B + sy];
    double m = 0.0, csum = 0.0;
    for (int p = P.a_rp[r]; p < P.a_rp[r + 1]; p++)
        m = fmax(m, fabs(aval[(long long)p * B + sy]) * sr * s_orig[(long long)P.a_ci[p] * B + sy]);
    for (int q = P.at_rp[r]; q < P.at_rp[r + 1]; q++) csum += fabs(aval[(long long)P.at_src[q] * B + sy]);
    if (isfinite(m)) atomic_max_nonneg(norms + (long long)NM_AMAX * B + sy, m);
    if (isfinite(csum)) atomic_max_nonneg(norms + (long long)NM_A1NORM * B + sy, csum);
}

// Batched refactorization: work items (row, system), rows deepest first and
// every system of a row together; each item is the single-system row body on
// that system's batch-innermost arrays (a warp per row of one system, its
// columns across the lanes).
template <typename T>
__global__ void __launch_bounds__(WARPS * 32, 2)
k_brefactor(DevPattern P, RunCfg rc, int B, const double *__restrict__ aval, const double *__restrict__ sp,
            const unsigned long long *__restrict__ norms, T *LU, T *LUT, T *rcp, double tau_rel) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T *sval = reinterpret_cast<T *>(smem) + (size_t)wid * rc.cap;
    int *scol = reinterpret_cast<int *>(smem + (size_t)nw * rc.cap * sizeof(T)) + (size_t)wid * rc.cap;
    const int e = rc.sched->epoch + 1;
    const int gw = blockIdx.x * nw + wid;
    for (;;) {
        const int slot = claim_row(rc, lane);
        if (slot >= P.n * B) break;
        const int i = P.order_f[slot / B], sy = slot % B;
        const double tau = tau_rel * __longlong_as_double((long long)norms[(long long)NM_AMAX * B + sy]);
        refactor_row<T>(P, rc, Strided<const double>{aval, B, sy}, Strided<const double>{sp, B, sy},
                        Strided<T>{LU, B, sy}, Strided<T>{LUT, B, sy}, Strided<T>{rcp, B, sy}, tau, i, sval,
                        scol, rc.cap, gw, lane);
    }
    if (lane == 0) finish_launch(rc, e);
}

// Batched triangular solves over tasks (see k_trisolve for the phases).
template <typename T, bool BACKWARD, bool TRANS>
__global__ void __launch_bounds__(WARPS * 32, 2)
k_btrisolve(DevPattern P, RunCfg rc, TaskCfg tk, int B, const T *__restrict__ F, const T *__restrict__ rcp,
            const double *__restrict__ rhs, const double *__restrict__ sp, const T *__restrict__ yin, T *yout,
            double *__restrict__ out, int accumulate) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T *loc = reinterpret_cast<T *>(smem) + (size_t)wid * tk.cap;
    const int e = rc.sched->epoch + 1;
    const int *order = BACKWARD ? tk.order_b : tk.order_topo;
    for (;;) {
        const int slot = claim_row(rc, lane);
        if (slot >= tk.ntasks * B) break;
        const int tid = order[slot / B], sy = slot % B;
        trisolve_task<T, BACKWARD, TRANS>(P, rc, tk, Strided<const T>{F, B, sy}, Strided<const T>{rcp, B, sy},
                                          Strided<const double>{rhs, B, sy}, Strided<const double>{sp, B, sy},
                                          Strided<const T>{yin, B, sy}, Strided<T>{yout, B, sy},
                                          Strided<double>{out, B, sy}, accumulate, tid, loc, lane);
    }
    if (lane == 0) finish_launch(rc, e);
}

// ===========================================================================
// Uneven batch: several contexts (different patterns) in one persistent
// launch per phase.  Work items are (system, row) or (system, task), ordered
// by level across systems (a topological order of every system), claimed from
// one counter; each item reads its system's structures from a table.

struct QSys {
    DevPattern P;
    TaskCfg tk;
    TaskCfg tkc[4];                    // CTA tasks of each solve phase (forward, backward, transposed)
    void *LU, *LUT, *rcp, *y;          // factor, transposed factor, reciprocal pivots, 2n work
    const double *sp;                  // scaling in permuted order
    const unsigned long long *norms;   // the context's norm words (NM_AMAX for tau)
    const double *values, *b, *rho;    // matrix values, right-hand side, residual
    double *x;                         // solution (assigned, then accumulated)
    const double *g;                   // transposed right-hand side
    double *lam;                       // transposed solution
    double tau_rel;
    int n;
};

template <typename T>
__global__ void __launch_bounds__(WARPS * 32, 2)
k_qrefactor(const QSys *__restrict__ sys, const int2 *__restrict__ items, int nitems, RunCfg rc) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T *sval = reinterpret_cast<T *>(smem) + (size_t)wid * rc.cap;
    int *scol = reinterpret_cast<int *>(smem + (size_t)nw * rc.cap * sizeof(T)) + (size_t)wid * rc.cap;
    const int e = rc.sched->epoch + 1;
    const int gw = blockIdx.x * nw + wid;
    for (;;) {
        const int slot = claim_row(rc, lane);
        if (slot >= nitems) break;
        const int2 it = items[slot];
        const QSys &q = sys[it.x];
        const double tau = q.tau_rel * __longlong_as_double((long long)q.norms[NM_AMAX]);
        refactor_row<T>(q.P, rc, q.values, q.sp, (T *)q.LU, (T *)q.LUT, (T *)q.rcp, tau, it.y, sval, scol,
                        rc.cap, gw, lane);
    }
    if (lane == 0) finish_launch(rc, e);
}

// phase: forward / backward; TRANS: transposed; refine: right-hand side is rho
// and the solution is accumulated
template <typename T, bool BACKWARD, bool TRANS>
__global__ void __launch_bounds__(WARPS * 32, 2)
k_qtrisolve(const QSys *__restrict__ sys, const int2 *__restrict__ items, int nitems, RunCfg rc, int refine,
            int tcap, const int2 *__restrict__ chains, int nch) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int e = rc.sched->epoch + 1;
    if ((int)blockIdx.x < nch) {            // a long task of one system on this whole CTA
        const int2 ch = chains[blockIdx.x];
        const QSys &q = sys[ch.x];
        const TaskCfg &tk = q.tkc[(TRANS ? 2 : 0) + (BACKWARD ? 1 : 0)];
        const int tid = tk.chain_task[ch.y];
        T *y = (T *)q.y, *z = y + q.n;
        const T *F = (const T *)(TRANS ? q.LUT : q.LU);
        if (BACKWARD)
            trisolve_chain<T, true, TRANS>(q.P, rc, tk, ch.y, tk.task_lo[tid], tk.task_hi[tid], F,
                                           (const T *)q.rcp, nullptr, q.sp, y, z, TRANS ? q.lam : q.x,
                                           TRANS ? 0 : refine, smem);
        else
            trisolve_chain<T, false, TRANS>(q.P, rc, tk, ch.y, tk.task_lo[tid], tk.task_hi[tid], F,
                                            (const T *)q.rcp, TRANS ? q.g : (refine ? q.rho : q.b), q.sp,
                                            nullptr, y, nullptr, 0, smem);
        if (lane == 0) finish_launch(rc, e);
        return;
    }
    // per-warp slice of the queue-wide capacity (at least every system's tk.cap)
    T *loc = reinterpret_cast<T *>(smem) + (size_t)wid * tcap;
    for (;;) {
        const int slot = claim_row(rc, lane);
        if (slot >= nitems) break;
        const int2 it = items[slot];
        const QSys &q = sys[it.x];
        T *y = (T *)q.y, *z = y + q.n;
        const T *F = (const T *)(TRANS ? q.LUT : q.LU);
        const double *rhs = TRANS ? q.g : (refine ? q.rho : q.b);
        double *out = TRANS ? q.lam : q.x;
        if (BACKWARD)
            trisolve_task<T, true, TRANS>(q.P, rc, q.tk, F, (const T *)q.rcp, (const double *)nullptr, q.sp,
                                          (const T *)y, z, out, TRANS ? 0 : refine, it.y, loc, lane);
        else
            trisolve_task<T, false, TRANS>(q.P, rc, q.tk, F, (const T *)q.rcp, rhs, q.sp, (const T *)nullptr, y,
                                           (double *)nullptr, 0, it.y, loc, lane);
    }
    if (lane == 0) finish_launch(rc, e);
}

// omega of one system from its norm words
__global__ void k_omega(const unsigned long long *__restrict__ norms, double *__restrict__ out) {
    const double an = __longlong_as_double((long long)norms[NM_ANORM]);
    const double xm = __longlong_as_double((long long)norms[NM_XMAX]);
    const double bm = __longlong_as_double((long long)norms[NM_BMAX]);
    const double rm = __longlong_as_double((long long)norms[NM_RMAX]);
    const double den = an * xm + bm;
    const double w = den > 0.0 ? rm / den : (rm > 0.0 ? INFINITY : 0.0);
    *out = isnan(w) ? INFINITY : w;        // inf / inf: a non-finite entry somewhere
}

// rho = b - A x (or A^T x) per system, with per-system norms
__global__ void k_bresid(DevPattern P, int B, const double *__restrict__ aval, const double *__restrict__ b,
                         const double *__restrict__ x, double *__restrict__ rho, unsigned long long *norms,
                         int transpose) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)P.n * B) return;
    const int r = (int)(gid / B), sy = (int)(gid % B);
    double acc = 0.0;
    if (!transpose) {
        for (int p = P.a_rp[r]; p < P.a_rp[r + 1]; p++)
            acc += aval[(long long)p * B + sy] * x[(long long)P.a_ci[p] * B + sy];
    } else {
        for (int q = P.at_rp[r]; q < P.at_rp[r + 1]; q++) {
            const int k = P.at_src[q];
            acc += aval[(long long)k * B + sy] * x[(long long)P.a_row[k] * B + sy];
        }
    }
    const double br = b[gid];
    const double rv = br - acc;
    rho[gid] = rv;
    atomic_max_nonneg(norms + (long long)NM_RMAX * B + sy, abs_nan_inf(rv));
    atomic_max_nonneg(norms + (long long)NM_XMAX * B + sy, abs_nan_inf(x[gid]));
    atomic_max_nonneg(norms + (long long)NM_BMAX * B + sy, abs_nan_inf(br));
}

// dA_k = -lam[row_k] x[col_k]
__global__ void k_adjoint(DevPattern P, const double *__restrict__ lam, const double *__restrict__ x,
                          double *__restrict__ dA) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P.nnz_a) dA[k] = -lam[P.a_row[k]] * x[P.a_ci[k]];
}

template <typename T>
__global__ void k_bexport(const T *__restrict__ LU, const int *__restrict__ slot, int B, int sys,
                          double *__restrict__ out, long long m) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < m) out[k] = (double)LU[(long long)slot[k] * B + sys];
}

template <typename T>
__global__ void k_export(const T *__restrict__ LU, const int *__restrict__ slot, double *__restrict__ out,
                         long long m) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < m) out[k] = (double)LU[slot[k]];
}

}  // namespace kkt

// ===========================================================================
// host side

using namespace kkt;

struct kkt_ctx {
    Analysis an;
    kkt_options opt{};
    bool host_only = true;
    int dev = -1;
    // device memory
    DevPattern P{};
    RunCfg rc{};
    int *d_ints = nullptr;
    void *d_lu = nullptr, *d_lut = nullptr, *d_rcp = nullptr;
    double *d_s = nullptr, *d_sp = nullptr, *d_rho = nullptr;
    void *d_y = nullptr;
    int *d_status = nullptr;
    unsigned long long *d_norms = nullptr;
    Sched *d_sched = nullptr;
    void *d_scratch = nullptr;
    void *d_maps = nullptr;
    int *d_task_orders = nullptr;
    unsigned long long *d_trace = nullptr;
    // caller-view copies of the pattern (built on first export)
    mutable std::vector<int> view_rp, view_ci, view_slot;
    // FGMRES workspace (refine modes fgmres / auto): V[(m+1) n], Z[m n], w[n],
    // partial dots, coefficients
    double *d_krylov = nullptr;
    int kry_m = 0, kry_blocks = 0;
    // batched workspace (capacity max_batch): factors, transposed factors,
    // reciprocal pivots, scaling, work vectors and norms, batch innermost
    int bcap = 0;
    void *b_lu = nullptr, *b_lut = nullptr, *b_rcp = nullptr, *b_y = nullptr;
    double *b_s = nullptr, *b_sp = nullptr, *b_rho = nullptr;
    unsigned long long *b_norms = nullptr, *hb_norms = nullptr;
    const double *b_values = nullptr;
    int b_factored = 0;
    int *d_view_slot = nullptr;
    TaskCfg tk{};             // all tasks (batched and queued solves)
    TaskCfg tk1{};            // single-system solves: CTA tasks + warp tasks
    const int *cs_fwd = nullptr, *csd_fwd = nullptr, *cs_bwd = nullptr, *csd_bwd = nullptr;
    const int *blk_info = nullptr;   // per block of the CTA tasks: lo, hi, block index
    int nblk = 0;                    // blocks of all CTA tasks
    void *d_tiles = nullptr;         // packed tiles, 4 phases x nblk x 2 x 32 x 32
    bool tiles_fresh = false;        // d_tiles match the current factors
    std::vector<int> chain_h;        // CTA tasks of the single-system solves (host copy)
    // outside items of CTA-task rows: splits and rows per direction, order lengths
    const int *ce_fwd = nullptr, *ce_bwd = nullptr, *xr_fwd = nullptr, *xr_bwd = nullptr;
    // far sources of CTA-task rows summed by partner CTAs: slot bounds, far
    // rows in step order, partner tables (see the task setup in upload)
    const int *cf_fwd = nullptr, *cf_bwd = nullptr, *fr_fwd = nullptr, *fr_bwd = nullptr;
    const int4 *part_fwd = nullptr, *part_bwd = nullptr;
    int npart = 0;
    int nord_f = 0, nord_b = 0;
    size_t solve_smem = 0, bsolve_smem = 0;
    unsigned long long *h_norms = nullptr;  // pinned
    int grid = 0, solve_grid = 0, bsolve_grid = 0, cta_warps = WARPS, solve_warps = SWARPS, cap = 0;
    size_t smem = 0, device_bytes = 0;
    int rgrid = 0;                   // CTAs of k_refactor
    size_t rsmem = 0;                // shared memory of k_refactor (big and small warp rows)
    long long nnz_lu = 0;
    std::vector<int> at_rp, at_src;
    const double *values = nullptr;  // values of the current factorization (caller-owned)
    // Value-aware row permutation (kkt_analyze_values / options.user_row_perm):
    // the context factors Q A, row j of which is row q[j] of the caller's A.
    // Values, right-hand sides and transposed solutions cross the boundary
    // through gather/scatter kernels; all other work sees Q A.
    bool rowperm = false;
    std::vector<int> q, qmap;        // q[j]: row of A; qmap[k]: entry of A stored at entry k of Q A
    int *d_q = nullptr, *d_qmap = nullptr;
    double *d_qvals = nullptr;       // values of Q A (nnz)
    double *d_qvec = nullptr;        // 2 n: Q b, and Q lambda
    double *d_qdA = nullptr;         // gradient on the entries of Q A (nnz)
    void *d_dense = nullptr;         // dense root block (dense_rows x dense_ld words)
    int *d_dense_ctl = nullptr;      // k_dense_lu: a published flag per block column
    int dense_ld = 0, dense_grid = 0;   // dense_grid: CTAs (block columns) of k_dense_lu
    int cap_r = 0;                   // row capacity of k_refactor's small warps
    int far_rows = 0;                // rows of CTA solve tasks whose far sources a partner sums
    bool factored = false;
    int last_iters = 0;
    double last_omega = -1.0;
    double tau_rel = 0.0;
    double auto_ratio = 0.5;  // refine mode auto: classic steps while omega falls at least this much
    long long launches = 0;  // kernels launched by this context
};

static thread_local std::string g_last_error;

namespace kkt {
void set_last_error(const std::string &msg) { g_last_error = msg; }
}  // namespace kkt

static kkt_status cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return KKT_ERR_CUDA;
}
#define CK(call)                                                   \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return cuda_fail(_e, #call);        \
    } while (0)

namespace {
// A named range around every entry point for profilers (NVTX; costs a few ns
// when no profiler is attached).
struct ApiRange {
    explicit ApiRange(const char *name) { nvtxRangePushA(name); }
    ~ApiRange() { nvtxRangePop(); }
};

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

inline int blocks_for(long long threads, int bs) { return (int)((threads + bs - 1) / bs); }
// CTAs of the row-norm kernels (k_scale, k_amax, k_resid): 8 lanes per row,
// grid-stride beyond 2,048 CTAs, so the per-CTA atomics stay few
inline int norm_blocks(long long n) { return std::max(1, std::min(blocks_for(8 * n, RTHREADS), 2048)); }

}  // namespace

// Raise a kernel's dynamic shared-memory limit on the current device to at
// least `bytes`.  The limit belongs to the kernel, not to a context, so it is
// only ever raised: a context created later with smaller needs must not break
// the launches of one created earlier.
cudaError_t kkt::ensure_smem(const void *f, size_t bytes) {
    static std::mutex m;
    static std::map<std::pair<const void *, int>, size_t> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(m);
    size_t &have = done[{f, dev}];
    if (bytes <= have) return cudaSuccess;
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
}

// The entry points below have C linkage through their declarations in kkt.h.

void kkt_default_options(kkt_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->factor_fp32 = 0;
    o->equilibrate = 1;
    o->ordering = KKT_ORDER_AMD;
    o->user_perm = nullptr;
    o->refine_mode = KKT_REFINE_CLASSIC;
    o->fgmres_restart = 20;
    o->max_refine = 20;
    o->tol = 1e-14;
    o->pivot_tau_rel = 0.0;
    o->spin_limit = 4000000;
    o->device = 0;
    o->max_batch = 1;
    o->cta_warps = 0;
    o->refactor_ctas = 0;
    o->solve_ctas = 0;
    o->update_map_budget = 0;
    o->trace = 0;
    o->unpublished_row = -1;
    o->poll_ns_max = 0;
    o->refactor_big_warps = 0;
    o->symmetric = 0;
    o->jacobi_sweeps = 8;
    o->user_row_perm = nullptr;
    o->dense_block = 0;
    o->refactor_row_cap = 0;
    o->refine_auto_ratio = 0.0;
    o->solve_far_blocks = 0;
    o->solve_far_ctas = 0;
}

const char *kkt_status_string(kkt_status s) {
    switch (s) {
        case KKT_OK: return "ok";
        case KKT_ERR_ARG: return "invalid argument";
        case KKT_ERR_PATTERN: return "malformed pattern";
        case KKT_ERR_ALLOC: return "allocation failed";
        case KKT_ERR_CUDA: return "CUDA error";
        case KKT_ERR_NONFINITE: return "non-finite value";
        case KKT_ERR_NOT_CONVERGED: return "refinement did not converge";
        case KKT_ERR_TIMEOUT: return "device wait timed out";
        case KKT_ERR_STATE: return "call out of order";
        case KKT_ERR_INTERNAL: return "internal error";
        case KKT_WARN_PERTURBED: return "perturbed pivots";
    }
    return "unknown status";
}

const char *kkt_last_error(void) { return g_last_error.c_str(); }

static kkt_status upload(kkt_ctx *c) {
    Analysis &a = c->an;
    const int n = a.n;
    const long long nnza = (long long)a.a_ci.size();
    const long long nlu = (long long)a.lu_ci.size();
    c->nnz_lu = nlu;
    // transpose of the user pattern: entry index of each (row, col) by column
    c->at_rp.assign(n + 1, 0);
    for (long long k = 0; k < nnza; k++) c->at_rp[a.a_ci[k] + 1]++;
    for (int i = 0; i < n; i++) c->at_rp[i + 1] += c->at_rp[i];
    c->at_src.resize(nnza);
    {
        std::vector<int> f(c->at_rp.begin(), c->at_rp.end() - 1);
        for (long long k = 0; k < nnza; k++) c->at_src[f[a.a_ci[k]]++] = (int)k;
    }
    // claim queues of the single-system refactorization (see k_refactor):
    // rows longer than the small per-warp buffer go to the big warps; rows
    // with no such row below them in the elimination tree come first
    const int cap_s = std::min(((std::max(a.max_row, 32) + 31) / 32) * 32, 1024);
    // the single-system refactorization's per-warp row capacity (an option)
    const int cap_r = c->opt.refactor_row_cap > 0
                          ? std::min(((std::max(c->opt.refactor_row_cap, 32) + 31) / 32) * 32,
                                     ((std::max(a.max_row, 32) + 31) / 32) * 32)
                          : cap_s;
    c->cap_r = cap_r;
    std::vector<int> ord_free, ord_long, ord_rest;
    {
        std::vector<char> is_long(n), below(n, 0);      // below: a long row in the subtree, excluding itself
        for (int r = 0; r < n; r++) is_long[r] = a.lu_rp[r + 1] - a.lu_rp[r] > cap_r;
        for (int r = 0; r < n; r++)                      // children before parents (postorder labels)
            if (a.parent[r] >= 0 && (below[r] || is_long[r])) below[a.parent[r]] = 1;
        ord_free.reserve(n);
        for (int r : a.order_f)
            (is_long[r] ? ord_long : below[r] ? ord_rest : ord_free).push_back(r);
    }
    struct Arr { const int *h; long long m; const int **dst; };
    std::vector<Arr> arrs = {
        {a.a_rp.data(), n + 1, &c->P.a_rp},     {a.a_ci.data(), nnza, &c->P.a_ci},
        {a.a_row.data(), nnza, &c->P.a_row},    {c->at_rp.data(), n + 1, &c->P.at_rp},
        {c->at_src.data(), nnza, &c->P.at_src}, {a.perm.data(), n, &c->P.perm},
        {a.iperm.data(), n, &c->P.iperm},       {a.lu_rp.data(), n + 1, &c->P.lu_rp},
        {a.lu_ci.data(), nlu, &c->P.lu_ci},     {a.diag.data(), n, &c->P.diag},
        {a.src.data(), nlu, &c->P.src},         {a.tpos.data(), nlu, &c->P.tpos},
        {a.order_f.data(), n, &c->P.order_f},   {a.order_b.data(), n, &c->P.order_b},
        {ord_free.data(), (long long)ord_free.size(), &c->P.order_free},
        {ord_long.data(), (long long)ord_long.size(), &c->P.order_long},
        {ord_rest.data(), (long long)ord_rest.size(), &c->P.order_rest},
        {a.task_lo.data(), (long long)a.task_lo.size(), &c->tk.task_lo},
        {a.task_hi.data(), (long long)a.task_hi.size(), &c->tk.task_hi},
    };
    long long total = 0;
    for (auto &r : arrs) total += (r.m + 31) / 32 * 32;
    CK(cudaMalloc(&c->d_ints, total * sizeof(int)));
    long long off = 0;
    for (auto &r : arrs) {
        int *d = c->d_ints + off;
        CK(cudaMemcpy(d, r.h, r.m * sizeof(int), cudaMemcpyHostToDevice));
        *r.dst = d;
        off += (r.m + 31) / 32 * 32;
    }
    c->device_bytes = total * sizeof(int);
    c->P.n = n;
    c->P.nnz_a = nnza;
    c->P.n_free = (int)ord_free.size();
    c->P.n_long = (int)ord_long.size();
    c->P.n_rest = (int)ord_rest.size();
    c->P.dense_lo = n - a.dense_rows;

    const bool f32 = c->opt.factor_fp32 != 0;
    const size_t tsz = f32 ? sizeof(float) : sizeof(double);
    CK(cudaMalloc(&c->d_lu, nlu * tsz + 64));     // + 64: 16-byte copies may round up past the end
    CK(cudaMalloc(&c->d_lut, nlu * tsz));
    CK(cudaMalloc(&c->d_rcp, (size_t)n * tsz));
    CK(cudaMalloc(&c->d_s, n * sizeof(double)));
    CK(cudaMalloc(&c->d_sp, n * sizeof(double)));
    CK(cudaMalloc(&c->d_rho, n * sizeof(double)));
    CK(cudaMalloc(&c->d_y, 6 * (size_t)n * sizeof(double)));   // y, z, outside sums, far sums (fwd, bwd)
    CK(cudaMalloc(&c->d_status, ST_WORDS * sizeof(int)));
    CK(cudaMalloc(&c->d_norms, NM_WORDS * sizeof(unsigned long long)));
    CK(cudaMalloc(&c->d_sched, sizeof(Sched)));
    CK(cudaMemset(c->d_status, 0, ST_WORDS * sizeof(int)));
    CK(cudaMemset(c->d_norms, 0, NM_WORDS * sizeof(unsigned long long)));
    CK(cudaMemset(c->d_sched, 0, sizeof(Sched)));
    CK(cudaMallocHost(&c->h_norms, NM_WORDS * sizeof(unsigned long long)));
    c->device_bytes += 2 * nlu * tsz + (size_t)n * tsz + 5 * n * sizeof(double) + 256;

    // persistent grids: as many CTAs as fit on the device at once, unless the
    // options fix the CTA count; a grid never exceeds one warp per row
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
    c->cta_warps = c->opt.cta_warps > 0 ? std::min(c->opt.cta_warps, WARPS) : WARPS;
    const int nw = c->cta_warps;
    const int cap = cap_s;
    c->cap = cap;
    c->smem = (size_t)nw * cap * (tsz + sizeof(int));      // batched kernels: uniform per-warp rows
    int per_sm = 0;
    if (f32) {
        CK(ensure_smem((const void *)k_refactor<float>, c->smem));
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_refactor<float>, nw * 32, c->smem));
    } else {
        CK(ensure_smem((const void *)k_refactor<double>, c->smem));
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_refactor<double>, nw * 32, c->smem));
    }
    if (per_sm < 1) { g_last_error = "refactor kernel does not fit on an SM"; return KKT_ERR_CUDA; }
    const int rows_cap = (n + nw - 1) / nw;
    int grid = c->opt.refactor_ctas > 0 ? std::min(c->opt.refactor_ctas, sms * per_sm) : sms * per_sm;
    c->grid = std::max(1, std::min(grid, rows_cap));
    // k_refactor: every warp owns a block of shared memory with its row buffer
    // (cap entries; big warps cap_big), then either the row's columns (no
    // update maps: targets are found by binary search) or its staging ring
    // (update maps: pivot rows fed ahead by cp.async, see Stage<T>).  Big warps
    // only when the options ask for them.
    {
        const bool mapped = !a.upd_off.empty();
        const bool staged = mapped;
        const size_t ring = f32 ? (size_t)Stage<float>::RING : (size_t)Stage<double>::RING;
        auto warp_bytes = [&](int capw) {
            const size_t vb = ((size_t)capw * tsz + 15) & ~(size_t)15;
            const size_t cb = ((size_t)capw * sizeof(int) + 15) & ~(size_t)15;
            return vb + (staged ? ring : (mapped ? 0 : cb));
        };
        const size_t cta_max = 227 * 1024;
        int nbig = 0, cap_big = cap_r;
        if (!ord_long.empty() && nw >= 2 && c->opt.refactor_big_warps > 0) {
            cap_big = ((a.max_row + 31) / 32) * 32;
            while (cap_big > cap_r && warp_bytes(cap_big) + (size_t)(nw - 1) * warp_bytes(cap_r) > cta_max)
                cap_big -= 32;
            if (cap_big > cap_r) {
                const long long each = (long long)warp_bytes(cap_big) - (long long)warp_bytes(cap_r);
                const long long most = ((long long)cta_max - (long long)nw * (long long)warp_bytes(cap_r)) / each;
                nbig = (int)std::max(1LL, std::min<long long>({(long long)c->opt.refactor_big_warps,
                                                               (long long)nw / 2, most}));
            } else {
                cap_big = cap_r;
            }
        }
        if (nbig == 0 && c->P.n_long > 0) {
            // no big warps: every row in one queue
            c->P.order_free = c->P.order_f;
            c->P.n_free = n;
            c->P.n_long = 0;
            c->P.n_rest = 0;
        }
        c->rc.nbig = nbig;
        c->rc.cap_big = cap_big;
        c->rc.smem_cols = mapped ? 0 : 1;
        c->rc.staged = staged ? 1 : 0;
        c->rc.symmetric = (staged && c->opt.symmetric) ? 1 : 0;   // LDL^T needs the update maps
        c->rc.warp_bytes_big = (int)warp_bytes(cap_big);
        c->rc.warp_bytes_small = (int)warp_bytes(cap_r);
        c->rsmem = (size_t)nbig * warp_bytes(cap_big) + (size_t)(nw - nbig) * warp_bytes(cap_r);
        int per_sm_r = 0;
        if (f32) {
            CK(ensure_smem((const void *)k_refactor<float>, c->rsmem));
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_r, k_refactor<float>, nw * 32, c->rsmem));
        } else {
            CK(ensure_smem((const void *)k_refactor<double>, c->rsmem));
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_r, k_refactor<double>, nw * 32, c->rsmem));
        }
        if (per_sm_r < 1) { g_last_error = "refactor kernel does not fit on an SM"; return KKT_ERR_CUDA; }
        const int rg = c->opt.refactor_ctas > 0 ? std::min(c->opt.refactor_ctas, sms * per_sm_r)
                                                : sms * per_sm_r;
        c->rgrid = std::max(1, std::min(rg, rows_cap));
    }
    // batched solves: 2 CTAs of cta_warps per SM; single-system solves: CTAs of
    // twice as many warps, one per SM (a CTA task gets the whole SM)
    c->bsolve_grid = std::max(1, std::min(sms * 2, rows_cap));
    c->solve_warps = 2 * nw;
    const int snw = c->solve_warps;
    int sgrid = c->opt.solve_ctas > 0 ? c->opt.solve_ctas : sms;
    c->solve_grid = std::max(1, std::min(sgrid, (n + snw - 1) / snw));
    // rows longer than the shared-memory capacity work in global scratch
    if (a.max_row > cap) {
        const size_t per = (size_t)a.max_row, warps = (size_t)std::max(c->grid, c->rgrid) * nw;
        CK(cudaMalloc(&c->d_scratch, per * tsz * warps));
        c->device_bytes += per * tsz * warps;
        c->rc.scratch_stride = (int)per;
    }
    // update maps
    if (!a.upd_off.empty()) {
        // the map starts on a 256-byte boundary and is readable 64 bytes past
        // its end (16-byte copies of the staged refactorization)
        const size_t off_b = ((size_t)nlu * sizeof(unsigned) + 255) & ~(size_t)255;
        const size_t map_b = a.upd_map.size() * sizeof(unsigned short);
        CK(cudaMalloc(&c->d_maps, off_b + map_b + 64));
        CK(cudaMemset(c->d_maps, 0, off_b + map_b + 64));
        CK(cudaMemcpy(c->d_maps, a.upd_off.data(), (size_t)nlu * sizeof(unsigned), cudaMemcpyHostToDevice));
        unsigned short *dm = (unsigned short *)((char *)c->d_maps + off_b);
        if (map_b) CK(cudaMemcpy(dm, a.upd_map.data(), map_b, cudaMemcpyHostToDevice));
        c->P.upd_off = (const unsigned *)c->d_maps;
        c->P.upd_map = dm;
        c->device_bytes += off_b + map_b;
    }
    // solve tasks: claim orders and shared-memory capacity
    {
        const int nt = (int)a.task_lo.size();
        std::vector<int> len(nt), top(nt), depth(nt);
        for (int T = 0; T < nt; T++) {
            len[T] = a.task_hi[T] - a.task_lo[T] + 1;
            top[T] = a.level[a.task_hi[T]];
            depth[T] = a.level_u[a.task_hi[T]];
        }
        // Claim orders over a set of tasks: forward = the longest tasks (fewer
        // than a quarter of the resident warps) first, then the deepest top
        // rows first (critical path first; a task depends only on deeper
        // tasks); backward = by height of the top row, from the root;
        // topological = deepest top rows first.
        auto orders = [&](const std::vector<int> &set, long long warps, std::vector<int> &of,
                          std::vector<int> &ob, std::vector<int> &ot, long long *nlong = nullptr) {
            std::vector<int> bylen(set);
            std::sort(bylen.begin(), bylen.end(), [&](int x, int y) { return len[x] > len[y]; });
            const long long max_long = std::max(0LL, warps / 4);
            int lmin = INT32_MAX;
            long long cnt = 0;
            size_t q = 0;
            while (q < bylen.size()) {
                size_t r = q;
                while (r < bylen.size() && len[bylen[r]] == len[bylen[q]]) r++;
                if (cnt + (long long)(r - q) > max_long || len[bylen[q]] < 2) break;
                cnt += (long long)(r - q);
                lmin = len[bylen[q]];
                q = r;
            }
            if (nlong) *nlong = cnt;
            of = set;
            ob = set;
            ot = set;
            std::stable_sort(of.begin(), of.end(), [&](int x, int y) {
                const bool lx = len[x] >= lmin, ly = len[y] >= lmin;
                if (lx != ly) return lx;
                return depth[x] > depth[y];
            });
            std::stable_sort(ob.begin(), ob.end(), [&](int x, int y) { return top[x] > top[y]; });
            std::stable_sort(ot.begin(), ot.end(), [&](int x, int y) { return depth[x] > depth[y]; });
        };
        std::vector<int> all(nt);
        std::iota(all.begin(), all.end(), 0);
        std::vector<int> of, ob, ot;
        orders(all, (long long)c->bsolve_grid * nw, of, ob, ot);
        // Single-system solves: the longest tasks (at least CHAIN_MIN rows, at
        // most a quarter of the CTAs) run on a CTA each; the rest are claimed
        // by warps.
        std::vector<int> chain, reg;
        if (snw >= 8 && c->solve_grid >= 6) {
            std::vector<int> bylen(all);
            std::stable_sort(bylen.begin(), bylen.end(), [&](int x, int y) { return len[x] > len[y]; });
            const int max_chain = c->solve_grid / 3;
            for (int T : bylen) {
                if ((int)chain.size() >= max_chain || len[T] < CHAIN_MIN) break;
                chain.push_back(T);
            }
        }
        {
            std::vector<char> is_chain(nt, 0);
            for (int T : chain) is_chain[T] = 1;
            for (int T = 0; T < nt; T++)
                if (!is_chain[T]) reg.push_back(T);
        }
        std::vector<int> of1, ob1, ot1;
        long long nlong1 = 0;
        orders(reg, (long long)(c->solve_grid - (int)chain.size()) * snw, of1, ob1, ot1, &nlong1);
        // Single-row tasks (leaves of the tree) in packs of 32, a lane per row:
        // forward they depend on nothing and follow the longest-first prefix;
        // backward they depend only on ancestors and come last.  An order entry
        // p < 0 stands for pack -1 - p.
        std::vector<int> pack_rows;
        {
            std::vector<int> leaves, f2, b2;
            for (int T : of1)
                if (len[T] == 1) leaves.push_back(T);
            const int npk = (int)((leaves.size() + 31) / 32);
            pack_rows.assign((size_t)npk * 32, -1);
            for (size_t q = 0; q < leaves.size(); q++) pack_rows[q] = a.task_lo[leaves[q]];
            for (long long q = 0; q < nlong1; q++) f2.push_back(of1[q]);
            for (int p = 0; p < npk; p++) f2.push_back(-1 - p);
            for (size_t q = (size_t)nlong1; q < of1.size(); q++)
                if (len[of1[q]] > 1) f2.push_back(of1[q]);
            for (int T : ob1)
                if (len[T] > 1) b2.push_back(T);
            for (int p = 0; p < npk; p++) b2.push_back(-1 - p);
            of1.swap(f2);
            ob1.swap(b2);
        }
        // Outside items: every row of a CTA task with dependencies in other
        // tasks gets a warp item for that part, claimed with the tasks:
        // forward by the row's depth among the depth-ordered tasks (its outside
        // sources are deeper), backward right after its task's position (its
        // outside sources are ancestors in earlier tasks).
        // Far sources (forward / backward phases alike): a row's sources in its
        // own task more than `far` blocks back, if there are at least FAR_MIN
        // of them, are summed by a partner CTA of the task (a CTA of its own,
        // streaming those entries on another SM while the task's CTA walks on)
        // and published in a per-row array; the task's CTA then reads only the
        // entries of the last blocks.  A partner's warps take the task's far
        // rows in step order and wait only for rows at least `far` blocks
        // back, which the task's CTA produces without them, so every wait ends.
        const int far = c->opt.solve_far_blocks < 0 ? 0 : (c->opt.solve_far_blocks == 0 ? 2
                                                                                         : c->opt.solve_far_blocks);
        constexpr int FAR_MIN = 32;
        std::vector<int> ce_f(n, 0), ce_b(n, 0), cf_f(n, 0), cf_b(n, 0), xr_f, xr_b;
        std::vector<int> fr_f, fr_b;                       // far rows of each CTA task, in step order
        std::vector<int> fo_f(chain.size() + 1, 0), fo_b(chain.size() + 1, 0);
        std::vector<double> far_load(chain.size(), 0.0);   // far entries of each CTA task
        {
            std::vector<int> task_of_row(n, -1);
            for (int T : chain)
                for (int i = a.task_lo[T]; i <= a.task_hi[T]; i++) task_of_row[i] = T;
            const int *ci = a.lu_ci.data();
            for (size_t qc = 0; qc < chain.size(); qc++) {
                const int T = chain[qc], lo = a.task_lo[T], hi = a.task_hi[T];
                for (int i = lo; i <= hi; i++) {
                    const int rb = a.lu_rp[i], dg = a.diag[i];
                    ce_f[i] = cf_f[i] = (int)(std::lower_bound(ci + rb, ci + dg, lo) - ci);
                    const int bf = (i - lo) / CB;
                    if (far > 0 && bf > far) {
                        const int e = (int)(std::lower_bound(ci + rb, ci + dg, lo + CB * (bf - far)) - ci);
                        if (e - ce_f[i] >= FAR_MIN) {
                            cf_f[i] = e;
                            fr_f.push_back(i);
                            far_load[qc] += e - ce_f[i];
                        }
                    }
                    if (ce_f[i] > rb) xr_f.push_back(i);
                }
                fo_f[qc + 1] = (int)fr_f.size();
                for (int i = hi; i >= lo; i--) {
                    const int dg = a.diag[i], re = a.lu_rp[i + 1];
                    ce_b[i] = cf_b[i] = (int)(std::upper_bound(ci + dg + 1, ci + re, hi) - ci);
                    const int bb = (hi - i) / CB;
                    if (far > 0 && bb > far) {
                        const int e = (int)(std::upper_bound(ci + dg + 1, ci + re, hi - CB * (bb - far)) - ci);
                        if (ce_b[i] - e >= FAR_MIN) {
                            cf_b[i] = e;
                            fr_b.push_back(i);
                            far_load[qc] += ce_b[i] - e;
                        }
                    }
                }
                for (int i = lo; i <= hi; i++)
                    if (ce_b[i] < a.lu_rp[i + 1]) xr_b.push_back(i);
                fo_b[qc + 1] = (int)fr_b.size();
            }
            // forward: merge into the depth-ordered part after the prefix and packs
            const size_t head = (size_t)nlong1 + (pack_rows.size() / 32);
            std::vector<std::pair<int, int>> tail;        // (depth key, entry)
            for (size_t q = head; q < of1.size(); q++) tail.push_back({depth[of1[q]], of1[q]});
            for (size_t k = 0; k < xr_f.size(); k++) tail.push_back({a.level_u[xr_f[k]], nt + (int)k});
            std::stable_sort(tail.begin(), tail.end(), [](const std::pair<int, int> &x, const std::pair<int, int> &y) {
                return x.first > y.first;
            });
            of1.resize(head);
            for (auto &e : tail) of1.push_back(e.second);
            // backward: by the height of the row's task's top, after the tasks
            // of that height (packs keep their place at the end)
            std::vector<std::array<int, 3>> bk;           // (height key, tie, entry)
            for (size_t q = 0; q < ob1.size(); q++) {
                const int e = ob1[q];
                bk.push_back({e >= 0 ? top[e] : -1, 0, e});
            }
            for (size_t k = 0; k < xr_b.size(); k++) bk.push_back({top[task_of_row[xr_b[k]]], 1, nt + (int)k});
            std::stable_sort(bk.begin(), bk.end(), [](const std::array<int, 3> &x, const std::array<int, 3> &y) {
                if (x[0] != y[0]) return x[0] > y[0];
                return x[1] < y[1];
            });
            ob1.clear();
            for (auto &e : bk) ob1.push_back(e[2]);
        }
        // Partner CTAs: up to `nfar` CTAs (at most a third of the CTAs left
        // after the CTA tasks), each given to the task with the most far
        // entries per partner; a task left without one keeps its far sources.
        std::vector<int> parts(chain.size(), 0);
        {
            const int want = c->opt.solve_far_ctas < 0 ? 0 : (c->opt.solve_far_ctas == 0 ? 8 : c->opt.solve_far_ctas);
            const int nfar = std::max(0, std::min(want, (c->solve_grid - (int)chain.size()) / 3));
            for (int k = 0; k < nfar; k++) {
                int best = -1;
                double bl = 0.0;
                for (size_t qc = 0; qc < chain.size(); qc++) {
                    const double l = far_load[qc] / (parts[qc] + 1);
                    if (l > bl) { bl = l; best = (int)qc; }
                }
                if (best < 0) break;
                parts[best]++;
            }
        }
        std::vector<int> part_f, part_b, fr_f2, fr_b2;
        c->far_rows = 0;
        for (size_t qc = 0; qc < chain.size(); qc++) {
            if (parts[qc] == 0) {                       // no partner: the CTA sums every source in its task
                for (int k = fo_f[qc]; k < fo_f[qc + 1]; k++) cf_f[fr_f[k]] = ce_f[fr_f[k]];
                for (int k = fo_b[qc]; k < fo_b[qc + 1]; k++) cf_b[fr_b[k]] = ce_b[fr_b[k]];
                continue;
            }
            const int of0 = (int)fr_f2.size(), ob0 = (int)fr_b2.size();
            fr_f2.insert(fr_f2.end(), fr_f.begin() + fo_f[qc], fr_f.begin() + fo_f[qc + 1]);
            fr_b2.insert(fr_b2.end(), fr_b.begin() + fo_b[qc], fr_b.begin() + fo_b[qc + 1]);
            c->far_rows += fo_f[qc + 1] - fo_f[qc];
            for (int r = 0; r < parts[qc]; r++) {
                part_f.insert(part_f.end(), {of0, fo_f[qc + 1] - fo_f[qc], r, parts[qc]});
                part_b.insert(part_b.end(), {ob0, fo_b[qc + 1] - fo_b[qc], r, parts[qc]});
            }
        }
        c->npart = (int)part_f.size() / 4;
        std::vector<int> blk0(chain.size() + 1, 0), binfo;
        for (size_t q = 0; q < chain.size(); q++) {
            const int T = chain[q], nbq = (len[T] + CB - 1) / CB;
            blk0[q + 1] = blk0[q] + nbq;
            for (int b = 0; b < nbq; b++) {
                binfo.push_back(a.task_lo[T]);
                binfo.push_back(a.task_hi[T]);
                binfo.push_back(b);
            }
        }
        // slot splits of the rows of CTA tasks (forward / backward phases share
        // them: cs_late and cs_diag are column bounds turned into slots)
        int zmax = 0;
        for (int T : chain) zmax = std::max(zmax, len[T]);
        // Forward and backward phases walk the task in opposite directions, so
        // the splits differ; both are stored: [0, n) forward, [n, 2n) backward.
        std::vector<int> csl(2 * (size_t)n, -1), csd(2 * (size_t)n, -1);
        for (int T : chain) {
            const int lo = a.task_lo[T], hi = a.task_hi[T];
            for (int i = lo; i <= hi; i++) {
                const int rb = a.lu_rp[i], dg = a.diag[i], re = a.lu_rp[i + 1];
                const int *ci = a.lu_ci.data();
                // forward: step k = i - lo, block b; sources with column >= lo + CB*max(b-1,0)
                // are late or diag, >= lo + CB*b diag
                {
                    const int k = i - lo, b = k / CB;
                    const int c_late = lo + CB * std::max(b - 1, 0), c_diag = lo + CB * b;
                    csl[i] = (int)(std::lower_bound(ci + rb, ci + dg, c_late) - ci);
                    csd[i] = (int)(std::lower_bound(ci + rb, ci + dg, c_diag) - ci);
                }
                // backward: step k = hi - i; sources with column <= hi - CB*max(b-1,0)
                // are late or diag, <= hi - CB*b diag (a head of the U slots)
                {
                    const int k = hi - i, b = k / CB;
                    const int c_late = hi - CB * std::max(b - 1, 0), c_diag = hi - CB * b;
                    csl[n + (size_t)i] = (int)(std::upper_bound(ci + dg + 1, ci + re, c_late) - ci);
                    csd[n + (size_t)i] = (int)(std::upper_bound(ci + dg + 1, ci + re, c_diag) - ci);
                }
            }
        }
        // The waits of the partner CTAs end only if every far range lies
        // among the early sources (at least one whole block back) and each
        // task's far rows are listed in step order; check both before any
        // kernel relies on them.
        {
            bool ok = true;
            for (int T : chain) {
                for (int i = a.task_lo[T]; ok && i <= a.task_hi[T]; i++) {
                    if (cf_f[i] != ce_f[i]) ok = ce_f[i] < cf_f[i] && cf_f[i] <= csl[i];
                    if (ok && cf_b[i] != ce_b[i]) ok = csl[n + (size_t)i] <= cf_b[i] && cf_b[i] < ce_b[i];
                }
            }
            for (size_t q = 0; ok && q + 4 <= part_f.size(); q += 4) {
                const int o0 = part_f[q], cnt = part_f[q + 1], b0 = part_b[q], cntb = part_b[q + 1];
                for (int r = 1; ok && r < cnt; r++) ok = fr_f2[o0 + r - 1] < fr_f2[o0 + r];
                for (int r = 1; ok && r < cntb; r++) ok = fr_b2[b0 + r - 1] > fr_b2[b0 + r];
            }
            if (!ok) {
                g_last_error = "internal: inconsistent far-source plan of the triangular solves";
                return KKT_ERR_ARG;
            }
        }
        int *d = nullptr;
        const size_t words = 3 * (size_t)nt + 3 * (size_t)(nt + xr_f.size() + xr_b.size()) + chain.size() +
                             4 * (size_t)n + blk0.size() + binfo.size() + pack_rows.size() + 2 * (size_t)n +
                             xr_f.size() + xr_b.size() + 2 * (size_t)n + fr_f2.size() + fr_b2.size() +
                             part_f.size() + part_b.size() + 4;
        CK(cudaMalloc(&d, words * sizeof(int)));
        size_t o = 0;
        auto put = [&](const std::vector<int> &v) -> const int * {
            const int *p = d + o;
            if (!v.empty()) {
                cudaError_t e = cudaMemcpy(d + o, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice);
                if (e != cudaSuccess) return nullptr;
            }
            o += v.size();
            return p;
        };
        c->d_task_orders = d;
        c->tk.ntasks = nt;
        c->tk.order_f = put(of);
        c->tk.order_b = put(ob);
        c->tk.order_topo = put(ot);
        c->tk1.task_lo = c->tk.task_lo;
        c->tk1.task_hi = c->tk.task_hi;
        c->tk1.ntasks = (int)of1.size();     // per phase in tasks_of
        c->tk1.order_f = put(of1);
        c->tk1.order_b = put(ob1);
        c->tk1.order_topo = put(ot1);
        c->tk1.nchain = (int)chain.size();
        c->tk1.chain_task = put(chain);
        c->chain_h = chain;
        c->tk1.chain_blk0 = put(blk0);
        c->tk1.pack_rows = put(pack_rows);
        c->ce_fwd = put(ce_f);
        c->ce_bwd = put(ce_b);
        c->xr_fwd = put(xr_f);
        c->xr_bwd = put(xr_b);
        c->cf_fwd = put(cf_f);
        c->cf_bwd = put(cf_b);
        c->fr_fwd = put(fr_f2);
        c->fr_bwd = put(fr_b2);
        o = (o + 3) & ~(size_t)3;                       // int4 tables: 16-byte aligned
        c->part_fwd = reinterpret_cast<const int4 *>(put(part_f));
        c->part_bwd = reinterpret_cast<const int4 *>(put(part_b));
        c->nord_f = (int)of1.size();
        c->nord_b = (int)ob1.size();
        c->tk1.ext_base = nt;
        c->blk_info = put(binfo);
        c->nblk = blk0.back();
        c->cs_fwd = put(std::vector<int>(csl.begin(), csl.begin() + n));
        c->cs_bwd = put(std::vector<int>(csl.begin() + n, csl.end()));
        c->csd_fwd = put(std::vector<int>(csd.begin(), csd.begin() + n));
        c->csd_bwd = put(std::vector<int>(csd.begin() + n, csd.end()));
        if (!c->tk.order_f || !c->tk1.order_f || !c->tk1.chain_task || !c->cs_fwd || !c->csd_bwd ||
            !c->tk1.chain_blk0 || !c->blk_info) {
            g_last_error = "copy of the task tables failed";
            return KKT_ERR_CUDA;
        }
        c->tk.cap = std::min(a.max_task, 1024);
        int max_reg = 1;
        for (int T : reg) max_reg = std::max(max_reg, len[T]);
        c->tk1.cap = std::min(max_reg, 1024);
        {   // rows of a CTA task cached in shared memory: all of the longest
            // task if the CTA's shared memory allows, a multiple of 4 (alignment)
            const size_t fixed = chain_smem_bytes(0, tsz), per = chain_smem_bytes(1, tsz) - fixed;
            const int zfit = (int)((CHAIN_SMEM - fixed) / per) & ~3;
            c->tk1.zcap = std::min((zmax + 3) & ~3, std::min(zfit, ZCAP_MAX));
        }
        c->device_bytes += words * sizeof(int);
        if (c->nblk > 0) {
            const size_t tb = 4 * (size_t)c->nblk * 2 * CB * CB * tsz;
            CK(cudaMalloc(&c->d_tiles, tb));
            c->device_bytes += tb;
        }
        c->solve_smem = std::max((size_t)snw * c->tk1.cap * tsz,
                                 c->tk1.nchain ? chain_smem_bytes(c->tk1.zcap, tsz) : 0);
        auto setsm = [&](const void *f) {
            return ensure_smem(f, c->solve_smem);
        };
        int per_sm_s = 0;
        if (f32) {
            CK(setsm((const void *)k_trisolve<float, false, false>));
            CK(setsm((const void *)k_trisolve<float, true, false>));
            CK(setsm((const void *)k_trisolve<float, false, true>));
            CK(setsm((const void *)k_trisolve<float, true, true>));
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_s, k_trisolve<float, false, false>,
                                                             snw * 32, c->solve_smem));
        } else {
            CK(setsm((const void *)k_trisolve<double, false, false>));
            CK(setsm((const void *)k_trisolve<double, true, false>));
            CK(setsm((const void *)k_trisolve<double, false, true>));
            CK(setsm((const void *)k_trisolve<double, true, true>));
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_s, k_trisolve<double, false, false>,
                                                             snw * 32, c->solve_smem));
        }
        // every CTA of a solve must be resident at once (CTA tasks and waiting warps)
        if ((long long)per_sm_s * sms < c->solve_grid) {
            g_last_error = "solve grid does not fit on the device at once";
            return KKT_ERR_CUDA;
        }
    }
    if (c->opt.refine_mode == KKT_REFINE_FGMRES || c->opt.refine_mode == KKT_REFINE_AUTO ||
        c->opt.refine_mode == KKT_REFINE_FGMRES_JACOBI) {
        const int m = std::min(c->opt.fgmres_restart, 63);
        c->kry_m = m;
        c->kry_blocks = std::max(1, std::min(1024, (n + 255) / 256));
        const size_t words = (size_t)(2 * m + 2) * n + (size_t)c->kry_blocks * (m + 1) + 4 * (m + 2);
        CK(cudaMalloc(&c->d_krylov, words * sizeof(double)));
        c->device_bytes += words * sizeof(double);
    }
    if (c->opt.max_batch > 1) {
        const size_t Bc = (size_t)c->opt.max_batch;
        c->bcap = c->opt.max_batch;
        CK(cudaMalloc(&c->b_lu, nlu * Bc * tsz));
        CK(cudaMalloc(&c->b_lut, nlu * Bc * tsz));
        CK(cudaMalloc(&c->b_rcp, (size_t)n * Bc * tsz));
        CK(cudaMalloc(&c->b_y, 2 * (size_t)n * Bc * tsz));
        CK(cudaMalloc(&c->b_s, (size_t)n * Bc * sizeof(double)));
        CK(cudaMalloc(&c->b_sp, (size_t)n * Bc * sizeof(double)));
        CK(cudaMalloc(&c->b_rho, (size_t)n * Bc * sizeof(double)));
        CK(cudaMalloc(&c->b_norms, NM_WORDS * Bc * sizeof(unsigned long long)));
        CK(cudaMallocHost(&c->hb_norms, NM_WORDS * Bc * sizeof(unsigned long long)));
        c->device_bytes += (2 * nlu + 3 * (size_t)n) * Bc * tsz + 3 * (size_t)n * Bc * sizeof(double);
        c->bsolve_smem = (size_t)nw * c->tk.cap * tsz;
        auto setb = [&](const void *f, size_t bytes) {
            return ensure_smem(f, bytes);
        };
        if (f32) {
            CK(setb((const void *)k_brefactor<float>, c->smem));
            CK(setb((const void *)k_btrisolve<float, false, false>, c->bsolve_smem));
            CK(setb((const void *)k_btrisolve<float, true, false>, c->bsolve_smem));
            CK(setb((const void *)k_btrisolve<float, false, true>, c->bsolve_smem));
            CK(setb((const void *)k_btrisolve<float, true, true>, c->bsolve_smem));
        } else {
            CK(setb((const void *)k_brefactor<double>, c->smem));
            CK(setb((const void *)k_btrisolve<double, false, false>, c->bsolve_smem));
            CK(setb((const void *)k_btrisolve<double, true, false>, c->bsolve_smem));
            CK(setb((const void *)k_btrisolve<double, false, true>, c->bsolve_smem));
            CK(setb((const void *)k_btrisolve<double, true, true>, c->bsolve_smem));
        }
        // every CTA of a batched solve must be resident at once (waiting warps)
        int per_sm_b = 0;
        if (f32) CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, k_btrisolve<float, false, false>,
                                                                  nw * 32, c->bsolve_smem));
        else CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, k_btrisolve<double, false, false>,
                                                              nw * 32, c->bsolve_smem));
        if ((long long)per_sm_b * sms < c->bsolve_grid) c->bsolve_grid = per_sm_b * sms;
    }
    if (c->opt.trace) {
        const long long items = std::max<long long>(n, c->tk.ntasks);
        c->rc.trace_stride = 2 * items;
        CK(cudaMalloc(&c->d_trace, TR_PHASES * 2 * items * sizeof(unsigned long long)));
        CK(cudaMemset(c->d_trace, 0, TR_PHASES * 2 * items * sizeof(unsigned long long)));
        c->rc.trace = c->d_trace;
    }
    c->rc.spin_limit = c->opt.spin_limit;
    c->rc.unpublished_row = -1;
    c->rc.poll_ns_max = c->opt.poll_ns_max > 0 ? (unsigned)c->opt.poll_ns_max : 128u;
    if (c->opt.unpublished_row >= 0 && c->opt.unpublished_row < n)
        c->rc.unpublished_row = a.internal_of[c->opt.unpublished_row];
    c->rc.status = c->d_status;
    c->rc.norms = c->d_norms;
    c->rc.sched = c->d_sched;
    c->rc.cap = cap;
    c->rc.scratch = c->d_scratch;
    // dense root block: its dense array (row-major, leading dimension a multiple
    // of 32 words) and the barrier word of k_dense_lu; the shared RunCfg keeps
    // the block off (the batched and queued kernels factor its rows as rows)
    c->rc.dense_lo = INT_MAX;
    c->rc.dense_ld = 0;
    c->rc.dense = nullptr;
    c->rc.dense_ctl = nullptr;
    if (a.dense_rows > 0) {
        const int sd = a.dense_rows;
        c->dense_ld = (sd + 31) / 32 * 32;
        const size_t db = (size_t)sd * c->dense_ld * tsz;
        const size_t cb = dense_lu_ctl_bytes(sd);
        CK(cudaMalloc(&c->d_dense, db));
        CK(cudaMalloc(&c->d_dense_ctl, cb));
        CK(cudaMemset(c->d_dense_ctl, 0, cb));
        c->device_bytes += db + cb;
        CK(dense_lu_prepare(f32 ? 1 : 0, sd, sms, &c->dense_grid));
    }
    if (c->rowperm) {
        const size_t nnz = c->qmap.size();
        CK(cudaMalloc(&c->d_q, (size_t)n * sizeof(int)));
        CK(cudaMalloc(&c->d_qmap, nnz * sizeof(int)));
        CK(cudaMalloc(&c->d_qvals, nnz * sizeof(double)));
        CK(cudaMalloc(&c->d_qvec, 2 * (size_t)n * sizeof(double)));
        CK(cudaMalloc(&c->d_qdA, nnz * sizeof(double)));
        CK(cudaMemcpy(c->d_q, c->q.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->d_qmap, c->qmap.data(), nnz * sizeof(int), cudaMemcpyHostToDevice));
        c->device_bytes += (size_t)n * 4 + nnz * 4 + nnz * 16 + 16 * (size_t)n;
    }
    return KKT_OK;
}

void kkt_destroy(kkt_ctx *c) {
    if (!c) return;
    if (!c->host_only) {
        DeviceGuard g(c->dev);
        cudaFree(c->d_q);
        cudaFree(c->d_qmap);
        cudaFree(c->d_qvals);
        cudaFree(c->d_qvec);
        cudaFree(c->d_qdA);
        cudaFree(c->d_ints);
        cudaFree(c->d_lu);
        cudaFree(c->d_lut);
        cudaFree(c->d_rcp);
        cudaFree(c->d_s);
        cudaFree(c->d_sp);
        cudaFree(c->d_rho);
        cudaFree(c->d_y);
        cudaFree(c->d_status);
        cudaFree(c->d_norms);
        cudaFree(c->d_sched);
        cudaFree(c->d_maps);
        cudaFree(c->d_task_orders);
        cudaFree(c->d_tiles);
        cudaFree(c->d_trace);
        cudaFree(c->d_view_slot);
        cudaFree(c->d_krylov);
        cudaFree(c->b_lu);
        cudaFree(c->b_lut);
        cudaFree(c->b_rcp);
        cudaFree(c->b_y);
        cudaFree(c->b_s);
        cudaFree(c->b_sp);
        cudaFree(c->b_rho);
        cudaFree(c->b_norms);
        cudaFreeHost(c->hb_norms);
        cudaFree(c->d_scratch);
        cudaFree(c->d_dense);
        cudaFree(c->d_dense_ctl);
        cudaFreeHost(c->h_norms);
    }
    delete c;
}

// Analysis of the pattern of A, or of Q A when a row permutation is given by
// the options or computed from values_host (max-product matching).
// Option ranges shared by kkt_analyze(_values) and kkt_load_analysis.
static bool options_valid(const kkt_options &o) {
    return o.fgmres_restart >= 1 && o.max_refine >= 0 && o.spin_limit >= 1 &&
           o.refine_mode >= KKT_REFINE_CLASSIC && o.refine_mode <= KKT_REFINE_FGMRES_JACOBI &&
           o.jacobi_sweeps >= 0 && o.dense_block >= -1 && o.refactor_row_cap >= 0 &&
           o.refine_auto_ratio >= 0.0 && o.refine_auto_ratio < 1.0 && o.max_batch >= 1 && o.cta_warps >= 0 &&
           o.refactor_ctas >= 0 && o.solve_ctas >= 0 && o.solve_far_blocks >= -1 && o.solve_far_ctas >= -1;
}

static kkt_status analyze_ctx(int n, const int *row_ptr, const int *col_idx, const double *values_host,
                              const kkt_options *opt, kkt_ctx **out) {
    ApiRange nvtx_range(values_host ? "kkt_analyze_values" : "kkt_analyze");
    if (!out) return KKT_ERR_ARG;
    *out = nullptr;
    std::unique_ptr<kkt_ctx> c(new (std::nothrow) kkt_ctx());
    if (!c) return KKT_ERR_ALLOC;
    if (opt) c->opt = *opt; else kkt_default_options(&c->opt);
    if (!options_valid(c->opt)) {
        g_last_error = "invalid option";
        return KKT_ERR_ARG;
    }
    std::string err;
    int rc;
    try {
        long long budget = 0;
        if (c->opt.device >= 0) {
            if (c->opt.update_map_budget > 0) {
                budget = (long long)c->opt.update_map_budget;
            } else {                          // a quarter of the free device memory, at most 16 GiB
                DeviceGuard g(c->opt.device);
                size_t fr = 0, tot = 0;
                if (g.ok && cudaMemGetInfo(&fr, &tot) == cudaSuccess)
                    budget = std::min<long long>((long long)(fr / 4), 16LL << 30);
                else
                    budget = 1LL << 30;
            }
        }
        const int *rp = row_ptr, *ci = col_idx;
        std::vector<int> qa_rp, qa_ci;
        if (c->opt.user_row_perm || values_host) {
            if (!row_ptr || !col_idx || validate_pattern(n, row_ptr, col_idx) != A_OK) {
                g_last_error = "malformed pattern";
                return KKT_ERR_PATTERN;
            }
            std::vector<int> &q = c->q;
            if (c->opt.user_row_perm) {
                q.assign(c->opt.user_row_perm, c->opt.user_row_perm + n);
                std::vector<char> seen(n, 0);
                for (int j = 0; j < n; j++) {
                    if (q[j] < 0 || q[j] >= n || seen[q[j]]) {
                        g_last_error = "user_row_perm is not a permutation";
                        return KKT_ERR_ARG;
                    }
                    seen[q[j]] = 1;
                }
            } else {
                rc = max_product_matching(n, row_ptr, col_idx, values_host, q, err);
                if (rc != A_OK) {
                    g_last_error = err;
                    return (kkt_status)rc;
                }
            }
            // Q A: row j is row q[j] of A; qmap[k] = entry of A at entry k of Q A
            qa_rp.assign(n + 1, 0);
            for (int j = 0; j < n; j++) qa_rp[j + 1] = qa_rp[j] + row_ptr[q[j] + 1] - row_ptr[q[j]];
            qa_ci.resize(qa_rp[n]);
            c->qmap.resize(qa_rp[n]);
            for (int j = 0; j < n; j++)
                for (int t = 0; t < qa_rp[j + 1] - qa_rp[j]; t++) {
                    qa_ci[qa_rp[j] + t] = col_idx[row_ptr[q[j]] + t];
                    c->qmap[qa_rp[j] + t] = row_ptr[q[j]] + t;
                }
            c->rowperm = true;
            rp = qa_rp.data();
            ci = qa_ci.data();
        }
        // The dense root block pays with FP32 factors (FP64 arithmetic is slow on
        // this GPU: the block's FP64 LU is not faster than its rows' own chain),
        // so the automatic choice applies to FP32 factors only; a requested block
        // is capped at what k_dense_lu holds in shared memory.
        int dreq = c->opt.dense_block;
        if (dreq == 0 && !c->opt.factor_fp32) dreq = -1;
        if (dreq > 0) dreq = std::min(dreq, dense_lu_max_rows(c->opt.factor_fp32 ? 1 : 0));
        rc = analyze(n, rp, ci, c->opt.ordering, c->opt.user_perm, c->an, err, budget, dreq,
                     dense_lu_max_rows(c->opt.factor_fp32 ? 1 : 0));
    } catch (const std::bad_alloc &) {
        g_last_error = "host allocation failed during analysis";
        return KKT_ERR_ALLOC;
    }
    if (rc != A_OK) {
        g_last_error = err;
        return (kkt_status)rc;
    }
    c->opt.user_perm = nullptr;  // copied
    c->opt.user_row_perm = nullptr;
    c->tau_rel = c->opt.pivot_tau_rel > 0 ? c->opt.pivot_tau_rel
                                          : (c->opt.factor_fp32 ? 0x1p-24 : 1e-14);
    c->auto_ratio = c->opt.refine_auto_ratio > 0 ? c->opt.refine_auto_ratio : 0.5;
    c->dev = c->opt.device;
    c->host_only = c->opt.device < 0;
    if (!c->host_only) {
        DeviceGuard g(c->dev);
        if (!g.ok) { g_last_error = "cannot select the CUDA device"; return KKT_ERR_CUDA; }
        kkt_status s = upload(c.get());
        if (s != KKT_OK) {
            kkt_destroy(c.release());
            return s;
        }
    }
    *out = c.release();
    return KKT_OK;
}

kkt_status kkt_analyze(int n, const int *row_ptr, const int *col_idx, const kkt_options *opt,
                       kkt_ctx **out) {
    return analyze_ctx(n, row_ptr, col_idx, nullptr, opt, out);
}

kkt_status kkt_analyze_values(int n, const int *row_ptr, const int *col_idx, const double *values_host,
                              const kkt_options *opt, kkt_ctx **out) {
    if (!values_host) return KKT_ERR_ARG;
    return analyze_ctx(n, row_ptr, col_idx, values_host, opt, out);
}

kkt_status kkt_export_row_perm(const kkt_ctx *c, int *row_of_col) {
    if (!c || !row_of_col) return KKT_ERR_ARG;
    const int n = c->an.n;
    for (int j = 0; j < n; j++) row_of_col[j] = c->rowperm ? c->q[j] : j;
    return KKT_OK;
}

#define REQUIRE_DEVICE(c)                                                              \
    do {                                                                               \
        if (!(c)) return KKT_ERR_ARG;                                                  \
        if ((c)->host_only) { g_last_error = "host-only context"; return KKT_ERR_STATE; } \
    } while (0)

// Packs the CTA tasks' tiles from the current factors (see k_pack_tiles).
template <typename T> static kkt_status pack_tiles(kkt_ctx *c, cudaStream_t s) {
    if (c->nblk > 0) {
        const long long threads = 4LL * c->nblk * 2 * CB * 32;
        k_pack_tiles<T><<<blocks_for(threads, 256), 256, 0, s>>>(
            c->P, c->blk_info, c->nblk, c->cs_fwd, c->csd_fwd, c->cs_bwd, c->csd_bwd, (const T *)c->d_lu,
            (const T *)c->d_lut, (const T *)c->d_rcp, (T *)c->d_tiles);
        CK(cudaGetLastError());
        c->launches++;
    }
    c->tiles_fresh = true;
    return KKT_OK;
}

template <typename T> static kkt_status launch_refactor(kkt_ctx *c, cudaStream_t s) {
    // every entry starts as the not-ready marker; published entries overwrite it
    CK(cudaMemsetAsync(c->d_lu, 0xff, (size_t)c->nnz_lu * sizeof(T), s));
    CK(cudaMemsetAsync(c->d_rcp, 0xff, (size_t)c->an.n * sizeof(T), s));
    RunCfg rc = c->rc;
    rc.cap = c->cap_r;
    if (c->an.dense_rows > 0) {          // rows of the dense root block stop below it
        rc.dense_lo = c->an.n - c->an.dense_rows;
        rc.dense_ld = c->dense_ld;
        rc.dense = c->d_dense;
        rc.dense_ctl = c->d_dense_ctl;
    }
    k_refactor<T><<<c->rgrid, c->cta_warps * 32, c->rsmem, s>>>(c->P, rc, c->values, c->d_sp,
                                                               (T *)c->d_lu, (T *)c->d_lut,
                                                               (T *)c->d_rcp, c->tau_rel);
    CK(cudaGetLastError());
    c->launches++;
    if (c->an.dense_rows > 0) {
        CK(launch_dense_lu<T>(c->P, rc, c->values, c->d_sp, (T *)c->d_lu, (T *)c->d_lut, (T *)c->d_rcp,
                              c->tau_rel, s));
        c->launches++;
    }
    return pack_tiles<T>(c, s);
}

// task configuration of a single-system solve phase (the slot splits of CTA
// tasks depend on the direction of the walk)
static TaskCfg tasks_of(const kkt_ctx *c, bool backward, bool trans) {
    TaskCfg t = c->tk1;
    t.cs_late = backward ? c->cs_bwd : c->cs_fwd;
    t.cs_diag = backward ? c->csd_bwd : c->csd_fwd;
    t.ntasks = backward ? c->nord_b : c->nord_f;
    t.cs_ext = backward ? c->ce_bwd : c->ce_fwd;
    t.ext_rows = backward ? c->xr_bwd : c->xr_fwd;
    {   // outside sums after y and z in the work vector (4n doubles)
        const size_t tsz_ = c->opt.factor_fp32 ? sizeof(float) : sizeof(double);
        const size_t n = (size_t)c->an.n;
        t.ext = (char *)c->d_y + (2 + (backward ? 1 : 0)) * n * tsz_;
        t.npart = c->npart;
        t.part = backward ? c->part_bwd : c->part_fwd;
        t.far_rows = backward ? c->fr_bwd : c->fr_fwd;
        t.cs_far = backward ? c->cf_bwd : c->cf_fwd;
        t.far = c->npart ? (char *)c->d_y + (4 + (backward ? 1 : 0)) * n * tsz_ : nullptr;
    }
    const int ph = (trans ? 2 : 0) + (backward ? 1 : 0);
    const size_t tsz = c->opt.factor_fp32 ? sizeof(float) : sizeof(double);
    t.tiles = c->d_tiles ? (const void *)((const char *)c->d_tiles + (size_t)ph * c->nblk * 2 * CB * CB * tsz)
                         : nullptr;
    return t;
}

template <typename T>
static kkt_status launch_solve(kkt_ctx *c, const double *b, double *x, int accumulate, cudaStream_t s) {
    const int n = c->an.n;
    T *y = (T *)c->d_y, *z = y + n;
    const T *L = (const T *)c->d_lu, *R = (const T *)c->d_rcp;
    CK(cudaMemsetAsync(y, 0xff, (c->npart ? 6 : 4) * (size_t)n * sizeof(T), s));   // y, z, outside and far sums
    k_trisolve<T, false, false><<<c->solve_grid, c->solve_warps * 32, c->solve_smem, s>>>(
        c->P, c->rc, tasks_of(c, false, false), L, R, b, c->d_sp, nullptr, y, nullptr, 0);
    CK(cudaGetLastError());
    c->launches++;
    k_trisolve<T, true, false><<<c->solve_grid, c->solve_warps * 32, c->solve_smem, s>>>(
        c->P, c->rc, tasks_of(c, true, false), L, R, nullptr, c->d_sp, y, z, x, accumulate);
    CK(cudaGetLastError());
    c->launches++;
    return KKT_OK;
}

template <typename T>
static kkt_status launch_solve_t(kkt_ctx *c, const double *g, double *lam, int accumulate,
                                 cudaStream_t s) {
    const int n = c->an.n;
    T *y = (T *)c->d_y, *z = y + n;
    const T *L = (const T *)c->d_lut, *R = (const T *)c->d_rcp;
    CK(cudaMemsetAsync(y, 0xff, (c->npart ? 6 : 4) * (size_t)n * sizeof(T), s));   // y, z, outside and far sums
    k_trisolve<T, false, true><<<c->solve_grid, c->solve_warps * 32, c->solve_smem, s>>>(
        c->P, c->rc, tasks_of(c, false, true), L, R, g, c->d_sp, nullptr, y, nullptr, 0);
    CK(cudaGetLastError());
    c->launches++;
    k_trisolve<T, true, true><<<c->solve_grid, c->solve_warps * 32, c->solve_smem, s>>>(
        c->P, c->rc, tasks_of(c, true, true), L, R, nullptr, c->d_sp, y, z, lam, accumulate);
    CK(cudaGetLastError());
    c->launches++;
    return KKT_OK;
}

// row permutation of a value-aware context: dst[j] = src[q[j]] (gather a
// vector into Q's order) or dst[q[j]] = src[j] (scatter it back)
static kkt_status q_vec(kkt_ctx *c, const double *src, double *dst, bool gather, cudaStream_t s) {
    const int n = c->an.n;
    if (gather) k_gather<<<blocks_for(n, 256), 256, 0, s>>>(n, c->d_q, src, dst);
    else k_scatter<<<blocks_for(n, 256), 256, 0, s>>>(n, c->d_q, src, dst);
    CK(cudaGetLastError());
    c->launches++;
    return KKT_OK;
}

kkt_status kkt_refactor(kkt_ctx *c, const double *values_dev, kkt_stream stream) {
    ApiRange nvtx_range("kkt_refactor");
    REQUIRE_DEVICE(c);
    if (!values_dev) return KKT_ERR_ARG;
    DeviceGuard g(c->dev);
    cudaStream_t s = (cudaStream_t)stream;
    if (c->rowperm) {                       // the values of Q A
        const long long m = (long long)c->qmap.size();
        k_gather<<<blocks_for(m, 256), 256, 0, s>>>(m, c->d_qmap, values_dev, c->d_qvals);
        CK(cudaGetLastError());
        c->launches++;
        values_dev = c->d_qvals;
    }
    c->values = values_dev;
    const int n = c->an.n;
    CK(cudaMemsetAsync(c->d_norms, 0, NM_WORDS * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(c->d_status + ST_NEGATIVE, 0, 2 * sizeof(int), s));   // this refactorization's inertia
    k_scale<<<norm_blocks(n), RTHREADS, 0, s>>>(c->P, values_dev, c->d_s, c->d_sp, c->d_norms,
                                                     c->d_status, c->opt.equilibrate);
    CK(cudaGetLastError());
    c->launches++;
    k_amax<<<norm_blocks(n), RTHREADS, 0, s>>>(c->P, values_dev, c->d_s, c->d_norms);
    CK(cudaGetLastError());
    c->launches++;
    kkt_status r = c->opt.factor_fp32 ? launch_refactor<float>(c, s) : launch_refactor<double>(c, s);
    if (r == KKT_OK) c->factored = true;
    return r;
}

static kkt_status solve_any(kkt_ctx *c, const double *b, double *x, int accumulate, int transpose,
                            cudaStream_t s) {
    if (!c->tiles_fresh) {                 // factors written by a queue since the last packing
        kkt_status r = c->opt.factor_fp32 ? pack_tiles<float>(c, s) : pack_tiles<double>(c, s);
        if (r != KKT_OK) return r;
    }
    if (transpose)
        return c->opt.factor_fp32 ? launch_solve_t<float>(c, b, x, accumulate, s)
                                  : launch_solve_t<double>(c, b, x, accumulate, s);
    return c->opt.factor_fp32 ? launch_solve<float>(c, b, x, accumulate, s)
                              : launch_solve<double>(c, b, x, accumulate, s);
}

// Approximate solve by Jacobi sweeps (k_jacobi): `sweeps` sweeps on each
// triangular factor; the work vectors are three n-vectors of the context's
// scratch (c, then ping-pong).  A' = L U: L stage then U stage; A'^T = U^T L^T
// on the transposed factor: U^T stage (scaled) then L^T stage.
template <typename T>
static kkt_status launch_jacobi(kkt_ctx *c, const double *b, double *x, int accumulate, int transpose,
                                int sweeps, cudaStream_t s) {
    const int n = c->an.n;
    T *buf[3] = {(T *)c->d_y, (T *)c->d_y + n, (T *)c->d_y + 2 * (size_t)n};
    const T *F = (const T *)(transpose ? c->d_lut : c->d_lu), *R = (const T *)c->d_rcp;
    const int gb = blocks_for(8LL * n, 256), nb = blocks_for(n, 256);
    k_perm_in<T><<<nb, 256, 0, s>>>(c->P, c->d_sp, b, buf[0]);
    CK(cudaGetLastError());
    c->launches++;
    // first stage: unit L (left slots, no scale) or U^T (left slots, scaled)
    int cur = 0;                                // buffer holding the current iterate
    if (transpose) {                            // w_0 = D^-1 c into buf[1]
        k_jacobi<T, false, true><<<gb, 256, 0, s>>>(c->P, F, R, buf[0], nullptr, buf[1]);
        CK(cudaGetLastError());
        c->launches++;
        cur = 1;
    }
    for (int k = 0; k < sweeps; k++) {
        const int nxt = (cur == 1) ? 2 : 1;
        if (transpose) k_jacobi<T, false, true><<<gb, 256, 0, s>>>(c->P, F, R, buf[0], buf[cur], buf[nxt]);
        else k_jacobi<T, false, false><<<gb, 256, 0, s>>>(c->P, F, R, buf[0], buf[cur], buf[nxt]);
        CK(cudaGetLastError());
        c->launches++;
        cur = nxt;
    }
    // second stage on w = buf[cur]: U (right slots, scaled) or unit L^T (right, no scale)
    const int w = cur;
    int z = -1;
    int fa = (w == 0) ? 1 : 0, fb = (w == 2) ? 1 : 2;   // the two buffers other than w
    if (!transpose) {                           // z_0 = D^-1 w
        k_jacobi<T, true, true><<<gb, 256, 0, s>>>(c->P, F, R, buf[w], nullptr, buf[fa]);
        CK(cudaGetLastError());
        c->launches++;
        z = fa;
    } else {
        z = w;                                  // z_0 = w
    }
    for (int k = 0; k < sweeps; k++) {
        const int nxt = (z == fa) ? fb : fa;
        if (transpose) k_jacobi<T, true, false><<<gb, 256, 0, s>>>(c->P, F, R, buf[w], buf[z], buf[nxt]);
        else k_jacobi<T, true, true><<<gb, 256, 0, s>>>(c->P, F, R, buf[w], buf[z], buf[nxt]);
        CK(cudaGetLastError());
        c->launches++;
        z = nxt;
    }
    k_perm_out<T><<<nb, 256, 0, s>>>(c->P, c->d_sp, buf[z], x, accumulate);
    CK(cudaGetLastError());
    c->launches++;
    return KKT_OK;
}

static kkt_status jacobi_any(kkt_ctx *c, const double *b, double *x, int accumulate, int transpose, int sweeps,
                             cudaStream_t s) {
    return c->opt.factor_fp32 ? launch_jacobi<float>(c, b, x, accumulate, transpose, sweeps, s)
                              : launch_jacobi<double>(c, b, x, accumulate, transpose, sweeps, s);
}

// the preconditioner of FGMRES: the exact triangular solves, or Jacobi sweeps
static kkt_status precond_any(kkt_ctx *c, const double *b, double *x, int transpose, cudaStream_t s) {
    if (c->opt.refine_mode == KKT_REFINE_FGMRES_JACOBI)
        return jacobi_any(c, b, x, 0, transpose, c->opt.jacobi_sweeps, s);
    return solve_any(c, b, x, 0, transpose, s);
}

kkt_status kkt_solve_jacobi(kkt_ctx *c, const double *b_dev, double *x_dev, int sweeps, int transpose,
                            kkt_stream stream) {
    ApiRange nvtx_range("kkt_solve_jacobi");
    REQUIRE_DEVICE(c);
    if (!b_dev || !x_dev || b_dev == x_dev || sweeps < 0) return KKT_ERR_ARG;
    if (!c->factored) return KKT_ERR_STATE;
    DeviceGuard g(c->dev);
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->rowperm) return jacobi_any(c, b_dev, x_dev, 0, transpose ? 1 : 0, sweeps, s);
    kkt_status st;
    if (!transpose) {                       // (Q A) x = Q b
        if ((st = q_vec(c, b_dev, c->d_qvec, true, s))) return st;
        return jacobi_any(c, c->d_qvec, x_dev, 0, 0, sweeps, s);
    }
    double *mu = c->d_qvec + c->an.n;       // (Q A)^T mu = g, lam = Q^T mu
    if ((st = jacobi_any(c, b_dev, mu, 0, 1, sweeps, s))) return st;
    return q_vec(c, mu, x_dev, false, s);
}

kkt_status kkt_solve(kkt_ctx *c, const double *b_dev, double *x_dev, kkt_stream stream) {
    ApiRange nvtx_range("kkt_solve");
    REQUIRE_DEVICE(c);
    if (!b_dev || !x_dev || b_dev == x_dev) return KKT_ERR_ARG;
    if (!c->factored) return KKT_ERR_STATE;
    DeviceGuard g(c->dev);
    cudaStream_t s = (cudaStream_t)stream;
    if (c->rowperm) {                       // (Q A) x = Q b: the columns, hence x, are not permuted
        kkt_status st = q_vec(c, b_dev, c->d_qvec, true, s);
        if (st) return st;
        b_dev = c->d_qvec;
    }
    return solve_any(c, b_dev, x_dev, 0, 0, s);
}

kkt_status kkt_solve_transpose(kkt_ctx *c, const double *g_dev, double *lam_dev, kkt_stream stream) {
    ApiRange nvtx_range("kkt_solve_transpose");
    REQUIRE_DEVICE(c);
    if (!g_dev || !lam_dev || g_dev == lam_dev) return KKT_ERR_ARG;
    if (!c->factored) return KKT_ERR_STATE;
    DeviceGuard g(c->dev);
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->rowperm) return solve_any(c, g_dev, lam_dev, 0, 1, s);
    double *mu = c->d_qvec + c->an.n;       // A^T lam = g  <=>  (Q A)^T (Q lam) = g
    kkt_status st = solve_any(c, g_dev, mu, 0, 1, s);
    if (st) return st;
    return q_vec(c, mu, lam_dev, false, s);
}

// residual + norms; returns omega on the host (synchronises the stream)
static kkt_status residual_omega(kkt_ctx *c, const double *b, const double *x, int transpose,
                                 cudaStream_t s, double *omega) {
    const int n = c->an.n;
    CK(cudaMemsetAsync(c->d_norms + NM_RMAX, 0, 3 * sizeof(unsigned long long), s));
    k_resid<<<norm_blocks(n), RTHREADS, 0, s>>>(c->P, c->values, b, x, c->d_rho, c->d_norms, transpose);
    CK(cudaGetLastError());
    c->launches++;
    CK(cudaMemcpyAsync(c->h_norms, c->d_norms, NM_WORDS * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    auto val = [&](int k) { double v; std::memcpy(&v, &c->h_norms[k], sizeof(v)); return v; };
    const double an = val(transpose ? NM_A1NORM : NM_ANORM);
    const double den = an * val(NM_XMAX) + val(NM_BMAX);
    const double r = val(NM_RMAX);
    *omega = den > 0 ? r / den : (r > 0 ? INFINITY : 0.0);
    if (std::isnan(*omega)) *omega = INFINITY;   // inf / inf: a non-finite entry somewhere
    return KKT_OK;
}

static kkt_status dot_to_host(kkt_ctx *c, const double *V, long long ld, int k, const double *w,
                              double *h_dev, int add, cudaStream_t s) {
    const int n = c->an.n;
    double *part = c->d_krylov + (size_t)(2 * c->kry_m + 2) * n;
    k_mdot<<<c->kry_blocks, 256, 0, s>>>(V, ld, k, w, n, part);
    CK(cudaGetLastError());
    c->launches++;
    k_mdot_fin<<<k, 256, 0, s>>>(part, c->kry_blocks, k, h_dev, add);
    CK(cudaGetLastError());
    c->launches++;
    return KKT_OK;
}

// One FGMRES(m) cycle from x (Saad 1993; Sec. 5.1: the LU factors as the
// preconditioner, classical Gram-Schmidt applied twice).  Uses at most
// max_apps preconditioner applications; returns the number used.
static kkt_status fgmres_cycle(kkt_ctx *c, const double *b, double *x, double tol, int max_apps,
                               int transpose, double anorm, double bnorm, double xnorm, double rinf,
                               int *used, cudaStream_t s) {
    const int n = c->an.n, m = std::min(c->kry_m, max_apps);
    *used = 0;
    if (m < 1) return KKT_OK;
    double *V = c->d_krylov, *Z = V + (size_t)(c->kry_m + 1) * n, *w = Z + (size_t)c->kry_m * n;
    double *coef = c->d_krylov + (size_t)(2 * c->kry_m + 2) * n + (size_t)c->kry_blocks * (c->kry_m + 1);
    double *h1 = coef, *h2 = coef + (c->kry_m + 2);
    const int nb = blocks_for(n, 256);
    kkt_status st;
    // r0 = b - A x (into w), beta = ||r0||_2
    k_spmv<<<blocks_for(8LL * n, 256), 256, 0, s>>>(c->P, c->values, x, w, transpose);
    CK(cudaGetLastError());
    c->launches++;
    {
        const double one = 1.0;
        CK(cudaMemcpyAsync(h1, &one, sizeof(double), cudaMemcpyHostToDevice, s));
    }
    // w = b - A x  via  w <- -(A x) + b : V[0] holds b temporarily
    CK(cudaMemcpyAsync(V, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    k_vcomb<<<nb, 256, 0, s>>>(V, w, 0, 1, h1, -1.0, n);    // V0 = b - Ax
    CK(cudaGetLastError());
    c->launches++;
    if ((st = dot_to_host(c, V, n, 1, V, h2, 0, s))) return st;
    double hb[2 * 66];
    CK(cudaMemcpyAsync(hb, h2, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double beta = std::sqrt(hb[0]);
    if (!(beta > 0.0)) return KKT_OK;
    k_vscale<<<nb, 256, 0, s>>>(V, V, 1.0 / beta, n);
    CK(cudaGetLastError());
    c->launches++;
    std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1, 0.0);
    g[0] = beta;
    int k_used = 0;
    for (int j = 0; j < m; j++) {
        double *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n;
        if ((st = precond_any(c, vj, zj, transpose, s))) return st;
        k_spmv<<<blocks_for(8LL * n, 256), 256, 0, s>>>(c->P, c->values, zj, w, transpose);
        CK(cudaGetLastError());
        c->launches++;
        // CGS2
        if ((st = dot_to_host(c, V, n, j + 1, w, h1, 0, s))) return st;
        k_vcomb<<<nb, 256, 0, s>>>(w, V, n, j + 1, h1, -1.0, n);
        CK(cudaGetLastError());
        c->launches++;
        if ((st = dot_to_host(c, V, n, j + 1, w, h2, 0, s))) return st;
        k_vcomb<<<nb, 256, 0, s>>>(w, V, n, j + 1, h2, -1.0, n);
        CK(cudaGetLastError());
        c->launches++;
        if ((st = dot_to_host(c, w, n, 1, w, h2 + j + 1, 0, s))) return st;
        CK(cudaMemcpyAsync(hb, h1, (j + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(hb + 66, h2, (j + 2) * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int q = 0; q <= j; q++) H[(size_t)q * m + j] = hb[q] + hb[66 + q];
        const double hnext = std::sqrt(hb[66 + j + 1]);
        H[(size_t)(j + 1) * m + j] = hnext;
        if (hnext > 0.0) {
            k_vscale<<<nb, 256, 0, s>>>(V + (size_t)(j + 1) * n, w, 1.0 / hnext, n);
            CK(cudaGetLastError());
            c->launches++;
        }
        for (int q = 0; q < j; q++) {
            const double t = cs[q] * H[(size_t)q * m + j] + sn[q] * H[(size_t)(q + 1) * m + j];
            H[(size_t)(q + 1) * m + j] = -sn[q] * H[(size_t)q * m + j] + cs[q] * H[(size_t)(q + 1) * m + j];
            H[(size_t)q * m + j] = t;
        }
        const double a0 = H[(size_t)j * m + j], a1 = H[(size_t)(j + 1) * m + j];
        const double den = std::hypot(a0, a1);
        cs[j] = den == 0.0 ? 1.0 : a0 / den;
        sn[j] = den == 0.0 ? 0.0 : a1 / den;
        H[(size_t)j * m + j] = cs[j] * a0 + sn[j] * a1;
        H[(size_t)(j + 1) * m + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        k_used = j + 1;
        // stop once the residual's infinity norm, estimated from its 2-norm |g|
        // times the ratio ||r0||_inf / ||r0||_2 of the cycle's first residual,
        // meets the target; the caller then measures omega itself (a 2-norm
        // test alone would overshoot by up to sqrt(n))
        if (std::fabs(g[j + 1]) * (rinf / beta) <= tol * (anorm * xnorm + bnorm) || hnext == 0.0) break;
    }
    // y = H^-1 g (upper triangular), x += Z y
    std::vector<double> y(k_used, 0.0);
    for (int q = k_used - 1; q >= 0; q--) {
        double t = g[q];
        for (int r = q + 1; r < k_used; r++) t -= H[(size_t)q * m + r] * y[r];
        y[q] = t / H[(size_t)q * m + q];
    }
    CK(cudaMemcpyAsync(h1, y.data(), k_used * sizeof(double), cudaMemcpyHostToDevice, s));
    k_vcomb<<<nb, 256, 0, s>>>(x, Z, n, k_used, h1, 1.0, n);
    CK(cudaGetLastError());
    c->launches++;
    CK(cudaStreamSynchronize(s));    // y lives on the host stack
    *used = k_used;
    return KKT_OK;
}

static double host_norm(const kkt_ctx *c, int k) {
    double v;
    std::memcpy(&v, &c->h_norms[k], sizeof(v));
    return v;
}

static kkt_status refine_any(kkt_ctx *c, const double *b, double *x, double tol, int max_it,
                             kkt_refine_info *info, int transpose, cudaStream_t s) {
    if (tol <= 0) tol = c->opt.tol;
    if (max_it < 0) max_it = c->opt.max_refine;
    if (info) std::memset(info, 0, sizeof(*info));
    const int mode = c->opt.refine_mode;
    double w;
    kkt_status st = residual_omega(c, b, x, transpose, s, &w);
    if (st) return st;
    int it = 0;
    if (info) info->omega_hist[info->n_hist++] = w;
    auto record = [&](double v) {
        if (info && info->n_hist < 64) info->omega_hist[info->n_hist++] = v;
    };
    if (mode == KKT_REFINE_CLASSIC || mode == KKT_REFINE_AUTO) {
        while (!(w <= tol) && it < max_it && std::isfinite(w)) {
            st = solve_any(c, c->d_rho, x, 1, transpose, s);
            if (st) return st;
            it++;
            const double prev = w;
            st = residual_omega(c, b, x, transpose, s, &w);
            if (st) return st;
            record(w);
            if (mode == KKT_REFINE_AUTO && !(w <= c->auto_ratio * prev) && !(w <= tol)) break;   // stalled
        }
    }
    if ((mode == KKT_REFINE_FGMRES || mode == KKT_REFINE_AUTO || mode == KKT_REFINE_FGMRES_JACOBI) &&
        c->d_krylov) {
        while (!(w <= tol) && it < max_it && std::isfinite(w)) {
            const double an = host_norm(c, transpose ? NM_A1NORM : NM_ANORM);
            int used = 0;
            st = fgmres_cycle(c, b, x, tol, max_it - it, transpose, an, host_norm(c, NM_BMAX),
                              host_norm(c, NM_XMAX), host_norm(c, NM_RMAX), &used, s);
            if (st) return st;
            it += used;
            st = residual_omega(c, b, x, transpose, s, &w);
            if (st) return st;
            record(w);
            if (used == 0) break;
        }
    }
    c->last_iters = it;
    c->last_omega = w;
    if (info) {
        info->iters = it;
        info->omega = w;
        info->converged = w <= tol;
    }
    int dst[ST_WORDS];
    CK(cudaMemcpy(dst, c->d_status, sizeof(dst), cudaMemcpyDeviceToHost));
    if (dst[ST_TIMEOUT]) return KKT_ERR_TIMEOUT;
    // a NaN or infinity in x, b or the residual (omega = inf), or one flagged
    // earlier by the refactorization, makes the result unusable
    if (!std::isfinite(w) || dst[ST_NONFINITE]) return KKT_ERR_NONFINITE;
    return (w <= tol) ? KKT_OK : KKT_ERR_NOT_CONVERGED;
}

kkt_status kkt_refine(kkt_ctx *c, const double *b_dev, double *x_dev, double tol, int max_it,
                      kkt_refine_info *info, kkt_stream stream) {
    ApiRange nvtx_range("kkt_refine");
    REQUIRE_DEVICE(c);
    if (!b_dev || !x_dev || b_dev == x_dev) return KKT_ERR_ARG;
    if (!c->factored) return KKT_ERR_STATE;
    DeviceGuard g(c->dev);
    cudaStream_t s = (cudaStream_t)stream;
    if (c->rowperm) {                       // the residual of Q A x = Q b has the norms of A x = b
        kkt_status st = q_vec(c, b_dev, c->d_qvec, true, s);
        if (st) return st;
        b_dev = c->d_qvec;
    }
    return refine_any(c, b_dev, x_dev, tol, max_it, info, 0, s);
}

kkt_status kkt_refine_transpose(kkt_ctx *c, const double *g_dev, double *lam_dev, double tol,
                                int max_it, kkt_refine_info *info, kkt_stream stream) {
    ApiRange nvtx_range("kkt_refine_transpose");
    REQUIRE_DEVICE(c);
    if (!g_dev || !lam_dev || g_dev == lam_dev) return KKT_ERR_ARG;
    if (!c->factored) return KKT_ERR_STATE;
    DeviceGuard g(c->dev);
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->rowperm) return refine_any(c, g_dev, lam_dev, tol, max_it, info, 1, s);
    double *mu = c->d_qvec + c->an.n;       // refine mu = Q lam on (Q A)^T mu = g
    kkt_status st = q_vec(c, lam_dev, mu, true, s);
    if (st) return st;
    const kkt_status r = refine_any(c, g_dev, mu, tol, max_it, info, 1, s);
    if (r == KKT_ERR_CUDA) return r;
    st = q_vec(c, mu, lam_dev, false, s);
    return st ? st : r;
}

// ---------------------------------------------------------------------------
// batched entry points

static void ensure_view(const kkt_ctx *c);

#define REQUIRE_BATCH(c, B)                                                                  \
    do {                                                                                     \
        REQUIRE_DEVICE(c);                                                                   \
        if ((c)->rowperm) {                                                                  \
            g_last_error = "batched calls do not support a row permutation";                 \
            return KKT_ERR_STATE;                                                            \
        }                                                                                    \
        if ((B) < 1 || (B) > (c)->bcap) {                                                    \
            g_last_error = "batch size outside 1..max_batch (set max_batch at analysis)";    \
            return KKT_ERR_ARG;                                                              \
        }                                                                                    \
    } while (0)

template <typename T> static kkt_status launch_brefactor(kkt_ctx *c, int B, cudaStream_t s) {
    const int n = c->an.n;
    // every entry starts as the not-ready marker; published entries overwrite it
    CK(cudaMemsetAsync(c->b_lu, 0xff, (size_t)c->nnz_lu * B * sizeof(T), s));
    CK(cudaMemsetAsync(c->b_rcp, 0xff, (size_t)n * B * sizeof(T), s));
    k_brefactor<T><<<c->grid, c->cta_warps * 32, c->smem, s>>>(c->P, c->rc, B, c->b_values, c->b_sp, c->b_norms,
                                                          (T *)c->b_lu, (T *)c->b_lut, (T *)c->b_rcp, c->tau_rel);
    CK(cudaGetLastError());
    c->launches++;
    return KKT_OK;
}

kkt_status kkt_batch_refactor(kkt_ctx *c, int B, const double *values_dev, kkt_stream stream) {
    ApiRange nvtx_range("kkt_batch_refactor");
    REQUIRE_BATCH(c, B);
    if (!values_dev) return KKT_ERR_ARG;
    DeviceGuard g(c->dev);
    cudaStream_t s = (cudaStream_t)stream;
    const int n = c->an.n;
    c->b_values = values_dev;
    CK(cudaMemsetAsync(c->b_norms, 0, NM_WORDS * (size_t)B * sizeof(unsigned long long), s));
    k_bscale<<<blocks_for((long long)n * B, 256), 256, 0, s>>>(c->P, B, values_dev, c->b_s, c->b_sp, c->b_norms,
                                                              c->d_status, c->opt.equilibrate);
    CK(cudaGetLastError());
    c->launches++;
    k_bamax<<<blocks_for((long long)n * B, 256), 256, 0, s>>>(c->P, B, values_dev, c->b_s, c->b_norms);
    CK(cudaGetLastError());
    c->launches++;
    kkt_status r = c->opt.factor_fp32 ? launch_brefactor<float>(c, B, s) : launch_brefactor<double>(c, B, s);
    if (r == KKT_OK) c->b_factored = B;
    return r;
}

template <typename T>
static kkt_status launch_bsolve(kkt_ctx *c, int B, const double *b, double *x, int accumulate, int transpose,
                                cudaStream_t s) {
    const int n = c->an.n;
    T *y = (T *)c->b_y, *z = y + (size_t)n * B;
    const T *F = (const T *)(transpose ? c->b_lut : c->b_lu), *R = (const T *)c->b_rcp;
    CK(cudaMemsetAsync(y, 0xff, 2 * (size_t)n * B * sizeof(T), s));
    if (transpose) {
        k_btrisolve<T, false, true><<<c->bsolve_grid, c->cta_warps * 32, c->bsolve_smem, s>>>(
            c->P, c->rc, c->tk, B, F, R, b, c->b_sp, nullptr, y, nullptr, 0);
        CK(cudaGetLastError());
        c->launches++;
        k_btrisolve<T, true, true><<<c->bsolve_grid, c->cta_warps * 32, c->bsolve_smem, s>>>(
            c->P, c->rc, c->tk, B, F, R, nullptr, c->b_sp, y, z, x, accumulate);
    } else {
        k_btrisolve<T, false, false><<<c->bsolve_grid, c->cta_warps * 32, c->bsolve_smem, s>>>(
            c->P, c->rc, c->tk, B, F, R, b, c->b_sp, nullptr, y, nullptr, 0);
        CK(cudaGetLastError());
        c->launches++;
        k_btrisolve<T, true, false><<<c->bsolve_grid, c->cta_warps * 32, c->bsolve_smem, s>>>(
            c->P, c->rc, c->tk, B, F, R, nullptr, c->b_sp, y, z, x, accumulate);
    }
    CK(cudaGetLastError());
    c->launches++;
    return KKT_OK;
}

static kkt_status bsolve_any(kkt_ctx *c, int B, const double *b, double *x, int accumulate, int transpose,
                             cudaStream_t s) {
    return c->opt.factor_fp32 ? launch_bsolve<float>(c, B, b, x, accumulate, transpose, s)
                              : launch_bsolve<double>(c, B, b, x, accumulate, transpose, s);
}

kkt_status kkt_batch_solve(kkt_ctx *c, int B, const double *b_dev, double *x_dev, kkt_stream stream) {
    ApiRange nvtx_range("kkt_batch_solve");
    REQUIRE_BATCH(c, B);
    if (!b_dev || !x_dev || b_dev == x_dev) return KKT_ERR_ARG;
    if (c->b_factored != B) return KKT_ERR_STATE;
    DeviceGuard g(c->dev);
    return bsolve_any(c, B, b_dev, x_dev, 0, 0, (cudaStream_t)stream);
}

kkt_status kkt_batch_solve_transpose(kkt_ctx *c, int B, const double *g_dev, double *lam_dev,
                                     kkt_stream stream) {
    ApiRange nvtx_range("kkt_batch_solve_transpose");
    REQUIRE_BATCH(c, B);
    if (!g_dev || !lam_dev || g_dev == lam_dev) return KKT_ERR_ARG;
    if (c->b_factored != B) return KKT_ERR_STATE;
    DeviceGuard g(c->dev);
    return bsolve_any(c, B, g_dev, lam_dev, 0, 1, (cudaStream_t)stream);
}

static kkt_status bresidual_omega(kkt_ctx *c, int B, const double *b, const double *x, int transpose,
                                  cudaStream_t s, double *omega) {
    const int n = c->an.n;
    for (int k = NM_RMAX; k <= NM_BMAX; k++)
        CK(cudaMemsetAsync(c->b_norms + (size_t)k * B, 0, B * sizeof(unsigned long long), s));
    k_bresid<<<blocks_for((long long)n * B, 256), 256, 0, s>>>(c->P, B, c->b_values, b, x, c->b_rho, c->b_norms,
                                                              transpose);
    CK(cudaGetLastError());
    c->launches++;
    CK(cudaMemcpyAsync(c->hb_norms, c->b_norms, NM_WORDS * (size_t)B * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    auto val = [&](int k, int sy) {
        double v;
        std::memcpy(&v, &c->hb_norms[(size_t)k * B + sy], sizeof(v));
        return v;
    };
    for (int sy = 0; sy < B; sy++) {
        const double an = val(transpose ? NM_A1NORM : NM_ANORM, sy);
        const double den = an * val(NM_XMAX, sy) + val(NM_BMAX, sy);
        const double r = val(NM_RMAX, sy);
        omega[sy] = den > 0 ? r / den : (r > 0 ? INFINITY : 0.0);
        if (std::isnan(omega[sy])) omega[sy] = INFINITY;
    }
    return KKT_OK;
}

static kkt_status brefine_any(kkt_ctx *c, int B, const double *b, double *x, double tol, int max_it,
                              double *omega_host, int *iters, int transpose, cudaStream_t s) {
    if (tol <= 0) tol = c->opt.tol;
    if (max_it < 0) max_it = c->opt.max_refine;
    std::vector<double> w(B);
    kkt_status st = bresidual_omega(c, B, b, x, transpose, s, w.data());
    if (st) return st;
    int it = 0;
    auto worst = [&]() {
        double m = 0.0;
        for (double v : w) m = std::isfinite(v) ? std::max(m, v) : INFINITY;
        return m;
    };
    while (!(worst() <= tol) && it < max_it && std::isfinite(worst())) {
        st = bsolve_any(c, B, c->b_rho, x, 1, transpose, s);
        if (st) return st;
        it++;
        st = bresidual_omega(c, B, b, x, transpose, s, w.data());
        if (st) return st;
    }
    if (omega_host) std::memcpy(omega_host, w.data(), B * sizeof(double));
    if (iters) *iters = it;
    int dst[ST_WORDS];
    CK(cudaMemcpy(dst, c->d_status, sizeof(dst), cudaMemcpyDeviceToHost));
    if (dst[ST_TIMEOUT]) return KKT_ERR_TIMEOUT;
    if (!std::isfinite(worst()) || dst[ST_NONFINITE]) return KKT_ERR_NONFINITE;
    return worst() <= tol ? KKT_OK : KKT_ERR_NOT_CONVERGED;
}

kkt_status kkt_batch_refine(kkt_ctx *c, int B, const double *b_dev, double *x_dev, double tol, int max_it,
                            double *omega_host, int *iters, kkt_stream stream) {
    ApiRange nvtx_range("kkt_batch_refine");
    REQUIRE_BATCH(c, B);
    if (!b_dev || !x_dev || b_dev == x_dev) return KKT_ERR_ARG;
    if (c->b_factored != B) return KKT_ERR_STATE;
    DeviceGuard g(c->dev);
    return brefine_any(c, B, b_dev, x_dev, tol, max_it, omega_host, iters, 0, (cudaStream_t)stream);
}

kkt_status kkt_batch_refine_transpose(kkt_ctx *c, int B, const double *g_dev, double *lam_dev, double tol,
                                      int max_it, double *omega_host, int *iters, kkt_stream stream) {
    ApiRange nvtx_range("kkt_batch_refine_transpose");
    REQUIRE_BATCH(c, B);
    if (!g_dev || !lam_dev || g_dev == lam_dev) return KKT_ERR_ARG;
    if (c->b_factored != B) return KKT_ERR_STATE;
    DeviceGuard g(c->dev);
    return brefine_any(c, B, g_dev, lam_dev, tol, max_it, omega_host, iters, 1, (cudaStream_t)stream);
}

kkt_status kkt_batch_export_factors(kkt_ctx *c, int sys, double *out_dev, kkt_stream stream) {
    REQUIRE_DEVICE(c);
    if (!out_dev || sys < 0 || sys >= c->b_factored) return KKT_ERR_ARG;
    DeviceGuard g(c->dev);
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->d_view_slot) {
        ensure_view(c);
        CK(cudaMalloc(&c->d_view_slot, c->view_slot.size() * sizeof(int)));
        CK(cudaMemcpy(c->d_view_slot, c->view_slot.data(), c->view_slot.size() * sizeof(int),
                      cudaMemcpyHostToDevice));
    }
    const int B = c->b_factored;
    if (c->opt.factor_fp32)
        k_bexport<float><<<blocks_for(c->nnz_lu, 256), 256, 0, s>>>((const float *)c->b_lu, c->d_view_slot, B, sys,
                                                                    out_dev, c->nnz_lu);
    else
        k_bexport<double><<<blocks_for(c->nnz_lu, 256), 256, 0, s>>>((const double *)c->b_lu, c->d_view_slot, B,
                                                                     sys, out_dev, c->nnz_lu);
    CK(cudaGetLastError());
    c->launches++;
    return KKT_OK;
}

// ---------------------------------------------------------------------------
// uneven-pattern queue

struct kkt_queue {
    std::vector<kkt_ctx *> ctx;
    int m = 0, dev = -1;
    bool f32 = false;
    QSys *d_sys = nullptr;
    std::vector<QSys> h_sys;
    int2 *d_items = nullptr;          // refactor | forward | backward items
    int n_ref = 0, n_fwd = 0, n_bwd = 0;
    // With CTAs of WARPS warps the solves run the longest tasks (from the
    // contexts' CTA tasks) on a CTA each: d_chains (system, chain index), and
    // d_items_reg the forward | backward items without them.
    int nch = 0, n_fwd_reg = 0, n_bwd_reg = 0;
    int2 *d_chains = nullptr, *d_items_reg = nullptr;
    size_t smem_chain = 0;
    // the candidates (longest first: length, system, chain index; at most
    // QCHAIN_MAX) and the solve items; kkt_queue_set_tiles picks how many
    // candidates run as CTA tasks
    std::vector<std::array<int, 3>> cand;
    std::vector<int2> fwd_items, bwd_items;
    int ctas_opt = 0;
    Sched *d_sched = nullptr;
    int *d_status = nullptr;
    void *d_scratch = nullptr;
    RunCfg rc{};
    int cta_warps = WARPS, grid = 0, sgrid = 0, cap = 32, tcap = 1;
    size_t smem_ref = 0, smem_sol = 0;
    cudaGraphExec_t graph = nullptr;
    std::vector<const void *> key;    // pointers and settings the captured graph was built with
    long long launches = 0;
};

template <typename T> static kkt_status q_set_smem(kkt_queue *q) {
    CK(ensure_smem((const void *)k_qrefactor<T>, q->smem_ref));
    CK(ensure_smem((const void *)k_qtrisolve<T, false, false>, q->smem_sol));
    CK(ensure_smem((const void *)k_qtrisolve<T, true, false>, q->smem_sol));
    CK(ensure_smem((const void *)k_qtrisolve<T, false, true>, q->smem_sol));
    CK(ensure_smem((const void *)k_qtrisolve<T, true, true>, q->smem_sol));
    return KKT_OK;
}

// The first k candidates run as CTA tasks (with CTAs of WARPS warps); the
// other tasks stay warp items.
static kkt_status q_set_chains(kkt_queue *q, int k) {
    k = std::max(0, std::min(k, (int)q->cand.size()));
    std::vector<int2> chains;
    std::set<std::pair<int, int>> taken;           // (system, task)
    const size_t tsz = q->f32 ? sizeof(float) : sizeof(double);
    q->smem_chain = 0;
    for (int j = 0; j < k; j++) {
        const auto &cd = q->cand[j];
        const kkt_ctx *c = q->ctx[cd[1]];
        chains.push_back(make_int2(cd[1], cd[2]));
        taken.insert({cd[1], c->chain_h[cd[2]]});
        q->smem_chain = std::max(q->smem_chain, chain_smem_bytes(c->tk1.zcap, tsz));
    }
    std::vector<int2> reg;
    for (auto &v : q->fwd_items)
        if (!taken.count({v.x, v.y})) reg.push_back(v);
    q->n_fwd_reg = (int)reg.size();
    for (auto &v : q->bwd_items)
        if (!taken.count({v.x, v.y})) reg.push_back(v);
    q->n_bwd_reg = (int)reg.size() - q->n_fwd_reg;
    q->nch = k;
    if (k > 0) CK(cudaMemcpy(q->d_chains, chains.data(), chains.size() * sizeof(int2), cudaMemcpyHostToDevice));
    if (!reg.empty()) CK(cudaMemcpy(q->d_items_reg, reg.data(), reg.size() * sizeof(int2), cudaMemcpyHostToDevice));
    if (q->graph) { cudaGraphExecDestroy(q->graph); q->graph = nullptr; }
    q->key.clear();
    return KKT_OK;
}

static kkt_status q_configure(kkt_queue *q, int cta_warps, int ctas) {
    const size_t tsz = q->f32 ? sizeof(float) : sizeof(double);
    q->cta_warps = std::max(1, std::min(cta_warps > 0 ? cta_warps : WARPS, WARPS));
    const int nw = q->cta_warps;
    q->smem_ref = (size_t)nw * q->cap * (tsz + sizeof(int));
    q->smem_sol = (size_t)nw * q->tcap * tsz;
    if (nw == WARPS && q->nch > 0) q->smem_sol = std::max(q->smem_sol, q->smem_chain);
    kkt_status st = q->f32 ? q_set_smem<float>(q) : q_set_smem<double>(q);
    if (st) return st;
    int sms = 0, per_sm = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, q->dev));
    if (q->f32)
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qrefactor<float>, nw * 32, q->smem_ref));
    else
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qrefactor<double>, nw * 32, q->smem_ref));
    if (per_sm < 1) { g_last_error = "queue refactor kernel does not fit on an SM"; return KKT_ERR_CUDA; }
    q->grid = ctas > 0 ? std::min(ctas, sms * per_sm) : sms * per_sm;
    int per_sm_s = 0;
    if (q->f32)
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_s, k_qtrisolve<float, false, false>, nw * 32, q->smem_sol));
    else
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_s, k_qtrisolve<double, false, false>, nw * 32, q->smem_sol));
    q->sgrid = ctas > 0 ? std::min(ctas, sms * std::max(per_sm_s, 1)) : sms * std::min(std::max(per_sm_s, 1), 2);
    // scratch for rows longer than the shared-memory row
    int longest = 0;
    for (auto *c : q->ctx) if (c->an.max_row > q->cap) longest = std::max(longest, c->an.max_row);
    cudaFree(q->d_scratch);
    q->d_scratch = nullptr;
    q->rc.scratch_stride = 0;
    if (longest > 0) {
        CK(cudaMalloc(&q->d_scratch, (size_t)longest * tsz * q->grid * nw));
        q->rc.scratch_stride = longest;
    }
    q->rc.scratch = q->d_scratch;
    q->rc.cap = q->cap;
    if (q->graph) { cudaGraphExecDestroy(q->graph); q->graph = nullptr; }
    q->key.clear();
    return KKT_OK;
}

kkt_status kkt_queue_create(kkt_ctx *const *ctxs, int m, kkt_queue **out) {
    if (!ctxs || m < 1 || !out) return KKT_ERR_ARG;
    *out = nullptr;
    std::unique_ptr<kkt_queue> q(new (std::nothrow) kkt_queue());
    if (!q) return KKT_ERR_ALLOC;
    q->m = m;
    for (int k = 0; k < m; k++) {
        kkt_ctx *c = ctxs[k];
        if (!c || c->host_only) { g_last_error = "queue needs device contexts"; return KKT_ERR_ARG; }
        if (c->rowperm) { g_last_error = "queue contexts cannot carry a row permutation"; return KKT_ERR_STATE; }
        if (k && (c->dev != ctxs[0]->dev || c->opt.factor_fp32 != ctxs[0]->opt.factor_fp32)) {
            g_last_error = "queue contexts must share the device and the factor precision";
            return KKT_ERR_ARG;
        }
        q->ctx.push_back(c);
    }
    q->dev = ctxs[0]->dev;
    q->f32 = ctxs[0]->opt.factor_fp32 != 0;
    DeviceGuard g(q->dev);
    // items: refactor rows deepest first (by distance to the root, across
    // systems), forward solve tasks by depth of their top row, deepest first;
    // backward solve tasks by height of their top row, from the root (each a
    // topological order of every system; see the single-system claim orders)
    std::vector<std::array<int, 4>> ref, fwd, bwd;
    for (int k = 0; k < m; k++) {
        const Analysis &a = q->ctx[k]->an;
        for (int r = 0; r < a.n; r++) ref.push_back({-a.level_u[a.order_f[r]], k, r, a.order_f[r]});
        for (int t = 0; t < (int)a.task_lo.size(); t++) {
            const int top = a.level[a.task_hi[t]];
            fwd.push_back({-a.level_u[a.task_hi[t]], k, t, t});
            bwd.push_back({-top, k, t, t});
        }
        q->cap = std::max(q->cap, q->ctx[k]->cap);
        q->tcap = std::max(q->tcap, q->ctx[k]->tk.cap);
    }
    std::sort(ref.begin(), ref.end());
    std::sort(fwd.begin(), fwd.end());
    std::sort(bwd.begin(), bwd.end());
    std::vector<int2> items;
    for (auto &v : ref) items.push_back(make_int2(v[1], v[3]));
    for (auto &v : fwd) items.push_back(make_int2(v[1], v[3]));
    for (auto &v : bwd) items.push_back(make_int2(v[1], v[3]));
    q->n_ref = (int)ref.size();
    q->n_fwd = (int)fwd.size();
    q->n_bwd = (int)bwd.size();
    CK(cudaMalloc(&q->d_items, items.size() * sizeof(int2)));
    CK(cudaMemcpy(q->d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice));
    {   // CTA-task candidates: the longest of the contexts' CTA tasks, at most QCHAIN_MAX
        for (int k = 0; k < m; k++) {
            const kkt_ctx *c = q->ctx[k];
            for (int ci = 0; ci < (int)c->chain_h.size(); ci++) {
                const int T = c->chain_h[ci];
                q->cand.push_back({c->an.task_hi[T] - c->an.task_lo[T] + 1, k, ci});
            }
        }
        std::stable_sort(q->cand.begin(), q->cand.end(),
                         [](const std::array<int, 3> &x, const std::array<int, 3> &y) { return x[0] > y[0]; });
        if ((int)q->cand.size() > QCHAIN_MAX) q->cand.resize(QCHAIN_MAX);
        for (auto &v : fwd) q->fwd_items.push_back(make_int2(v[1], v[3]));
        for (auto &v : bwd) q->bwd_items.push_back(make_int2(v[1], v[3]));
        CK(cudaMalloc(&q->d_chains, std::max<size_t>(1, q->cand.size()) * sizeof(int2)));
        CK(cudaMalloc(&q->d_items_reg, std::max<size_t>(1, q->fwd_items.size() + q->bwd_items.size()) * sizeof(int2)));
    }
    CK(cudaMalloc(&q->d_sys, m * sizeof(QSys)));
    CK(cudaMalloc(&q->d_sched, sizeof(Sched)));
    CK(cudaMemset(q->d_sched, 0, sizeof(Sched)));
    CK(cudaMalloc(&q->d_status, ST_WORDS * sizeof(int)));
    CK(cudaMemset(q->d_status, 0, ST_WORDS * sizeof(int)));
    q->h_sys.resize(m);
    for (int k = 0; k < m; k++) {
        kkt_ctx *c = q->ctx[k];
        QSys &s = q->h_sys[k];
        std::memset(&s, 0, sizeof(s));
        s.P = c->P;
        s.tk = c->tk;
        s.LU = c->d_lu;
        s.LUT = c->d_lut;
        s.rcp = c->d_rcp;
        s.y = c->d_y;
        s.sp = c->d_sp;
        s.norms = c->d_norms;
        s.rho = c->d_rho;
        s.tau_rel = c->tau_rel;
        s.n = c->an.n;
        for (int ph = 0; ph < 4; ph++) {
            s.tkc[ph] = tasks_of(c, ph & 1, ph >= 2);
            s.tkc[ph].ext = nullptr;           // a queue's CTA tasks sum their outside parts themselves
            s.tkc[ph].far = nullptr;           // and their far sources
            s.tkc[ph].npart = 0;
        }
    }
    q->rc = ctxs[0]->rc;
    q->rc.status = q->d_status;
    q->rc.sched = q->d_sched;
    q->rc.trace = nullptr;
    q->rc.unpublished_row = -1;
    kkt_status st = q_set_chains(q.get(), (int)q->cand.size());
    if (st == KKT_OK) st = q_configure(q.get(), 0, 0);
    if (st) { kkt_queue_destroy(q.release()); return st; }
    *out = q.release();
    return KKT_OK;
}

void kkt_queue_destroy(kkt_queue *q) {
    if (!q) return;
    DeviceGuard g(q->dev);
    if (q->graph) cudaGraphExecDestroy(q->graph);
    cudaFree(q->d_items);
    cudaFree(q->d_chains);
    cudaFree(q->d_items_reg);
    cudaFree(q->d_sys);
    cudaFree(q->d_sched);
    cudaFree(q->d_status);
    cudaFree(q->d_scratch);
    delete q;
}

kkt_status kkt_queue_set_launch(kkt_queue *q, int cta_warps, int ctas) {
    if (!q || cta_warps < 0 || ctas < 0) return KKT_ERR_ARG;
    DeviceGuard g(q->dev);
    q->ctas_opt = ctas;
    return q_configure(q, cta_warps, ctas);
}

kkt_status kkt_queue_set_tiles(kkt_queue *q, int cta_tasks) {
    if (!q || cta_tasks < -1) return KKT_ERR_ARG;
    DeviceGuard g(q->dev);
    kkt_status st = q_set_chains(q, cta_tasks < 0 ? (int)q->cand.size() : cta_tasks);
    if (st) return st;
    return q_configure(q, q->cta_warps, q->ctas_opt);
}

template <typename T>
static kkt_status q_record(kkt_queue *q, int n_refine, double *omega_dev, cudaStream_t s) {
    const int nw = q->cta_warps;
    const int2 *ir = q->d_items, *iff = ir + q->n_ref, *ib = iff + q->n_fwd;
    for (int k = 0; k < q->m; k++) {
        kkt_ctx *c = q->ctx[k];
        const QSys &h = q->h_sys[k];
        const int n = c->an.n;
        CK(cudaMemsetAsync(c->d_norms, 0, NM_WORDS * sizeof(unsigned long long), s));
        k_scale<<<norm_blocks(n), RTHREADS, 0, s>>>(c->P, h.values, c->d_s, c->d_sp, c->d_norms, q->d_status,
                                                         c->opt.equilibrate);
        CK(cudaGetLastError());
        k_amax<<<norm_blocks(n), RTHREADS, 0, s>>>(c->P, h.values, c->d_s, c->d_norms);
        CK(cudaGetLastError());
        CK(cudaMemsetAsync(c->d_lu, 0xff, (size_t)c->nnz_lu * sizeof(T), s));
        CK(cudaMemsetAsync(c->d_rcp, 0xff, (size_t)n * sizeof(T), s));
        q->launches += 2;
    }
    k_qrefactor<T><<<q->grid, nw * 32, q->smem_ref, s>>>(q->d_sys, ir, q->n_ref, q->rc);
    CK(cudaGetLastError());
    q->launches++;
    // tiles of the contexts' CTA tasks from the new factors
    for (int k = 0; k < q->m; k++) {
        kkt_ctx *c = q->ctx[k];
        if (c->nblk == 0) continue;
        const long long threads = 4LL * c->nblk * 2 * CB * 32;
        k_pack_tiles<T><<<blocks_for(threads, 256), 256, 0, s>>>(
            c->P, c->blk_info, c->nblk, c->cs_fwd, c->csd_fwd, c->cs_bwd, c->csd_bwd, (const T *)c->d_lu,
            (const T *)c->d_lut, (const T *)c->d_rcp, (T *)c->d_tiles);
        CK(cudaGetLastError());
        q->launches++;
    }
    const bool cta = (nw == WARPS && q->nch > 0);
    const int nch = cta ? q->nch : 0;
    const int2 *sf = cta ? q->d_items_reg : iff, *sb = cta ? q->d_items_reg + q->n_fwd_reg : ib;
    const int nf = cta ? q->n_fwd_reg : q->n_fwd, nbk = cta ? q->n_bwd_reg : q->n_bwd;
    for (int pass = 0; pass <= n_refine; pass++) {
        if (pass > 0) {
            for (int k = 0; k < q->m; k++) {
                kkt_ctx *c = q->ctx[k];
                const QSys &h = q->h_sys[k];
                CK(cudaMemsetAsync(c->d_norms + NM_RMAX, 0, 3 * sizeof(unsigned long long), s));
                k_resid<<<norm_blocks(c->an.n), RTHREADS, 0, s>>>(c->P, h.values, h.b, h.x, c->d_rho,
                                                                      c->d_norms, 0);
                CK(cudaGetLastError());
                q->launches++;
            }
        }
        for (int k = 0; k < q->m; k++)
            CK(cudaMemsetAsync(q->ctx[k]->d_y, 0xff, 2 * (size_t)q->ctx[k]->an.n * sizeof(T), s));
        k_qtrisolve<T, false, false><<<q->sgrid, nw * 32, q->smem_sol, s>>>(q->d_sys, sf, nf, q->rc, pass > 0,
                                                                            q->tcap, q->d_chains, nch);
        CK(cudaGetLastError());
        k_qtrisolve<T, true, false><<<q->sgrid, nw * 32, q->smem_sol, s>>>(q->d_sys, sb, nbk, q->rc, pass > 0,
                                                                           q->tcap, q->d_chains, nch);
        CK(cudaGetLastError());
        q->launches += 2;
    }
    if (omega_dev) {
        for (int k = 0; k < q->m; k++) {
            kkt_ctx *c = q->ctx[k];
            const QSys &h = q->h_sys[k];
            CK(cudaMemsetAsync(c->d_norms + NM_RMAX, 0, 3 * sizeof(unsigned long long), s));
            k_resid<<<norm_blocks(c->an.n), RTHREADS, 0, s>>>(c->P, h.values, h.b, h.x, c->d_rho, c->d_norms, 0);
            CK(cudaGetLastError());
            k_omega<<<1, 1, 0, s>>>(c->d_norms, omega_dev + k);
            CK(cudaGetLastError());
            q->launches += 2;
        }
    }
    return KKT_OK;
}

kkt_status kkt_queue_run(kkt_queue *q, const double *const *values, const double *const *b, double *const *x,
                         int n_refine, double *omega_dev, kkt_stream stream) {
    ApiRange nvtx_range("kkt_queue_run");
    if (!q || !values || !b || !x || n_refine < 0) return KKT_ERR_ARG;
    DeviceGuard g(q->dev);
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<const void *> key;
    for (int k = 0; k < q->m; k++) {
        if (!values[k] || !b[k] || !x[k] || (const void *)b[k] == (const void *)x[k]) return KKT_ERR_ARG;
        key.push_back(values[k]);
        key.push_back(b[k]);
        key.push_back(x[k]);
    }
    key.push_back((const void *)(intptr_t)n_refine);
    key.push_back(omega_dev);
    if (!q->graph || key != q->key) {
        // new buffers or settings: refresh the system table and record the graph again
        for (int k = 0; k < q->m; k++) {
            q->h_sys[k].values = values[k];
            q->h_sys[k].b = b[k];
            q->h_sys[k].x = x[k];
        }
        CK(cudaStreamSynchronize(s));
        CK(cudaMemcpy(q->d_sys, q->h_sys.data(), q->m * sizeof(QSys), cudaMemcpyHostToDevice));
        if (q->graph) { cudaGraphExecDestroy(q->graph); q->graph = nullptr; }
        cudaStream_t cs;
        CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t gr;
        CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        kkt_status st = q->f32 ? q_record<float>(q, n_refine, omega_dev, cs) : q_record<double>(q, n_refine, omega_dev, cs);
        cudaError_t e = cudaStreamEndCapture(cs, &gr);
        cudaStreamDestroy(cs);
        if (st) return st;
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&q->graph, gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        q->key = key;
    }
    // every run writes new factors and packs the contexts' tiles from them
    for (int k = 0; k < q->m; k++) {
        q->ctx[k]->values = values[k];
        q->ctx[k]->factored = true;
        q->ctx[k]->tiles_fresh = true;
    }
    CK(cudaGraphLaunch(q->graph, s));
    return KKT_OK;
}

kkt_status kkt_queue_solve_transpose(kkt_queue *q, const double *const *g_, double *const *lam, kkt_stream stream) {
    ApiRange nvtx_range("kkt_queue_solve_transpose");
    if (!q || !g_ || !lam) return KKT_ERR_ARG;
    DeviceGuard g(q->dev);
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < q->m; k++) {
        if (!g_[k] || !lam[k] || (const void *)g_[k] == (const void *)lam[k]) return KKT_ERR_ARG;
        q->h_sys[k].g = g_[k];
        q->h_sys[k].lam = lam[k];
    }
    CK(cudaStreamSynchronize(s));
    CK(cudaMemcpy(q->d_sys, q->h_sys.data(), q->m * sizeof(QSys), cudaMemcpyHostToDevice));
    const int nw = q->cta_warps;
    const int2 *iff = q->d_items + q->n_ref, *ib = iff + q->n_fwd;
    for (int k = 0; k < q->m; k++) {
        kkt_ctx *c = q->ctx[k];
        if (!c->tiles_fresh) {              // factors of a single-system refactor not yet packed
            kkt_status r = q->f32 ? pack_tiles<float>(c, s) : pack_tiles<double>(c, s);
            if (r != KKT_OK) return r;
        }
        CK(cudaMemsetAsync(c->d_y, 0xff, 2 * (size_t)c->an.n * (q->f32 ? sizeof(float) : sizeof(double)), s));
    }
    const bool cta = (nw == WARPS && q->nch > 0);
    const int nch = cta ? q->nch : 0;
    const int2 *sf = cta ? q->d_items_reg : iff, *sb = cta ? q->d_items_reg + q->n_fwd_reg : ib;
    const int nf = cta ? q->n_fwd_reg : q->n_fwd, nbk = cta ? q->n_bwd_reg : q->n_bwd;
    if (q->f32) {
        k_qtrisolve<float, false, true><<<q->sgrid, nw * 32, q->smem_sol, s>>>(q->d_sys, sf, nf, q->rc, 0, q->tcap,
                                                                               q->d_chains, nch);
        CK(cudaGetLastError());
        k_qtrisolve<float, true, true><<<q->sgrid, nw * 32, q->smem_sol, s>>>(q->d_sys, sb, nbk, q->rc, 0, q->tcap,
                                                                              q->d_chains, nch);
    } else {
        k_qtrisolve<double, false, true><<<q->sgrid, nw * 32, q->smem_sol, s>>>(q->d_sys, sf, nf, q->rc, 0, q->tcap,
                                                                                q->d_chains, nch);
        CK(cudaGetLastError());
        k_qtrisolve<double, true, true><<<q->sgrid, nw * 32, q->smem_sol, s>>>(q->d_sys, sb, nbk, q->rc, 0, q->tcap,
                                                                               q->d_chains, nch);
    }
    CK(cudaGetLastError());
    q->launches += 2;
    return KKT_OK;
}

kkt_status kkt_queue_status_sync(kkt_queue *q, kkt_stream stream, int *n_perturbed) {
    if (!q) return KKT_ERR_ARG;
    DeviceGuard g(q->dev);
    int st[ST_WORDS];
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    CK(cudaMemcpy(st, q->d_status, sizeof(st), cudaMemcpyDeviceToHost));
    CK(cudaMemset(q->d_status, 0, sizeof(st)));
    if (n_perturbed) *n_perturbed = st[ST_PERTURBED];
    if (st[ST_INTERNAL]) return KKT_ERR_INTERNAL;
    if (st[ST_TIMEOUT]) return KKT_ERR_TIMEOUT;
    if (st[ST_NONFINITE]) return KKT_ERR_NONFINITE;
    if (st[ST_PERTURBED]) return KKT_WARN_PERTURBED;
    return KKT_OK;
}

kkt_status kkt_adjoint_gather(kkt_ctx *c, const double *lam_dev, const double *x_dev, double *dA_dev,
                              kkt_stream stream) {
    ApiRange nvtx_range("kkt_adjoint_gather");
    REQUIRE_DEVICE(c);
    if (!lam_dev || !x_dev || !dA_dev) return KKT_ERR_ARG;
    DeviceGuard g(c->dev);
    cudaStream_t s = (cudaStream_t)stream;
    const long long m = c->P.nnz_a;
    if (!c->rowperm) {
        k_adjoint<<<blocks_for(m, 256), 256, 0, s>>>(c->P, lam_dev, x_dev, dA_dev);
        CK(cudaGetLastError());
        c->launches++;
        return KKT_OK;
    }
    // entry k of Q A is entry qmap[k] of A, in row q[j] of A: dA = -lam[q[j]] x[col]
    double *mu = c->d_qvec + c->an.n;
    kkt_status st = q_vec(c, lam_dev, mu, true, s);
    if (st) return st;
    k_adjoint<<<blocks_for(m, 256), 256, 0, s>>>(c->P, mu, x_dev, c->d_qdA);
    CK(cudaGetLastError());
    k_scatter<<<blocks_for(m, 256), 256, 0, s>>>(m, c->d_qmap, c->d_qdA, dA_dev);
    CK(cudaGetLastError());
    c->launches += 2;
    return KKT_OK;
}

kkt_status kkt_status_sync(kkt_ctx *c, kkt_stream stream, int *n_perturbed) {
    REQUIRE_DEVICE(c);
    DeviceGuard g(c->dev);
    cudaStream_t s = (cudaStream_t)stream;
    int st[ST_WORDS];
    CK(cudaStreamSynchronize(s));
    CK(cudaMemcpy(st, c->d_status, sizeof(st), cudaMemcpyDeviceToHost));
    // the accumulated conditions are cleared; the inertia counters of the last
    // refactorization (ST_NEGATIVE, ST_PERT_LAST) stay for kkt_inertia
    CK(cudaMemset(c->d_status, 0, ST_NEGATIVE * sizeof(int)));
    if (n_perturbed) *n_perturbed = st[ST_PERTURBED];
    if (st[ST_INTERNAL]) { g_last_error = "factor pattern not closed under fill"; return KKT_ERR_INTERNAL; }
    if (st[ST_TIMEOUT]) return KKT_ERR_TIMEOUT;
    if (st[ST_NONFINITE]) return KKT_ERR_NONFINITE;
    if (st[ST_PERTURBED]) return KKT_WARN_PERTURBED;
    return KKT_OK;
}

kkt_status kkt_inertia(kkt_ctx *c, kkt_stream stream, int *n_pos, int *n_neg, int *n_perturbed) {
    REQUIRE_DEVICE(c);
    if (!c->opt.symmetric) {
        g_last_error = "kkt_inertia: the context was not created for symmetric values";
        return KKT_ERR_STATE;
    }
    if (!c->factored) return KKT_ERR_STATE;
    DeviceGuard g(c->dev);
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    int st[ST_WORDS];
    CK(cudaMemcpy(st, c->d_status, sizeof(st), cudaMemcpyDeviceToHost));
    if (n_neg) *n_neg = st[ST_NEGATIVE];
    if (n_pos) *n_pos = c->an.n - st[ST_NEGATIVE];
    if (n_perturbed) *n_perturbed = st[ST_PERT_LAST];
    return KKT_OK;
}

// The pattern of L+U in the caller's labelling (rows and columns numbered by
// the caller-view ordering) and, per entry, its slot in the internal layout.
static void ensure_view(const kkt_ctx *c) {
    if (!c->view_rp.empty()) return;
    const Analysis &a = c->an;
    const int n = a.n;
    c->view_rp.assign(n + 1, 0);
    c->view_ci.resize(a.lu_ci.size());
    c->view_slot.resize(a.lu_ci.size());
    std::vector<std::pair<int, int>> row;
    size_t q = 0;
    for (int v = 0; v < n; v++) {
        const int u = a.internal_of[v];
        row.clear();
        for (int t = a.lu_rp[u]; t < a.lu_rp[u + 1]; t++) row.push_back({a.view_of[a.lu_ci[t]], t});
        std::sort(row.begin(), row.end());
        for (auto &e : row) { c->view_ci[q] = e.first; c->view_slot[q] = e.second; q++; }
        c->view_rp[v + 1] = (int)q;
    }
}

kkt_status kkt_get_stats(const kkt_ctx *c, kkt_stats *o) {
    if (!c || !o) return KKT_ERR_ARG;
    std::memset(o, 0, sizeof(*o));
    const Analysis &a = c->an;
    const int n = a.n;
    o->n = n;
    o->nnz_a = (long long)a.a_ci.size();
    o->nnz_sym = a.nnz_sym;
    o->nnz_lu = (long long)a.lu_ci.size();
    o->n_levels = a.n_levels;
    o->n_levels_u = a.n_levels_u;
    o->max_row = a.max_row;
    o->flops_refactor = a.flops;
    const double W = c->opt.factor_fp32 ? 4.0 : 8.0;
    // refactor: values + scatter map read once, factor written once, factor
    // structure (column indices, row pointers) read once
    o->bytes_refactor = 12.0 * o->nnz_a + (W + 4.0) * o->nnz_lu + 4.0 * (n + 1) + 4.0 * o->nnz_lu;
    // solve: factor values and indices read once, b, x and the work vector, perm and scale
    o->bytes_solve = (W + 4.0) * o->nnz_lu + 3.0 * 8.0 * n + 8.0 * n;
    o->bytes_spmv = 12.0 * o->nnz_a + 32.0 * n;
    o->device_bytes = c->device_bytes;
    o->grid_ctas = c->rgrid;
    o->refactor_big_warps = c->rc.nbig;
    o->refactor_big_cap = c->rc.cap_big;
    o->solve_ctas = c->solve_grid;
    o->warps_per_cta = c->cta_warps;
    o->last_refine_iters = c->last_iters;
    o->last_omega = c->last_omega;
    o->factor_fp32 = c->opt.factor_fp32;
    o->kernel_launches = c->launches;
    o->update_map_entries = (long long)a.upd_map.size();
    o->n_tasks = (int)a.task_lo.size();
    o->max_task = a.max_task;
    o->dense_rows = a.dense_rows;
    o->refactor_row_cap = c->cap_r;
    o->solve_far_rows = c->far_rows;
    o->solve_far_ctas = c->npart;
    return KKT_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint of the analysis: a flat image of everything kkt_analyze computed
// (and the row permutation of a value-aware context), so a later run can skip
// the host analysis.  Layout: "KKTA", version, then for every array its
// length (int64) and contents, then the scalars, then a 64-bit FNV-1a checksum
// of all preceding bytes.
namespace {
constexpr unsigned kImgMagic = 0x41544b4bu;   // "KKTA"
constexpr unsigned kImgVersion = 2;

struct ImgWriter {
    std::vector<unsigned char> out;
    void raw(const void *p, size_t b) {
        const unsigned char *q = static_cast<const unsigned char *>(p);
        out.insert(out.end(), q, q + b);
    }
    template <typename T> void val(T v) { raw(&v, sizeof(v)); }
    template <typename T> void vec(const std::vector<T> &v) {
        val<long long>((long long)v.size());
        if (!v.empty()) raw(v.data(), v.size() * sizeof(T));
    }
};
struct ImgReader {
    const unsigned char *p;
    size_t left;
    bool ok = true;
    void raw(void *d, size_t b) {
        if (!ok || b > left) { ok = false; return; }
        std::memcpy(d, p, b);
        p += b;
        left -= b;
    }
    template <typename T> T val() { T v{}; raw(&v, sizeof(v)); return v; }
    template <typename T> void vec(std::vector<T> &v, long long expect = -1) {
        const long long m = val<long long>();
        if (!ok || m < 0 || (expect >= 0 && m != expect) || (unsigned long long)m * sizeof(T) > left) {
            ok = false;
            return;
        }
        v.resize((size_t)m);
        if (m) raw(v.data(), (size_t)m * sizeof(T));
    }
};
unsigned long long fnv1a(const unsigned char *p, size_t b) {
    unsigned long long h = 1469598103934665603ull;
    for (size_t i = 0; i < b; i++) { h ^= p[i]; h *= 1099511628211ull; }
    return h;
}
}  // namespace

kkt_status kkt_save_analysis(const kkt_ctx *c, void *buf, size_t cap, size_t *size) {
    if (!c || !size) return KKT_ERR_ARG;
    const Analysis &a = c->an;
    ImgWriter w;
    w.val(kImgMagic);
    w.val(kImgVersion);
    w.val(a.n);
    w.vec(a.a_rp); w.vec(a.a_ci); w.vec(a.a_row); w.vec(a.perm); w.vec(a.iperm);
    w.vec(a.view_perm); w.vec(a.view_of); w.vec(a.internal_of); w.vec(a.parent);
    w.vec(a.lu_rp); w.vec(a.lu_ci); w.vec(a.diag); w.vec(a.src); w.vec(a.tpos);
    w.vec(a.level); w.vec(a.level_u); w.vec(a.order_f); w.vec(a.order_b);
    w.vec(a.task_lo); w.vec(a.task_hi); w.vec(a.upd_off); w.vec(a.upd_map);
    w.val(a.n_levels); w.val(a.n_levels_u); w.val(a.nnz_sym); w.val(a.max_row); w.val(a.flops);
    w.val(a.max_task);
    w.val(a.dense_rows);
    w.val<int>(c->rowperm ? 1 : 0);
    w.vec(c->q); w.vec(c->qmap);
    w.val(fnv1a(w.out.data(), w.out.size()));
    *size = w.out.size();
    if (!buf) return KKT_OK;
    if (cap < w.out.size()) { g_last_error = "kkt_save_analysis: buffer too small"; return KKT_ERR_ARG; }
    std::memcpy(buf, w.out.data(), w.out.size());
    return KKT_OK;
}

kkt_status kkt_load_analysis(const void *buf, size_t size, const kkt_options *opt, kkt_ctx **out) {
    if (!buf || !out || size < 8 + 16) return KKT_ERR_ARG;
    *out = nullptr;
    ApiRange nvtx_range("kkt_load_analysis");
    const unsigned char *b = static_cast<const unsigned char *>(buf);
    unsigned long long sum = 0;
    std::memcpy(&sum, b + size - 8, 8);
    if (fnv1a(b, size - 8) != sum) { g_last_error = "analysis image: checksum mismatch"; return KKT_ERR_ARG; }
    std::unique_ptr<kkt_ctx> c(new (std::nothrow) kkt_ctx());
    if (!c) return KKT_ERR_ALLOC;
    if (opt) c->opt = *opt; else kkt_default_options(&c->opt);
    if (!options_valid(c->opt)) {
        g_last_error = "invalid option";
        return KKT_ERR_ARG;
    }
    Analysis &a = c->an;
    try {
        ImgReader r{b, size - 8};
        if (r.val<unsigned>() != kImgMagic || r.val<unsigned>() != kImgVersion) {
            g_last_error = "analysis image: not a kkt analysis of this version";
            return KKT_ERR_ARG;
        }
        a.n = r.val<int>();
        const long long n = a.n;
        if (!r.ok || n <= 0) { g_last_error = "analysis image: bad size"; return KKT_ERR_ARG; }
        r.vec(a.a_rp, n + 1); r.vec(a.a_ci); r.vec(a.a_row); r.vec(a.perm, n); r.vec(a.iperm, n);
        r.vec(a.view_perm, n); r.vec(a.view_of, n); r.vec(a.internal_of, n); r.vec(a.parent, n);
        r.vec(a.lu_rp, n + 1); r.vec(a.lu_ci); r.vec(a.diag, n); r.vec(a.src); r.vec(a.tpos);
        r.vec(a.level, n); r.vec(a.level_u, n); r.vec(a.order_f, n); r.vec(a.order_b, n);
        r.vec(a.task_lo); r.vec(a.task_hi); r.vec(a.upd_off); r.vec(a.upd_map);
        a.n_levels = r.val<int>(); a.n_levels_u = r.val<int>(); a.nnz_sym = r.val<long long>();
        a.max_row = r.val<int>(); a.flops = r.val<double>(); a.max_task = r.val<int>();
        a.dense_rows = r.val<int>();
        c->rowperm = r.val<int>() != 0;
        r.vec(c->q); r.vec(c->qmap);
        // the sizes the kernels rely on
        const long long nlu = (long long)a.lu_ci.size(), nna = (long long)a.a_ci.size();
        bool ok = r.ok && r.left == 0 && a.lu_rp[0] == 0 && a.lu_rp[n] == nlu && a.a_rp[0] == 0 &&
                  a.a_rp[n] == nna && (long long)a.a_row.size() == nna && (long long)a.src.size() == nlu &&
                  (long long)a.tpos.size() == nlu && a.task_lo.size() == a.task_hi.size() &&
                  (a.upd_off.empty() || (long long)a.upd_off.size() == nlu) &&
                  (!c->rowperm || ((long long)c->q.size() == n && (long long)c->qmap.size() == nna));
        for (long long i = 0; ok && i < n; i++)
            ok = a.lu_rp[i] <= a.lu_rp[i + 1] && a.a_rp[i] <= a.a_rp[i + 1] && a.diag[i] >= a.lu_rp[i] &&
                 a.diag[i] < a.lu_rp[i + 1] && a.perm[i] >= 0 && a.perm[i] < n && a.order_f[i] >= 0 &&
                 a.order_f[i] < n && a.order_b[i] >= 0 && a.order_b[i] < n;
        for (long long k = 0; ok && k < nlu; k++)
            ok = a.lu_ci[k] >= 0 && a.lu_ci[k] < n && a.src[k] >= -1 && a.src[k] < nna && a.tpos[k] >= 0 &&
                 a.tpos[k] < nlu && (a.upd_off.empty() || a.upd_off[k] <= a.upd_map.size());
        // the dense root block: every one of its rows ends in all of its columns
        ok = ok && a.dense_rows >= 0 && a.dense_rows <= n;
        for (long long i = n - a.dense_rows; ok && i < n; i++) {
            const long long t0 = (long long)a.lu_rp[i + 1] - a.dense_rows;
            ok = t0 >= a.lu_rp[i];
            for (long long q = 0; ok && q < a.dense_rows; q++) ok = a.lu_ci[t0 + q] == n - a.dense_rows + q;
        }
        if (!ok) { g_last_error = "analysis image: inconsistent arrays"; return KKT_ERR_ARG; }
    } catch (const std::bad_alloc &) {
        g_last_error = "host allocation failed while loading an analysis";
        return KKT_ERR_ALLOC;
    }
    c->opt.user_perm = nullptr;
    c->opt.user_row_perm = nullptr;
    c->tau_rel = c->opt.pivot_tau_rel > 0 ? c->opt.pivot_tau_rel : (c->opt.factor_fp32 ? 0x1p-24 : 1e-14);
    c->auto_ratio = c->opt.refine_auto_ratio > 0 ? c->opt.refine_auto_ratio : 0.5;
    c->dev = c->opt.device;
    c->host_only = c->opt.device < 0;
    if (!c->host_only) {
        DeviceGuard g(c->dev);
        if (!g.ok) { g_last_error = "cannot select the CUDA device"; return KKT_ERR_CUDA; }
        kkt_status st = upload(c.get());
        if (st != KKT_OK) {
            kkt_destroy(c.release());
            return st;
        }
    }
    *out = c.release();
    return KKT_OK;
}

kkt_status kkt_export_symbolic(const kkt_ctx *c, int *perm, int *lu_row_ptr, int *lu_col_idx,
                               int *level, int *level_u) {
    if (!c) return KKT_ERR_ARG;
    const Analysis &a = c->an;
    if (perm) std::memcpy(perm, a.view_perm.data(), a.n * sizeof(int));
    if (lu_row_ptr || lu_col_idx) ensure_view(c);
    if (lu_row_ptr) std::memcpy(lu_row_ptr, c->view_rp.data(), (a.n + 1) * sizeof(int));
    if (lu_col_idx) std::memcpy(lu_col_idx, c->view_ci.data(), c->view_ci.size() * sizeof(int));
    for (int v = 0; v < a.n; v++) {
        if (level) level[v] = a.level[a.internal_of[v]];
        if (level_u) level_u[v] = a.level_u[a.internal_of[v]];
    }
    return KKT_OK;
}

kkt_status kkt_export_dense_rows(const kkt_ctx *c, int *rows) {
    if (!c || (!rows && c->an.dense_rows > 0)) return KKT_ERR_ARG;
    const Analysis &a = c->an;
    for (int r = 0; r < a.dense_rows; r++) rows[r] = a.view_of[a.n - a.dense_rows + r];
    return KKT_OK;
}

kkt_status kkt_export_factors(kkt_ctx *c, double *out_dev, kkt_stream stream) {
    REQUIRE_DEVICE(c);
    if (!out_dev) return KKT_ERR_ARG;
    if (!c->factored) return KKT_ERR_STATE;
    DeviceGuard g(c->dev);
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->d_view_slot) {
        ensure_view(c);
        CK(cudaMalloc(&c->d_view_slot, c->view_slot.size() * sizeof(int)));
        CK(cudaMemcpy(c->d_view_slot, c->view_slot.data(), c->view_slot.size() * sizeof(int),
                      cudaMemcpyHostToDevice));
    }
    if (c->opt.factor_fp32)
        k_export<float><<<blocks_for(c->nnz_lu, 256), 256, 0, s>>>((const float *)c->d_lu, c->d_view_slot,
                                                                   out_dev, c->nnz_lu);
    else
        k_export<double><<<blocks_for(c->nnz_lu, 256), 256, 0, s>>>((const double *)c->d_lu, c->d_view_slot,
                                                                    out_dev, c->nnz_lu);
    CK(cudaGetLastError());
    c->launches++;
    return KKT_OK;
}

kkt_status kkt_export_trace(kkt_ctx *c, int phase, unsigned long long *out_host, long long max_items,
                            long long *n_items) {
    REQUIRE_DEVICE(c);
    if (!out_host || phase < 0 || phase >= TR_PHASES || max_items < 0) return KKT_ERR_ARG;
    if (!c->d_trace) { g_last_error = "tracing was not enabled at analysis"; return KKT_ERR_STATE; }
    DeviceGuard g(c->dev);
    const long long items = phase == TR_REFACTOR ? c->an.n : phase == TR_DENSE ? c->dense_grid : c->tk.ntasks;
    const long long m = std::min(items, max_items);
    CK(cudaDeviceSynchronize());
    if (phase == TR_REFACTOR) {
        // recorded by internal row; returned by row in the caller's numbering
        std::vector<unsigned long long> h(2 * (size_t)items);
        CK(cudaMemcpy(h.data(), c->d_trace, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
        for (long long i = 0; i < items; i++) {
            const long long v = c->an.view_of[i];
            if (v < m) {
                out_host[2 * v] = h[2 * i];
                out_host[2 * v + 1] = h[2 * i + 1];
            }
        }
    } else {
        CK(cudaMemcpy(out_host, c->d_trace + phase * c->rc.trace_stride, 2 * m * sizeof(unsigned long long),
                      cudaMemcpyDeviceToHost));
    }
    if (n_items) *n_items = m;
    return KKT_OK;
}

kkt_status kkt_export_scaling(kkt_ctx *c, double *out_dev, kkt_stream stream) {
    REQUIRE_DEVICE(c);
    if (!out_dev) return KKT_ERR_ARG;
    if (!c->factored) return KKT_ERR_STATE;
    DeviceGuard g(c->dev);
    CK(cudaMemcpyAsync(out_dev, c->d_s, c->an.n * sizeof(double), cudaMemcpyDeviceToDevice,
                       (cudaStream_t)stream));
    return KKT_OK;
}
