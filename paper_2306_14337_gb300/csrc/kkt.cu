// kkt.cu -- CUDA kernels and C entry points of the fixed-pattern KKT
// refactorization library (see include/kkt.h for the interface).
//
// arXiv 2306.14337 maps onto this file as follows:
//   Sec. 5.2 "fill the values of A into the combined storage for L and U"
//       -> k_scale / k_amax (power-of-two scaling, norms) and the value gather
//          at the start of every row of k_refactor;
//   Sec. 5.2 Algorithm 1 (row-wise, dependency-driven LU)
//       -> k_refactor: one warp per row of the combined L+U (CSR), rows
//          claimed in level order, ready flags on the rows it depends on,
//          the row staged in shared memory, updates placed by a binary search
//          of the row's sorted column list (no atomics);
//   Sec. 5.2 Algorithm 2 (dependency-driven triangular solve)
//       -> k_fsolve / k_bsolve and the transposed pair k_tfsolve / k_tbsolve,
//          one warp per row, permutation and scaling fused at entry and exit;
//   Sec. 5.1 iterative refinement rho = r - K dx, K delta = rho, dx += delta
//       -> k_resid (FP64 CSR residual fused with the infinity norms) and the
//          refinement loop in kkt_refine (the update is fused into k_bsolve).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "kkt.h"
#include "analysis.h"
#include "kernels.cuh"

namespace kkt {

constexpr unsigned FULL = 0xffffffffu;
constexpr int WARPS = 8;  // warps per CTA of the persistent kernels

// ---------------------------------------------------------------------------
// synchronisation helpers

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename T> __device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }

// Wait until flags[d] == e.  Bounded: after spin_limit polls the wait sets
// the timeout and abort words and returns false; once abort is set every
// other wait returns false at its next check.
__device__ bool wait_ready(const RunCfg &rc, int d, int e) {
    if (ld_relaxed(rc.flags + d) != e) {
        long long it = 0;
        while (ld_relaxed(rc.flags + d) != e) {
            ++it;
            if ((it & 31) == 0) {
                if (ld_relaxed(rc.status + ST_ABORT)) return false;
                if (it > rc.spin_limit) {
                    atomicExch(rc.status + ST_TIMEOUT, 1);
                    atomicExch(rc.status + ST_ABORT, 1);
                    return false;
                }
                __nanosleep(32);
            }
        }
    }
    (void)ld_acquire(rc.flags + d);  // synchronises with the producer's release
    return true;
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
        rc.sched->done = 0;
        __threadfence();
        rc.sched->epoch = e;
    }
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *p, double v) {
    atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ int floor_half(int e) { return e >= 0 ? e / 2 : -((1 - e) / 2); }

// ---------------------------------------------------------------------------
// scaling and norms (8 lanes per row)

// s_i = 2^-floor(floor(log2 r_i) / 2), r_i = max_j |a_ij| (1 for a zero or
// non-finite row); sp[new] = s[old]; ||A||_inf; non-finite input flagged.
__global__ void k_scale(DevPattern P, const double *__restrict__ aval, double *__restrict__ s_orig,
                        double *__restrict__ sp, unsigned long long *norms, int *status, int equil) {
    const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int sub = threadIdx.x & 7;
    double rmax = 0.0, rsum = 0.0;
    bool bad = false;
    const int r = g;
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
        else atomic_max_nonneg(norms + NM_ANORM, rsum);
    }
}

// max |A'| (for the pivot threshold) and ||A||_1 (for transposed residuals)
__global__ void k_amax(DevPattern P, const double *__restrict__ aval, const double *__restrict__ s_orig,
                       unsigned long long *norms) {
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int sub = threadIdx.x & 7;
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
        if (isfinite(m)) atomic_max_nonneg(norms + NM_AMAX, m);
        if (isfinite(csum)) atomic_max_nonneg(norms + NM_A1NORM, csum);
    }
}

// ---------------------------------------------------------------------------
// numeric refactorization: one warp per row of L+U

template <typename T>
__global__ void __launch_bounds__(WARPS * 32)
k_refactor(DevPattern P, RunCfg rc, const double *__restrict__ aval, const double *__restrict__ sp,
           T *__restrict__ LU, double tau_rel) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int *scol = reinterpret_cast<int *>(smem) + (size_t)wid * rc.cap;
    T *sval = reinterpret_cast<T *>(smem + (size_t)nw * rc.cap * sizeof(int)) + (size_t)wid * rc.cap;
    const int e = rc.sched->epoch + 1;
    const int gw = blockIdx.x * nw + wid;
    const double tau = tau_rel * __longlong_as_double((long long)rc.norms[NM_AMAX]);
    for (;;) {
        const int slot = claim_row(rc, lane);
        if (slot >= P.n) break;
        const int i = P.order_f[slot];
        const int rb = P.lu_rp[i], len = P.lu_rp[i + 1] - rb, dp = P.diag[i] - rb;
        const int *c;
        T *w;
        if (len <= rc.cap) {
            for (int t = lane; t < len; t += 32) scol[t] = P.lu_ci[rb + t];
            c = scol;
            w = sval;
        } else {
            c = P.lu_ci + rb;
            w = reinterpret_cast<T *>(rc.scratch) + (size_t)gw * rc.scratch_stride;
        }
        // gather A'(i,:) = s_i a_ij s_j into the row (structural zeros elsewhere)
        const double si = sp[i];
        for (int t = lane; t < len; t += 32) {
            const int k = P.src[rb + t];
            w[t] = (T)((k >= 0) ? si * sp[P.lu_ci[rb + t]] * aval[k] : 0.0);
        }
        __syncwarp();
        // eliminate with every U row d < i the row depends on, in increasing d
        for (int t = 0; t < dp; t++) {
            const int d = c[t];
            const int ub = P.diag[d], ue = P.lu_rp[d + 1];   // static: issued before the wait
            if (lane == 0) wait_ready(rc, d, e);
            __syncwarp();
            const T l = w[t] / ldcg(LU + ub);
            for (int u = ub + 1 + lane; u < ue; u += 32) {
                const int j = P.lu_ci[u];
                const T uv = ldcg(LU + u);
                int lo = t + 1, hi = len;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (c[mid] < j) lo = mid + 1; else hi = mid;
                }
                if (lo < len && c[lo] == j) w[lo] -= l * uv;
                else atomicExch(rc.status + ST_INTERNAL, 1);   // pattern not closed under fill
            }
            __syncwarp();
            if (lane == 0) w[t] = l;
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
            }
            w[dp] = (T)pv;
        }
        __syncwarp();
        for (int t = lane; t < len; t += 32) LU[rb + t] = w[t];
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release(rc.flags + i, e);
    }
    if (lane == 0) finish_launch(rc, e);
}

// ---------------------------------------------------------------------------
// triangular solves: one warp per row, lanes over the row's entries.
//
// Ready signal (the idea of Algorithm 2: a value that is not yet computed
// marks the unknown as not ready): the output vector is filled with an
// all-ones bit pattern before the launch, a row's unknown is published with a
// single relaxed store of its value, and a dependent row polls that word
// until it changes.  One memory round trip per dependency, no flag and no
// fence (an aligned 32/64-bit access is single-copy atomic).  A computed value
// whose bits equal the marker is replaced by a canonical NaN and flagged.

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

template <typename T> __device__ __forceinline__ void publish(const RunCfg &rc, T *p, T v) {
    if (is_marker(v)) {
        v = T(NAN);
        atomicExch(rc.status + ST_NONFINITE, 1);
    }
    st_relaxed_v(p, v);
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Forward, unit L: y_i = b'_i - sum_{d<i} L(i,d) y_d,  b'_i = s_i b[perm[i]].
template <typename T>
__global__ void __launch_bounds__(WARPS * 32)
k_fsolve(DevPattern P, RunCfg rc, const T *__restrict__ LU, const double *__restrict__ b,
         const double *__restrict__ sp, T *y) {
    const int lane = threadIdx.x & 31;
    const int e = rc.sched->epoch + 1;
    for (;;) {
        const int slot = claim_row(rc, lane);
        if (slot >= P.n) break;
        const int i = P.order_f[slot];
        const int rb = P.lu_rp[i], de = P.diag[i];
        const T bi = (lane == 0) ? (T)(sp[i] * b[P.perm[i]]) : T(0);   // issued before the waits
        T acc = 0;
        for (int t = rb + lane; t < de; t += 32) {
            const T l = LU[t];
            const int d = P.lu_ci[t];
            acc += l * wait_value(rc, y + d);
        }
        acc = warp_sum(acc);
        if (lane == 0) publish(rc, y + i, bi - acc);
    }
    if (lane == 0) finish_launch(rc, e);
}

// Backward, U: z_j = (y_j - sum_{k>j} U(j,k) z_k) / U(j,j);
// x[perm[j]] = s_j z_j (accumulate != 0: +=, the refinement update).
template <typename T>
__global__ void __launch_bounds__(WARPS * 32)
k_bsolve(DevPattern P, RunCfg rc, const T *__restrict__ LU, const double *__restrict__ sp,
         const T *__restrict__ y, T *z, double *__restrict__ x, int accumulate) {
    const int lane = threadIdx.x & 31;
    const int e = rc.sched->epoch + 1;
    for (;;) {
        const int slot = claim_row(rc, lane);
        if (slot >= P.n) break;
        const int j = P.order_b[slot];
        const int dg = P.diag[j], re = P.lu_rp[j + 1];
        const T yj = (lane == 0) ? y[j] : T(0);
        const T uj = (lane == 0) ? LU[dg] : T(1);
        T acc = 0;
        for (int t = dg + 1 + lane; t < re; t += 32) {
            const T u = LU[t];
            const int k = P.lu_ci[t];
            acc += u * wait_value(rc, z + k);
        }
        acc = warp_sum(acc);
        if (lane == 0) {
            const T zj = (yj - acc) / uj;
            publish(rc, z + j, zj);
            const double v = sp[j] * (double)zj;
            const int o = P.perm[j];
            x[o] = accumulate ? x[o] + v : v;
        }
    }
    if (lane == 0) finish_launch(rc, e);
}

// Transposed forward, U^T: w_j = (g'_j - sum_{d<j} U(d,j) w_d) / U(j,j);
// U(d,j) sits in row d at the transposed slot of L-slot (j,d).
template <typename T>
__global__ void __launch_bounds__(WARPS * 32)
k_tfsolve(DevPattern P, RunCfg rc, const T *__restrict__ LU, const double *__restrict__ g,
          const double *__restrict__ sp, T *y) {
    const int lane = threadIdx.x & 31;
    const int e = rc.sched->epoch + 1;
    for (;;) {
        const int slot = claim_row(rc, lane);
        if (slot >= P.n) break;
        const int j = P.order_f[slot];
        const int rb = P.lu_rp[j], dg = P.diag[j];
        const T gj = (lane == 0) ? (T)(sp[j] * g[P.perm[j]]) : T(0);
        const T uj = (lane == 0) ? LU[dg] : T(1);
        T acc = 0;
        for (int t = rb + lane; t < dg; t += 32) {
            const T u = LU[P.tpos[t]];
            const int d = P.lu_ci[t];
            acc += u * wait_value(rc, y + d);
        }
        acc = warp_sum(acc);
        if (lane == 0) publish(rc, y + j, (gj - acc) / uj);
    }
    if (lane == 0) finish_launch(rc, e);
}

// Transposed backward, unit L^T: z_j = w_j - sum_{i>j} L(i,j) z_i;
// lam[perm[j]] = s_j z_j (accumulate != 0: +=).
template <typename T>
__global__ void __launch_bounds__(WARPS * 32)
k_tbsolve(DevPattern P, RunCfg rc, const T *__restrict__ LU, const double *__restrict__ sp,
          const T *__restrict__ y, T *z, double *__restrict__ lam, int accumulate) {
    const int lane = threadIdx.x & 31;
    const int e = rc.sched->epoch + 1;
    for (;;) {
        const int slot = claim_row(rc, lane);
        if (slot >= P.n) break;
        const int j = P.order_b[slot];
        const int dg = P.diag[j], re = P.lu_rp[j + 1];
        const T yj = (lane == 0) ? y[j] : T(0);
        T acc = 0;
        for (int t = dg + 1 + lane; t < re; t += 32) {
            const T l = LU[P.tpos[t]];
            const int i = P.lu_ci[t];
            acc += l * wait_value(rc, z + i);
        }
        acc = warp_sum(acc);
        if (lane == 0) {
            const T zj = yj - acc;
            publish(rc, z + j, zj);
            const double v = sp[j] * (double)zj;
            const int o = P.perm[j];
            lam[o] = accumulate ? lam[o] + v : v;
        }
    }
    if (lane == 0) finish_launch(rc, e);
}

// ---------------------------------------------------------------------------
// FP64 residual rho = b - A x (or b - A^T x), 8 lanes per row, fused with
// ||rho||_inf, ||x||_inf, ||b||_inf.
__global__ void k_resid(DevPattern P, const double *__restrict__ aval, const double *__restrict__ b,
                        const double *__restrict__ x, double *__restrict__ rho,
                        unsigned long long *norms, int transpose) {
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
    double rv = 0.0, xv = 0.0, bv = 0.0;
    if (r < P.n && sub == 0) {
        const double br = b[r];
        rv = br - acc;
        rho[r] = rv;
        rv = fabs(rv);
        xv = fabs(x[r]);
        bv = fabs(br);
    }
    for (int o = 16; o > 0; o >>= 1) {
        rv = fmax(rv, __shfl_xor_sync(FULL, rv, o));
        xv = fmax(xv, __shfl_xor_sync(FULL, xv, o));
        bv = fmax(bv, __shfl_xor_sync(FULL, bv, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(norms + NM_RMAX, rv);
        atomic_max_nonneg(norms + NM_XMAX, xv);
        atomic_max_nonneg(norms + NM_BMAX, bv);
    }
}

// dA_k = -lam[row_k] x[col_k]
__global__ void k_adjoint(DevPattern P, const double *__restrict__ lam, const double *__restrict__ x,
                          double *__restrict__ dA) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P.nnz_a) dA[k] = -lam[P.a_row[k]] * x[P.a_ci[k]];
}

template <typename T>
__global__ void k_export(const T *__restrict__ LU, double *__restrict__ out, long long m) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < m) out[k] = (double)LU[k];
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
    void *d_lu = nullptr;
    double *d_s = nullptr, *d_sp = nullptr, *d_rho = nullptr;
    void *d_y = nullptr;
    int *d_status = nullptr;
    unsigned long long *d_norms = nullptr;
    Sched *d_sched = nullptr;
    int *d_flags = nullptr;
    void *d_scratch = nullptr;
    unsigned long long *h_norms = nullptr;  // pinned
    int grid = 0, solve_grid = 0, cta_warps = WARPS, cap = 0;
    size_t smem = 0, device_bytes = 0;
    long long nnz_lu = 0;
    std::vector<int> at_rp, at_src;
    const double *values = nullptr;  // values of the current factorization (caller-owned)
    bool factored = false;
    int last_iters = 0;
    double last_omega = -1.0;
    double tau_rel = 0.0;
    long long launches = 0;  // kernels launched by this context
};

static thread_local std::string g_last_error;

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
}  // namespace

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
    struct Arr { const int *h; long long m; const int **dst; };
    std::vector<Arr> arrs = {
        {a.a_rp.data(), n + 1, &c->P.a_rp},     {a.a_ci.data(), nnza, &c->P.a_ci},
        {a.a_row.data(), nnza, &c->P.a_row},    {c->at_rp.data(), n + 1, &c->P.at_rp},
        {c->at_src.data(), nnza, &c->P.at_src}, {a.perm.data(), n, &c->P.perm},
        {a.iperm.data(), n, &c->P.iperm},       {a.lu_rp.data(), n + 1, &c->P.lu_rp},
        {a.lu_ci.data(), nlu, &c->P.lu_ci},     {a.diag.data(), n, &c->P.diag},
        {a.src.data(), nlu, &c->P.src},         {a.tpos.data(), nlu, &c->P.tpos},
        {a.order_f.data(), n, &c->P.order_f},   {a.order_b.data(), n, &c->P.order_b},
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

    const bool f32 = c->opt.factor_fp32 != 0;
    const size_t tsz = f32 ? sizeof(float) : sizeof(double);
    CK(cudaMalloc(&c->d_lu, nlu * tsz));
    CK(cudaMalloc(&c->d_s, n * sizeof(double)));
    CK(cudaMalloc(&c->d_sp, n * sizeof(double)));
    CK(cudaMalloc(&c->d_rho, n * sizeof(double)));
    CK(cudaMalloc(&c->d_y, 2 * (size_t)n * sizeof(double)));
    CK(cudaMalloc(&c->d_status, ST_WORDS * sizeof(int)));
    CK(cudaMalloc(&c->d_norms, NM_WORDS * sizeof(unsigned long long)));
    CK(cudaMalloc(&c->d_sched, sizeof(Sched)));
    CK(cudaMalloc(&c->d_flags, n * sizeof(int)));
    CK(cudaMemset(c->d_status, 0, ST_WORDS * sizeof(int)));
    CK(cudaMemset(c->d_norms, 0, NM_WORDS * sizeof(unsigned long long)));
    CK(cudaMemset(c->d_sched, 0, sizeof(Sched)));
    CK(cudaMemset(c->d_flags, 0, n * sizeof(int)));
    CK(cudaMallocHost(&c->h_norms, NM_WORDS * sizeof(unsigned long long)));
    c->device_bytes += nlu * tsz + 4 * n * sizeof(double) + n * sizeof(int) + 256;

    // persistent grids: as many CTAs as fit on the device at once, unless the
    // options fix the CTA count; a grid never exceeds one warp per row
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
    c->cta_warps = c->opt.cta_warps > 0 ? std::min(c->opt.cta_warps, WARPS) : WARPS;
    const int nw = c->cta_warps;
    int cap = ((std::max(a.max_row, 32) + 31) / 32) * 32;
    cap = std::min(cap, 1024);
    c->cap = cap;
    c->smem = (size_t)nw * cap * (sizeof(int) + tsz);
    int per_sm = 0;
    if (f32) {
        CK(cudaFuncSetAttribute(k_refactor<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem));
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_refactor<float>, nw * 32, c->smem));
    } else {
        CK(cudaFuncSetAttribute(k_refactor<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem));
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_refactor<double>, nw * 32, c->smem));
    }
    if (per_sm < 1) { g_last_error = "refactor kernel does not fit on an SM"; return KKT_ERR_CUDA; }
    const int rows_cap = (n + nw - 1) / nw;
    int grid = c->opt.refactor_ctas > 0 ? std::min(c->opt.refactor_ctas, sms * per_sm) : sms * per_sm;
    c->grid = std::max(1, std::min(grid, rows_cap));
    int sgrid = c->opt.solve_ctas > 0 ? c->opt.solve_ctas : sms * 2;
    c->solve_grid = std::max(1, std::min(sgrid, rows_cap));
    // rows longer than the shared-memory capacity work in global scratch
    if (a.max_row > cap) {
        size_t per = (size_t)a.max_row;
        CK(cudaMalloc(&c->d_scratch, per * tsz * c->grid * nw));
        c->device_bytes += per * tsz * c->grid * nw;
        c->rc.scratch_stride = (int)per;
    }
    c->rc.spin_limit = c->opt.spin_limit;
    c->rc.status = c->d_status;
    c->rc.norms = c->d_norms;
    c->rc.sched = c->d_sched;
    c->rc.flags = c->d_flags;
    c->rc.cap = cap;
    c->rc.scratch = c->d_scratch;
    return KKT_OK;
}

void kkt_destroy(kkt_ctx *c) {
    if (!c) return;
    if (!c->host_only) {
        DeviceGuard g(c->dev);
        cudaFree(c->d_ints);
        cudaFree(c->d_lu);
        cudaFree(c->d_s);
        cudaFree(c->d_sp);
        cudaFree(c->d_rho);
        cudaFree(c->d_y);
        cudaFree(c->d_status);
        cudaFree(c->d_norms);
        cudaFree(c->d_sched);
        cudaFree(c->d_flags);
        cudaFree(c->d_scratch);
        cudaFreeHost(c->h_norms);
    }
    delete c;
}

kkt_status kkt_analyze(int n, const int *row_ptr, const int *col_idx, const kkt_options *opt,
                       kkt_ctx **out) {
    if (!out) return KKT_ERR_ARG;
    *out = nullptr;
    std::unique_ptr<kkt_ctx> c(new (std::nothrow) kkt_ctx());
    if (!c) return KKT_ERR_ALLOC;
    if (opt) c->opt = *opt; else kkt_default_options(&c->opt);
    if (c->opt.fgmres_restart < 1 || c->opt.max_refine < 0 || c->opt.spin_limit < 1 ||
        c->opt.max_batch < 1 || c->opt.cta_warps < 0 || c->opt.refactor_ctas < 0 ||
        c->opt.solve_ctas < 0) {
        g_last_error = "invalid option";
        return KKT_ERR_ARG;
    }
    std::string err;
    int rc;
    try {
        rc = analyze(n, row_ptr, col_idx, c->opt.ordering, c->opt.user_perm, c->an, err);
    } catch (const std::bad_alloc &) {
        g_last_error = "host allocation failed during analysis";
        return KKT_ERR_ALLOC;
    }
    if (rc != A_OK) {
        g_last_error = err;
        return (kkt_status)rc;
    }
    c->opt.user_perm = nullptr;  // copied
    c->tau_rel = c->opt.pivot_tau_rel > 0 ? c->opt.pivot_tau_rel
                                          : (c->opt.factor_fp32 ? 0x1p-24 : 1e-14);
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

#define REQUIRE_DEVICE(c)                                                              \
    do {                                                                               \
        if (!(c)) return KKT_ERR_ARG;                                                  \
        if ((c)->host_only) { g_last_error = "host-only context"; return KKT_ERR_STATE; } \
    } while (0)

template <typename T> static kkt_status launch_refactor(kkt_ctx *c, cudaStream_t s) {
    k_refactor<T><<<c->grid, c->cta_warps * 32, c->smem, s>>>(c->P, c->rc, c->values, c->d_sp,
                                                               (T *)c->d_lu, c->tau_rel);
    CK(cudaGetLastError());
    c->launches++;
    return KKT_OK;
}

kkt_status kkt_refactor(kkt_ctx *c, const double *values_dev, kkt_stream stream) {
    REQUIRE_DEVICE(c);
    if (!values_dev) return KKT_ERR_ARG;
    DeviceGuard g(c->dev);
    cudaStream_t s = (cudaStream_t)stream;
    c->values = values_dev;
    const int n = c->an.n;
    CK(cudaMemsetAsync(c->d_norms, 0, NM_WORDS * sizeof(unsigned long long), s));
    k_scale<<<blocks_for(8LL * n, 256), 256, 0, s>>>(c->P, values_dev, c->d_s, c->d_sp, c->d_norms,
                                                     c->d_status, c->opt.equilibrate);
    CK(cudaGetLastError());
    c->launches++;
    k_amax<<<blocks_for(8LL * n, 256), 256, 0, s>>>(c->P, values_dev, c->d_s, c->d_norms);
    CK(cudaGetLastError());
    c->launches++;
    kkt_status r = c->opt.factor_fp32 ? launch_refactor<float>(c, s) : launch_refactor<double>(c, s);
    if (r == KKT_OK) c->factored = true;
    return r;
}

template <typename T>
static kkt_status launch_solve(kkt_ctx *c, const double *b, double *x, int accumulate, cudaStream_t s) {
    const int n = c->an.n;
    T *y = (T *)c->d_y, *z = y + n;
    CK(cudaMemsetAsync(y, 0xff, 2 * (size_t)n * sizeof(T), s));
    k_fsolve<T><<<c->solve_grid, c->cta_warps * 32, 0, s>>>(c->P, c->rc, (const T *)c->d_lu, b, c->d_sp, y);
    CK(cudaGetLastError());
    c->launches++;
    k_bsolve<T><<<c->solve_grid, c->cta_warps * 32, 0, s>>>(c->P, c->rc, (const T *)c->d_lu, c->d_sp, y, z,
                                                            x, accumulate);
    CK(cudaGetLastError());
    c->launches++;
    return KKT_OK;
}

template <typename T>
static kkt_status launch_solve_t(kkt_ctx *c, const double *g, double *lam, int accumulate,
                                 cudaStream_t s) {
    const int n = c->an.n;
    T *y = (T *)c->d_y, *z = y + n;
    CK(cudaMemsetAsync(y, 0xff, 2 * (size_t)n * sizeof(T), s));
    k_tfsolve<T><<<c->solve_grid, c->cta_warps * 32, 0, s>>>(c->P, c->rc, (const T *)c->d_lu, g, c->d_sp, y);
    CK(cudaGetLastError());
    c->launches++;
    k_tbsolve<T><<<c->solve_grid, c->cta_warps * 32, 0, s>>>(c->P, c->rc, (const T *)c->d_lu, c->d_sp, y, z,
                                                             lam, accumulate);
    CK(cudaGetLastError());
    c->launches++;
    return KKT_OK;
}

static kkt_status solve_any(kkt_ctx *c, const double *b, double *x, int accumulate, int transpose,
                            cudaStream_t s) {
    if (transpose)
        return c->opt.factor_fp32 ? launch_solve_t<float>(c, b, x, accumulate, s)
                                  : launch_solve_t<double>(c, b, x, accumulate, s);
    return c->opt.factor_fp32 ? launch_solve<float>(c, b, x, accumulate, s)
                              : launch_solve<double>(c, b, x, accumulate, s);
}

kkt_status kkt_solve(kkt_ctx *c, const double *b_dev, double *x_dev, kkt_stream stream) {
    REQUIRE_DEVICE(c);
    if (!b_dev || !x_dev || b_dev == x_dev) return KKT_ERR_ARG;
    if (!c->factored) return KKT_ERR_STATE;
    DeviceGuard g(c->dev);
    return solve_any(c, b_dev, x_dev, 0, 0, (cudaStream_t)stream);
}

kkt_status kkt_solve_transpose(kkt_ctx *c, const double *g_dev, double *lam_dev, kkt_stream stream) {
    REQUIRE_DEVICE(c);
    if (!g_dev || !lam_dev || g_dev == lam_dev) return KKT_ERR_ARG;
    if (!c->factored) return KKT_ERR_STATE;
    DeviceGuard g(c->dev);
    return solve_any(c, g_dev, lam_dev, 0, 1, (cudaStream_t)stream);
}

// residual + norms; returns omega on the host (synchronises the stream)
static kkt_status residual_omega(kkt_ctx *c, const double *b, const double *x, int transpose,
                                 cudaStream_t s, double *omega) {
    const int n = c->an.n;
    CK(cudaMemsetAsync(c->d_norms + NM_RMAX, 0, 3 * sizeof(unsigned long long), s));
    k_resid<<<blocks_for(8LL * n, 256), 256, 0, s>>>(c->P, c->values, b, x, c->d_rho, c->d_norms, transpose);
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
    return KKT_OK;
}

static kkt_status refine_any(kkt_ctx *c, const double *b, double *x, double tol, int max_it,
                             kkt_refine_info *info, int transpose, cudaStream_t s) {
    if (tol <= 0) tol = c->opt.tol;
    if (max_it < 0) max_it = c->opt.max_refine;
    if (info) std::memset(info, 0, sizeof(*info));
    double w;
    kkt_status st = residual_omega(c, b, x, transpose, s, &w);
    if (st) return st;
    int it = 0;
    if (info) info->omega_hist[info->n_hist++] = w;
    while (!(w <= tol) && it < max_it && std::isfinite(w)) {
        st = solve_any(c, c->d_rho, x, 1, transpose, s);
        if (st) return st;
        it++;
        st = residual_omega(c, b, x, transpose, s, &w);
        if (st) return st;
        if (info && info->n_hist < 64) info->omega_hist[info->n_hist++] = w;
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
    return (w <= tol) ? KKT_OK : KKT_ERR_NOT_CONVERGED;
}

kkt_status kkt_refine(kkt_ctx *c, const double *b_dev, double *x_dev, double tol, int max_it,
                      kkt_refine_info *info, kkt_stream stream) {
    REQUIRE_DEVICE(c);
    if (!b_dev || !x_dev || b_dev == x_dev) return KKT_ERR_ARG;
    if (!c->factored) return KKT_ERR_STATE;
    DeviceGuard g(c->dev);
    return refine_any(c, b_dev, x_dev, tol, max_it, info, 0, (cudaStream_t)stream);
}

kkt_status kkt_refine_transpose(kkt_ctx *c, const double *g_dev, double *lam_dev, double tol,
                                int max_it, kkt_refine_info *info, kkt_stream stream) {
    REQUIRE_DEVICE(c);
    if (!g_dev || !lam_dev || g_dev == lam_dev) return KKT_ERR_ARG;
    if (!c->factored) return KKT_ERR_STATE;
    DeviceGuard g(c->dev);
    return refine_any(c, g_dev, lam_dev, tol, max_it, info, 1, (cudaStream_t)stream);
}

kkt_status kkt_adjoint_gather(kkt_ctx *c, const double *lam_dev, const double *x_dev, double *dA_dev,
                              kkt_stream stream) {
    REQUIRE_DEVICE(c);
    if (!lam_dev || !x_dev || !dA_dev) return KKT_ERR_ARG;
    DeviceGuard g(c->dev);
    const long long m = c->P.nnz_a;
    k_adjoint<<<blocks_for(m, 256), 256, 0, (cudaStream_t)stream>>>(c->P, lam_dev, x_dev, dA_dev);
    CK(cudaGetLastError());
    c->launches++;
    return KKT_OK;
}

kkt_status kkt_status_sync(kkt_ctx *c, kkt_stream stream, int *n_perturbed) {
    REQUIRE_DEVICE(c);
    DeviceGuard g(c->dev);
    cudaStream_t s = (cudaStream_t)stream;
    int st[ST_WORDS];
    CK(cudaStreamSynchronize(s));
    CK(cudaMemcpy(st, c->d_status, sizeof(st), cudaMemcpyDeviceToHost));
    CK(cudaMemset(c->d_status, 0, sizeof(st)));
    if (n_perturbed) *n_perturbed = st[ST_PERTURBED];
    if (st[ST_INTERNAL]) { g_last_error = "factor pattern not closed under fill"; return KKT_ERR_INTERNAL; }
    if (st[ST_TIMEOUT]) return KKT_ERR_TIMEOUT;
    if (st[ST_NONFINITE]) return KKT_ERR_NONFINITE;
    if (st[ST_PERTURBED]) return KKT_WARN_PERTURBED;
    return KKT_OK;
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
    o->grid_ctas = c->grid;
    o->solve_ctas = c->solve_grid;
    o->warps_per_cta = c->cta_warps;
    o->last_refine_iters = c->last_iters;
    o->last_omega = c->last_omega;
    o->factor_fp32 = c->opt.factor_fp32;
    o->kernel_launches = c->launches;
    return KKT_OK;
}

kkt_status kkt_export_symbolic(const kkt_ctx *c, int *perm, int *lu_row_ptr, int *lu_col_idx,
                               int *level, int *level_u) {
    if (!c) return KKT_ERR_ARG;
    const Analysis &a = c->an;
    if (perm) std::memcpy(perm, a.perm.data(), a.n * sizeof(int));
    if (lu_row_ptr) std::memcpy(lu_row_ptr, a.lu_rp.data(), (a.n + 1) * sizeof(int));
    if (lu_col_idx) std::memcpy(lu_col_idx, a.lu_ci.data(), a.lu_ci.size() * sizeof(int));
    if (level) std::memcpy(level, a.level.data(), a.n * sizeof(int));
    if (level_u) std::memcpy(level_u, a.level_u.data(), a.n * sizeof(int));
    return KKT_OK;
}

kkt_status kkt_export_factors(kkt_ctx *c, double *out_dev, kkt_stream stream) {
    REQUIRE_DEVICE(c);
    if (!out_dev) return KKT_ERR_ARG;
    if (!c->factored) return KKT_ERR_STATE;
    DeviceGuard g(c->dev);
    cudaStream_t s = (cudaStream_t)stream;
    if (c->opt.factor_fp32)
        k_export<float><<<blocks_for(c->nnz_lu, 256), 256, 0, s>>>((const float *)c->d_lu, out_dev, c->nnz_lu);
    else
        k_export<double><<<blocks_for(c->nnz_lu, 256), 256, 0, s>>>((const double *)c->d_lu, out_dev, c->nnz_lu);
    CK(cudaGetLastError());
    c->launches++;
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
