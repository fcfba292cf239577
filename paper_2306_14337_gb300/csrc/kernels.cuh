// kernels.cuh -- device kernels of the fixed-pattern KKT refactorization.
//
// Scheduling.  Every triangular phase (the refactorization and the four
// triangular solves) is one persistent launch.  Its warps claim rows in a
// topological order (by dependency level, arXiv 2306.14337 Sec. 5.2 and
// Algorithms 1-2: work on a row starts once the rows it depends on are done)
// from an atomic counter, and wait for each dependency on a per-row ready
// flag.  A row is only ever waited on after it was claimed by a running warp,
// so the schedule cannot deadlock whatever the residency; every wait is
// bounded (spin_limit polls) and on expiry raises KKT_ERR_TIMEOUT in the
// device status word and lets all warps drain.
//
// Flags carry an epoch number that is read from device memory at kernel start
// and advanced by the last warp to finish, so flags never need clearing and a
// launch can be replayed from a CUDA graph.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace kkt {

enum StatusSlot { ST_PERTURBED = 0, ST_NONFINITE = 1, ST_TIMEOUT = 2, ST_ABORT = 3, ST_INTERNAL = 4,
                  ST_WORDS = 8 };

// Norms kept on the device as the bit patterns of non-negative doubles, so
// that atomicMax on unsigned 64-bit integers orders them correctly.
enum NormSlot { NM_ANORM = 0, NM_A1NORM = 1, NM_AMAX = 2, NM_RMAX = 3, NM_XMAX = 4, NM_BMAX = 5,
                NM_WORDS = 8 };

struct Sched {
    int next;   // row-claim counter
    int done;   // warps that found the queue empty
    int epoch;  // epoch of the last completed triangular launch (shared by all phases)
    int pad;
};

struct DevPattern {
    int n;
    long long nnz_a;
    const int *a_rp, *a_ci, *a_row;      // user CSR and row of each entry
    const int *at_rp, *at_src;           // user pattern by columns: entry index per slot
    const int *perm, *iperm;             // new -> old, old -> new
    const int *lu_rp, *lu_ci, *diag, *src, *tpos;
    const int *order_f, *order_b;
};

struct RunCfg {
    long long spin_limit;
    int *status;                 // ST_WORDS ints
    unsigned long long *norms;   // NM_WORDS
    Sched *sched;                // one scheduler record per context (phases are stream-ordered)
    int *flags;                  // n ints
    int cap;                     // shared-memory capacity per warp (entries)
    void *scratch;               // per-warp global rows for rows longer than cap
    int scratch_stride;          // entries per warp in scratch
};

}  // namespace kkt
