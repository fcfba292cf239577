// kernels.cuh -- device kernels of the fixed-pattern KKT refactorization.
//
// Scheduling.  Every triangular phase (the refactorization and the four
// triangular solves) is one persistent launch.  Its warps claim work (rows of
// the refactorization, longest-path tasks of the solves) in a topological
// order from an atomic counter (arXiv 2306.14337 Sec. 5.2, Algorithms 1-2:
// work on a row starts once the rows it depends on are done) and wait for each
// dependency on the dependency's value itself.  Work is only ever waited on
// after it was claimed by a running warp, so the schedule cannot deadlock;
// every wait is bounded (spin_limit polls) and on expiry raises
// KKT_ERR_TIMEOUT in the device status word and lets all warps drain.
//
// The claim queue resets itself: the last warp to find it empty zeroes it for
// the next launch, so launches need no host-side preparation and can be
// replayed from a CUDA graph.
//
// Kinds of work in a solve phase (see TaskCfg): the longest tasks each run on
// a whole CTA (one walker warp, one warp for late updates, helper warps over
// packed 32 x 32 tiles); short tasks run on one warp; single-row tasks run 32
// to a warp as packs; and the parts of a CTA task's rows that depend on other
// tasks are summed ahead of time by warp items, so the walker only adds them.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

namespace kkt {

// ST_NEGATIVE / ST_PERT_LAST: negative and perturbed pivots of the last
// symmetric (LDL^T) refactorization, cleared at its start (the inertia).
enum StatusSlot { ST_PERTURBED = 0, ST_NONFINITE = 1, ST_TIMEOUT = 2, ST_ABORT = 3, ST_INTERNAL = 4,
                  ST_NEGATIVE = 5, ST_PERT_LAST = 6, ST_WORDS = 8 };

// Norms kept on the device as the bit patterns of non-negative doubles, so
// that atomicMax on unsigned 64-bit integers orders them correctly.
enum NormSlot { NM_ANORM = 0, NM_A1NORM = 1, NM_AMAX = 2, NM_RMAX = 3, NM_XMAX = 4, NM_BMAX = 5,
                NM_WORDS = 8 };

struct Sched {
    int next;       // row-claim counter (the refactorization: its free-row queue)
    int done;       // warps that found the queue empty
    int epoch;      // epoch of the last completed triangular launch (shared by all phases)
    int next_long;  // claim counters of the refactorization's long-row and
    int next_rest;  //   remaining-row queues
    int pad[3];
};

struct DevPattern {
    int n;
    long long nnz_a;
    const int *a_rp, *a_ci, *a_row;      // user CSR and row of each entry
    const int *at_rp, *at_src;           // user pattern by columns: entry index per slot
    const int *perm, *iperm;             // new -> old, old -> new
    const int *lu_rp, *lu_ci, *diag, *src, *tpos;
    const int *order_f, *order_b;        // rows by forward / backward level
    // The single-system refactorization splits order_f in three subsequences
    // (see k_refactor): rows without a long descendant (order_free), rows
    // longer than the small per-warp buffer (order_long), and the other rows
    // (order_rest), of n_free / n_long / n - n_free - n_long rows.
    const int *order_free, *order_long, *order_rest;
    int n_free, n_long, n_rest;
    const unsigned *upd_off;             // update maps (null when not built)
    const unsigned short *upd_map;
    // First row of the dense root block (n: none).  The update maps hold no
    // entries for the block's own pivot steps (row and pivot both >= dense_lo);
    // kernels that take those steps as sparse steps search the row instead.
    int dense_lo;
};

struct TaskCfg {
    int ntasks;
    int cap;                             // task results kept in shared memory per warp
    const int *task_lo, *task_hi;        // rows of task t: [lo, hi], bottom to top
    const int *order_f, *order_b;        // claim orders of the forward / backward phases
    const int *order_topo;               // forward order without the longest-first prefix
    // Long tasks of the single-system solves run on a whole CTA each: CTA b <
    // nchain takes task chain_task[b]; the claim orders above then hold the
    // other tasks only.  cs_late / cs_diag: per row of such a task, the slot
    // splits of its dependency range by source block (see trisolve_chain).
    int nchain;
    int zcap;                            // results of a CTA task kept in shared memory
    const int *chain_task;
    const int *cs_late, *cs_diag;
    // Per refactorization, the 32 x 32 tiles of every block of every CTA task
    // are packed for each solve phase (see k_pack_tiles): block b of CTA task
    // c is block chain_blk0[c] + b of this phase's tile array.
    const int *chain_blk0;
    const void *tiles;
    // Claim-order entries p < 0 are packs of single-row tasks: pack -1 - p
    // holds the rows pack_rows[32 (-1 - p) + lane] (-1: empty lane).
    const int *pack_rows;
    // Outside parts of CTA-task rows (optional, ext != null): claim-order
    // entries e >= ext_base are warp items that sum row ext_rows[e - ext_base]
    // over its dependencies outside its task and publish the sum in ext[row];
    // cs_ext[row] splits the row's dependency slots (forward: outside
    // [row start, cs_ext), backward: outside [cs_ext, row end)).
    int ext_base;
    const int *ext_rows;
    const int *cs_ext;
    void *ext;
    // Far sources of CTA-task rows (optional, far != null): CTAs nchain ..
    // nchain + npart - 1 are partners; partner p sums, for the far rows
    // far_rows[part[p].x + r] (r = part[p].z * warps + warp, stepping by
    // part[p].w * warps, r < part[p].y), the slots between cs_ext[row] and
    // cs_far[row] (forward: [cs_ext, cs_far), backward: [cs_far, cs_ext)) and
    // publishes the sum in far[row].
    int npart;
    const int4 *part;
    const int *far_rows;
    const int *cs_far;
    void *far;
};

struct RunCfg {
    long long spin_limit;
    int *status;                 // ST_WORDS ints
    unsigned long long *norms;   // NM_WORDS
    Sched *sched;                // one scheduler record per context (phases are stream-ordered)
    int cap;                     // shared-memory row capacity per warp of the refactorization
                                 // (batched and queued kernels; small warps of k_refactor)
    int cap_big;                 // k_refactor: row capacity of its big warps
    int nbig;                    // k_refactor: big warps per CTA (warps 0 .. nbig-1; 0 = none)
    int smem_cols;               // k_refactor: 1 if the row's columns are staged too (no update maps)
    int staged;                  // k_refactor: 1 = pivot rows fed through each warp's staging ring
    int symmetric;               // k_refactor: 1 = LDL^T of symmetric values (refactor_row_sym)
    int warp_bytes_big;          // k_refactor: shared-memory bytes of a big / small warp's block
    int warp_bytes_small;
    void *scratch;               // per-warp global rows for rows longer than cap
    int scratch_stride;          // entries per warp in scratch
    unsigned long long *trace;   // optional: per work item {claim, done} %globaltimer (ns)
    long long trace_stride;      // words per phase region
    int unpublished_row;         // failure-detection test: this row is never published (-1: none)
    unsigned poll_ns_max;        // backoff cap of a waiting lane (ns)
    // Dense root block (single-system refactorization only): rows >= dense_lo
    // take only their pivot steps below the block and leave their partly
    // reduced block row in dense (row-major, leading dimension dense_ld);
    // k_dense_lu then factors the block.  dense_lo = INT_MAX: no block.
    int dense_lo;
    int dense_ld;
    void *dense;
    int *dense_ctl;              // k_dense_lu: one published flag per block column
};

// Launch k_dense_lu<T> (csrc/dense.cu): the LU of the dense root block left
// in rc.dense by the refactorization, with the pivot test; the block's factors
// go to LU (and the transposed copy LUT), its reciprocal pivots to rcp.
// dense_lu_prepare (once per context) sets the kernel's shared-memory limit
// for a block of s rows and returns its CTA count, or an error if they do not
// all fit on the device at once; dense_lu_max_rows is the largest block it
// takes; dense_lu_ctl_bytes the size of rc.dense_ctl.
template <typename T>
cudaError_t launch_dense_lu(const DevPattern &P, const RunCfg &rc, const double *aval, const double *sp,
                            T *LU, T *LUT, T *rcp, double tau_rel, cudaStream_t stream);
int dense_lu_threads();
int dense_lu_max_rows(int fp32);
size_t dense_lu_ctl_bytes(int s);
cudaError_t dense_lu_prepare(int fp32, int s, int sms, int *ctas);

// Raise a kernel's dynamic shared-memory limit on the current device to at
// least `bytes` (never lowers it; thread-safe).
cudaError_t ensure_smem(const void *f, size_t bytes);

// Record the text returned by kkt_last_error() on the calling thread (every
// translation unit of the library reports through this one store).
void set_last_error(const std::string &msg);

// Trace regions, one per phase, each (max work items) x 2 words.
// TR_DENSE: the block columns of k_dense_lu (start of its own work, publication).
enum TracePhase { TR_REFACTOR = 0, TR_FWD = 1, TR_BWD = 2, TR_TFWD = 3, TR_TBWD = 4, TR_DENSE = 5, TR_PHASES = 6 };

}  // namespace kkt
