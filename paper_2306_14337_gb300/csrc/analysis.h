// analysis.h -- host-side pattern analysis (one per sparsity pattern).
//
// Produces everything the device kernels need to refactor and solve a matrix
// of a fixed pattern (arXiv 2306.14337, Sec. 4 symbolic phase, Sec. 5.2
// preprocessing): a symmetric fill-reducing permutation, the pattern of the
// combined L+U factor stored row by row, the dependency levels, and the maps
// that place user values and transposed entries.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace kkt {

struct Analysis {
    int n = 0;
    // user pattern (copied)
    std::vector<int> a_rp, a_ci;
    std::vector<int> a_row;        // row of every user entry
    // ordering: perm[new] = old, iperm[old] = new (internal labelling, see below)
    std::vector<int> perm, iperm;
    // The caller's view: view_perm is the ordering as given (or as computed by
    // the minimum-degree code).  Internally the rows are relabelled by a
    // postorder of the elimination tree that visits each node's deepest child
    // last, which keeps the fill and the tree but makes every solve task a
    // contiguous index range.  view_of[internal] = view index.
    std::vector<int> view_perm, view_of, internal_of;
    // elimination tree of the permuted symmetric pattern
    std::vector<int> parent;
    // combined L+U pattern of the permuted matrix, CSR, columns ascending
    std::vector<int> lu_rp, lu_ci;
    std::vector<int> diag;         // position of the diagonal in each row
    std::vector<int> src;          // user entry stored in each slot, or -1
    std::vector<int> tpos;         // slot of the transposed entry (diagonal: itself)
    // levels and schedules
    std::vector<int> level, level_u;
    std::vector<int> order_f;      // rows by depth, deepest first (refactorization claim order)
    std::vector<int> order_b;      // rows by depth, root first
    int n_levels = 0, n_levels_u = 0;
    long long nnz_sym = 0;
    int max_row = 0;
    double flops = 0.0;
    // Longest-path decomposition of the elimination tree (solve tasks): every
    // task is the path that starts at a node which is not its parent's deepest
    // child and follows deepest children down to a leaf.  After relabelling,
    // task t covers the contiguous rows [task_lo[t], task_hi[t]] (bottom to top).
    std::vector<int> task_lo, task_hi;
    int max_task = 0;
    // Update maps of the refactorization: for L slot t of row i (pivot row d),
    // upd_off[t] is where the relative positions in row i of the entries of
    // U(d, >d) start inside upd_map (empty when over budget).
    std::vector<unsigned> upd_off;
    std::vector<unsigned short> upd_map;
    // Dense root block: the last dense_rows rows (internal labelling) are
    // stored as a full square block of the combined pattern (its structural
    // zeros become explicit slots), so that their elimination among
    // themselves runs as a blocked dense LU.  0 = no such block.  The block
    // is the top of a path of the elimination tree (at most as many rows as
    // the path from the last root down its deepest children).  Rows below
    // the block never depend on it; the update maps hold no entries for the
    // block's own pivot steps (rows and pivots both inside the block).
    int dense_rows = 0;
};

// Largest trailing block the automatic choice considers, the density it
// requires and the smallest block it keeps.
constexpr int DENSE_MAX_ROWS = 2048;
constexpr double DENSE_MIN_DENSITY = 0.8;
constexpr int DENSE_MIN_ROWS = 96;

// Status codes match kkt_status.
enum { A_OK = 0, A_ERR_ARG = 1, A_ERR_PATTERN = 2, A_ERR_ALLOC = 3 };

int validate_pattern(int n, const int *rp, const int *ci);

// Adjacency of A + A^T without the diagonal (CSR, sorted, unique).
void symmetric_graph(int n, const int *rp, const int *ci, std::vector<int> &grp,
                     std::vector<int> &gci);

// Approximate minimum degree ordering of a symmetric graph (no self loops).
void amd_order(int n, const std::vector<int> &grp, const std::vector<int> &gci,
               std::vector<int> &perm);

// Value-aware row permutation (Sec. 5.2: MC64 matching before the ordering):
// row_of_col[j] = the row matched to column j in a perfect matching of the
// nonzeros of A that maximizes the product of |a_{row_of_col[j], j}|, so the
// row-permuted matrix Q A (row j of Q A = row row_of_col[j] of A) has a
// nonzero diagonal with the largest possible product.  Returns A_OK, or
// A_ERR_PATTERN (err set) when A has no perfect matching (structurally
// singular).
int max_product_matching(int n, const int *rp, const int *ci, const double *val,
                         std::vector<int> &row_of_col, std::string &err);

// Full analysis.  ordering: 0 AMD, 1 natural, 2 user (user_perm, new -> old).
// dense_req: -1 no dense root block; 0 the automatic choice (the largest
// trailing block of at most DENSE_MAX_ROWS rows whose pattern is at least
// DENSE_MIN_DENSITY full, if it has DENSE_MIN_ROWS rows or more); k > 0
// k rows.  Either is capped at the length of the path of the elimination
// tree that ends the internal order; the automatic choice also at dense_max.
int analyze(int n, const int *rp, const int *ci, int ordering, const int *user_perm,
            Analysis &out, std::string &err, long long map_budget_bytes = 0, int dense_req = -1,
            int dense_max = DENSE_MAX_ROWS);

}  // namespace kkt
