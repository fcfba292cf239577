// analysis.cpp -- host-side analysis of a fixed sparsity pattern.
//
// arXiv 2306.14337: the symbolic phase runs once on the host (Sec. 4); the
// matrix is reordered with a symmetric fill-reducing ordering of A + A^T
// (Sec. 5.2) and the pattern of the combined L+U storage is computed once and
// reused by every later refactorization (Sec. 5.2, "symbolic factorization").
//
// This file uses its own algorithms: an approximate-minimum-degree ordering on
// a quotient graph (elements, supervariables, approximate external degrees,
// element absorption), the elimination tree by path compression, and the row
// patterns of L as row subtrees of that tree.  Levels are elimination-tree
// heights (forward) and depths (backward).
#include "analysis.h"

#include <algorithm>
#include <cmath>
#include <limits>
#include <queue>
#include <cstring>
#include <numeric>
#include <atomic>
#include <thread>

namespace kkt {

int validate_pattern(int n, const int *rp, const int *ci) {
    if (n <= 0 || !rp || !ci) return A_ERR_PATTERN;
    if (rp[0] != 0) return A_ERR_PATTERN;
    for (int i = 0; i < n; i++) {
        if (rp[i + 1] < rp[i]) return A_ERR_PATTERN;
        for (int p = rp[i]; p < rp[i + 1]; p++) {
            if (ci[p] < 0 || ci[p] >= n) return A_ERR_PATTERN;
            if (p > rp[i] && ci[p] <= ci[p - 1]) return A_ERR_PATTERN;
        }
    }
    return A_OK;
}

void symmetric_graph(int n, const int *rp, const int *ci, std::vector<int> &grp,
                     std::vector<int> &gci) {
    std::vector<int> cnt(n + 1, 0);
    for (int i = 0; i < n; i++)
        for (int p = rp[i]; p < rp[i + 1]; p++)
            if (ci[p] != i) { cnt[i + 1]++; cnt[ci[p] + 1]++; }
    for (int i = 0; i < n; i++) cnt[i + 1] += cnt[i];
    std::vector<int> tmp(cnt[n]);
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    for (int i = 0; i < n; i++)
        for (int p = rp[i]; p < rp[i + 1]; p++)
            if (ci[p] != i) { tmp[fill[i]++] = ci[p]; tmp[fill[ci[p]]++] = i; }
    grp.assign(n + 1, 0);
    gci.clear();
    gci.reserve(tmp.size());
    for (int i = 0; i < n; i++) {
        auto b = tmp.begin() + cnt[i], e = tmp.begin() + cnt[i + 1];
        std::sort(b, e);
        auto u = std::unique(b, e);
        gci.insert(gci.end(), b, u);
        grp[i + 1] = (int)gci.size();
    }
}

// ---------------------------------------------------------------------------
// Approximate minimum degree.
//
// Quotient graph: every index is either a variable (not yet eliminated) or an
// element (an eliminated pivot, standing for the clique it created).  A
// variable i keeps the variables it is still directly adjacent to (A[i]) and
// the elements it belongs to (E[i]); an element e keeps its variables (Le[e]).
// Eliminating pivot p turns it into an element whose variable set is the union
// of A[p] and of the sets of the elements around p, which are absorbed.  The
// external degree of each affected variable is bounded from above by
//   |A_i| + |L_p \ i| + sum_{e in E_i, e != p} |L_e \ L_p|
// (weighted by supervariable size), the approximation of Amestoy, Davis and
// Duff (1996); |L_e \ L_p| is obtained by subtracting from |L_e| the weights
// of the variables of L_p that lie in e.  Elements with |L_e \ L_p| = 0 are
// absorbed into p.  Variables of L_p with identical adjacency are merged into
// supervariables and eliminated together.
void amd_order(int n, const std::vector<int> &grp, const std::vector<int> &gci,
               std::vector<int> &perm) {
    enum : char { VAR = 0, ELEM = 1, DEAD = 2, MERGED = 3 };
    std::vector<std::vector<int>> A(n), E(n), Le(n);
    std::vector<int> nv(n, 1), deg(n, 0), rep(n, -1);
    std::vector<long long> wsz(n, 0), w(n, 0);
    std::vector<char> st(n, VAR);
    std::vector<int> head(n + 1, -1), nxt(n, -1), prv(n, -1);
    std::vector<int> mark(n, 0), wtag(n, 0);
    int tag = 0;

    auto bucket_insert = [&](int i, int d) {
        deg[i] = d;
        nxt[i] = head[d];
        prv[i] = -1;
        if (head[d] >= 0) prv[head[d]] = i;
        head[d] = i;
    };
    auto bucket_remove = [&](int i) {
        int d = deg[i];
        if (prv[i] >= 0) nxt[prv[i]] = nxt[i]; else head[d] = nxt[i];
        if (nxt[i] >= 0) prv[nxt[i]] = prv[i];
        nxt[i] = prv[i] = -1;
    };
    for (int i = 0; i < n; i++) {
        A[i].assign(gci.begin() + grp[i], gci.begin() + grp[i + 1]);
        bucket_insert(i, std::min((int)A[i].size(), n));
    }
    std::vector<int> elim;
    elim.reserve(n);
    std::vector<int> Lp, nd(n, 0);
    int mindeg = 0;
    long long k = 0;
    while (k < n) {
        while (mindeg <= n && head[mindeg] < 0) mindeg++;
        if (mindeg > n) break;  // cannot happen: weights sum to n
        int p = head[mindeg];
        bucket_remove(p);
        elim.push_back(p);
        k += nv[p];
        ++tag;
        // variables of the new element
        Lp.clear();
        mark[p] = tag;
        for (int e : E[p]) {
            if (st[e] != ELEM) continue;
            for (int i : Le[e])
                if (st[i] == VAR && mark[i] != tag) { mark[i] = tag; Lp.push_back(i); }
            st[e] = DEAD;
            std::vector<int>().swap(Le[e]);
        }
        for (int i : A[p])
            if (st[i] == VAR && mark[i] != tag) { mark[i] = tag; Lp.push_back(i); }
        st[p] = ELEM;
        std::vector<int>().swap(A[p]);
        std::vector<int>().swap(E[p]);
        long long lpw = 0;
        for (int i : Lp) { lpw += nv[i]; bucket_remove(i); }
        // |L_e \ L_p| for every element touching L_p
        for (int i : Lp)
            for (int e : E[i]) {
                if (st[e] != ELEM) continue;
                if (wtag[e] != tag) { wtag[e] = tag; w[e] = wsz[e]; }
                w[e] -= nv[i];
            }
        // prune adjacency, absorb covered elements, bound the degree
        for (int i : Lp) {
            std::vector<int> ne;
            ne.reserve(E[i].size() + 1);
            long long de = 0;
            for (int e : E[i]) {
                if (st[e] != ELEM) continue;
                if (w[e] == 0) { st[e] = DEAD; std::vector<int>().swap(Le[e]); continue; }
                ne.push_back(e);
                de += w[e];
            }
            ne.push_back(p);
            std::sort(ne.begin(), ne.end());
            std::vector<int> na;
            na.reserve(A[i].size());
            long long da = 0;
            for (int j : A[i])
                if (st[j] == VAR && mark[j] != tag) { na.push_back(j); da += nv[j]; }
            std::sort(na.begin(), na.end());
            A[i].swap(na);
            E[i].swap(ne);
            long long rest = (long long)n - k - nv[i];
            long long d = da + de + (lpw - nv[i]);
            d = std::min(d, (long long)deg[i] + lpw - nv[i]);
            d = std::min(d, rest);
            nd[i] = (int)std::max(0LL, d);
        }
        // supervariables: identical A and E among the variables of L_p
        if (Lp.size() > 1) {
            std::vector<std::pair<unsigned long long, int>> key;
            key.reserve(Lp.size());
            for (int i : Lp) {
                unsigned long long h = 1469598103934665603ULL;
                for (int j : A[i]) h = (h ^ (unsigned)j) * 1099511628211ULL;
                h = (h ^ 0x9e3779b9ULL) * 1099511628211ULL;
                for (int e : E[i]) h = (h ^ (unsigned)e) * 1099511628211ULL;
                key.push_back({h, i});
            }
            std::sort(key.begin(), key.end());
            for (size_t a = 0; a < key.size();) {
                size_t b = a;
                while (b < key.size() && key[b].first == key[a].first) b++;
                for (size_t x = a; x < b; x++) {
                    int i = key[x].second;
                    if (st[i] != VAR) continue;
                    for (size_t y = x + 1; y < b; y++) {
                        int j = key[y].second;
                        if (st[j] != VAR) continue;
                        if (A[i] == A[j] && E[i] == E[j]) {
                            nv[i] += nv[j];
                            nd[i] -= nv[j];
                            nv[j] = 0;
                            st[j] = MERGED;
                            rep[j] = i;
                            std::vector<int>().swap(A[j]);
                            std::vector<int>().swap(E[j]);
                        }
                    }
                }
                a = b;
            }
        }
        Le[p] = Lp;
        wsz[p] = lpw;
        for (int i : Lp) {
            if (st[i] != VAR) continue;
            int d = std::min(std::max(nd[i], 0), n);
            bucket_insert(i, d);
            if (d < mindeg) mindeg = d;
        }
    }
    // pivots in elimination order, each followed by the variables merged into it
    std::vector<std::vector<int>> kids(n);
    for (int j = 0; j < n; j++)
        if (rep[j] >= 0) kids[rep[j]].push_back(j);
    perm.clear();
    perm.reserve(n);
    std::vector<int> stack;
    for (int p : elim) {
        stack.assign(1, p);
        while (!stack.empty()) {
            int v = stack.back();
            stack.pop_back();
            perm.push_back(v);
            for (auto it = kids[v].rbegin(); it != kids[v].rend(); ++it) stack.push_back(*it);
        }
    }
}

// ---------------------------------------------------------------------------

static int find_slot(const std::vector<int> &rp, const std::vector<int> &ci, int row, int col) {
    auto b = ci.begin() + rp[row], e = ci.begin() + rp[row + 1];
    auto it = std::lower_bound(b, e, col);
    if (it == e || *it != col) return -1;
    return (int)(it - ci.begin());
}

// Elimination tree (parent) and heights (leaves 0) of the symmetric graph
// (grp, gci) under the ordering perm / iperm.
static void etree_heights(int n, const std::vector<int> &grp, const std::vector<int> &gci,
                          const std::vector<int> &perm, const std::vector<int> &iperm,
                          std::vector<int> &parent, std::vector<int> &height) {
    parent.assign(n, -1);
    std::vector<int> anc(n, -1), nb;
    for (int i = 0; i < n; i++) {
        const int o = perm[i];
        nb.clear();
        for (int p = grp[o]; p < grp[o + 1]; p++) nb.push_back(iperm[gci[p]]);
        for (int r : nb) {
            if (r >= i) continue;
            while (anc[r] != -1 && anc[r] != i) {
                const int t = anc[r];
                anc[r] = i;
                r = t;
            }
            if (anc[r] == -1) { anc[r] = i; parent[r] = i; }
        }
    }
    height.assign(n, 0);
    for (int i = 0; i < n; i++)
        if (parent[i] >= 0) height[parent[i]] = std::max(height[parent[i]], height[i] + 1);
}

int analyze(int n, const int *rp, const int *ci, int ordering, const int *user_perm,
            Analysis &out, std::string &err, long long map_budget_bytes, int dense_req, int dense_max) {
    int rc = validate_pattern(n, rp, ci);
    if (rc) { err = "malformed CSR pattern (n <= 0, unsorted, duplicate or out-of-range index)"; return rc; }
    if (rp[n] > (1 << 30)) { err = "too many entries"; return A_ERR_ARG; }
    Analysis &a = out;
    a.n = n;
    a.a_rp.assign(rp, rp + n + 1);
    a.a_ci.assign(ci, ci + rp[n]);
    a.a_row.resize(rp[n]);
    for (int i = 0; i < n; i++)
        for (int p = rp[i]; p < rp[i + 1]; p++) a.a_row[p] = i;

    std::vector<int> grp, gci;
    symmetric_graph(n, rp, ci, grp, gci);
    a.nnz_sym = (long long)gci.size() + n;

    // ordering
    if (ordering == 0) {
        amd_order(n, grp, gci, a.perm);
    } else if (ordering == 1) {
        a.perm.resize(n);
        std::iota(a.perm.begin(), a.perm.end(), 0);
    } else if (ordering == 2) {
        if (!user_perm) { err = "user ordering requested without user_perm"; return A_ERR_ARG; }
        a.perm.assign(user_perm, user_perm + n);
    } else {
        err = "unknown ordering";
        return A_ERR_ARG;
    }
    if ((int)a.perm.size() != n) { err = "ordering has wrong length"; return A_ERR_ARG; }
    a.iperm.assign(n, -1);
    for (int i = 0; i < n; i++) {
        int o = a.perm[i];
        if (o < 0 || o >= n || a.iperm[o] >= 0) { err = "ordering is not a permutation"; return A_ERR_ARG; }
        a.iperm[o] = i;
    }
    // Relabel by a postorder of the elimination tree of the given ordering in
    // which every node's deepest child (most levels below it; ties: smallest
    // index) is visited last.  A postorder keeps the fill and the tree; this
    // one places each deepest child directly before its parent.
    a.view_perm = a.perm;
    {
        std::vector<int> par, hgt;
        etree_heights(n, grp, gci, a.perm, a.iperm, par, hgt);
        std::vector<int> heavy(n, -1), first(n, -1), next(n, -1);
        for (int j = n - 1; j >= 0; j--) {            // child lists ascending
            const int p = par[j];
            if (p < 0) continue;
            next[j] = first[p];
            first[p] = j;
            const int h = heavy[p];
            if (h < 0 || hgt[j] > hgt[h] || (hgt[j] == hgt[h] && j < h)) heavy[p] = j;
        }
        a.internal_of.assign(n, -1);
        int pos = 0;
        std::vector<std::pair<int, int>> st;           // (node, stage)
        for (int r = 0; r < n; r++) {
            if (par[r] >= 0) continue;
            st.push_back({r, 0});
            while (!st.empty()) {
                auto &top = st.back();
                const int v = top.first;
                if (top.second == 0) {                  // push children: heavy deepest in stack order
                    top.second = 1;
                    if (heavy[v] >= 0) st.push_back({heavy[v], 0});
                    std::vector<int> light;
                    for (int c = first[v]; c >= 0; c = next[c]) if (c != heavy[v]) light.push_back(c);
                    for (auto it = light.rbegin(); it != light.rend(); ++it) st.push_back({*it, 0});
                } else {
                    a.internal_of[v] = pos++;
                    st.pop_back();
                }
            }
        }
        a.view_of.assign(n, -1);
        for (int v = 0; v < n; v++) a.view_of[a.internal_of[v]] = v;
        std::vector<int> ip(n);
        for (int u = 0; u < n; u++) ip[u] = a.view_perm[a.view_of[u]];
        a.perm = ip;
        for (int u = 0; u < n; u++) a.iperm[a.perm[u]] = u;
    }

    // permuted symmetric graph: neighbours of new vertex i, sorted
    std::vector<int> prp(n + 1, 0), pci(gci.size());
    for (int i = 0; i < n; i++) prp[i + 1] = prp[i] + (grp[a.perm[i] + 1] - grp[a.perm[i]]);
    for (int i = 0; i < n; i++) {
        int o = a.perm[i], q = prp[i];
        for (int p = grp[o]; p < grp[o + 1]; p++) pci[q++] = a.iperm[gci[p]];
        std::sort(pci.begin() + prp[i], pci.begin() + prp[i + 1]);
    }

    // elimination tree by path compression over virtual ancestors
    a.parent.assign(n, -1);
    std::vector<int> anc(n, -1);
    for (int i = 0; i < n; i++) {
        for (int p = prp[i]; p < prp[i + 1]; p++) {
            int r = pci[p];
            if (r >= i) break;
            while (anc[r] != -1 && anc[r] != i) {
                int t = anc[r];
                anc[r] = i;
                r = t;
            }
            if (anc[r] == -1) { anc[r] = i; a.parent[r] = i; }
        }
    }

    // row patterns of L: row subtree of i = union of tree paths from each
    // j < i adjacent to i up to i
    std::vector<int> lrp(n + 1, 0);
    std::vector<int> lci;
    lci.reserve(gci.size() * 3);
    std::vector<int> mk(n, -1);
    for (int i = 0; i < n; i++) {
        size_t start = lci.size();
        mk[i] = i;
        for (int p = prp[i]; p < prp[i + 1]; p++) {
            int r = pci[p];
            if (r >= i) break;
            while (r >= 0 && mk[r] != i) {
                mk[r] = i;
                lci.push_back(r);
                r = a.parent[r];
            }
            if (r < 0) { err = "internal: elimination tree path does not reach its row"; return A_ERR_ARG; }
        }
        std::sort(lci.begin() + start, lci.end());
        lrp[i + 1] = (int)lci.size();
    }
    // Dense root block (Sec. 4: supernodal factorizations; the top of the
    // elimination tree of these KKT matrices is a chain of separator rows
    // whose trailing block is nearly full).  Rows [lo, n) get every column of
    // [lo, i) in their L part, so the trailing s x s block is full; fill stays
    // closed (a pivot d >= lo only updates rows and columns >= lo), rows below
    // lo are unchanged, and the block becomes a chain of the tree.
    {
        int s = 0;
        if (dense_req > 0) {
            s = std::min(dense_req, n);
        } else if (dense_req == 0) {
            // entries of the trailing block of t rows: t + 2 |{L(i,j): i, j >= n - t}|;
            // adding row n - t - 1 adds the entries of its L column
            std::vector<int> lcol(n, 0);
            for (size_t q = 0; q < lci.size(); q++) lcol[lci[q]]++;
            long long cnt = 0;
            const int tmax = std::min({n, DENSE_MAX_ROWS, dense_max});
            for (int t = 1; t <= tmax; t++) {
                cnt += lcol[n - t];
                if ((double)(t + 2 * cnt) >= DENSE_MIN_DENSITY * (double)t * (double)t) s = t;
            }
            if (s < DENSE_MIN_ROWS) s = 0;
        }
        // The block must be a chain of the elimination tree (each row the
        // child of the next): then every order of the tree's postorders and
        // of the caller's ordering agrees on it, and the full block changes
        // the factorization of that order by explicit zeros only.  The
        // relabelling put the longest path from the last root at the end.
        int chain = 1;
        while (chain < n && a.parent[n - chain - 1] == n - chain) chain++;
        s = std::min(s, chain);
        if (dense_req == 0 && s < DENSE_MIN_ROWS) s = 0;
        a.dense_rows = s;
        if (s > 0) {
            const int lo = n - s;
            std::vector<int> nrp(n + 1, 0), nci;
            nci.reserve(lci.size() + (size_t)s * (size_t)s / 2);
            for (int i = 0; i < n; i++) {
                for (int p = lrp[i]; p < lrp[i + 1]; p++)
                    if (i < lo || lci[p] < lo) nci.push_back(lci[p]);
                if (i >= lo)
                    for (int j = lo; j < i; j++) nci.push_back(j);
                nrp[i + 1] = (int)nci.size();
            }
            lrp.swap(nrp);
            lci.swap(nci);
            for (int i = lo; i < n - 1; i++) a.parent[i] = i + 1;
            a.parent[n - 1] = -1;
        }
    }
    // rows of U = columns of L (pattern symmetric)
    std::vector<int> ucnt(n + 1, 0);
    for (size_t q = 0; q < lci.size(); q++) ucnt[lci[q] + 1]++;
    for (int i = 0; i < n; i++) ucnt[i + 1] += ucnt[i];
    std::vector<int> uci(lci.size()), ufill(ucnt.begin(), ucnt.end() - 1);
    for (int i = 0; i < n; i++)
        for (int p = lrp[i]; p < lrp[i + 1]; p++) uci[ufill[lci[p]]++] = i;  // ascending i
    // combined rows
    long long nnz = (long long)lci.size() * 2 + n;
    if (nnz > (1LL << 31) - 1) { err = "factor too large for 32-bit indices"; return A_ERR_ARG; }
    a.lu_rp.assign(n + 1, 0);
    a.lu_ci.resize(nnz);
    a.diag.resize(n);
    {
        long long q = 0;
        for (int i = 0; i < n; i++) {
            for (int p = lrp[i]; p < lrp[i + 1]; p++) a.lu_ci[q++] = lci[p];
            a.diag[i] = (int)q;
            a.lu_ci[q++] = i;
            for (int p = ucnt[i]; p < ucnt[i + 1]; p++) a.lu_ci[q++] = uci[p];
            a.lu_rp[i + 1] = (int)q;
        }
    }
    a.max_row = 0;
    for (int i = 0; i < n; i++) a.max_row = std::max(a.max_row, a.lu_rp[i + 1] - a.lu_rp[i]);

    // user entry -> slot
    a.src.assign(nnz, -1);
    for (int r = 0; r < n; r++)
        for (int p = rp[r]; p < rp[r + 1]; p++) {
            int s = find_slot(a.lu_rp, a.lu_ci, a.iperm[r], a.iperm[ci[p]]);
            if (s < 0) { err = "internal: user entry outside the filled pattern"; return A_ERR_ARG; }
            a.src[s] = p;
        }
    // transposed slots
    a.tpos.resize(nnz);
    for (int i = 0; i < n; i++)
        for (int p = a.lu_rp[i]; p < a.lu_rp[i + 1]; p++) {
            int j = a.lu_ci[p];
            int s = (j == i) ? p : find_slot(a.lu_rp, a.lu_ci, j, i);
            if (s < 0) { err = "internal: pattern not symmetric"; return A_ERR_ARG; }
            a.tpos[p] = s;
        }

    // levels: height (leaves 0) and depth (roots 0) in the elimination tree
    a.level.assign(n, 0);
    for (int i = 0; i < n; i++)
        if (a.parent[i] >= 0) a.level[a.parent[i]] = std::max(a.level[a.parent[i]], a.level[i] + 1);
    a.level_u.assign(n, 0);
    for (int i = n - 1; i >= 0; i--)
        if (a.parent[i] >= 0) a.level_u[i] = a.level_u[a.parent[i]] + 1;
    a.n_levels = *std::max_element(a.level.begin(), a.level.end()) + 1;
    a.n_levels_u = *std::max_element(a.level_u.begin(), a.level_u.end()) + 1;
    auto by_level = [n](const std::vector<int> &lev, int nl, std::vector<int> &ord) {
        std::vector<int> c(nl + 1, 0);
        for (int i = 0; i < n; i++) c[lev[i] + 1]++;
        for (int l = 0; l < nl; l++) c[l + 1] += c[l];
        ord.resize(n);
        for (int i = 0; i < n; i++) ord[c[lev[i]]++] = i;
    };
    // Refactorization claim order: deepest rows first (distance to the root,
    // descending; Hu's critical-path-first list schedule for an in-tree).  A
    // row depends only on its descendants, which are deeper, so the order is
    // topological; unlike an order by height it starts the long paths of the
    // tree first instead of every leaf of the tree.
    {
        std::vector<int> neg(n);
        for (int i = 0; i < n; i++) neg[i] = a.n_levels_u - 1 - a.level_u[i];
        by_level(neg, a.n_levels_u, a.order_f);
    }
    by_level(a.level_u, a.n_levels_u, a.order_b);

    // flops of one refactorization: each pivot d eliminated from the rows of
    // L(:,d) costs one division and a multiply-add per entry of U(d, >d)
    double fl = 0.0;
    for (int d = 0; d < n; d++) {
        double lcol = ucnt[d + 1] - ucnt[d];       // |L(:,d)| = |U(d,:)| off-diagonal
        fl += lcol * (1.0 + 2.0 * lcol);
    }
    a.flops = fl;

    // longest-path tasks: after the relabelling every node's deepest child is
    // the node just below it, so a task is a maximal run v, v-1, v-2, ... with
    // parent(x - 1) = x and x - 1 the deepest child of x.
    {
        std::vector<int> heavy(n, -1);
        for (int j = 0; j < n; j++) {
            const int p = a.parent[j];
            if (p < 0) continue;
            const int h = heavy[p];
            if (h < 0 || a.level[j] > a.level[h] || (a.level[j] == a.level[h] && j > h)) heavy[p] = j;
        }
        a.task_lo.clear();
        a.task_hi.clear();
        a.max_task = 0;
        for (int t = 0; t < n; t++) {
            const int p = a.parent[t];
            if (p >= 0 && heavy[p] == t) continue;       // not a task top
            int lo = t;
            while (heavy[lo] >= 0) {
                if (heavy[lo] != lo - 1) { err = "internal: task rows are not contiguous"; return A_ERR_ARG; }
                lo = heavy[lo];
            }
            a.task_lo.push_back(lo);
            a.task_hi.push_back(t);
            a.max_task = std::max(a.max_task, t - lo + 1);
        }
    }

    // update maps: one uint16 per multiply-add of the refactorization; rows
    // are independent, so they are filled in parallel after a prefix sum
    // (the dense root block's own pivot steps -- row and pivot both in the
    // block -- run in the dense kernel and have no map entries)
    a.upd_off.clear();
    a.upd_map.clear();
    {
        const int dlo = n - a.dense_rows;
        std::vector<long long> rowq(n + 1, 0);
        for (int i = 0; i < n; i++) {
            long long c = 0;
            for (int t = a.lu_rp[i]; t < a.diag[i]; t++) {
                const int d = a.lu_ci[t];
                if (i >= dlo && d >= dlo) break;
                c += a.lu_rp[d + 1] - a.diag[d] - 1;
            }
            rowq[i + 1] = rowq[i] + c;
        }
        const double entries = (double)rowq[n];
        const bool fits = a.max_row <= 65535 && entries < 4.0e9 &&
                          entries * 2.0 + 4.0 * (double)nnz <= (double)map_budget_bytes;
        if (fits) {
            a.upd_off.assign(nnz, 0);
            a.upd_map.resize((size_t)rowq[n]);
            std::atomic<int> bad{0};
            auto fill = [&](int r0, int r1) {
                for (int i = r0; i < r1; i++) {
                    const int rb = a.lu_rp[i], re = a.lu_rp[i + 1];
                    size_t q = (size_t)rowq[i];
                    for (int t = rb; t < a.diag[i]; t++) {
                        const int d = a.lu_ci[t];
                        a.upd_off[t] = (unsigned)q;
                        if (i >= dlo && d >= dlo) continue;
                        int w = t + 1;               // merge U(d, >d) into row i (both sorted)
                        for (int u = a.diag[d] + 1; u < a.lu_rp[d + 1]; u++) {
                            const int j = a.lu_ci[u];
                            while (w < re && a.lu_ci[w] < j) w++;
                            if (w >= re || a.lu_ci[w] != j) { bad = 1; return; }
                            a.upd_map[q++] = (unsigned short)(w - rb);
                        }
                    }
                }
            };
            unsigned nth = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
            if (rowq[n] < (1LL << 22)) nth = 1;
            std::vector<std::thread> th;
            int r0 = 0;
            for (unsigned k = 0; k < nth; k++) {
                const long long target = rowq[n] * (long long)(k + 1) / nth;
                int r1 = r0;
                while (r1 < n && (k + 1 == nth || rowq[r1] < target)) r1++;
                if (k + 1 == nth) r1 = n;
                th.emplace_back(fill, r0, r1);
                r0 = r1;
            }
            for (auto &t : th) t.join();
            if (bad) { err = "internal: update target outside the filled row"; return A_ERR_ARG; }
        }
    }
    return A_OK;
}


// ---------------------------------------------------------------------------
// Maximum-product matching (the weighted bipartite matching of Duff and
// Koster's MC64, which the paper's Ginkgo path runs before AMD, Sec. 5.2).
// Costs c(j,i) = log max_k |a_kj| - log |a_ij| >= 0 per column j over the
// nonzero entries; a perfect matching of minimum total cost maximizes the
// product of the matched |a_ij|.  Successive shortest augmenting paths with
// dual potentials (Hungarian method): column potentials p, row potentials q,
// reduced costs c - p - q >= 0 and 0 on matched edges; a greedy pass matches
// every column it can on a zero reduced cost, then each free column finds the
// nearest free row by Dijkstra over alternating paths and the potentials of
// the nodes settled before it move by D - dist, which keeps every reduced
// cost non-negative and makes the new path tight.
int max_product_matching(int n, const int *rp, const int *ci, const double *val,
                         std::vector<int> &row_of_col, std::string &err) {
    // column-wise copy of the nonzero entries with their costs
    std::vector<int> cp(n + 1, 0);
    for (int r = 0; r < n; r++)
        for (int p = rp[r]; p < rp[r + 1]; p++)
            if (val[p] != 0.0 && std::isfinite(val[p])) cp[ci[p] + 1]++;
    for (int j = 0; j < n; j++) cp[j + 1] += cp[j];
    std::vector<int> crow(cp[n]);
    std::vector<double> cost(cp[n]);
    {
        std::vector<int> fill(cp.begin(), cp.end() - 1);
        for (int r = 0; r < n; r++)
            for (int p = rp[r]; p < rp[r + 1]; p++)
                if (val[p] != 0.0 && std::isfinite(val[p])) {
                    const int j = ci[p];
                    crow[fill[j]] = r;
                    cost[fill[j]++] = std::log(std::fabs(val[p]));
                }
    }
    for (int j = 0; j < n; j++) {
        if (cp[j] == cp[j + 1]) { err = "matching: an empty column (structurally singular)"; return A_ERR_PATTERN; }
        double m = -INFINITY;
        for (int t = cp[j]; t < cp[j + 1]; t++) m = std::max(m, cost[t]);
        for (int t = cp[j]; t < cp[j + 1]; t++) cost[t] = m - cost[t];
    }
    const double INF = std::numeric_limits<double>::infinity();
    std::vector<double> pcol(n, 0.0), qrow(n, INF);
    for (int j = 0; j < n; j++)
        for (int t = cp[j]; t < cp[j + 1]; t++) qrow[crow[t]] = std::min(qrow[crow[t]], cost[t]);
    for (int i = 0; i < n; i++)
        if (!(qrow[i] < INF)) { err = "matching: an empty row (structurally singular)"; return A_ERR_PATTERN; }
    row_of_col.assign(n, -1);
    std::vector<int> col_of_row(n, -1);
    for (int j = 0; j < n; j++)                       // greedy on tight edges
        for (int t = cp[j]; t < cp[j + 1]; t++) {
            const int i = crow[t];
            if (col_of_row[i] < 0 && cost[t] - pcol[j] - qrow[i] <= 0.0) {
                row_of_col[j] = i;
                col_of_row[i] = j;
                break;
            }
        }
    std::vector<double> dist(n, INF);
    std::vector<int> pred(n, -1);                     // row -> column it was reached from
    std::vector<char> done(n, 0);
    std::vector<int> touched, settled_rows, settled_cols;
    typedef std::pair<double, int> QE;
    for (int s = 0; s < n; s++) {
        if (row_of_col[s] >= 0) continue;
        std::priority_queue<QE, std::vector<QE>, std::greater<QE>> pq;
        touched.clear();
        settled_rows.clear();
        settled_cols.clear();
        auto relax = [&](int j, double dj) {
            for (int t = cp[j]; t < cp[j + 1]; t++) {
                const int i = crow[t];
                if (done[i]) continue;
                const double nd = dj + std::max(0.0, cost[t] - pcol[j] - qrow[i]);
                if (nd < dist[i]) {
                    if (!(dist[i] < INF)) touched.push_back(i);
                    dist[i] = nd;
                    pred[i] = j;
                    pq.push(QE(nd, i));
                }
            }
        };
        std::vector<double> dcol_settled;
        settled_cols.push_back(s);
        dcol_settled.push_back(0.0);
        relax(s, 0.0);
        int t_row = -1;
        double D = 0.0;
        while (!pq.empty()) {
            const QE e = pq.top();
            pq.pop();
            const int i = e.second;
            if (done[i] || e.first > dist[i]) continue;
            done[i] = 1;
            settled_rows.push_back(i);
            if (col_of_row[i] < 0) { t_row = i; D = dist[i]; break; }
            const int j = col_of_row[i];
            settled_cols.push_back(j);
            dcol_settled.push_back(dist[i]);
            relax(j, dist[i]);
        }
        if (t_row < 0) { err = "matching: no perfect matching (structurally singular)"; return A_ERR_PATTERN; }
        // potentials of the nodes settled before the free row
        for (size_t k = 0; k < settled_cols.size(); k++) pcol[settled_cols[k]] += D - dcol_settled[k];
        for (int i : settled_rows)
            if (i != t_row) qrow[i] -= D - dist[i];
        // augment along the path back to s
        int i = t_row;
        while (i >= 0) {
            const int j = pred[i];
            const int prev = row_of_col[j];
            row_of_col[j] = i;
            col_of_row[i] = j;
            i = (j == s) ? -1 : prev;
        }
        for (int r : touched) { dist[r] = INF; done[r] = 0; pred[r] = -1; }
    }
    return A_OK;
}

}  // namespace kkt
