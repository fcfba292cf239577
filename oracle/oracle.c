/*
 * oracle.c -- plain, slow, single-threaded CPU reference for the fixed-pivot
 * sparse LU refactorization of KKT systems and its solves.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load this file's library.  It shares no
 * source, header, table or helper with the CUDA library it checks.
 *
 * Passages followed (arXiv 2306.14337):
 *   Sec. 4  : three phases -- symbolic, numeric, solve; refactorization reuses
 *             the permutation and the L/U patterns (no pivoting on the device).
 *   Sec. 5.1: the first system is factored by KLU, whose numeric kernel is the
 *             Gilbert-Peierls left-looking LU; the pattern of each column is
 *             the reach of A(:,j) in the graph of the L columns found so far.
 *   Sec. 5  : IPM regularization acts as static-pivot perturbation -> one
 *             pivot sequence is reused; here the diagonal of the symmetrically
 *             permuted matrix is the pivot sequence.
 *   Sec. 5.1: iterative refinement rho = r - K dx, K delta = rho, dx += delta.
 *
 * Readings where the paper is silent (all listed in the design notes):
 *   - Doolittle form: L unit lower triangular (diagonal not stored), pivots
 *     in U (the garbled alpha <- a_id / a_ii of Algorithm 1 read as a_id/u_dd).
 *   - Pivot perturbation: tau = tau_rel * max|A'|; a computed pivot p with
 *     !(|p| >= tau) or |p| infinite becomes sign(A'_jj) * tau (+ if A'_jj == 0)
 *     and is counted.
 *   - Fill is structural: explicit zeros keep their slots.
 *   - Equilibration: r_i = max_j |a_ij|, e_i = floor(log2 r_i) (exact, ilogb),
 *     s_i = 2^-floor(e_i / 2); s_i = 1 when r_i is zero or not finite.
 *   - Level of column j: 0 when U(:,j) holds only the diagonal, else
 *     1 + max level of the k < j in U(:,j).  Backward level of row j: 0 when
 *     U(j,:) holds only the diagonal, else 1 + max backward level of the
 *     k > j in U(j,:).
 *
 * Index convention: all arrays int32 / float64, compressed sparse column for
 * the factors, rows ascending within each column.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* growable arrays                                                          */
typedef struct { int *i; double *x; double *t; double *e; long n, cap; } orc_vec;

static int vec_push(orc_vec *v, int i, double x, double t, double e) {
    if (v->n == v->cap) {
        long nc = v->cap ? 2 * v->cap : 1024;
        int *ni = (int *)realloc(v->i, nc * sizeof(int));
        if (!ni) return -1;
        v->i = ni;
        double *nx = (double *)realloc(v->x, nc * sizeof(double));
        if (!nx) return -1;
        v->x = nx;
        double *nt = (double *)realloc(v->t, nc * sizeof(double));
        if (!nt) return -1;
        v->t = nt;
        double *ne = (double *)realloc(v->e, nc * sizeof(double));
        if (!ne) return -1;
        v->e = ne;
        v->cap = nc;
    }
    v->i[v->n] = i; v->x[v->n] = x; v->t[v->n] = t; v->e[v->n] = e; v->n++;
    return 0;
}

static double gamma_m(int m, double u) { return (m * u) / (1.0 - m * u); }

static int cmp_int(const void *a, const void *b) {
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/* ------------------------------------------------------------------------ */
/* Factor handle                                                            */
typedef struct {
    int n;
    int *Lp; orc_vec L;   /* strict lower part, unit diagonal implied */
    int *Up; orc_vec U;   /* upper part, diagonal is the last entry of each column */
    int n_perturbed;
    double tau;
} orc_lu;

void orc_lu_free(orc_lu *f) {
    if (!f) return;
    free(f->Lp); free(f->Up);
    free(f->L.i); free(f->L.x); free(f->L.t); free(f->L.e);
    free(f->U.i); free(f->U.x); free(f->U.t); free(f->U.e);
    free(f);
}

/*
 * Gilbert-Peierls left-looking LU of A' (n x n, CSC: Ap, Ai, Ax; every column
 * must hold its diagonal) with the diagonal pivot sequence (Sec. 5.1, KLU's
 * numeric phase; Sec. 4 "numeric phase").  For column j:
 *   1. reach = nodes reachable from struct(A'(:,j)) in the graph with edges
 *      k -> i for i in struct(L(:,k)), k < j; a depth-first search gives a
 *      topological order (reverse postorder).
 *   2. x = A'(:,j); for k in reach (topological order), k < j:
 *        x[i] -= L(i,k) * x[k] for i in struct(L(:,k));
 *      t accumulates |A'(i,j)| + sum |L(i,k) x[k]| (the magnitude of the terms
 *      that formed each entry).
 *   3. pivot p = x[j], perturbation test (see header).
 *   4. U(k,j) = x[k] for k <= j;  L(i,j) = x[i] / p for i > j.
 *
 * Alongside, a first-order running rounding-error bound e (Wilkinson's running
 * error analysis) is kept for every entry so that a result computed with
 * another summation order can be compared entry by entry:
 *   e(x_i) = gamma_{m_i + 1} t_i + sum_k ( |L(i,k)| e(U(k,j)) + e(L(i,k)) |U(k,j)| ),
 *   m_i = number of update terms of the entry, gamma_m = m u / (1 - m u),
 *   e(L(i,j)) = ( e(x_i) + |L(i,j)| e(x_j) ) / |p| + u |L(i,j)|.
 * gamma_m t bounds the error of a sum of m+1 terms in any order (Higham,
 * Sec. 3.1); the second part carries the errors of the factor entries used.
 * Returns NULL on allocation failure.
 */
orc_lu *orc_lu_factor(int n, const int *Ap, const int *Ai, const double *Ax, double tau_rel) {
    orc_lu *f = (orc_lu *)calloc(1, sizeof(orc_lu));
    if (!f) return NULL;
    f->n = n;
    f->Lp = (int *)calloc((size_t)n + 1, sizeof(int));
    f->Up = (int *)calloc((size_t)n + 1, sizeof(int));
    double *x = (double *)calloc((size_t)n, sizeof(double));
    double *t = (double *)calloc((size_t)n, sizeof(double));
    double *ea = (double *)calloc((size_t)n, sizeof(double));   /* propagated error */
    int *nterm = (int *)calloc((size_t)n, sizeof(int));
    const double u = 0x1p-53;
    int *mark = (int *)malloc((size_t)n * sizeof(int));
    int *stack = (int *)malloc((size_t)n * sizeof(int));
    int *child = (int *)malloc((size_t)n * sizeof(int));
    int *topo = (int *)malloc((size_t)n * sizeof(int));
    int *tmp = (int *)malloc((size_t)n * sizeof(int));
    if (!f->Lp || !f->Up || !x || !t || !ea || !nterm || !mark || !stack || !child || !topo || !tmp) goto fail;
    for (int i = 0; i < n; i++) mark[i] = -1;

    double amax = 0.0;
    for (long p = 0; p < Ap[n]; p++) {
        double a = fabs(Ax[p]);
        if (a > amax) amax = a;
    }
    f->tau = tau_rel * amax;

    for (int j = 0; j < n; j++) {
        /* 1. reach of struct(A'(:,j)), postorder into topo[top..n-1] reversed */
        int top = n;
        for (int p = Ap[j]; p < Ap[j + 1]; p++) {
            int r = Ai[p];
            if (mark[r] == j) continue;
            int sp = 0;
            stack[sp++] = r;
            mark[r] = j;
            child[r] = (r < j) ? f->Lp[r] : -1;
            while (sp > 0) {
                int k = stack[sp - 1];
                int advanced = 0;
                if (k < j) {
                    while (child[k] < f->Lp[k + 1]) {
                        int i = f->L.i[child[k]++];
                        if (mark[i] != j) {
                            mark[i] = j;
                            child[i] = (i < j) ? f->Lp[i] : -1;
                            stack[sp++] = i;
                            advanced = 1;
                            break;
                        }
                    }
                }
                if (!advanced) {
                    sp--;
                    topo[--top] = k;   /* postorder, stored back to front */
                }
            }
        }
        /* 2. numeric: scatter A'(:,j), then eliminate in topological order */
        for (int q = top; q < n; q++) {
            int r = topo[q];
            x[r] = 0.0; t[r] = 0.0; ea[r] = 0.0; nterm[r] = 0;
        }
        double ajj = 0.0;
        for (int p = Ap[j]; p < Ap[j + 1]; p++) {
            x[Ai[p]] = Ax[p];
            t[Ai[p]] = fabs(Ax[p]);
            if (Ai[p] == j) ajj = Ax[p];
        }
        for (int q = top; q < n; q++) {
            int k = topo[q];
            if (k >= j) continue;
            double xk = x[k];
            /* x[k] is final: its bound is complete */
            double ek = ea[k] + gamma_m(nterm[k] + 1, u) * t[k];
            for (int p = f->Lp[k]; p < f->Lp[k + 1]; p++) {
                int i = f->L.i[p];
                double term = f->L.x[p] * xk;
                x[i] -= term;
                t[i] += fabs(term);
                ea[i] += fabs(f->L.x[p]) * ek + f->L.e[p] * fabs(xk);
                nterm[i]++;
            }
        }
        /* 3. pivot perturbation test */
        double piv = x[j];
        if (!(fabs(piv) >= f->tau) || isinf(piv)) {
            piv = (ajj < 0.0) ? -f->tau : f->tau;
            f->n_perturbed++;
        }
        /* 4. store U(:,j) (rows ascending, diagonal last) and L(:,j) */
        int nt = 0;
        for (int q = top; q < n; q++) tmp[nt++] = topo[q];
        qsort(tmp, nt, sizeof(int), cmp_int);
        double ej = ea[j] + gamma_m(nterm[j] + 1, u) * t[j];
        for (int q = 0; q < nt; q++) {
            int i = tmp[q];
            if (i < j) {
                double ei = ea[i] + gamma_m(nterm[i] + 1, u) * t[i];
                if (vec_push(&f->U, i, x[i], t[i], ei)) goto fail;
            }
        }
        if (vec_push(&f->U, j, piv, t[j], ej)) goto fail;
        f->Up[j + 1] = (int)f->U.n;
        for (int q = 0; q < nt; q++) {
            int i = tmp[q];
            if (i > j) {
                double l = x[i] / piv;
                double ei = ea[i] + gamma_m(nterm[i] + 1, u) * t[i];
                double el = (ei + fabs(l) * ej) / fabs(piv) + u * fabs(l);
                if (vec_push(&f->L, i, l, t[i] / fabs(piv), el)) goto fail;
            }
        }
        f->Lp[j + 1] = (int)f->L.n;
    }
    free(x); free(t); free(ea); free(nterm); free(mark); free(stack); free(child); free(topo); free(tmp);
    return f;
fail:
    free(x); free(t); free(ea); free(nterm); free(mark); free(stack); free(child); free(topo); free(tmp);
    orc_lu_free(f);
    return NULL;
}

long orc_lu_nnz_l(const orc_lu *f) { return f->L.n; }
long orc_lu_nnz_u(const orc_lu *f) { return f->U.n; }
int orc_lu_n_perturbed(const orc_lu *f) { return f->n_perturbed; }
double orc_lu_tau(const orc_lu *f) { return f->tau; }

void orc_lu_export(const orc_lu *f, int *Lp, int *Li, double *Lx, double *Lt, double *Le,
                   int *Up, int *Ui, double *Ux, double *Ut, double *Ue) {
    memcpy(Lp, f->Lp, sizeof(int) * (f->n + 1));
    memcpy(Up, f->Up, sizeof(int) * (f->n + 1));
    if (f->L.n) {
        memcpy(Li, f->L.i, sizeof(int) * f->L.n);
        memcpy(Lx, f->L.x, sizeof(double) * f->L.n);
        memcpy(Lt, f->L.t, sizeof(double) * f->L.n);
        memcpy(Le, f->L.e, sizeof(double) * f->L.n);
    }
    memcpy(Ui, f->U.i, sizeof(int) * f->U.n);
    memcpy(Ux, f->U.x, sizeof(double) * f->U.n);
    memcpy(Ut, f->U.t, sizeof(double) * f->U.n);
    memcpy(Ue, f->U.e, sizeof(double) * f->U.n);
}

/* Solve A' z = y in place: forward with unit L, then backward with U. */
void orc_lu_solve(const orc_lu *f, double *y) {
    int n = f->n;
    for (int j = 0; j < n; j++) {
        double yj = y[j];
        for (int p = f->Lp[j]; p < f->Lp[j + 1]; p++) y[f->L.i[p]] -= f->L.x[p] * yj;
    }
    for (int j = n - 1; j >= 0; j--) {
        int d = f->Up[j + 1] - 1;               /* diagonal is last */
        y[j] /= f->U.x[d];
        double yj = y[j];
        for (int p = f->Up[j]; p < d; p++) y[f->U.i[p]] -= f->U.x[p] * yj;
    }
}

/* Solve A'^T z = y in place: A'^T = U^T L^T, U^T lower (forward), L^T unit upper (backward). */
void orc_lu_solve_t(const orc_lu *f, double *y) {
    int n = f->n;
    for (int j = 0; j < n; j++) {
        int d = f->Up[j + 1] - 1;
        double s = y[j];
        for (int p = f->Up[j]; p < d; p++) s -= f->U.x[p] * y[f->U.i[p]];
        y[j] = s / f->U.x[d];
    }
    for (int j = n - 1; j >= 0; j--) {
        double s = y[j];
        for (int p = f->Lp[j]; p < f->Lp[j + 1]; p++) s -= f->L.x[p] * y[f->L.i[p]];
        y[j] = s;
    }
}

/* Levels from the U pattern (definition in the header). lev, levu: int[n]. */
int orc_lu_levels(const orc_lu *f, int *lev, int *levu) {
    int n = f->n;
    for (int j = 0; j < n; j++) {
        int d = f->Up[j + 1] - 1, m = -1;
        for (int p = f->Up[j]; p < d; p++) if (lev[f->U.i[p]] > m) m = lev[f->U.i[p]];
        lev[j] = m + 1;
    }
    /* rows of U: entries (i, j) with i < j live in column j; row i needs max over those j */
    for (int i = 0; i < n; i++) levu[i] = 0;
    /* process columns from the right: when row i is finished, all U(i, j>i) were seen */
    int *best = (int *)malloc(sizeof(int) * (size_t)n);
    if (!best) return -1;
    for (int i = 0; i < n; i++) best[i] = -1;
    for (int j = n - 1; j >= 0; j--) {
        levu[j] = best[j] + 1;           /* all j' > j already processed */
        int d = f->Up[j + 1] - 1;
        for (int p = f->Up[j]; p < d; p++) {
            int i = f->U.i[p];
            if (levu[j] > best[i]) best[i] = levu[j];
        }
    }
    free(best);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* residual rho = b - A x (A in CSR, FP64), and infinity norms.            */
void orc_residual(int n, const int *rp, const int *ci, const double *ax, const double *b,
                  const double *x, double *rho) {
    for (int i = 0; i < n; i++) {
        double s = b[i];
        for (int p = rp[i]; p < rp[i + 1]; p++) s -= ax[p] * x[ci[p]];
        rho[i] = s;
    }
}

double orc_norm_inf_matrix(int n, const int *rp, const double *ax) {
    double m = 0.0;
    for (int i = 0; i < n; i++) {
        double s = 0.0;
        for (int p = rp[i]; p < rp[i + 1]; p++) s += fabs(ax[p]);
        if (s > m) m = s;
    }
    return m;
}

/* ------------------------------------------------------------------------ */
/* power-of-two symmetric equilibration (reading in the header)             */
static int floor_half(int e) { return e >= 0 ? e / 2 : -((1 - e) / 2); }

void orc_equilibrate(int n, const int *rp, const double *ax, double *s) {
    for (int i = 0; i < n; i++) {
        double r = 0.0;
        int bad = 0;
        for (int p = rp[i]; p < rp[i + 1]; p++) {
            double a = fabs(ax[p]);
            if (!isfinite(a)) bad = 1;
            if (a > r) r = a;
        }
        if (bad || r == 0.0) { s[i] = 1.0; continue; }
        s[i] = ldexp(1.0, -floor_half(ilogb(r)));
    }
}

/* ------------------------------------------------------------------------ */
/* Textbook minimum degree on the explicit elimination graph (used only to  */
/* produce test permutations independently of the library's ordering).      */
/* Input: symmetric pattern without the diagonal requirement (CSR).          */
/* At every step the uneliminated vertex of least current degree (smallest   */
/* index on ties) is eliminated and its neighbours are made a clique.        */
typedef struct { int deg, v; } heap_item;
static void heap_push(heap_item *h, long *hn, heap_item it) {
    long i = (*hn)++;
    h[i] = it;
    while (i > 0) {
        long p = (i - 1) / 2;
        if (h[p].deg < h[i].deg || (h[p].deg == h[i].deg && h[p].v <= h[i].v)) break;
        heap_item tmp = h[p]; h[p] = h[i]; h[i] = tmp; i = p;
    }
}
static heap_item heap_pop(heap_item *h, long *hn) {
    heap_item top = h[0];
    h[0] = h[--(*hn)];
    long i = 0;
    for (;;) {
        long l = 2 * i + 1, r = l + 1, m = i;
        if (l < *hn && (h[l].deg < h[m].deg || (h[l].deg == h[m].deg && h[l].v < h[m].v))) m = l;
        if (r < *hn && (h[r].deg < h[m].deg || (h[r].deg == h[m].deg && h[r].v < h[m].v))) m = r;
        if (m == i) break;
        heap_item tmp = h[m]; h[m] = h[i]; h[i] = tmp; i = m;
    }
    return top;
}

int orc_min_degree(int n, const int *rp, const int *ci, int *perm) {
    int **adj = (int **)calloc((size_t)n, sizeof(int *));
    int *deg = (int *)calloc((size_t)n, sizeof(int));
    int *cap = (int *)calloc((size_t)n, sizeof(int));
    char *gone = (char *)calloc((size_t)n, 1);
    int *mark = (int *)malloc(sizeof(int) * (size_t)n);
    int *buf = (int *)malloc(sizeof(int) * (size_t)n);
    long hcap = 4L * n + 16, hn = 0;
    heap_item *h = (heap_item *)malloc(sizeof(heap_item) * hcap);
    int rc = -1;
    if (!adj || !deg || !cap || !gone || !mark || !buf || !h) goto out;
    for (int i = 0; i < n; i++) {
        mark[i] = -1;
        int c = rp[i + 1] - rp[i];
        adj[i] = (int *)malloc(sizeof(int) * (size_t)(c > 0 ? c : 1));
        if (!adj[i]) goto out;
        cap[i] = c > 0 ? c : 1;
        int m = 0;
        for (int p = rp[i]; p < rp[i + 1]; p++) if (ci[p] != i) adj[i][m++] = ci[p];
        deg[i] = m;
        heap_push(h, &hn, (heap_item){m, i});
    }
    for (int k = 0; k < n; k++) {
        heap_item it;
        do { it = heap_pop(h, &hn); } while (gone[it.v] || it.deg != deg[it.v]);
        int v = it.v;
        perm[k] = v;
        gone[v] = 1;
        /* live neighbours of v */
        int nv = 0;
        for (int q = 0; q < deg[v]; q++) if (!gone[adj[v][q]]) buf[nv++] = adj[v][q];
        for (int q = 0; q < nv; q++) mark[buf[q]] = k;
        /* each neighbour u: adj(u) = (adj(u) u N(v)) \ {u, v}, eliminated vertices dropped */
        for (int q = 0; q < nv; q++) {
            int u = buf[q];
            int m = 0;
            /* keep live old neighbours that are not in N(v) (those are re-added below) */
            for (int r = 0; r < deg[u]; r++) {
                int w = adj[u][r];
                if (!gone[w] && mark[w] != k) adj[u][m++] = w;
            }
            int need = m + nv - 1;
            if (need > cap[u]) {
                int nc = need * 2;
                int *na = (int *)realloc(adj[u], sizeof(int) * (size_t)nc);
                if (!na) goto out;
                adj[u] = na; cap[u] = nc;
            }
            for (int r = 0; r < nv; r++) if (buf[r] != u) adj[u][m++] = buf[r];
            deg[u] = m;
            if (hn + 1 > hcap) {
                hcap *= 2;
                heap_item *nh = (heap_item *)realloc(h, sizeof(heap_item) * hcap);
                if (!nh) goto out;
                h = nh;
            }
            heap_push(h, &hn, (heap_item){m, u});
        }
    }
    rc = 0;
out:
    if (adj) for (int i = 0; i < n; i++) free(adj[i]);
    free(adj); free(deg); free(cap); free(gone); free(mark); free(buf); free(h);
    return rc;
}
