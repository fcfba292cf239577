"""Oracle: a plain, slow CPU reference for fixed-pattern KKT refactorization.

TEST INFRASTRUCTURE ONLY.  The product library never imports this package;
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA library.

What it computes (arXiv 2306.14337):
  * Sec. 2 (Eq. 4): every K_k of a run shares one sparsity pattern.
  * Sec. 4 / Sec. 5.1 / Sec. 5.2: analyse once (fill-reducing symmetric
    ordering of A + A^T, Sec. 5.2), then for each value set a numeric LU with
    the same pivot sequence, followed by triangular solves.
  * Sec. 5.1: iterative refinement rho = r - K dx, K delta = rho,
    dx <- dx + delta; FGMRES with the LU factors as a right preconditioner
    and CGS2 orthogonalization as the alternative; tolerance 1e-14 and at most
    20 iterations (Sec. 5.3).

Numbers are float64 throughout.  The numeric kernel is ``oracle.c``
(Gilbert-Peierls left-looking LU).  The ordering used by parity tests comes
from the textbook minimum-degree routine in ``oracle.c`` (not from the
library), so the oracle never takes an input from the product path.

Readings of points the paper leaves open are stated in ``oracle.c``'s header
and next to each function below.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with gcc into ``oracle/_build/liboracle.so``."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_lu_factor.restype = C.c_void_p
            L.orc_lu_factor.argtypes = [C.c_int, _ip, _ip, _dp, C.c_double]
            L.orc_lu_free.argtypes = [C.c_void_p]
            for f in ("orc_lu_nnz_l", "orc_lu_nnz_u"):
                getattr(L, f).restype = C.c_long
                getattr(L, f).argtypes = [C.c_void_p]
            L.orc_lu_n_perturbed.restype = C.c_int
            L.orc_lu_n_perturbed.argtypes = [C.c_void_p]
            L.orc_lu_tau.restype = C.c_double
            L.orc_lu_tau.argtypes = [C.c_void_p]
            L.orc_lu_export.argtypes = [C.c_void_p, _ip, _ip, _dp, _dp, _dp, _ip, _ip, _dp, _dp, _dp]
            L.orc_lu_solve.argtypes = [C.c_void_p, _dp]
            L.orc_lu_solve_t.argtypes = [C.c_void_p, _dp]
            L.orc_lu_levels.restype = C.c_int
            L.orc_lu_levels.argtypes = [C.c_void_p, _ip, _ip]
            L.orc_residual.argtypes = [C.c_int, _ip, _ip, _dp, _dp, _dp, _dp]
            L.orc_norm_inf_matrix.restype = C.c_double
            L.orc_norm_inf_matrix.argtypes = [C.c_int, _ip, _dp]
            L.orc_equilibrate.argtypes = [C.c_int, _ip, _dp, _dp]
            L.orc_min_degree.restype = C.c_int
            L.orc_min_degree.argtypes = [C.c_int, _ip, _ip, _ip]
            _lib = L
    return _lib


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# Pattern helpers (Sec. 5.2: the ordering is computed on A + A^T)

def symmetrized_pattern(n, indptr, indices):
    """Pattern of A + A^T + I as CSR (int32, sorted, unique), via SciPy."""
    P = sp.csr_matrix((np.ones(len(indices), dtype=np.int8), _i32(indices), _i32(indptr)),
                      shape=(n, n))
    S = (P + P.T + sp.identity(n, dtype=np.int8, format="csr")).tocsr()
    S.sort_indices()
    return _i32(S.indptr), _i32(S.indices)


def min_degree(n, indptr, indices):
    """Permutation (new -> old) from textbook minimum degree on A + A^T.

    Used by the tests to hand the same ordering to the oracle and the library.
    """
    rp, ci = symmetrized_pattern(n, indptr, indices)
    perm = np.zeros(n, dtype=np.int32)
    if lib().orc_min_degree(n, rp, ci, perm) != 0:
        raise MemoryError("orc_min_degree")
    return perm


def max_product_matching(n, indptr, indices, values):
    """Row permutation q of a perfect matching of the nonzeros of A that
    maximizes prod_j |a_{q[j], j}| (row j of Q A is row q[j] of A): the
    weighted bipartite matching MC64 computes, which the paper's Ginkgo path
    applies before the ordering (Sec. 5.2).  Plain definition: minimize
    sum_j c(q[j], j) with c(i, j) = log max_k |a_kj| - log |a_ij| over the
    nonzeros, solved by SciPy's min_weight_full_bipartite_matching as the step
    (costs shifted by 1, which adds n to every perfect matching).  Raises
    ValueError when A has no perfect matching."""
    from scipy.sparse.csgraph import min_weight_full_bipartite_matching
    A = sp.csr_matrix((np.array(values, dtype=np.float64), np.array(indices, dtype=np.int32),
                       np.array(indptr, dtype=np.int32)), shape=(n, n))    # copies: the caller's arrays stay as they are
    A.eliminate_zeros()
    Ac = abs(A).tocsc()
    colmax = np.zeros(n)
    for j in range(n):
        seg = Ac.data[Ac.indptr[j]:Ac.indptr[j + 1]]
        colmax[j] = seg.max() if seg.size else 0.0
    C = Ac.copy()
    C.data = np.log(np.repeat(colmax, np.diff(Ac.indptr))) - np.log(Ac.data) + 1.0
    r, c = min_weight_full_bipartite_matching(C.tocsr())
    q = np.empty(n, dtype=np.int32)
    q[c] = r
    return q


def row_permuted(n, indptr, indices, values, q):
    """Q A as CSR (row j = row q[j] of A), values in the new row order."""
    A = sp.csr_matrix((_f64(values), _i32(indices), _i32(indptr)), shape=(n, n))
    B = A[np.asarray(q), :].tocsr()
    B.sort_indices()
    return _i32(B.indptr), _i32(B.indices), _f64(B.data)


def equilibrate(n, indptr, values):
    """Power-of-two symmetric scaling s (reading: s_i = 2^-floor(floor(log2 r_i)/2),
    r_i = max_j |a_ij|); s_i = 1 for a zero or non-finite row."""
    s = np.zeros(n)
    lib().orc_equilibrate(n, _i32(indptr), _f64(values), s)
    return s


def permuted_matrix(n, indptr, indices, values, perm, s):
    """A' = S P A_sym P^T S as CSC with structural zeros kept.

    perm[i'] = original index of permuted index i'.  A'[i', j'] =
    s[perm[i']] * A[perm[i'], perm[j']] * s[perm[j']]; entries of A + A^T + I
    that A does not store are explicit zeros.
    """
    indptr = _i32(indptr); indices = _i32(indices); values = _f64(values)
    perm = _i32(perm)
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    rows = np.repeat(np.arange(n), np.diff(indptr))
    srp, sci = symmetrized_pattern(n, indptr, indices)
    srows = np.repeat(np.arange(n), np.diff(srp))
    # value of every symmetrized slot: user value if stored, else 0
    ukey = rows.astype(np.int64) * n + indices
    skey = srows.astype(np.int64) * n + sci
    pos = np.searchsorted(ukey, skey)
    pos_c = np.minimum(pos, len(ukey) - 1)
    hit = (pos < len(ukey)) & (ukey[pos_c] == skey)
    sval = np.zeros(len(skey))
    sval[hit] = values[pos_c[hit]] * s[srows[hit]] * s[sci[hit]]
    pr = iperm[srows]
    pc = iperm[sci]
    order = np.lexsort((pr, pc))           # column-major, rows ascending
    pr, pc, sval = pr[order], pc[order], sval[order]
    colptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(colptr, pc + 1, 1)
    colptr = np.cumsum(colptr)
    return _i32(colptr), _i32(pr), _f64(sval)


# --------------------------------------------------------------------------

class Factor:
    """LU of A' (Doolittle, unit L, diagonal pivots) from ``oracle.c``."""

    def __init__(self, n, colptr, rowidx, vals, tau_rel):
        self.n = n
        L = lib()
        self._h = L.orc_lu_factor(n, _i32(colptr), _i32(rowidx), _f64(vals), float(tau_rel))
        if not self._h:
            raise MemoryError("orc_lu_factor")
        nl, nu = L.orc_lu_nnz_l(self._h), L.orc_lu_nnz_u(self._h)
        self.Lp = np.zeros(n + 1, np.int32); self.Li = np.zeros(max(nl, 1), np.int32)
        self.Lx = np.zeros(max(nl, 1)); self.Lt = np.zeros(max(nl, 1)); self.Le = np.zeros(max(nl, 1))
        self.Up = np.zeros(n + 1, np.int32); self.Ui = np.zeros(nu, np.int32)
        self.Ux = np.zeros(nu); self.Ut = np.zeros(nu); self.Ue = np.zeros(nu)
        L.orc_lu_export(self._h, self.Lp, self.Li, self.Lx, self.Lt, self.Le,
                        self.Up, self.Ui, self.Ux, self.Ut, self.Ue)
        self.Li, self.Lx, self.Lt, self.Le = self.Li[:nl], self.Lx[:nl], self.Lt[:nl], self.Le[:nl]
        self.n_perturbed = L.orc_lu_n_perturbed(self._h)
        self.tau = L.orc_lu_tau(self._h)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_lu_free(self._h)
            self._h = None

    @property
    def nnz(self):
        """Stored entries of combined L+U (diagonal once)."""
        return int(self.Lp[-1] + self.Up[-1])

    def levels(self):
        """(lev, levu): column levels of the refactorization / forward solve and
        backward levels of the U solve (definitions in oracle.c)."""
        lev = np.zeros(self.n, np.int32); levu = np.zeros(self.n, np.int32)
        if lib().orc_lu_levels(self._h, lev, levu) != 0:
            raise MemoryError
        return lev, levu

    def solve(self, y):
        y = _f64(y).copy()
        lib().orc_lu_solve(self._h, y)
        return y

    def solve_t(self, y):
        y = _f64(y).copy()
        lib().orc_lu_solve_t(self._h, y)
        return y

    def jacobi_solve(self, y, sweeps):
        """Approximate U^-1 L^-1 y by Jacobi sweeps on each triangular factor
        (Sec. 6: iterative approximation of the triangular solves, the method
        of Anzt, Chow and Dongarra 2015).  With L = I + L_s (L_s strictly
        lower) and U = D + U_s (D its diagonal, U_s strictly upper):
            w_0 = y,        w_{k+1} = y - L_s w_k,            k < sweeps,
            z_0 = D^-1 w,   z_{k+1} = D^-1 (w - U_s z_k),     k < sweeps.
        Each sweep is one sparse product, with no dependency between rows.
        Since L_s and D^-1 U_s are nilpotent, the result is the exact solve
        once sweeps + 1 reaches the number of levels of the factor's
        dependency graph."""
        return self._jacobi(_f64(y), sweeps, transpose=False)

    def jacobi_solve_t(self, y, sweeps):
        """The same for A'^T = U^T L^T: Jacobi sweeps on U^T = D + U_s^T, then on
        L^T = I + L_s^T."""
        return self._jacobi(_f64(y), sweeps, transpose=True)

    def _jacobi(self, y, sweeps, transpose):
        L = self.L_csc().tocsr()
        U = self.U_csc()
        D = U.diagonal()
        Us = sp.triu(U, 1, format="csr")
        if not transpose:
            w = y.copy()
            for _ in range(sweeps):
                w = y - L @ w
            z = w / D
            for _ in range(sweeps):
                z = (w - Us @ z) / D
            return z
        UsT = Us.T.tocsr()
        LT = L.T.tocsr()
        w = y / D
        for _ in range(sweeps):
            w = (y - UsT @ w) / D
        z = w.copy()
        for _ in range(sweeps):
            z = w - LT @ z
        return z

    def L_csc(self):
        return sp.csc_matrix((self.Lx, self.Li, self.Lp), shape=(self.n, self.n))

    def U_csc(self):
        return sp.csc_matrix((self.Ux, self.Ui, self.Up), shape=(self.n, self.n))

    def lu_csr(self):
        """Combined L+U row by row: (row_ptr, col_idx, values, error bounds),
        L strictly below the diagonal, U on and above it, columns ascending."""
        n = self.n
        lcol = np.repeat(np.arange(n), np.diff(self.Lp))
        ucol = np.repeat(np.arange(n), np.diff(self.Up))
        rows = np.concatenate([self.Li, self.Ui]).astype(np.int64)
        cols = np.concatenate([lcol, ucol]).astype(np.int64)
        vals = np.concatenate([self.Lx, self.Ux])
        errs = np.concatenate([self.Le, self.Ue])
        order = np.argsort(rows * n + cols, kind="stable")
        rp = np.zeros(n + 1, dtype=np.int64)
        np.add.at(rp, rows + 1, 1)
        return _i32(np.cumsum(rp)), _i32(cols[order]), vals[order], errs[order]

    def lu_pattern_csr(self):
        """Combined L+U pattern as CSR (row-wise), the layout used for
        comparisons with the library's analysis."""
        M = (sp.csc_matrix((np.ones_like(self.Lx), self.Li, self.Lp), shape=(self.n, self.n))
             + sp.csc_matrix((np.ones_like(self.Ux), self.Ui, self.Up), shape=(self.n, self.n))).tocsr()
        M.sort_indices()
        return _i32(M.indptr), _i32(M.indices)


def omega(n, indptr, indices, values, b, x, anorm=None):
    """Scaled residual ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf), FP64,
    on the original (unscaled, unpermuted) A."""
    rho = residual(n, indptr, indices, values, b, x)
    if anorm is None:
        anorm = lib().orc_norm_inf_matrix(n, _i32(indptr), _f64(values))
    den = anorm * np.max(np.abs(x), initial=0.0) + np.max(np.abs(b), initial=0.0)
    return float(np.max(np.abs(rho), initial=0.0) / den) if den > 0 else 0.0


def residual(n, indptr, indices, values, b, x):
    rho = np.zeros(n)
    lib().orc_residual(n, _i32(indptr), _i32(indices), _f64(values), _f64(b), _f64(x), rho)
    return rho


class Oracle:
    """Full reference pipeline for one value set on a fixed pattern.

    perm: new -> old permutation (required; the ordering is not a parity
    matter).  equilibrate: apply the power-of-two scaling.  tau_rel: pivot
    perturbation threshold relative to max|A'|.
    """

    def __init__(self, n, indptr, indices, values, perm, equil=True, tau_rel=1e-14,
                 factor_values=None):
        self.n = n
        self.indptr, self.indices, self.values = _i32(indptr), _i32(indices), _f64(values)
        self.perm = _i32(perm)
        if sorted(self.perm.tolist()) != list(range(n)):
            raise ValueError("perm is not a permutation")
        # factor_values: factor a different value set (a preconditioner for
        # refinement tests); residuals always use ``values``.
        fv = self.values if factor_values is None else _f64(factor_values)
        self.s = equilibrate(n, self.indptr, fv) if equil else np.ones(n)
        cp, ri, vx = permuted_matrix(n, self.indptr, self.indices, fv, self.perm, self.s)
        self.Ap = (cp, ri, vx)
        self.F = Factor(n, cp, ri, vx, tau_rel)
        self.anorm = lib().orc_norm_inf_matrix(n, self.indptr, self.values)

    # Solve A x = b: b' = S P b; A' z = b'; x = S P^T z (Sec. 5.2: permute and
    # scale the right-hand side and the solution).
    def solve(self, b):
        sp_ = self.s[self.perm]
        z = self.F.solve(sp_ * _f64(b)[self.perm])
        x = np.empty(self.n)
        x[self.perm] = sp_ * z
        return x

    # Solve A^T lam = g with the same factors: A'^T = U^T L^T.
    def solve_t(self, g):
        sp_ = self.s[self.perm]
        z = self.F.solve_t(sp_ * _f64(g)[self.perm])
        lam = np.empty(self.n)
        lam[self.perm] = sp_ * z
        return lam

    # Jacobi-sweep approximation of solve() (Sec. 6), same permutation and scaling.
    def solve_jacobi(self, b, sweeps):
        sp_ = self.s[self.perm]
        z = self.F.jacobi_solve(sp_ * _f64(b)[self.perm], sweeps)
        x = np.empty(self.n)
        x[self.perm] = sp_ * z
        return x

    def omega(self, b, x):
        return omega(self.n, self.indptr, self.indices, self.values, b, x, self.anorm)

    def refine(self, b, x0=None, tol=1e-14, max_it=20, mode="auto", restart=20, sweeps=0):
        """Iterative refinement (Sec. 5.1) to omega <= tol with at most max_it
        solves with the factors.

        mode "classic": x <- x + solve(b - A x) until converged.
        mode "fgmres": FGMRES(restart) right-preconditioned by the LU solve,
        CGS2 orthogonalization (Sec. 5.1).
        mode "auto" (reading): classic, switching to FGMRES for the remaining
        budget once an iteration fails to halve omega.
        mode "fgmres_jacobi": FGMRES(restart) whose preconditioner applies
        ``sweeps`` Jacobi sweeps per triangular factor instead of the exact
        solves (Sec. 6); FGMRES allows a preconditioner that is not an exact
        inverse (Saad 1993).
        Returns (x, iterations, omega history, converged).
        """
        b = _f64(b)
        x = np.zeros(self.n) if x0 is None else _f64(x0).copy()
        hist = []
        it = 0
        w = self.omega(b, x)
        hist.append(w)
        if mode in ("classic", "auto"):
            while w > tol and it < max_it:
                rho = residual(self.n, self.indptr, self.indices, self.values, b, x)
                x = x + self.solve(rho)
                it += 1
                w_new = self.omega(b, x)
                hist.append(w_new)
                stalled = not (w_new <= 0.5 * w)
                w = w_new
                if mode == "auto" and stalled and w > tol:
                    break
        if w > tol and it < max_it and mode in ("fgmres", "auto", "fgmres_jacobi"):
            prec = (lambda v: self.solve_jacobi(v, sweeps)) if mode == "fgmres_jacobi" else self.solve
            while w > tol and it < max_it:
                m = min(restart, max_it - it)
                x, used = self._fgmres_cycle(b, x, m, tol, prec)
                it += used
                w = self.omega(b, x)
                hist.append(w)
                if used == 0:
                    break
        return x, it, hist, w <= tol

    def _fgmres_cycle(self, b, x0, m, tol, prec=None):
        """One FGMRES(m) cycle (Saad 1993), right preconditioner M^-1 = LU solve
        (or ``prec``), CGS2 (classical Gram-Schmidt applied twice).  Stops early
        when the least-squares residual estimate meets the scaled tolerance.
        Returns (x, preconditioner applications)."""
        prec = self.solve if prec is None else prec
        n = self.n
        r0 = residual(n, self.indptr, self.indices, self.values, b, x0)
        beta = np.linalg.norm(r0)
        if beta == 0.0:
            return x0, 0
        A = sp.csr_matrix((self.values, self.indices, self.indptr), shape=(n, n))
        V = np.zeros((m + 1, n)); Z = np.zeros((m, n)); H = np.zeros((m + 1, m))
        V[0] = r0 / beta
        cs = np.zeros(m); sn = np.zeros(m)
        gvec = np.zeros(m + 1); gvec[0] = beta
        bn = np.max(np.abs(b))
        k_used = 0
        for j in range(m):
            Z[j] = prec(V[j])
            w = A @ Z[j]
            h1 = V[: j + 1] @ w
            w = w - V[: j + 1].T @ h1
            h2 = V[: j + 1] @ w
            w = w - V[: j + 1].T @ h2
            H[: j + 1, j] = h1 + h2
            hnext = np.linalg.norm(w)
            H[j + 1, j] = hnext
            if hnext != 0.0:
                V[j + 1] = w / hnext
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = (1.0, 0.0) if den == 0.0 else (H[j, j] / den, H[j + 1, j] / den)
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            gvec[j + 1] = -sn[j] * gvec[j]
            gvec[j] = cs[j] * gvec[j]
            k_used = j + 1
            # estimate: ||r||_2 >= ||r||_inf; stop once it meets the omega target
            xk_norm = np.max(np.abs(x0))
            if abs(gvec[j + 1]) <= tol * (self.anorm * xk_norm + bn) or hnext == 0.0:
                break
        k = k_used
        y = np.linalg.solve(np.triu(H[:k, :k]), gvec[:k]) if k else np.zeros(0)
        return x0 + Z[:k].T @ y, k

    def ldlt(self):
        """(L, D) with A' = L D L^T for symmetric values (Sec. 3 inertia; the
        MA57 form of Sec. 5.3's CPU baseline).  Plain definition: without row
        or column exchanges the Doolittle factors of a symmetric matrix satisfy
        U = D L^T with D = diag(U), so L is the unit lower factor of the LU and
        D its pivots (perturbed pivots included)."""
        return self.F.L_csc(), self.F.U_csc().diagonal().copy()

    def inertia(self):
        """(n_pos, n_neg) of A for symmetric values: the signs of the pivots D
        of A' = L D L^T.  A' = S P A P^T S is congruent to A, so by Sylvester's
        law of inertia these are the numbers of positive and negative
        eigenvalues of A (when no pivot was perturbed)."""
        _, D = self.ldlt()
        neg = int(np.sum(D < 0))
        return self.n - neg, neg

    def adjoint(self, x, g):
        """Backward of x = A^-1 b for the upstream gradient g:
        lam = A^-T g, dA_k = -lam[row_k] x[col_k] per stored entry, db = lam."""
        lam = self.solve_t(g)
        rows = np.repeat(np.arange(self.n), np.diff(self.indptr))
        return -lam[rows] * _f64(x)[self.indices], lam
