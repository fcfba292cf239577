"""Pins of the oracle against facts fixed by the mathematics (no GPU).

Each test checks the oracle against something other than itself: dense
Doolittle elimination, the Rose-Tarjan path theorem, elimination-tree
heights, SciPy's SuperLU, dense NumPy/torch solves, closed forms and finite
differences.  A dropped term, a wrong sign or index, or a transposed operand
anywhere in the oracle fails at least one of them.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
from kktgen import config_sequence, random_dd_values, random_sparse_pattern, kkt_sequence


def _random_case(n, density, seed, drop_diag=0.0):
    rp, ci = random_sparse_pattern(n, density, seed, drop_diag=drop_diag)
    v = random_dd_values(rp, ci, seed + 1)
    return rp, ci, v


def _dense_permuted(n, rp, ci, v, perm, s):
    A = sp.csr_matrix((v, ci, rp), shape=(n, n)).toarray()
    S = np.diag(s)
    Ap = (S @ A @ S)[np.ix_(perm, perm)]
    return Ap


def _dense_doolittle(A):
    """Textbook Doolittle elimination without exchanges: returns unit L and U."""
    n = A.shape[0]
    U = A.astype(np.float64).copy()
    L = np.eye(n)
    for k in range(n):
        for i in range(k + 1, n):
            L[i, k] = U[i, k] / U[k, k]
            U[i, k:] -= L[i, k] * U[k, k:]
            U[i, k] = 0.0
    return L, U


@pytest.mark.parametrize("n,density,seed", [(1, 1.0, 1), (2, 0.5, 2), (5, 0.4, 3),
                                            (17, 0.2, 4), (40, 0.08, 5), (60, 0.05, 6)])
def test_oracle_matches_dense_doolittle(n, density, seed):
    rp, ci, v = _random_case(n, density, seed)
    perm = np.random.default_rng(seed).permutation(n).astype(np.int32)
    o = oracle.Oracle(n, rp, ci, v, perm, equil=True)
    Ad = _dense_permuted(n, rp, ci, v, perm, o.s)
    Ld, Ud = _dense_doolittle(Ad)
    L = o.F.L_csc().toarray() + np.eye(n)
    U = o.F.U_csc().toarray()
    scale = max(1.0, np.abs(Ud).max())
    np.testing.assert_allclose(L, Ld, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(U, Ud, rtol=1e-13, atol=1e-13 * scale)
    assert o.F.n_perturbed == 0


def _path_theorem_fill(G):
    """Rose-Tarjan: (i, j) is in the filled pattern iff G has a path from i to
    j whose intermediate vertices are all < min(i, j)."""
    n = G.shape[0]
    F = np.zeros_like(G, dtype=bool)
    for i in range(n):
        for j in range(n):
            if i == j:
                F[i, j] = True
                continue
            lim = min(i, j)
            seen = {i}
            stack = [i]
            found = False
            while stack and not found:
                u = stack.pop()
                for w in np.nonzero(G[u])[0]:
                    if w == j:
                        found = True
                        break
                    if w < lim and w not in seen:
                        seen.add(w)
                        stack.append(w)
            F[i, j] = found
    return F


@pytest.mark.parametrize("n,density,seed", [(8, 0.25, 11), (25, 0.1, 12), (40, 0.06, 13),
                                            (60, 0.04, 14)])
def test_oracle_fill_matches_path_theorem(n, density, seed):
    rp, ci, v = _random_case(n, density, seed, drop_diag=0.2)
    perm = np.random.default_rng(seed).permutation(n).astype(np.int32)
    o = oracle.Oracle(n, rp, ci, v, perm)
    srp, sci = oracle.symmetrized_pattern(n, rp, ci)
    G = sp.csr_matrix((np.ones(len(sci)), sci, srp), shape=(n, n)).toarray() != 0
    G = G[np.ix_(perm, perm)]
    F = _path_theorem_fill(G)
    lrp, lci = o.F.lu_pattern_csr()
    P = sp.csr_matrix((np.ones(len(lci)), lci, lrp), shape=(n, n)).toarray() != 0
    assert np.array_equal(P, F)
    assert np.array_equal(P, P.T)          # symmetric structure: struct(L) = struct(U^T)


def _etree_heights(F):
    """Elimination tree from the filled pattern: parent(j) = min{i > j : L(i,j) != 0};
    height(j) = 0 for a leaf else 1 + max child height; depth(root) = 0."""
    n = F.Lp.size - 1
    parent = -np.ones(n, dtype=np.int64)
    for j in range(n):
        rows = F.Li[F.Lp[j]:F.Lp[j + 1]]
        if rows.size:
            parent[j] = rows.min()
    height = np.zeros(n, dtype=np.int64)
    for j in range(n):            # children have smaller index
        if parent[j] >= 0:
            height[parent[j]] = max(height[parent[j]], height[j] + 1)
    depth = np.zeros(n, dtype=np.int64)
    for j in range(n - 1, -1, -1):
        if parent[j] >= 0:
            depth[j] = depth[parent[j]] + 1
    return height, depth


def _longest_paths(F):
    """Brute-force longest path into / out of each vertex of the dependency DAG
    k -> j (U(k, j) != 0, k < j), by explicit relaxation over all edges."""
    n = F.Up.size - 1
    edges = []
    for j in range(n):
        for p in range(F.Up[j], F.Up[j + 1]):
            k = F.Ui[p]
            if k != j:
                edges.append((k, j))
    into = np.zeros(n, dtype=np.int64)
    out = np.zeros(n, dtype=np.int64)
    changed = True
    while changed:
        changed = False
        for k, j in edges:
            if into[k] + 1 > into[j]:
                into[j] = into[k] + 1; changed = True
            if out[j] + 1 > out[k]:
                out[k] = out[j] + 1; changed = True
    return into, out


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_oracle_levels_equal_longest_path_and_etree(seed):
    n = 50
    rp, ci, v = _random_case(n, 0.05, seed)
    perm = np.random.default_rng(seed).permutation(n).astype(np.int32)
    o = oracle.Oracle(n, rp, ci, v, perm)
    lev, levu = o.F.levels()
    into, out = _longest_paths(o.F)
    assert np.array_equal(lev, into)
    assert np.array_equal(levu, out)
    h, d = _etree_heights(o.F)
    assert np.array_equal(lev, h)
    assert np.array_equal(levu, d)


def test_oracle_levels_etree_on_kkt():
    s = config_sequence(0)
    p = oracle.min_degree(s.n, s.indptr, s.indices)
    o = oracle.Oracle(s.n, s.indptr, s.indices, s.values(0), p)
    lev, levu = o.F.levels()
    h, d = _etree_heights(o.F)
    assert np.array_equal(lev, h) and np.array_equal(levu, d)


def test_oracle_invariant_PAPt_equals_LU():
    """Componentwise backward error of the factorization: |A' - L U| <= gamma |L||U|
    (Higham, Thm 9.3) with gamma = n_k u / (1 - n_k u), n_k = length of the
    longest inner product; checked on a KKT matrix with non-symmetric values."""
    s = config_sequence(0, asym=0.1)
    v = s.values(4)
    p = oracle.min_degree(s.n, s.indptr, s.indices)
    o = oracle.Oracle(s.n, s.indptr, s.indices, v, p)
    L = o.F.L_csc() + sp.identity(s.n, format="csc")
    U = o.F.U_csc()
    cp, ri, vx = o.Ap
    Ap = sp.csc_matrix((vx, ri, cp), shape=(s.n, s.n))
    R = abs(Ap - L @ U).toarray()
    B = (abs(L) @ abs(U)).toarray()
    u = np.finfo(float).eps / 2
    nk = s.n
    gamma = nk * u / (1 - nk * u)
    assert np.all(R <= gamma * B + 1e-300)
    # and the factors carry information: the bound is far from trivial
    assert np.abs(R).max() > 0


def test_oracle_matches_superlu_natural():
    """SciPy SuperLU with the natural column order and diagonal pivoting
    threshold 0 keeps the diagonal pivots; its L and U agree with the oracle's
    entry by entry within 1e-11 relative or, where cancellation makes that
    unattainable for any summation order, within twice the oracle's
    first-order running error bound (which this also pins from below)."""
    s = config_sequence(0, asym=0.1)
    p = oracle.min_degree(s.n, s.indptr, s.indices)
    for step in (2, 9):
        v = s.values(step)
        o = oracle.Oracle(s.n, s.indptr, s.indices, v, p)
        cp, ri, vx = o.Ap
        Ap = sp.csc_matrix((vx, ri, cp), shape=(s.n, s.n))
        lu = spla.splu(Ap, permc_spec="NATURAL", diag_pivot_thresh=0.0,
                       options=dict(SymmetricMode=True))
        assert np.array_equal(lu.perm_r, np.arange(s.n))
        assert np.array_equal(lu.perm_c, np.arange(s.n))
        F = o.F
        Ls, Us = lu.L.toarray(), lu.U.toarray()
        lcol = np.repeat(np.arange(s.n), np.diff(F.Lp))
        ucol = np.repeat(np.arange(s.n), np.diff(F.Up))
        dL = np.abs(Ls[F.Li, lcol] - F.Lx)
        dU = np.abs(Us[F.Ui, ucol] - F.Ux)
        assert np.all(dL <= np.maximum(1e-11 * np.abs(F.Lx), 2 * F.Le))
        assert np.all(dU <= np.maximum(1e-11 * np.abs(F.Ux), 2 * F.Ue))
        # nothing outside the oracle's pattern
        Lmask = np.zeros((s.n, s.n), bool); Lmask[F.Li, lcol] = True
        Umask = np.zeros((s.n, s.n), bool); Umask[F.Ui, ucol] = True
        assert np.all(Ls[~Lmask & ~np.eye(s.n, dtype=bool)] == 0)
        assert np.all(Us[~Umask] == 0)


def test_oracle_error_bound_is_not_vacuous():
    """The running bound stays at rounding level where no cancellation occurs:
    on a diagonally dominant random matrix E <= 1e-12 (|x| + t) everywhere."""
    n = 60
    rp, ci, v = _random_case(n, 0.08, 41)
    perm = np.random.default_rng(41).permutation(n).astype(np.int32)
    o = oracle.Oracle(n, rp, ci, v, perm)
    F = o.F
    assert np.all(F.Le <= 1e-12 * (np.abs(F.Lx) + F.Lt))
    assert np.all(F.Ue <= 1e-12 * (np.abs(F.Ux) + F.Ut))


def test_oracle_manufactured_solution_and_dense_solve():
    s = config_sequence(0, asym=0.05)
    k = 6
    v = s.values(k)
    A = s.csr(k)
    xt = s.x_true(k)
    b = A @ xt
    p = oracle.min_degree(s.n, s.indptr, s.indices)
    o = oracle.Oracle(s.n, s.indptr, s.indices, v, p)
    x, it, hist, ok = o.refine(b, tol=1e-14, max_it=20)
    assert ok and hist[-1] <= 1e-14 and it <= 20
    xd = np.linalg.solve(A.toarray(), b)
    # both are backward stable; forward error bounded by cond * eps
    cond = np.linalg.cond(A.toarray(), p=np.inf)
    fe = np.abs(x - xd).max() / np.abs(xd).max()
    assert fe <= max(1e3 * cond * np.finfo(float).eps, 1e-14)
    assert np.abs(x - xt).max() / np.abs(xt).max() <= max(1e3 * cond * np.finfo(float).eps, 1e-14)


def test_oracle_solve_transpose_dense():
    s = config_sequence(0, asym=0.1)
    v = s.values(1)
    A = s.csr(1).toarray()
    g = np.random.default_rng(5).standard_normal(s.n)
    p = oracle.min_degree(s.n, s.indptr, s.indices)
    o = oracle.Oracle(s.n, s.indptr, s.indices, v, p)
    lam = o.solve_t(g)
    ref = np.linalg.solve(A.T, g)
    cond = np.linalg.cond(A, p=np.inf)
    assert np.abs(lam - ref).max() / np.abs(ref).max() <= 1e3 * cond * np.finfo(float).eps
    # the transpose is really used: A^-1 g differs from A^-T g for non-symmetric values
    assert np.abs(np.linalg.solve(A, g) - ref).max() > 1e-6 * np.abs(ref).max()


def test_oracle_pivot_perturbation_closed_form():
    """3x3 with a zero first pivot: exactly one perturbation to +tau, the rest
    of the factors in closed form (Doolittle with p1 = tau)."""
    a12, a13, a21, a22, a23, a31, a32, a33 = 2.0, -1.0, 3.0, 5.0, 1.0, -2.0, 4.0, 7.0
    A = np.array([[0.0, a12, a13], [a21, a22, a23], [a31, a32, a33]])
    Asp = sp.csr_matrix(A)
    Asp.eliminate_zeros()
    # keep the structural (0,0) slot: pattern with diagonal
    rp = np.array([0, 3, 6, 9], dtype=np.int32)
    ci = np.array([0, 1, 2] * 3, dtype=np.int32)
    v = A.reshape(-1)
    tau_rel = 1e-3
    o = oracle.Oracle(3, rp, ci, v, np.arange(3, dtype=np.int32), equil=False, tau_rel=tau_rel)
    tau = tau_rel * 7.0
    assert o.F.n_perturbed == 1
    assert o.F.tau == pytest.approx(tau, rel=0, abs=0)
    l21, l31 = a21 / tau, a31 / tau
    u22 = a22 - l21 * a12
    u23 = a23 - l21 * a13
    l32 = (a32 - l31 * a12) / u22
    u33 = a33 - l31 * a13 - l32 * u23
    L = o.F.L_csc().toarray() + np.eye(3)
    U = o.F.U_csc().toarray()
    np.testing.assert_allclose(L, [[1, 0, 0], [l21, 1, 0], [l31, l32, 1]], rtol=1e-15)
    np.testing.assert_allclose(U, [[tau, a12, a13], [0, u22, u23], [0, 0, u33]], rtol=1e-13)


def test_oracle_refine_fixed_point():
    s = config_sequence(0)
    v = s.values(0)
    b = s.rhs(0)
    p = oracle.min_degree(s.n, s.indptr, s.indices)
    o = oracle.Oracle(s.n, s.indptr, s.indices, v, p)
    x, it, hist, ok = o.refine(b)
    assert ok
    x2, it2, hist2, ok2 = o.refine(b, x0=x)
    assert it2 == 0 and ok2 and np.array_equal(x2, x)


@pytest.mark.parametrize("d", [0.3, 0.5, 1.0])
def test_oracle_fgmres_finite_termination(d):
    """GMRES-type methods terminate in at most n steps in exact arithmetic
    (Saad 1993).  With a poor preconditioner (factors of a matrix whose
    entries are perturbed by d N(0,1)) the classic iteration diverges while
    FGMRES(n) meets omega <= 1e-14 within n preconditioner applications."""
    n = 30
    rp, ci = random_sparse_pattern(n, 0.15, 51)
    v = random_dd_values(rp, ci, 52, dominance=0.05)
    b = np.random.default_rng(2).standard_normal(n)
    fv = v * (1 + d * np.random.default_rng(3).standard_normal(v.size))
    o = oracle.Oracle(n, rp, ci, v, np.arange(n, dtype=np.int32), factor_values=fv)
    xf, itf, hf, okf = o.refine(b, mode="fgmres", max_it=n, restart=n)
    xc, itc, hc, okc = o.refine(b, mode="classic", max_it=n)
    assert okf and itf <= n and hf[-1] <= 1e-14
    assert not okc
    A = sp.csr_matrix((v, ci, rp), shape=(n, n)).toarray()
    np.testing.assert_allclose(xf, np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)


def test_oracle_classic_refinement_contracts_with_nearby_factors():
    """With factors of a nearby matrix (relative perturbation 1e-3) classic
    refinement converges to omega <= 1e-14, and the mode "auto" path agrees."""
    s = config_sequence(0, asym=0.05)
    p = oracle.min_degree(s.n, s.indptr, s.indices)
    v = s.values(5)
    b = s.csr(5) @ s.x_true(5)
    fv = v * (1 + 1e-3 * np.random.default_rng(1).standard_normal(v.size))
    o = oracle.Oracle(s.n, s.indptr, s.indices, v, p, factor_values=fv)
    for mode in ("classic", "auto", "fgmres"):
        x, it, h, ok = o.refine(b, mode=mode)
        assert ok and h[-1] <= 1e-14 and 2 <= it <= 20


def test_oracle_equilibration_closed_form():
    r = np.array([1.0, 3.0, 4.0, 0.25, 0.2, 0.0, np.inf, 1e-300, 6e15])
    n = r.size
    rp = np.arange(n + 1, dtype=np.int32)
    s = oracle.equilibrate(n, rp, r)
    # e = floor(log2 r) by hand: 0, 1, 2, -2, -3, -, -, -997, 52
    want = [1.0, 1.0, 0.5, 2.0, 4.0, 1.0, 1.0, 2.0 ** 499, 2.0 ** -26]
    assert list(s) == want
    # s_i^2 r_i in [1, 4) for finite non-zero rows
    ok = np.isfinite(r) & (r > 0)
    assert np.all((s[ok] ** 2 * r[ok] >= 1.0) & (s[ok] ** 2 * r[ok] < 4.0))


def test_oracle_adjoint_vs_dense_torch_autograd():
    torch = pytest.importorskip("torch")
    s = kkt_sequence(40, 52, 8, seed=77, steps=3, W=4.0, asym=0.1)
    v = s.values(1)
    b = s.rhs(1)
    g = np.random.default_rng(3).standard_normal(s.n)
    p = oracle.min_degree(s.n, s.indptr, s.indices)
    o = oracle.Oracle(s.n, s.indptr, s.indices, v, p)
    x, *_ = o.refine(b)
    dA, db = o.adjoint(x, g)
    A = torch.tensor(s.csr(1).toarray(), dtype=torch.float64, requires_grad=True)
    bt = torch.tensor(b, dtype=torch.float64, requires_grad=True)
    xt = torch.linalg.solve(A, bt)
    (xt * torch.tensor(g)).sum().backward()
    rows = np.repeat(np.arange(s.n), np.diff(s.indptr))
    gA = A.grad.numpy()[rows, s.indices]
    np.testing.assert_allclose(db, bt.grad.numpy(), rtol=1e-7, atol=1e-9 * np.abs(db).max())
    np.testing.assert_allclose(dA, gA, rtol=1e-7, atol=1e-9 * np.abs(gA).max())


def test_oracle_adjoint_finite_differences():
    s = kkt_sequence(30, 39, 6, seed=78, steps=3, W=2.0, asym=0.1)
    v = s.values(0)
    b = s.rhs(0)
    g = np.random.default_rng(4).standard_normal(s.n)
    p = oracle.min_degree(s.n, s.indptr, s.indices)

    def loss(vals, bb):
        oo = oracle.Oracle(s.n, s.indptr, s.indices, vals, p)
        x, *_ = oo.refine(bb)
        return float(g @ x)

    o = oracle.Oracle(s.n, s.indptr, s.indices, v, p)
    x, *_ = o.refine(b)
    dA, db = o.adjoint(x, g)
    rng = np.random.default_rng(9)
    for k in rng.choice(len(v), 12, replace=False):
        h = 1e-6 * max(1.0, abs(v[k]))
        vp, vm = v.copy(), v.copy()
        vp[k] += h; vm[k] -= h
        fd = (loss(vp, b) - loss(vm, b)) / (2 * h)
        assert abs(fd - dA[k]) <= 1e-5 * max(1.0, abs(dA[k]))
    for i in rng.choice(s.n, 8, replace=False):
        h = 1e-6
        bp, bm = b.copy(), b.copy()
        bp[i] += h; bm[i] -= h
        fd = (loss(v, bp) - loss(v, bm)) / (2 * h)
        assert abs(fd - db[i]) <= 1e-5 * max(1.0, abs(db[i]))


def _md_bruteforce(G):
    """Minimum degree on a dense boolean elimination graph (ties: smallest index)."""
    G = G.copy()
    n = G.shape[0]
    np.fill_diagonal(G, False)
    alive = np.ones(n, dtype=bool)
    order = []
    for _ in range(n):
        deg = np.where(alive, (G & alive[None, :]).sum(axis=1), n + 1)
        v = int(np.argmin(deg))
        order.append(v)
        nb = np.nonzero(G[v] & alive)[0]
        for a in nb:
            for c in nb:
                if a != c:
                    G[a, c] = True
        alive[v] = False
    return np.array(order)


@pytest.mark.parametrize("seed", [31, 32])
def test_oracle_min_degree_bruteforce(seed):
    n = 30
    rp, ci, _ = _random_case(n, 0.08, seed)
    srp, sci = oracle.symmetrized_pattern(n, rp, ci)
    G = sp.csr_matrix((np.ones(len(sci)), sci, srp), shape=(n, n)).toarray() != 0
    assert np.array_equal(oracle.min_degree(n, rp, ci), _md_bruteforce(G))


def test_generator_shape_and_quasidefinite():
    s = config_sequence(0)
    assert s.n == 1400 and s.nnz == 14040
    A = s.csr(9).toarray()
    assert np.array_equal(A, A.T)
    nx = s.n_x
    H = A[:nx, :nx]
    assert np.linalg.eigvalsh(H).min() > 0
    C = A[nx:, nx:]
    assert np.all(np.diag(C) < 0) and np.count_nonzero(C - np.diag(np.diag(C))) == 0
    for cfg, n in ((1, 14000), (2, 70000)):
        assert config_sequence(cfg).n == n


def test_oracle_scaled_residual_hand_computed_3x3():
    """omega = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) on a 3x3
    case worked by hand (the scaled residual of the refinement target, Sec. 5.3
    tolerance 1e-14).

        A = [[4, -1, 0], [-2, 5, 1], [0, 3, -6]], x = [1, -2, 1/2],
        b = [7, -11, -8]
        A x = [4 + 2, -2 - 10 + 1/2, -6 - 3] = [6, -23/2, -9]
        rho = b - A x = [1, 1/2, 1]               -> ||rho||_inf = 1
        row sums of |A|: 5, 8, 9                  -> ||A||_inf = 9
        ||x||_inf = 2, ||b||_inf = 11             -> omega = 1 / (18 + 11) = 1/29

    A largest-entry norm (6) would give 1/23 and a sum over all entries (22)
    1/55; a residual of the wrong sign fails the rho check.
    """
    rp = np.array([0, 2, 5, 7], dtype=np.int32)
    ci = np.array([0, 1, 0, 1, 2, 1, 2], dtype=np.int32)
    v = np.array([4.0, -1.0, -2.0, 5.0, 1.0, 3.0, -6.0])
    x = np.array([1.0, -2.0, 0.5])
    b = np.array([7.0, -11.0, -8.0])
    assert np.array_equal(oracle.residual(3, rp, ci, v, b, x), [1.0, 0.5, 1.0])
    assert oracle.lib().orc_norm_inf_matrix(3, rp, v) == 9.0
    assert oracle.omega(3, rp, ci, v, b, x) == 1.0 / 29.0
    # through the pipeline object as well (its norm is computed once per value set)
    o = oracle.Oracle(3, rp, ci, v, np.arange(3, dtype=np.int32))
    assert o.anorm == 9.0 and o.omega(b, x) == 1.0 / 29.0


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_oracle_norm_inf_matches_dense_numpy(seed):
    """||A||_inf of the oracle equals NumPy's dense matrix infinity norm (the
    maximum absolute row sum).  Integer-valued entries make every sum exact, so
    the comparison is exact; a largest-entry or all-entry mutation differs."""
    n = 80
    rp, ci = random_sparse_pattern(n, 0.06, seed)
    v = np.random.default_rng(seed).integers(-9, 10, size=ci.size).astype(np.float64)
    A = sp.csr_matrix((v, ci, rp), shape=(n, n)).toarray()
    ref = np.linalg.norm(A, np.inf)
    assert oracle.lib().orc_norm_inf_matrix(n, rp, v) == ref
    assert ref != np.abs(A).max() and ref != np.abs(A).sum()
    # and omega against its definition written with NumPy's norms
    x = np.random.default_rng(seed + 10).integers(-5, 6, size=n).astype(np.float64)
    b = np.random.default_rng(seed + 20).integers(-50, 51, size=n).astype(np.float64)
    rho = b - A @ x
    want = np.linalg.norm(rho, np.inf) / (ref * np.linalg.norm(x, np.inf) + np.linalg.norm(b, np.inf))
    assert oracle.omega(n, rp, ci, v, b, x) == want


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_oracle_inertia_matches_dense_eigenvalues(seed):
    """Sylvester's law of inertia: the pivot signs of A' = L D L^T (A' = S P A
    P^T S, congruent to A) equal the eigenvalue signs of A.  On a small KKT
    matrix (quasi-definite: n_x + ... positive, the constraint rows negative)
    and on a random symmetric indefinite matrix, against numpy.linalg.eigvalsh."""
    s = kkt_sequence(12, 16, 3, seed=seed, steps=2, W=3.0)
    A = s.csr(1)
    p = oracle.min_degree(s.n, s.indptr, s.indices)
    o = oracle.Oracle(s.n, s.indptr, s.indices, A.data, p)
    assert o.F.n_perturbed == 0
    ev = np.linalg.eigvalsh(A.toarray())
    assert o.inertia() == (int(np.sum(ev > 0)), int(np.sum(ev < 0)))
    # random symmetric indefinite with a strong diagonal of random signs
    n = 40
    rp, ci = random_sparse_pattern(n, 0.1, seed)
    M = sp.csr_matrix((np.random.default_rng(seed).standard_normal(ci.size), ci, rp), shape=(n, n))
    M = (M + M.T).tocsr()
    M.setdiag(np.random.default_rng(seed + 9).choice([-1.0, 1.0], n) * (3.0 + np.abs(M).sum(axis=1).A1))
    M = M.tocsr(); M.sort_indices()
    perm = np.random.default_rng(seed).permutation(n).astype(np.int32)
    o = oracle.Oracle(n, M.indptr, M.indices, M.data, perm)
    ev = np.linalg.eigvalsh(M.toarray())
    assert o.inertia() == (int(np.sum(ev > 0)), int(np.sum(ev < 0)))


def test_oracle_ldlt_is_lu_of_symmetric_matrix():
    """For symmetric A', U = D L^T: every U entry equals the pivot times the
    mirrored L entry, to rounding (bounded by the oracle's running error
    bounds of both entries), on the 200-bus KKT (n = 1,400)."""
    s = config_sequence(0)
    k = 9
    A = s.csr(k)
    p = oracle.min_degree(s.n, s.indptr, s.indices)
    o = oracle.Oracle(s.n, s.indptr, s.indices, A.data, p)
    L, D = o.ldlt()
    U = o.F.U_csc().tocsr()
    Lt = L.T.tocsr()
    Ue = sp.csr_matrix((o.F.Ue, o.F.Ui, o.F.Up), shape=(s.n, s.n)).tocsc().T.tocsc().T  # same layout as U
    DLt = sp.diags(D) @ Lt
    diff = abs(sp.triu(U, 1) - sp.triu(DLt, 1))
    Ub = sp.csc_matrix((o.F.Ue, o.F.Ui, o.F.Up), shape=(s.n, s.n))
    Lb = sp.csc_matrix((o.F.Le, o.F.Li, o.F.Lp), shape=(s.n, s.n))
    bound = sp.triu(Ub, 1) + sp.diags(np.abs(D)) @ Lb.T.tocsr() + sp.diags(Ub.diagonal()) @ abs(Lt)
    d = diff.toarray(); bnd = 4 * bound.toarray()
    assert np.all(d <= bnd + 1e-300)


def _dense_ldlt(A):
    """Textbook LDL^T without pivoting: d_j = a_jj - sum_k l_jk^2 d_k,
    l_ij = (a_ij - sum_k l_ik l_jk d_k) / d_j."""
    n = A.shape[0]
    L = np.eye(n)
    d = np.zeros(n)
    for j in range(n):
        d[j] = A[j, j] - np.sum(L[j, :j] ** 2 * d[:j])
        for i in range(j + 1, n):
            L[i, j] = (A[i, j] - np.sum(L[i, :j] * L[j, :j] * d[:j])) / d[j]
    return L, d


@pytest.mark.parametrize("seed", [4, 5])
def test_oracle_ldlt_matches_dense_textbook_ldlt(seed):
    """The oracle's (L, D) against the textbook dense LDL^T of A' = S P A P^T S
    on a small KKT matrix (D_x, D_s within [0.1, 10]).  Both compute the same
    sums in different orders; each entry differs from the exact one by at most
    the oracle's running error bound E of that entry (first order, any
    summation order), so they agree within 2 E (the -1e-8 regularization block
    still cancels several digits in the last pivots)."""
    s = kkt_sequence(10, 13, 2, seed=seed, steps=2, W=1.0)
    A = s.csr(1)
    p = oracle.min_degree(s.n, s.indptr, s.indices)
    o = oracle.Oracle(s.n, s.indptr, s.indices, A.data, p)
    Ap = oracle.permuted_matrix(s.n, s.indptr, s.indices, A.data, p, o.s)
    Apd = sp.csc_matrix((Ap[2], Ap[1], Ap[0]), shape=(s.n, s.n)).toarray()
    Lr, dr = _dense_ldlt(Apd)
    L, D = o.ldlt()
    Ue = sp.csc_matrix((o.F.Ue, o.F.Ui, o.F.Up), shape=(s.n, s.n)).diagonal()
    Le = sp.csc_matrix((o.F.Le, o.F.Li, o.F.Lp), shape=(s.n, s.n)).toarray()
    assert np.all(np.abs(D - dr) <= 2 * Ue + 1e-15 * np.abs(dr))
    assert np.all(np.abs(L.toarray() + np.eye(s.n) - Lr) <= 2 * Le + 1e-15 * np.abs(Lr))


def test_oracle_jacobi_sweeps_exact_at_level_count():
    """L_s and D^-1 U_s are nilpotent: with m nodes on the longest dependency
    chain (m = max level + 1), (L_s)^m = 0, so m - 1 = max level sweeps give
    the exact triangular solves (to rounding); three sweeps fewer leave a visible
    error.  Checked for A' and A'^T against the oracle's own substitution
    solves (the levels are pinned against brute-force longest paths above)."""
    s = kkt_sequence(15, 20, 3, seed=7, steps=2, W=2.0)
    A = s.csr(1)
    p = oracle.min_degree(s.n, s.indptr, s.indices)
    o = oracle.Oracle(s.n, s.indptr, s.indices, A.data, p)
    lev, levu = o.F.levels()
    y = np.random.default_rng(1).standard_normal(s.n)
    ref, reft = o.F.solve(y), o.F.solve_t(y)
    # the L (forward) and U (backward) chains have the same length on A + A^T
    k = int(max(lev.max(), levu.max()))
    for fn, r in ((o.F.jacobi_solve, ref), (o.F.jacobi_solve_t, reft)):
        assert np.abs(fn(y, k) - r).max() <= 1e-9 * np.abs(r).max()
        assert np.abs(fn(y, k - 3) - r).max() > 1e-7 * np.abs(r).max()


def test_oracle_jacobi_closed_form_2x2():
    """A = [[2, 1], [4, 5]] (natural order, no scaling): L = [[1, 0], [2, 1]],
    U = [[2, 1], [0, 3]].  For y = (1, 1): w_0 = y, w_1 = (1, 1 - 2) = (1, -1);
    z_0 = D^-1 w = (1/2, -1/3), z_1 = ((1 - (-1/3)) / 2, -1/3) = (2/3, -1/3),
    the exact A^-1 y.  With 0 sweeps: (1/2, 1/3)."""
    rp = np.array([0, 2, 4], np.int32)
    ci = np.array([0, 1, 0, 1], np.int32)
    o = oracle.Oracle(2, rp, ci, np.array([2.0, 1.0, 4.0, 5.0]), np.arange(2, dtype=np.int32), equil=False)
    y = np.array([1.0, 1.0])
    np.testing.assert_allclose(o.F.jacobi_solve(y, 1), [2 / 3, -1 / 3], rtol=1e-15)
    np.testing.assert_allclose(o.F.jacobi_solve(y, 0), [1 / 2, 1 / 3], rtol=1e-15)
    np.testing.assert_allclose(o.F.jacobi_solve_t(y, 1), np.linalg.solve(np.array([[2.0, 1], [4, 5]]).T, y),
                               rtol=1e-15)


def test_oracle_fgmres_with_jacobi_preconditioner_converges():
    """FGMRES with a Jacobi-sweep preconditioner reaches omega <= 1e-14 on a
    well-conditioned system (diagonally dominant, so the sweeps contract);
    with 0 sweeps it needs more preconditioner applications than with 4."""
    n = 200
    rp, ci = random_sparse_pattern(n, 0.03, 61)
    v = random_dd_values(rp, ci, 62, dominance=1.0)
    b = np.random.default_rng(63).standard_normal(n)
    o = oracle.Oracle(n, rp, ci, v, oracle.min_degree(n, rp, ci))
    x4, it4, h4, ok4 = o.refine(b, mode="fgmres_jacobi", sweeps=4, max_it=60)
    x0, it0, h0, ok0 = o.refine(b, mode="fgmres_jacobi", sweeps=0, max_it=60)
    assert ok4 and ok0 and it4 < it0
    A = sp.csr_matrix((v, ci, rp), shape=(n, n)).toarray()
    np.testing.assert_allclose(x4, np.linalg.solve(A, b), rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_oracle_matching_is_the_max_product_permutation(seed):
    """Brute force over all n! row permutations (n = 6): the oracle's matching
    attains the largest |product| of a diagonal of Q A."""
    import itertools
    n = 6
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n)) * (rng.random((n, n)) < 0.5)
    M[np.arange(n), rng.permutation(n)] = 1.0 + rng.random(n)     # a perfect matching exists
    A = sp.csr_matrix(M)
    q = oracle.max_product_matching(n, A.indptr, A.indices, A.data)
    best = max(abs(np.prod([M[p[j], j] for j in range(n)])) for p in itertools.permutations(range(n)))
    got = abs(np.prod([M[q[j], j] for j in range(n)]))
    assert got == pytest.approx(best, rel=1e-12) and best > 0
    rp, ci, v = oracle.row_permuted(n, A.indptr, A.indices, A.data, q)
    assert np.array_equal(sp.csr_matrix((v, ci, rp), shape=(n, n)).toarray(), M[q, :])


def test_library_matching_reaches_the_oracle_optimum():
    """The library's own matching (kkt_analyze_values, host-only analysis)
    attains the same optimal sum of log |a| as the oracle's on random sparse
    matrices and on a KKT matrix with a zero equality block (no -1e-8
    regularization), and gives Q A a nonzero diagonal."""
    from paper_2306_14337_gb300 import KKTSolver
    cases = []
    for seed in (5, 6):
        rp, ci = random_sparse_pattern(300, 0.02, seed)
        cases.append((300, rp, ci, np.random.default_rng(seed).standard_normal(ci.size)))
    s = kkt_sequence(60, 78, 12, seed=3, steps=2, W=4.0, reg=0.0)
    cases.append((s.n, s.indptr, s.indices, s.values(1)))
    for n, rp, ci, v in cases:
        S = KKTSolver(n, rp, ci, values=v, device=None)
        q = S.export_row_perm()
        rp0, ci0, v0 = rp.copy(), ci.copy(), v.copy()
        qo = oracle.max_product_matching(n, rp, ci, v)
        assert np.array_equal(rp, rp0) and np.array_equal(ci, ci0) and np.array_equal(v, v0)
        A = sp.csr_matrix((v, ci, rp), shape=(n, n)).toarray()
        dl, do = A[q, np.arange(n)], A[qo, np.arange(n)]
        assert np.all(dl != 0) and sorted(q.tolist()) == list(range(n))
        assert np.sum(np.log(np.abs(dl))) == pytest.approx(np.sum(np.log(np.abs(do))), rel=1e-10, abs=1e-9)
