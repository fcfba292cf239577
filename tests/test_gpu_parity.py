"""GPU parity: the CUDA path through the C interface against the oracle.

Tolerances (written out per test):
  * fill pattern, levels, permutation: bit-exact (with a dense root block:
    the fill pattern plus the block, whose added slots hold exact zeros);
  * scaling s: bit-exact (powers of two);
  * FP64 factor entries: |gpu - ref| <= max(1e-11 |ref|, 4 E), E = the
    oracle's first-order running error bound of that entry (the KKT matrices
    here lose up to 8 digits to cancellation, so 1e-11 relative cannot hold
    for every entry under any summation order);
  * FP32 factor entries: the same rule with u = 2^-24 (E scaled by 2^29) and
    1e-5 relative;
  * solves: scaled residual omega <= 1e-14 after refinement, recomputed on
    the CPU by the oracle from the GPU's solution;
  * the adjoint gather: bit-exact (one product per entry).
"""
import numpy as np
import pytest
import torch

import oracle
from kktgen import config_sequence, kkt_sequence, random_dd_values, random_sparse_pattern
from paper_2306_14337_gb300 import KKTSolver, kkt_solve, _capi
from fill_split import on_fill

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)

_PERM = {}


def _seq(cfg, asym=0.0):
    return config_sequence(cfg, asym=asym)


def _perm(s, key):
    if key not in _PERM:
        _PERM[key] = oracle.min_degree(s.n, s.indptr, s.indices)
    return _PERM[key]


def _t(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device=DEV)


def _check_factors(S, o, fp32=False):
    rp, ci, ref, E = o.F.lu_csr()
    got = on_fill(S, rp, ci, S.export_factors().cpu().numpy())
    d = np.abs(got - ref)
    if fp32:
        tol = np.maximum(1e-5 * np.abs(ref), 4 * E * 2.0 ** 29)
    else:
        tol = np.maximum(1e-11 * np.abs(ref), 4 * E)
    bad = np.nonzero(~(d <= tol))[0]
    assert bad.size == 0, (f"{bad.size} entries off; worst ratio "
                           f"{np.max(d[bad] / tol[bad]):.3g} at slot {bad[0]}")
    return int(np.sum(d > 1e-11 * np.abs(ref)))


@pytest.mark.parametrize("step", [0, 5, 9])
@pytest.mark.parametrize("equil", [True, False])
def test_refactor_parity_200bus(step, equil):
    s = _seq(0, asym=0.1)
    p = _perm(s, ("cfg0",))
    v = s.values(step)
    S = KKTSolver(s.n, s.indptr, s.indices, perm=p, equilibrate=equil)
    o = oracle.Oracle(s.n, s.indptr, s.indices, v, p, equil=equil)
    vt = _t(v)
    S.refactor(vt)
    st, npert = S.status()
    assert st in (_capi.KKT_OK, _capi.KKT_WARN_PERTURBED)
    assert npert == o.F.n_perturbed
    assert np.array_equal(S.export_scaling().cpu().numpy(), o.s)
    _check_factors(S, o)


@pytest.mark.parametrize("step", [0, 29])
@pytest.mark.parametrize("budget", [0, 1])
def test_refactor_parity_2000bus(step, budget):
    """budget = 1 byte leaves the update maps out, so every update target is
    found by the binary search of the row's sorted columns (the path that
    systems whose maps exceed the budget take)."""
    s = _seq(1)
    p = _perm(s, ("cfg1",))
    v = s.values(step)
    S = KKTSolver(s.n, s.indptr, s.indices, perm=p, update_map_budget=budget)
    assert (S.stats()["update_map_entries"] == 0) == (budget == 1)
    o = oracle.Oracle(s.n, s.indptr, s.indices, v, p)
    S.refactor(_t(v))
    assert S.status()[1] == o.F.n_perturbed
    _check_factors(S, o)


@pytest.mark.parametrize("equil", [True, False])
@pytest.mark.parametrize("fp32", [False, True])
def test_refactor_parity_200bus_without_update_maps(equil, fp32):
    s = _seq(0, asym=0.1)
    p = _perm(s, ("cfg0",))
    v = s.values(9)
    S = KKTSolver(s.n, s.indptr, s.indices, perm=p, equilibrate=equil, fp32=fp32, update_map_budget=1)
    assert S.stats()["update_map_entries"] == 0
    o = oracle.Oracle(s.n, s.indptr, s.indices, v, p, equil=equil, tau_rel=2.0 ** -24 if fp32 else 1e-14)
    S.refactor(_t(v))
    assert S.status()[1] == o.F.n_perturbed
    _check_factors(S, o, fp32=fp32)


def test_contexts_of_different_sizes_coexist():
    """A kernel's shared-memory limit is per kernel, not per context: creating
    a context with smaller rows after a larger one must not break the larger
    one's launches."""
    big_s, small_s = _seq(1), _seq(0)
    big = KKTSolver(big_s.n, big_s.indptr, big_s.indices)
    small = KKTSolver(small_s.n, small_s.indptr, small_s.indices, cta_warps=2)
    for S, s in ((big, big_s), (small, small_s), (big, big_s)):
        b = _t(s.csr(1) @ s.x_true(1))
        S.refactor(_t(s.values(1)))
        x = S.solve(b)
        info = S.refine(b, x, tol=1e-14, max_it=20)
        assert info["converged"] and S.status()[0] == _capi.KKT_OK, info


@pytest.mark.parametrize("cfg,steps", [(0, range(10)), (1, (0, 7, 15, 29))])
def test_solve_refine_sequence(cfg, steps):
    """Refactor and solve a whole value sequence on one context (flags and
    epochs advance across calls); every step reaches omega <= 1e-14 as
    recomputed on the CPU, and the solution agrees with the oracle's."""
    s = _seq(cfg, asym=0.05)
    S = KKTSolver(s.n, s.indptr, s.indices)          # library's own ordering
    for k in steps:
        v = s.values(k)
        b = s.csr(k) @ s.x_true(k)
        vt, bt = _t(v), _t(b)
        S.refactor(vt)
        x = S.solve(bt)
        info = S.refine(bt, x, tol=1e-14, max_it=20)
        assert info["converged"], info
        xh = x.cpu().numpy()
        w = oracle.omega(s.n, s.indptr, s.indices, v, b, xh)
        assert w <= 1e-14, (k, w, info)
        if k == steps[0] or k == list(steps)[-1]:
            # Both solutions have omega <= 1e-14; their difference is bounded by
            # cond(A) * 1e-14, and cond(A) reaches ~1e10 once D spans [1e-8, 1e8].
            o = oracle.Oracle(s.n, s.indptr, s.indices, v, _perm(s, ("cfg%d" % cfg, "asym05")))
            xo, *_ = o.refine(b)
            assert np.abs(xh - xo).max() <= 1e-4 * np.abs(xo).max()


@pytest.mark.parametrize("cfg", [0, 1])
def test_transpose_solve_and_refine(cfg):
    s = _seq(cfg, asym=0.1)
    k = 3
    v = s.values(k)
    p = _perm(s, ("cfg%d" % cfg, "asym"))
    S = KKTSolver(s.n, s.indptr, s.indices, perm=p)
    S.refactor(_t(v))
    g = np.random.default_rng(11).standard_normal(s.n)
    gt = _t(g)
    lam = S.solve_transpose(gt)
    o = oracle.Oracle(s.n, s.indptr, s.indices, v, p)
    lo = o.solve_t(g)
    # unrefined transposed solves agree with the oracle's up to the factors' error
    rel = np.abs(lam.cpu().numpy() - lo).max() / np.abs(lo).max()
    assert rel <= 1e-3, rel
    info = S.refine_transpose(gt, lam, tol=1e-14, max_it=20)
    assert info["converged"], info
    At = s.csr(k).T.tocsr()
    lh = lam.cpu().numpy()
    w = oracle.omega(s.n, At.indptr, At.indices, At.data, g, lh)
    assert w <= 1e-14, w


def test_adjoint_gather_bit_exact():
    s = _seq(0, asym=0.1)
    S = KKTSolver(s.n, s.indptr, s.indices)
    rng = np.random.default_rng(3)
    lam, x = rng.standard_normal(s.n), rng.standard_normal(s.n)
    dA = S.adjoint_gather(_t(lam), _t(x)).cpu().numpy()
    rows = np.repeat(np.arange(s.n), np.diff(s.indptr))
    assert np.array_equal(dA, -lam[rows] * x[s.indices])


def test_autograd_matches_dense_torch():
    s = kkt_sequence(60, 78, 12, seed=21, steps=3, W=4.0, asym=0.1)
    v, b = s.values(1), s.rhs(1)
    g = np.random.default_rng(5).standard_normal(s.n)
    S = KKTSolver(s.n, s.indptr, s.indices)
    vt = _t(v).requires_grad_(True)
    bt = _t(b).requires_grad_(True)
    x = kkt_solve(S, vt, bt)
    (x * _t(g)).sum().backward()
    A = torch.tensor(s.csr(1).toarray(), dtype=torch.float64, requires_grad=True)
    bc = torch.tensor(b, dtype=torch.float64, requires_grad=True)
    xd = torch.linalg.solve(A, bc)
    (xd * torch.tensor(g)).sum().backward()
    rows = np.repeat(np.arange(s.n), np.diff(s.indptr))
    gA = A.grad.numpy()[rows, s.indices]
    np.testing.assert_allclose(x.detach().cpu().numpy(), xd.detach().numpy(), rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(bt.grad.cpu().numpy(), bc.grad.numpy(), rtol=1e-8,
                               atol=1e-10 * np.abs(bc.grad.numpy()).max())
    np.testing.assert_allclose(vt.grad.cpu().numpy(), gA, rtol=1e-8, atol=1e-10 * np.abs(gA).max())


def test_adjoint_matches_oracle_across_sequence_2000bus():
    """The GPU gradient against the oracle's adjoint at late steps of the
    2,000-bus sequence (D up to [1e-8, 1e8])."""
    s = _seq(1, asym=0.0)
    g = np.random.default_rng(1).standard_normal(s.n)
    S = KKTSolver(s.n, s.indptr, s.indices)
    p = _perm(s, ("cfg1",))
    for k in (12, 29):
        v, b = s.values(k), s.rhs(k)
        vt = _t(v).requires_grad_(True)
        bt = _t(b).requires_grad_(True)
        x = kkt_solve(S, vt, bt)
        (x * _t(g)).sum().backward()
        o = oracle.Oracle(s.n, s.indptr, s.indices, v, p)
        xo, *_ = o.refine(b)
        dAo, dbo = o.adjoint(xo, g)
        # both adjoints carry forward errors of order cond(A) * 1e-14
        np.testing.assert_allclose(vt.grad.cpu().numpy(), dAo, rtol=1e-4, atol=1e-7 * np.abs(dAo).max())
        np.testing.assert_allclose(bt.grad.cpu().numpy(), dbo, rtol=1e-4, atol=1e-7 * np.abs(dbo).max())


def test_autograd_finite_differences_2000bus():
    """Config of the 2,000-bus adjoint workload: dA and db against central
    differences (h = 1e-6, relative) of the oracle's solution on 64 random
    entries of the values and of b, and against the oracle's adjoint."""
    s = _seq(1, asym=0.0)
    k = 3          # D in [0.09, 12]: a central difference with h = 1e-6 is accurate here
    v, b = s.values(k), s.rhs(k)
    g = np.random.default_rng(1).standard_normal(s.n)
    S = KKTSolver(s.n, s.indptr, s.indices)          # library's own ordering
    p = _perm(s, ("cfg1",))                          # the oracle's own ordering
    vt = _t(v).requires_grad_(True)
    bt = _t(b).requires_grad_(True)
    x = kkt_solve(S, vt, bt)
    (x * _t(g)).sum().backward()
    dA = vt.grad.cpu().numpy()
    db = bt.grad.cpu().numpy()
    o = oracle.Oracle(s.n, s.indptr, s.indices, v, p)
    xo, *_ = o.refine(b)
    dAo, dbo = o.adjoint(xo, g)
    np.testing.assert_allclose(dA, dAo, rtol=1e-6, atol=1e-9 * np.abs(dAo).max())
    np.testing.assert_allclose(db, dbo, rtol=1e-6, atol=1e-9 * np.abs(dbo).max())

    def loss(vals, bb):
        oo = oracle.Oracle(s.n, s.indptr, s.indices, vals, p)
        xx, *_ = oo.refine(bb)
        return float(g @ xx)

    # Central differences with h = 1e-6 (relative).  Their own error (rounding
    # noise of the two solves / 2h, plus O(h^2) truncation) is estimated by
    # repeating with h/2; the gradient must agree within 1e-5 relative or
    # within 4x that estimate.
    def fd_entry(f, h):
        return (f(+h) - f(-h)) / (2 * h)

    rng = np.random.default_rng(2)
    for kk in rng.choice(len(v), 64, replace=False):
        def f(dv, kk=kk):
            vv = v.copy(); vv[kk] += dv
            return loss(vv, b)
        h = 1e-6 * max(1.0, abs(v[kk]))
        f1, f2 = fd_entry(f, h), fd_entry(f, h / 2)
        assert abs(f1 - dA[kk]) <= max(1e-5 * max(1.0, abs(dA[kk])), 4 * abs(f1 - f2)), (kk, f1, f2, dA[kk])
    for i in rng.choice(s.n, 64, replace=False):
        def f(db_, i=i):
            bb = b.copy(); bb[i] += db_
            return loss(v, bb)
        h = 1e-6 * max(1.0, abs(b[i]))
        f1, f2 = fd_entry(f, h), fd_entry(f, h / 2)
        assert abs(f1 - db[i]) <= max(1e-5 * max(1.0, abs(db[i])), 4 * abs(f1 - f2)), (i, f1, f2, db[i])


@pytest.mark.parametrize("cfg", [0, 1])
def test_fp32_factors_refine_to_fp64_accuracy(cfg):
    s = _seq(cfg, asym=0.05)
    k = s.steps - 1
    v = s.values(k)
    b = s.csr(k) @ s.x_true(k)
    p = _perm(s, ("cfg%d" % cfg, "asym05"))
    S = KKTSolver(s.n, s.indptr, s.indices, perm=p, fp32=True, refine_mode="auto")
    S.refactor(_t(v))
    o = oracle.Oracle(s.n, s.indptr, s.indices, v, p, tau_rel=2.0 ** -24)
    assert S.status()[1] == o.F.n_perturbed
    _check_factors(S, o, fp32=True)
    bt = _t(b)
    x = S.solve(bt)
    info = S.refine(bt, x, tol=1e-14, max_it=20)
    w = oracle.omega(s.n, s.indptr, s.indices, v, b, x.cpu().numpy())
    assert info["converged"] and w <= 1e-14, (info, w)


@pytest.mark.parametrize("mode", ["classic", "fgmres", "auto"])
@pytest.mark.parametrize("fp32", [False, True])
def test_refine_modes_reach_target(mode, fp32):
    """Every refinement mode (Sec. 5.1: classic, FGMRES with the LU
    preconditioner and CGS2, classic then FGMRES) reaches omega <= 1e-14 on the
    200-bus sequence's last step, for A and A^T, with FP64 or FP32 factors
    (classic with FP32 factors may stall: the paper's reason for FGMRES)."""
    s = _seq(0, asym=0.05)
    k = s.steps - 1
    v = s.values(k)
    A = s.csr(k)
    b = A @ s.x_true(k)
    g = np.random.default_rng(4).standard_normal(s.n)
    S = KKTSolver(s.n, s.indptr, s.indices, fp32=fp32, refine_mode=mode)
    S.refactor(_t(v))
    bt, gt = _t(b), _t(g)
    x = torch.zeros_like(bt)
    info = S.refine(bt, x, tol=1e-14, max_it=20)
    lam = torch.zeros_like(gt)
    info_t = S.refine_transpose(gt, lam, tol=1e-14, max_it=20)
    if fp32 and mode == "classic":
        return
    assert info["converged"] and info_t["converged"], (info, info_t)
    assert oracle.omega(s.n, s.indptr, s.indices, v, b, x.cpu().numpy()) <= 1e-14
    At = A.T.tocsr()
    assert oracle.omega(s.n, At.indptr, At.indices, At.data, g, lam.cpu().numpy()) <= 1e-14


def test_perturbed_pivot_closed_form():
    A = np.array([[0.0, 2.0, -1.0], [3.0, 5.0, 1.0], [-2.0, 4.0, 7.0]])
    rp = np.array([0, 3, 6, 9], np.int32)
    ci = np.array([0, 1, 2] * 3, np.int32)
    tau_rel = 1e-3
    S = KKTSolver(3, rp, ci, ordering="natural", equilibrate=False, pivot_tau_rel=tau_rel)
    S.refactor(_t(A.reshape(-1)))
    st, npert = S.status()
    assert st == _capi.KKT_WARN_PERTURBED and npert == 1
    tau = tau_rel * 7.0
    l21, l31 = 3.0 / tau, -2.0 / tau
    u22, u23 = 5.0 - l21 * 2.0, 1.0 - l21 * -1.0
    l32 = (4.0 - l31 * 2.0) / u22
    u33 = 7.0 - l31 * -1.0 - l32 * u23
    want = np.array([tau, 2.0, -1.0, l21, u22, u23, l31, l32, u33])
    np.testing.assert_allclose(S.export_factors().cpu().numpy(), want, rtol=1e-13)


def test_nonfinite_input_flagged():
    s = kkt_sequence(20, 26, 4, seed=2)
    v = s.values(0)
    v[5] = np.nan
    S = KKTSolver(s.n, s.indptr, s.indices)
    S.refactor(_t(v))
    st, _ = S.status()
    assert st == _capi.KKT_ERR_NONFINITE


def test_one_by_one_and_diagonal():
    S = KKTSolver(1, [0, 1], [0])
    S.refactor(_t([4.0]))
    x = S.solve(_t([2.0]))
    assert x.item() == 0.5
    n = 300
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    d = np.random.default_rng(0).uniform(0.5, 2.0, n) * np.where(np.arange(n) % 2, -1, 1)
    S = KKTSolver(n, rp, ci)
    S.refactor(_t(d))
    b = np.random.default_rng(1).standard_normal(n)
    x = S.solve(_t(b)).cpu().numpy()
    np.testing.assert_allclose(x, b / d, rtol=1e-15)


def test_missing_diagonal_and_empty_row():
    """Missing diagonal entries become structural zeros; an all-zero row is
    caught by the pivot test (perturbed and counted) like in the oracle."""
    n = 40
    rp, ci = random_sparse_pattern(n, 0.1, 17, drop_diag=0.3)
    v = random_dd_values(rp, ci, 18)
    # empty the last row
    last = rp[-2]
    rp2 = rp.copy(); rp2[-1] = last
    ci2, v2 = ci[:last], v[:last]
    p = np.random.default_rng(3).permutation(n).astype(np.int32)
    S = KKTSolver(n, rp2, ci2, perm=p)
    S.refactor(_t(v2))
    o = oracle.Oracle(n, rp2, ci2, v2, p)
    assert S.status()[1] == o.F.n_perturbed >= 1
    _check_factors(S, o)


def test_rows_longer_than_shared_memory():
    """An arrow matrix (dense last row and column) has rows longer than the
    per-warp shared-memory capacity, exercising the global scratch path."""
    n = 1500
    rows = [np.array([i, n - 1]) if i < n - 1 else np.arange(n) for i in range(n)]
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum([len(np.unique(r)) for r in rows])
    ci = np.concatenate([np.unique(r) for r in rows]).astype(np.int32)
    v = random_dd_values(rp, ci, 4)
    o = oracle.Oracle(n, rp, ci, v, np.arange(n, dtype=np.int32))
    b = np.random.default_rng(0).standard_normal(n)
    for budget in (0, 1):                # with and without the update maps
        S = KKTSolver(n, rp, ci, ordering="natural", update_map_budget=budget)
        assert S.stats()["max_row"] > 1024
        S.refactor(_t(v))
        _check_factors(S, o)
        x = S.solve(_t(b))
        S.refine(_t(b), x)
        assert oracle.omega(n, rp, ci, v, b, x.cpu().numpy()) <= 1e-14


@pytest.mark.parametrize("n,density,seed", [(2, 1.0, 1), (33, 0.2, 2), (257, 0.02, 3), (1000, 0.004, 4)])
def test_random_patterns(n, density, seed):
    """Random non-symmetric patterns (symmetrized by the analysis) with
    diagonally dominant values, random orderings, heavy fill."""
    rp, ci = random_sparse_pattern(n, density, seed, drop_diag=0.0)
    v = random_dd_values(rp, ci, seed)
    p = np.random.default_rng(seed).permutation(n).astype(np.int32)
    S = KKTSolver(n, rp, ci, perm=p)
    S.refactor(_t(v))
    o = oracle.Oracle(n, rp, ci, v, p)
    _check_factors(S, o)
    b = np.random.default_rng(seed).standard_normal(n)
    x = S.solve(_t(b))
    S.refine(_t(b), x)
    assert oracle.omega(n, rp, ci, v, b, x.cpu().numpy()) <= 1e-14


def test_loaded_analysis_factors_bit_identically():
    """A context resumed from a saved analysis image (kkt_load_analysis) gives
    the same factors, bit for bit, as the context that saved it (the row
    updates are applied in a fixed order, so the refactorization is
    deterministic)."""
    s = _seq(1)
    A = KKTSolver(s.n, s.indptr, s.indices)
    B = KKTSolver.from_analysis(A.save_analysis(), s.indptr, s.indices)
    v = _t(s.values(5))
    A.refactor(v)
    B.refactor(v)
    assert torch.equal(A.export_factors(), B.export_factors())
    b = _t(s.rhs(5))
    x = B.solve(b)
    assert B.refine(b, x)["converged"]
