"""The GPU's raw (unrefined) triangular solves, row by row, against the
rounding-error bound of a triangular solve with the GPU's own factors.

Refinement hides a slightly wrong solve (for instance a stale read in the
dependency-driven protocol of Algorithm 2, Sec. 5.2), so these tests look at
one kkt_solve / kkt_solve_transpose before any refinement.

Why a backward-error bound and not an element-wise forward comparison: the
triangular factors of these KKT matrices are very ill-conditioned.  Two correct
solves with identical factors (the oracle's C solve and SciPy's
spsolve_triangular, 2,000-bus system, last step) differ by up to 2.4e-4
relative, and the componentwise forward-error bound built from comparison
matrices exceeds |z| by up to 1e30.  What does hold at rounding level, row by
row, is the classical backward-error result for substitution (Higham,
"Accuracy and Stability of Numerical Algorithms", Thm. 8.5 and Sec. 9.4): with
the factors L, U the GPU exported and its computed solution z of (L U) z = c,

    |c - L (U z)|_i <= u |c|_i + gamma_m (2 + gamma_m) (|L| |U| |z|)_i,
    gamma_m = m u / (1 - m u), m = longest row of L+U plus 2,

with u the unit roundoff of the factor precision (the |c| term is the
rounding of the scaled right-hand side to FP32).  A stale read in row i (a
dependency taken as 0) adds |l_id y_d| to row i of the left side; on the
2,000-bus system all of 84 such planted errors exceed the bound (smallest by
7.6x) while correct solves stay below 0.003 of it.  The same holds for the
transposed solve with A'^T = U^T L^T.

Everything here is computed from the library's exports (factors, ordering,
scaling) with NumPy/SciPy in FP64; the oracle is not involved, so the
orderings may be the library's own (the benchmark's configuration).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from kktgen import config_sequence, random_dd_values, random_sparse_pattern
from paper_2306_14337_gb300 import KKTSolver

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def _t(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device=DEV)


def backward_error_ratios(S, b, fp32, transpose=False):
    """Max over rows of |c - L U z| / bound (see the module docstring) for
    the GPU's unrefined solve of A x = b (or A^T x = b)."""
    n = S.n
    sym = S.export_symbolic()
    perm = sym["perm"].astype(np.int64)
    F = sp.csr_matrix((S.export_factors().cpu().numpy(), sym["lu_ci"], sym["lu_rp"]), shape=(n, n))
    s = S.export_scaling().cpu().numpy()
    bt = _t(b)
    x = (S.solve_transpose(bt) if transpose else S.solve(bt)).cpu().numpy()
    L = (sp.tril(F, -1) + sp.identity(n)).tocsr()
    U = sp.triu(F, 0).tocsr()
    if transpose:                        # A'^T = U^T L^T: first factor U^T, second L^T
        L, U = U.T.tocsr(), L.T.tocsr()
    sp_ = s[perm]
    c = sp_ * b[perm]                    # S P b, exact (powers of two)
    z = x[perm] / sp_                    # exact inverse of x = S P^T z
    u = 2.0 ** -24 if fp32 else 2.0 ** -53
    m = int(np.diff(sym["lu_rp"]).max()) + 2
    g = m * u / (1 - m * u)
    r = np.abs(c - L @ (U @ z))
    bound = u * np.abs(c) + g * (2 + g) * (abs(L) @ (abs(U) @ np.abs(z)))
    assert np.all(np.isfinite(x)), "non-finite entries in the solution"
    with np.errstate(divide="ignore", invalid="ignore"):
        q = np.where(r == 0, 0.0, r / bound)
    return float(q.max())


def _check(S, b, fp32):
    for tr in (False, True):
        q = backward_error_ratios(S, b, fp32, transpose=tr)
        assert q <= 1.0, f"{'transposed ' if tr else ''}solve: backward error {q:.3g} x the bound"


@pytest.mark.parametrize("cfg,step", [(0, 0), (0, 9), (1, 0), (1, 29)])
@pytest.mark.parametrize("fp32", [False, True])
def test_raw_solves_config_sequences(cfg, step, fp32):
    s = config_sequence(cfg, asym=0.05)
    S = KKTSolver(s.n, s.indptr, s.indices, fp32=fp32)
    S.refactor(_t(s.values(step)))
    b = np.random.default_rng(step).standard_normal(s.n)
    _check(S, b, fp32)


@pytest.mark.parametrize("n,density,seed", [(33, 0.2, 2), (257, 0.02, 3), (1000, 0.004, 4)])
def test_raw_solves_random_patterns(n, density, seed):
    rp, ci = random_sparse_pattern(n, density, seed, drop_diag=0.0)
    v = random_dd_values(rp, ci, seed)
    p = np.random.default_rng(seed).permutation(n).astype(np.int32)
    S = KKTSolver(n, rp, ci, perm=p)
    S.refactor(_t(v))
    _check(S, np.random.default_rng(seed + 1).standard_normal(n), False)


def test_raw_solves_arrow_rows_longer_than_shared_memory():
    n = 1500
    rows = [np.array([i, n - 1]) if i < n - 1 else np.arange(n) for i in range(n)]
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum([len(np.unique(r)) for r in rows])
    ci = np.concatenate([np.unique(r) for r in rows]).astype(np.int32)
    v = random_dd_values(rp, ci, 4)
    for fp32 in (False, True):
        S = KKTSolver(n, rp, ci, ordering="natural", fp32=fp32)
        S.refactor(_t(v))
        _check(S, np.random.default_rng(0).standard_normal(n), fp32)


def test_raw_solves_70000bus_fp32_full_size():
    """The 70,000-bus late-IPM system (n = 490,000) with the library's own
    ordering and FP32 factors: the benchmark's configuration."""
    s = config_sequence(3)
    S = KKTSolver(s.n, s.indptr, s.indices, fp32=True)
    S.refactor(_t(s.values(0)))
    _check(S, s.rhs(0), True)


@pytest.mark.parametrize("far_blocks,far_ctas", [(1, 0), (3, 1), (1, 6), (-1, 0), (3, -1)])
@pytest.mark.parametrize("fp32", [False, True])
def test_raw_solves_far_sources_on_partner_ctas(far_blocks, far_ctas, fp32):
    """Long solve tasks hand the sums over their own sources more than a few
    blocks back to partner CTAs (Algorithm 2's dependency-driven substitution
    with the far part of a row summed on another SM).  Every split -- one
    block back, three, one or six partners, none -- solves within the
    backward-error bound, and the partner tables are in use exactly when
    the options ask for them."""
    s = config_sequence(1, asym=0.05)
    S = KKTSolver(s.n, s.indptr, s.indices, fp32=fp32, solve_far_blocks=far_blocks, solve_far_ctas=far_ctas)
    st = S.stats()
    if far_blocks < 0 or far_ctas < 0:
        assert st["solve_far_ctas"] == 0 and st["solve_far_rows"] == 0
    else:
        assert st["solve_far_ctas"] >= 1 and st["solve_far_rows"] > 0, st
        if far_ctas > 0:
            assert st["solve_far_ctas"] <= far_ctas
    S.refactor(_t(s.values(29)))
    _check(S, np.random.default_rng(3).standard_normal(s.n), fp32)
    # refinement on top of the split solves still reaches the target
    b = _t(s.csr(29) @ s.x_true(29))
    x = S.solve(b)
    info = S.refine(b, x, tol=1e-14, max_it=60)
    assert info["converged"], info


def test_raw_solves_far_sources_smallest_case():
    """The 200-bus system has a handful of far rows only one block back
    (solve_far_blocks = 1): the partner path at its smallest."""
    s = config_sequence(0, asym=0.05)
    S = KKTSolver(s.n, s.indptr, s.indices, solve_far_blocks=1)
    assert S.stats()["solve_far_rows"] > 0
    S.refactor(_t(s.values(9)))
    _check(S, np.random.default_rng(9).standard_normal(s.n), False)
