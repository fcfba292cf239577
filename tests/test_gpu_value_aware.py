"""Value-aware analysis (kkt_analyze_values / user_row_perm): a max-product
matching row permutation Q before the ordering (Sec. 5.2 MC64; Sec. 5.1 the
pivot sequence chosen on the first system's values, re-analysis when
refinement fails).

Test family: KKT matrices without the -1e-8 regularization, whose equality
block is a zero diagonal block (not quasi-definite).  The pattern-only
analysis then meets exactly zero pivots (perturbed, counted); with Q the
diagonal of Q A is nonzero and nothing is perturbed.

Against the oracle (its own matching and ordering handed to both sides):
factors of Q A within the LU parity tolerance, perturbation counts equal.
In the caller's numbering: solutions, transposed solutions and the adjoint,
with omega recomputed by the oracle on A and A^T.
"""
import numpy as np
import pytest
import torch

import oracle
from kktgen import kkt_sequence
from paper_2306_14337_gb300 import KKTSolver, _capi, kkt_solve
from fill_split import on_fill

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def _t(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device=DEV)


def _family(nb=200, seed=77):
    return kkt_sequence(nb, int(1.3 * nb), nb // 5, seed=seed, steps=10, W=6.0, reg=0.0)


@pytest.mark.parametrize("fp32", [False, True])
def test_value_aware_factors_match_oracle(fp32):
    s = _family()
    k = 9
    v = s.values(k)
    q = oracle.max_product_matching(s.n, s.indptr, s.indices, v)
    qrp, qci, qv = oracle.row_permuted(s.n, s.indptr, s.indices, v, q)
    p = oracle.min_degree(s.n, qrp, qci)
    S = KKTSolver(s.n, s.indptr, s.indices, row_perm=q, perm=p, fp32=fp32)
    assert np.array_equal(S.export_row_perm(), q)
    S.refactor(_t(v))
    o = oracle.Oracle(s.n, qrp, qci, qv, p, tau_rel=2.0 ** -24 if fp32 else 1e-14)
    # no zero pivot is left; FP32's threshold 2^-24 max|A'| still perturbs small ones, equally on both sides
    assert S.status()[1] == o.F.n_perturbed
    if not fp32:
        assert o.F.n_perturbed == 0
    rp, ci, ref, E = o.F.lu_csr()
    got = on_fill(S, rp, ci, S.export_factors().cpu().numpy())
    tol = np.maximum(1e-5 * np.abs(ref), 4 * E * 2.0 ** 29) if fp32 else np.maximum(1e-11 * np.abs(ref), 4 * E)
    assert np.all(np.abs(got - ref) <= tol)


@pytest.mark.parametrize("nb", [200, 2000])
def test_value_aware_solves_transposed_solves_and_adjoint(nb):
    s = _family(nb)
    k = 9
    v, b = s.values(k), s.rhs(k)
    S = KKTSolver(s.n, s.indptr, s.indices, values=v)          # the library's matching and ordering
    S.refactor(_t(v))
    assert S.status()[1] == 0
    x = S.solve(_t(b))
    info = S.refine(_t(b), x, 1e-14, 20)
    assert info["converged"], info
    xh = x.cpu().numpy()
    assert oracle.omega(s.n, s.indptr, s.indices, v, b, xh) <= 1e-14
    g = np.random.default_rng(2).standard_normal(s.n)
    lam = S.solve_transpose(_t(g))
    info = S.refine_transpose(_t(g), lam, 1e-14, 20)
    assert info["converged"], info
    lh = lam.cpu().numpy()
    At = s.csr(k).T.tocsr()
    assert oracle.omega(s.n, At.indptr, At.indices, At.data, g, lh) <= 1e-14
    # the gather in the caller's numbering: one product per stored entry
    dA = S.adjoint_gather(lam, x).cpu().numpy()
    rows = np.repeat(np.arange(s.n), np.diff(s.indptr))
    assert np.array_equal(dA, -lh[rows] * xh[s.indices])


def test_value_aware_autograd_matches_dense_torch():
    s = kkt_sequence(30, 39, 6, seed=5, steps=3, W=3.0, reg=0.0)
    v, b = s.values(1), s.rhs(1)
    g = np.random.default_rng(5).standard_normal(s.n)
    S = KKTSolver(s.n, s.indptr, s.indices, values=v)
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


def test_zero_pivots_perturbed_without_values_and_reanalysis_policy():
    """Pattern-only analysis of the zero-block family meets zero pivots
    (perturbed, counted).  The re-analysis policy (Sec. 5.1): a stale pivot
    sequence -- an ordering that eliminates every zero-diagonal constraint row
    first, so all of them are perturbed -- needs 3 solves in classic
    refinement (oracle: omega 1.1e-11 after 2) where the value-aware analysis
    needs 2; with one refinement step after the first solve, solve_robust's
    first attempt misses the target, it analyzes again on the values, and the
    second attempt meets omega <= 1e-14."""
    s = _family(200)
    k = 9
    v, b = s.values(k), s.rhs(k)
    plain = KKTSolver(s.n, s.indptr, s.indices)
    plain.refactor(_t(v))
    assert plain.status()[1] > 0
    nx = s.n_x
    stale = np.concatenate([np.arange(nx, s.n), np.arange(nx)]).astype(np.int32)
    S = KKTSolver(s.n, s.indptr, s.indices, perm=stale, refine_mode="classic")
    info = S.solve_robust(_t(v), _t(b), 1e-14, 1)
    assert info["reanalyzed"] and info["converged"], info
    assert S.export_row_perm().tolist() != list(range(s.n))
    assert oracle.omega(s.n, s.indptr, s.indices, v, b, info["x"].cpu().numpy()) <= 1e-14


def test_batched_calls_refuse_a_row_permutation():
    s = _family()
    S = KKTSolver(s.n, s.indptr, s.indices, values=s.values(0), max_batch=2)
    vb = _t(np.stack([s.values(0)] * 2, axis=1))
    with pytest.raises(_capi.KKTError) as e:
        S.batch_refactor(vb)
    assert e.value.status == _capi.KKT_ERR_STATE
