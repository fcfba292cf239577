"""Jacobi-sweep approximate triangular solves (Sec. 6; kkt_solve_jacobi) and
FGMRES with them as the preconditioner (refine_mode "fgmres_jacobi").

Parity of the sweeps: the GPU result against the same recurrence computed
here in FP64 with the GPU's exported factors, element by element, within a
first-order bound of the rounding of both computations: for w_{k+1} = c - L_s w_k
the error e obeys e_{k+1} <= |L_s| e_k + gamma (|c| + |L_s| |w_k|), e_0 = u |c|,
and the U stage likewise with the division by the pivots; the bound used is 2x
the propagated e (GPU and reference each within it), u = 2^-53 or 2^-24.
Exactness: with as many sweeps as the longest dependency chain minus one the
sweeps equal substitution (L_s and D^-1 U_s are nilpotent).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
from kktgen import config_sequence, random_dd_values, random_sparse_pattern
from paper_2306_14337_gb300 import KKTSolver, _capi

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def _t(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device=DEV)


def _reference(S, b, sweeps, transpose, fp32):
    """The sweeps in FP64 on the exported factors, and the first-order
    rounding bound of a computation in the factor precision."""
    n = S.n
    sym = S.export_symbolic()
    perm = sym["perm"].astype(np.int64)
    F = sp.csr_matrix((S.export_factors().cpu().numpy(), sym["lu_ci"], sym["lu_rp"]), shape=(n, n))
    s = S.export_scaling().cpu().numpy()
    u = 2.0 ** -24 if fp32 else 2.0 ** -53
    m = int(np.diff(sym["lu_rp"]).max()) + 2
    g = m * u / (1 - m * u)
    Ls = sp.tril(F, -1, format="csr")
    Us = sp.triu(F, 1, format="csr")
    D = F.diagonal()
    sp_ = s[perm]
    c = sp_ * b[perm]
    ec = u * np.abs(c) if fp32 else np.zeros(n)     # c rounded to FP32 on entry
    if not transpose:
        A1, A2, scale1 = Ls, Us, False               # unit L, then U (scaled by 1/D)
    else:
        A1, A2, scale1 = Us.T.tocsr(), Ls.T.tocsr(), True   # U^T (scaled), then unit L^T
    aA1, aA2, aD = abs(A1), abs(A2), np.abs(D)

    def stage(rhs, erhs, A, aA, scaled):
        inv = (1.0 / D) if scaled else np.ones(n)
        z = rhs * inv
        e = (erhs / aD + 2 * u * np.abs(z)) if scaled else erhs.copy()
        for _ in range(sweeps):
            zn = (rhs - A @ z) * inv
            en = erhs + aA @ e + g * (np.abs(rhs) + aA @ np.abs(z))
            e = (en / aD + 2 * u * np.abs(zn)) if scaled else en
            z = zn
        return z, e

    w, ew = stage(c, ec, A1, aA1, scale1)
    z, ez = stage(w, ew, A2, aA2, not scale1)
    x = np.empty(n)
    x[perm] = sp_ * z
    ex = np.empty(n)
    ex[perm] = sp_ * ez
    return x, ex


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("sweeps", [0, 2, 8])
@pytest.mark.parametrize("transpose", [False, True])
def test_jacobi_sweeps_match_reference_on_exported_factors(fp32, sweeps, transpose):
    s = config_sequence(0, asym=0.05)
    S = KKTSolver(s.n, s.indptr, s.indices, fp32=fp32)
    S.refactor(_t(s.values(2)))
    b = np.random.default_rng(sweeps).standard_normal(s.n)
    got = S.solve_jacobi(_t(b), sweeps, transpose=transpose).cpu().numpy()
    ref, err = _reference(S, b, sweeps, transpose, fp32)
    assert np.all(np.isfinite(got))
    bad = np.nonzero(~(np.abs(got - ref) <= 2 * err + 1e-300))[0]
    assert bad.size == 0, (bad.size, np.max(np.abs(got - ref)[bad] / (2 * err[bad] + 1e-300)))


def test_jacobi_sweeps_exact_at_chain_length():
    """Well-conditioned random pattern: max-level sweeps reproduce the
    substitution solve to rounding, for A and A^T, and the error falls with
    every one of the first sweeps (the Neumann series of a diagonally dominant
    factor decays quickly, so a few sweeps short of the chain length it is
    already below rounding)."""
    n = 400
    rp, ci = random_sparse_pattern(n, 0.01, 8)
    v = random_dd_values(rp, ci, 9)
    S = KKTSolver(n, rp, ci)
    S.refactor(_t(v))
    k = int(max(S.export_symbolic()["level"].max(), S.export_symbolic()["level_u"].max()))
    b = _t(np.random.default_rng(1).standard_normal(n))
    for tr in (False, True):
        exact = (S.solve_transpose(b) if tr else S.solve(b)).cpu().numpy()
        approx = S.solve_jacobi(b, k, transpose=tr).cpu().numpy()
        assert np.abs(approx - exact).max() <= 1e-12 * np.abs(exact).max()
        errs = [np.abs(S.solve_jacobi(b, q, transpose=tr).cpu().numpy() - exact).max() for q in (0, 1, 2)]
        assert errs[0] > errs[1] > errs[2] > 1e-12 * np.abs(exact).max(), errs


@pytest.mark.parametrize("fp32", [False, True])
def test_fgmres_with_jacobi_preconditioner_reaches_target(fp32):
    """FGMRES (Saad 1993) right-preconditioned by Jacobi sweeps reaches omega
    <= 1e-14 (recomputed by the oracle) where the sweeps contract: a random
    diagonally dominant system.  (On the KKT matrices they do not: the
    factors' off-diagonal entries are large, the sweeps diverge, and FGMRES
    stalls -- measured, 200-bus first step, 32 sweeps: omega 0.02 after 100
    iterations, against 2 iterations with the exact solves.)"""
    n = 1000
    rp, ci = random_sparse_pattern(n, 0.004, 4)
    v = random_dd_values(rp, ci, 4)
    b = np.random.default_rng(4).standard_normal(n)
    cases = [(n, rp, ci, v, b)]
    for (nn, r, c, vv, bb) in cases:
        S = KKTSolver(nn, r, c, fp32=fp32, refine_mode="fgmres_jacobi", jacobi_sweeps=8, max_refine=200)
        S.refactor(_t(vv))
        x = torch.zeros(nn, dtype=torch.float64, device=DEV)
        info = S.refine(_t(bb), x, 1e-14, 200)
        assert info["converged"], (nn, info["iters"], info["omega"])
        assert oracle.omega(nn, r, c, vv, bb, x.cpu().numpy()) <= 1e-14


def test_fgmres_jacobi_status_is_honest_when_it_stalls():
    """On the late 2,000-bus system (D over 16 decades) a few sweeps are a poor
    preconditioner: whatever happens, the reported status matches omega."""
    s = config_sequence(1)
    S = KKTSolver(s.n, s.indptr, s.indices, refine_mode="fgmres_jacobi", jacobi_sweeps=4)
    S.refactor(_t(s.values(29)))
    b = s.rhs(29)
    x = torch.zeros(s.n, dtype=torch.float64, device=DEV)
    info = S.refine(_t(b), x, 1e-14, 20)
    w = oracle.omega(s.n, s.indptr, s.indices, s.values(29), b, x.cpu().numpy())
    assert info["converged"] == (w <= 1e-14) or not np.isfinite(w)
    assert info["status"] in (_capi.KKT_OK, _capi.KKT_ERR_NOT_CONVERGED, _capi.KKT_ERR_NONFINITE)
