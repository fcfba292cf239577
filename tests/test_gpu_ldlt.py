"""Symmetric refactorization A' = L D L^T with inertia (options.symmetric).

Against the oracle: factor entries with the tolerance of the LU parity tests
(|gpu - ref| <= max(1e-11 |ref|, 4 E); FP32: 1e-5 and E scaled to u = 2^-24)
-- for symmetric A' the Doolittle L and U of the oracle are the L and D L^T of
the LDL^T -- and the inertia (the pivot signs) bit-exact.  Independently of the
oracle: the inertia against dense eigenvalues (Sylvester's law), and against the
closed form of these quasi-definite KKT matrices (H + D_x positive definite, the
constraint block negative definite): n_x positive, n - n_x negative pivots.
Solutions refined to omega <= 1e-14 (recomputed by the oracle), and the raw
solves with the GPU's own factors within the substitution backward-error bound.
"""
import numpy as np
import pytest
import torch

import oracle
from kktgen import config_sequence
from paper_2306_14337_gb300 import KKTSolver, _capi
from test_gpu_raw_solves import backward_error_ratios
from fill_split import on_fill

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
_PERM = {}


def _t(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device=DEV)


def _perm(cfg, s):
    if cfg not in _PERM:
        _PERM[cfg] = oracle.min_degree(s.n, s.indptr, s.indices)
    return _PERM[cfg]


def _n_x(s):
    return 2 * s.grid.nb + 2 * s.grid.ng


@pytest.mark.parametrize("cfg,step", [(0, 0), (0, 9), (1, 29)])
@pytest.mark.parametrize("fp32", [False, True])
def test_symmetric_factors_and_inertia_match_oracle(cfg, step, fp32):
    s = config_sequence(cfg)
    p = _perm(cfg, s)
    v = s.values(step)
    S = KKTSolver(s.n, s.indptr, s.indices, perm=p, symmetric=True, fp32=fp32)
    S.refactor(_t(v))
    o = oracle.Oracle(s.n, s.indptr, s.indices, v, p, tau_rel=2.0 ** -24 if fp32 else 1e-14)
    pos, neg, pert = S.inertia()
    assert pert == o.F.n_perturbed
    assert (pos, neg) == o.inertia() == (_n_x(s), s.n - _n_x(s))
    rp, ci, ref, E = o.F.lu_csr()
    got = on_fill(S, rp, ci, S.export_factors().cpu().numpy())
    tol = np.maximum(1e-5 * np.abs(ref), 4 * E * 2.0 ** 29) if fp32 else np.maximum(1e-11 * np.abs(ref), 4 * E)
    bad = np.nonzero(~(np.abs(got - ref) <= tol))[0]
    assert bad.size == 0, f"{bad.size} entries off"


def test_symmetric_inertia_matches_dense_eigenvalues():
    s = config_sequence(0)
    A = s.csr(9)
    S = KKTSolver(s.n, s.indptr, s.indices, symmetric=True)
    S.refactor(_t(A.data))
    ev = np.linalg.eigvalsh(A.toarray())
    assert S.inertia() == (int(np.sum(ev > 0)), int(np.sum(ev < 0)), 0)


@pytest.mark.parametrize("fp32", [False, True])
def test_symmetric_sequence_refines_to_target(fp32):
    s = config_sequence(1)
    S = KKTSolver(s.n, s.indptr, s.indices, symmetric=True, fp32=fp32, refine_mode="auto")
    for k in (0, 14, 29):
        v, b = s.values(k), s.rhs(k)
        S.refactor(_t(v))
        x = S.solve(_t(b))
        info = S.refine(_t(b), x, 1e-14, 20)
        assert info["converged"], info
        assert oracle.omega(s.n, s.indptr, s.indices, v, b, x.cpu().numpy()) <= 1e-14
        g = np.random.default_rng(k).standard_normal(s.n)
        lam = S.solve_transpose(_t(g))
        info = S.refine_transpose(_t(g), lam, 1e-14, 20)
        assert info["converged"], info
        assert S.inertia()[:2] == (_n_x(s), s.n - _n_x(s))


@pytest.mark.parametrize("fp32", [False, True])
def test_symmetric_raw_solves_backward_error(fp32):
    s = config_sequence(1)
    S = KKTSolver(s.n, s.indptr, s.indices, symmetric=True, fp32=fp32)
    S.refactor(_t(s.values(20)))
    b = np.random.default_rng(3).standard_normal(s.n)
    for tr in (False, True):
        assert backward_error_ratios(S, b, fp32, transpose=tr) <= 1.0


def test_symmetric_70000bus_fp32_full_size():
    """The 70,000-bus late-IPM system, FP32 LDL^T in the benchmark's
    configuration: inertia (n_x, n - n_x), refined omega by the oracle."""
    s = config_sequence(3)
    v, b = s.values(0), s.rhs(0)
    S = KKTSolver(s.n, s.indptr, s.indices, symmetric=True, fp32=True, refine_mode="auto")
    S.refactor(_t(v))
    assert S.inertia()[:2] == (_n_x(s), s.n - _n_x(s))
    bt = _t(b)
    x = S.solve(bt)
    info = S.refine(bt, x, 1e-14, 20)
    assert info["converged"], info
    assert oracle.omega(s.n, s.indptr, s.indices, v, b, x.cpu().numpy()) <= 1e-14


def test_inertia_needs_symmetric_context():
    s = config_sequence(0)
    S = KKTSolver(s.n, s.indptr, s.indices)
    S.refactor(_t(s.values(0)))
    with pytest.raises(_capi.KKTError) as e:
        S.inertia()
    assert e.value.status == _capi.KKT_ERR_STATE
