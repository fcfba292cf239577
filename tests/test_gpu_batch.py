"""Batched same-pattern systems (batch-innermost layout) against the oracle.

Scenario systems share the pattern and differ in values (bus loads scaled by
U(0.8, 1.2), the batched workload of the paper's 10,000-bus configuration);
B = 40 exercises one full group of 32 systems and a ragged group of 8.
Tolerances as in test_gpu_parity: factors within max(1e-11 rel, 4x the
oracle's running error bound) (FP32: u = 2^-24), solutions refined to scaled
residual <= 1e-14 recomputed on the CPU per system.
"""
import numpy as np
import pytest
import torch

import oracle
from kktgen import config_sequence
from paper_2306_14337_gb300 import KKTSolver
from fill_split import on_fill

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def _batch(s, k, B):
    vals = np.stack([s.values(k, sc) for sc in range(1, B + 1)], axis=1)
    bs = np.stack([s.csr(k, sc) @ s.x_true(k, sc) for sc in range(1, B + 1)], axis=1)
    return vals, bs


def _check_factor(S, got, o, fp32):
    rp, ci, ref, E = o.F.lu_csr()
    got = on_fill(S, rp, ci, got)
    d = np.abs(got - ref)
    tol = np.maximum(1e-5 * np.abs(ref), 4 * E * 2.0 ** 29) if fp32 else np.maximum(1e-11 * np.abs(ref), 4 * E)
    assert np.all(d <= tol), int(np.sum(~(d <= tol)))


@pytest.mark.parametrize("fp32", [False, True])
def test_batched_factors_and_refined_solves(fp32):
    s = config_sequence(0, asym=0.05)
    k = 6
    B = 40
    vals, bs = _batch(s, k, B)
    p = oracle.min_degree(s.n, s.indptr, s.indices)
    S = KKTSolver(s.n, s.indptr, s.indices, perm=p, fp32=fp32, max_batch=64)
    vt = torch.tensor(vals, device=DEV)
    bt = torch.tensor(bs, device=DEV)
    S.batch_refactor(vt)
    for sc in (0, 17, 31, 32, 39):
        o = oracle.Oracle(s.n, s.indptr, s.indices, vals[:, sc], p, tau_rel=2.0 ** -24 if fp32 else 1e-14)
        _check_factor(S, S.batch_export_factors(sc).cpu().numpy(), o, fp32)
    x = S.batch_solve(bt)
    info = S.batch_refine(bt, x, tol=1e-14, max_it=40)
    xh = x.cpu().numpy()
    for sc in range(B):
        w = oracle.omega(s.n, s.indptr, s.indices, vals[:, sc], bs[:, sc], xh[:, sc])
        assert w <= 1e-14, (sc, w, info["iters"])
    # transposed systems
    g = np.random.default_rng(3).standard_normal((s.n, B))
    gt = torch.tensor(g, device=DEV)
    lam = S.batch_solve_transpose(gt)
    info_t = S.batch_refine_transpose(gt, lam, tol=1e-14, max_it=40)
    lh = lam.cpu().numpy()
    for sc in (0, 31, 39):
        At = s.csr(k, sc + 1).T.tocsr()
        assert oracle.omega(s.n, At.indptr, At.indices, At.data, g[:, sc], lh[:, sc]) <= 1e-14, info_t


def test_batched_matches_single_system_path():
    """A batch of one system gives the single-system path's factors (both
    within tolerance of the oracle) and the same refined solution."""
    s = config_sequence(0, asym=0.05)
    vals, bs = _batch(s, 2, 3)
    S = KKTSolver(s.n, s.indptr, s.indices, max_batch=3)
    S.batch_refactor(torch.tensor(vals, device=DEV))
    xb = S.batch_solve(torch.tensor(bs, device=DEV))
    S.batch_refine(torch.tensor(bs, device=DEV), xb)
    for sc in range(3):
        S1 = KKTSolver(s.n, s.indptr, s.indices)
        v1 = torch.tensor(vals[:, sc], device=DEV)
        b1 = torch.tensor(bs[:, sc], device=DEV)
        S1.refactor(v1)
        x1 = S1.solve(b1)
        S1.refine(b1, x1)
        f1 = S1.export_factors().cpu().numpy()
        fb = S.batch_export_factors(sc).cpu().numpy()
        np.testing.assert_allclose(fb, f1, rtol=1e-9, atol=1e-12 * np.abs(f1).max())
        np.testing.assert_allclose(xb[:, sc].cpu().numpy(), x1.cpu().numpy(), rtol=1e-6,
                                   atol=1e-9 * np.abs(x1.cpu().numpy()).max())


def test_batch_size_checked():
    s = config_sequence(0)
    S = KKTSolver(s.n, s.indptr, s.indices, max_batch=4)
    from paper_2306_14337_gb300 import KKTError
    with pytest.raises(KKTError):
        S.batch_refactor(torch.zeros((s.nnz, 5), dtype=torch.float64, device=DEV))
