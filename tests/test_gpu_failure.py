"""Failure detection on the GPU without a fault: every device wait is bounded.

A row that is never published (testing option) makes the rows depending on
it exhaust their spin limit; the kernel then raises KKT_ERR_TIMEOUT in the
device status word, every other wait gives up, the launch completes, and the
context and device stay usable.  No trap, assert or invalid access is used.
"""
import numpy as np
import pytest
import torch

from kktgen import config_sequence
from paper_2306_14337_gb300 import KKTSolver, _capi

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def test_wait_that_never_ends_reports_timeout_and_device_stays_usable():
    s = config_sequence(0)
    v = torch.tensor(s.values(0), device=DEV)
    b = torch.tensor(s.rhs(0), device=DEV)
    probe = KKTSolver(s.n, s.indptr, s.indices, device=0)
    lev = probe.export_symbolic()["level"]
    row = int(np.argmin(lev))            # a leaf: many rows above depend on it
    S = KKTSolver(s.n, s.indptr, s.indices, spin_limit=2000, unpublished_row=row)
    S.refactor(v)
    st, _ = S.status()
    assert st == _capi.KKT_ERR_TIMEOUT
    # the same context works again once the status is read (the row stays
    # unpublished, so it times out again rather than hanging)
    S.refactor(v)
    assert S.status()[0] == _capi.KKT_ERR_TIMEOUT
    # and the device is healthy: a normal context solves to full accuracy
    T = KKTSolver(s.n, s.indptr, s.indices)
    T.refactor(v)
    x = T.solve(b)
    info = T.refine(b, x)
    assert info["converged"] and T.status()[0] == _capi.KKT_OK


def test_nan_in_solution_is_not_reported_as_converged():
    """fmax(NaN, y) = y would drop a NaN entry from the infinity norms and let a
    broken x pass omega <= tol.  NaN counts as +infinity: omega is +inf and
    refinement returns KKT_ERR_NONFINITE, for A and for A^T, single and batched."""
    s = config_sequence(0)
    v = torch.tensor(s.values(1), device=DEV)
    b = torch.tensor(s.rhs(1), device=DEV)
    S = KKTSolver(s.n, s.indptr, s.indices, max_batch=2)
    S.refactor(v)
    x = S.solve(b)
    assert S.refine(b, x)["converged"]
    for fn in (S.refine, S.refine_transpose):
        y = x.clone()
        y[7] = float("nan")
        r = fn(b, y, 1e-14, 0)
        assert r["status"] == _capi.KKT_ERR_NONFINITE and r["omega"] == np.inf and not r["converged"]
        r = fn(b, y, 1e-14, 3)            # refinement cannot repair it either
        assert r["status"] == _capi.KKT_ERR_NONFINITE and not r["converged"]
    # batched: the NaN system reports +inf, the other its true residual
    vb = torch.stack([v, v], dim=1).contiguous()
    bb = torch.stack([b, b], dim=1).contiguous()
    S.batch_refactor(vb)
    xb = S.batch_solve(bb)
    xb[3, 1] = float("nan")
    r = S.batch_refine(bb, xb, 1e-14, 0)
    assert r["status"] == _capi.KKT_ERR_NONFINITE
    assert r["omega"][1] == np.inf and r["omega"][0] < 1e-6
    assert S.status()[0] == _capi.KKT_OK      # the status word saw no device fault
