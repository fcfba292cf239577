"""The allocation-free scaled residual (kkt_scaled_residual_noalloc).

That entry point serves callers that cannot call cudaMalloc where they need a
residual, e.g. programs that hand their whole device-memory budget to their
own pool allocator at start-up, or loops that cannot afford the device-wide
synchronization of an allocation; it uses a fixed scratch array compiled into
the library instead of a context.  Here it is checked, through
the C interface, against the context-based residual that kkt_refine reports
(max_it = 0 evaluates omega for the given x without changing it), on two
calls in a row so that contents left in the shared scratch by the first call
cannot leak into the second.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from kktgen import config_sequence
from paper_2306_14337_gb300 import KKTSolver, _capi

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def _p(t):
    return C.c_void_p(t.data_ptr())


def test_noalloc_residual_matches_context_residual_twice():
    s = config_sequence(0, asym=0.05)
    k = 3
    v, b = s.values(k), s.rhs(k)
    n = s.n
    vt = torch.tensor(v, dtype=torch.float64, device=DEV)
    bt = torch.tensor(b, dtype=torch.float64, device=DEV)
    rp = torch.tensor(s.indptr, dtype=torch.int32, device=DEV)
    ci = torch.tensor(s.indices, dtype=torch.int32, device=DEV)
    S = KKTSolver(n, s.indptr, s.indices)
    S.refactor(vt)
    x1 = S.solve(bt)                    # one solve: omega around 1e-9
    x2 = x1.clone()
    S.refine(bt, x2)                    # refined: omega near 1e-16
    L = _capi.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    A = s.csr(k)
    for x in (x1, x2):                  # two calls in a row on the shared scratch
        ref = S.refine(bt, x.clone(), tol=1e-300, max_it=0)["omega"]
        rho = torch.full((n,), np.nan, dtype=torch.float64, device=DEV)
        out = torch.full((5,), np.nan, dtype=torch.float64, device=DEV)
        st = L.kkt_scaled_residual_noalloc(n, _p(rp), _p(ci), _p(vt), _p(bt), _p(x), _p(rho),
                                           _p(out), stream)
        assert st == _capi.KKT_OK
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert o[0] == pytest.approx(ref, rel=1e-12, abs=0.0)
        xh = x.cpu().numpy()
        rh = b - A @ xh
        np.testing.assert_allclose(rho.cpu().numpy(), rh, rtol=0, atol=1e-12 * np.abs(b).max())
        assert o[2] == np.abs(xh).max() and o[3] == np.abs(b).max()
        assert o[4] == pytest.approx(np.abs(A).sum(axis=1).max(), rel=1e-14)


def test_noalloc_residual_rejects_sizes_beyond_its_scratch():
    L = _capi.load()
    d = C.c_void_p(16)                  # never dereferenced: the size check comes first
    st = L.kkt_scaled_residual_noalloc(4_194_305, d, d, d, d, d, d, d, C.c_void_p(0))
    assert st == _capi.KKT_ERR_ARG
    assert b"4,194,304" in L.kkt_last_error()


def test_noalloc_residual_reports_nan_as_infinite_omega():
    """A NaN in x must not drop out of ||x||_inf or ||rho||_inf: omega is +inf,
    as the context's refinement reports it (KKT_ERR_NONFINITE)."""
    s = config_sequence(0)
    v, b = s.values(2), s.rhs(2)
    n = s.n
    vt = torch.tensor(v, dtype=torch.float64, device=DEV)
    bt = torch.tensor(b, dtype=torch.float64, device=DEV)
    rp = torch.tensor(s.indptr, dtype=torch.int32, device=DEV)
    ci = torch.tensor(s.indices, dtype=torch.int32, device=DEV)
    S = KKTSolver(n, s.indptr, s.indices)
    S.refactor(vt)
    x = S.solve(bt)
    S.refine(bt, x)
    x[n // 2] = float("nan")
    L = _capi.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rho = torch.empty(n, dtype=torch.float64, device=DEV)
    out = torch.zeros(5, dtype=torch.float64, device=DEV)
    assert L.kkt_scaled_residual_noalloc(n, _p(rp), _p(ci), _p(vt), _p(bt), _p(x), _p(rho), _p(out),
                                         stream) == _capi.KKT_OK
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert o[0] == np.inf and o[2] == np.inf
    r = S.refine(bt, x.clone(), tol=1e-14, max_it=0)
    assert r["status"] == _capi.KKT_ERR_NONFINITE and r["omega"] == np.inf
