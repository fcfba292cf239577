"""Torch-facing wrapper of the C interface: device memory and streams come
from PyTorch, all arithmetic runs in ``libkkt.so``.

``KKTSolver`` mirrors the C calls one to one; ``kkt_solve`` is the
differentiable solve (forward: refactor + solve + refine; backward: the
transposed solve with the same factors, then the adjoint gather kernel).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _capi
from ._capi import check

_ORDER = {"amd": _capi.ORDER_AMD, "natural": _capi.ORDER_NATURAL, "user": _capi.ORDER_USER}
_REFINE = {"classic": _capi.REFINE_CLASSIC, "fgmres": _capi.REFINE_FGMRES, "auto": _capi.REFINE_AUTO,
           "fgmres_jacobi": _capi.REFINE_FGMRES_JACOBI}


def _ptr(t: torch.Tensor):
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _i32(a):
    return np.ascontiguousarray(np.asarray(a), dtype=np.int32)


class KKTSolver:
    """One analysed sparsity pattern and its device-resident factors.

    indptr, indices: CSR pattern (host arrays, sorted and unique per row).
    device: CUDA device index, or None for a host-only analysis (no CUDA call;
    only ``stats`` and ``export_symbolic`` work).
    values: host values (CSR order) for a value-aware analysis
    (kkt_analyze_values: a max-product matching row permutation before the
    ordering); row_perm: a row permutation to use instead (row j of the
    factored matrix is row row_perm[j] of A).
    """

    def __init__(self, n, indptr, indices, *, fp32=False, equilibrate=True, ordering="amd",
                 perm=None, refine_mode="classic", tol=1e-14, max_refine=20,
                 pivot_tau_rel=0.0, spin_limit=4_000_000, cta_warps=0, refactor_ctas=0,
                 solve_ctas=0, update_map_budget=0, trace=False, max_batch=1, unpublished_row=-1,
                 poll_ns_max=0, refactor_big_warps=0, symmetric=False, jacobi_sweeps=8, values=None,
                 row_perm=None, dense_block=0, refactor_row_cap=0, refine_auto_ratio=0.0,
                 solve_far_blocks=0, solve_far_ctas=0, device=0):
        self._lib = _capi.load()
        self.n = int(n)
        self._rp = _i32(indptr)
        self._ci = _i32(indices)
        self.nnz = int(self._ci.size)
        opt = _capi.Options()
        self._lib.kkt_default_options(C.byref(opt))
        opt.factor_fp32 = int(bool(fp32))
        opt.equilibrate = int(bool(equilibrate))
        opt.ordering = _ORDER["user" if perm is not None else ordering]
        self._perm = None
        if perm is not None:
            self._perm = _i32(perm)
            opt.user_perm = self._perm.ctypes.data_as(C.POINTER(C.c_int))
        opt.refine_mode = _REFINE[refine_mode]
        opt.tol = float(tol)
        opt.max_refine = int(max_refine)
        opt.pivot_tau_rel = float(pivot_tau_rel)
        opt.spin_limit = int(spin_limit)
        opt.cta_warps = int(cta_warps)
        opt.refactor_ctas = int(refactor_ctas)
        opt.solve_ctas = int(solve_ctas)
        opt.update_map_budget = int(update_map_budget)
        opt.trace = int(bool(trace))
        opt.max_batch = int(max_batch)
        opt.unpublished_row = int(unpublished_row)
        opt.poll_ns_max = int(poll_ns_max)
        opt.refactor_big_warps = int(refactor_big_warps)
        opt.symmetric = int(bool(symmetric))
        opt.jacobi_sweeps = int(jacobi_sweeps)
        opt.dense_block = int(dense_block)
        opt.refactor_row_cap = int(refactor_row_cap)
        opt.refine_auto_ratio = float(refine_auto_ratio)
        opt.solve_far_blocks = int(solve_far_blocks)
        opt.solve_far_ctas = int(solve_far_ctas)
        self._row_perm = None
        if row_perm is not None:
            self._row_perm = _i32(row_perm)
            opt.user_row_perm = self._row_perm.ctypes.data_as(C.POINTER(C.c_int))
        self.device = None if device is None else torch.device("cuda", int(device)) if not isinstance(
            device, torch.device) else device
        opt.device = -1 if self.device is None else (self.device.index or 0)
        self.fp32 = bool(fp32)
        self._opt = opt
        h = C.c_void_p()
        if values is not None:
            vals = np.ascontiguousarray(np.asarray(values), dtype=np.float64)
            st = self._lib.kkt_analyze_values(self.n, self._rp.ctypes.data_as(C.POINTER(C.c_int)),
                                              self._ci.ctypes.data_as(C.POINTER(C.c_int)),
                                              vals.ctypes.data_as(C.POINTER(C.c_double)), C.byref(opt),
                                              C.byref(h))
            check(st, "kkt_analyze_values")
        else:
            st = self._lib.kkt_analyze(self.n, self._rp.ctypes.data_as(C.POINTER(C.c_int)),
                                       self._ci.ctypes.data_as(C.POINTER(C.c_int)), C.byref(opt),
                                       C.byref(h))
            check(st, "kkt_analyze")
        self._h = h
        self._values = None
        self.version = 0           # bumped by every refactor

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.kkt_destroy(h)
            self._h = None

    # ----------------------------------------------------------------- info
    def stats(self) -> dict:
        s = _capi.Stats()
        check(self._lib.kkt_get_stats(self._h, C.byref(s)), "kkt_get_stats")
        return {name: getattr(s, name) for name, _ in _capi.Stats._fields_}

    def export_symbolic(self):
        st = self.stats()
        n, m = st["n"], st["nnz_lu"]
        perm = np.zeros(n, np.int32)
        rp = np.zeros(n + 1, np.int32)
        ci = np.zeros(m, np.int32)
        lev = np.zeros(n, np.int32)
        levu = np.zeros(n, np.int32)
        P = lambda a: a.ctypes.data_as(C.POINTER(C.c_int))
        check(self._lib.kkt_export_symbolic(self._h, P(perm), P(rp), P(ci), P(lev), P(levu)),
              "kkt_export_symbolic")
        return dict(perm=perm, lu_rp=rp, lu_ci=ci, level=lev, level_u=levu)

    def export_dense_rows(self) -> np.ndarray:
        """Rows of the dense root block in elimination order, numbered like
        export_symbolic (empty without a block)."""
        m = self.stats()["dense_rows"]
        rows = np.zeros(max(m, 1), np.int32)
        check(self._lib.kkt_export_dense_rows(self._h, rows.ctypes.data_as(C.POINTER(C.c_int))),
              "kkt_export_dense_rows")
        return rows[:m]

    def export_row_perm(self) -> np.ndarray:
        """Row permutation of the factored matrix (identity without one)."""
        q = np.zeros(self.n, np.int32)
        check(self._lib.kkt_export_row_perm(self._h, q.ctypes.data_as(C.POINTER(C.c_int))),
              "kkt_export_row_perm")
        return q

    def save_analysis(self) -> bytes:
        """The analysis as a checksummed image (kkt_save_analysis)."""
        size = C.c_size_t(0)
        check(self._lib.kkt_save_analysis(self._h, None, 0, C.byref(size)), "kkt_save_analysis")
        buf = C.create_string_buffer(size.value)
        check(self._lib.kkt_save_analysis(self._h, buf, size.value, C.byref(size)), "kkt_save_analysis")
        return buf.raw[: size.value]

    @classmethod
    def from_analysis(cls, image: bytes, indptr, indices, **opts):
        """A context from a saved analysis image (kkt_load_analysis) instead of
        a new analysis; indptr/indices are the caller's pattern (kept for the
        binding's checks); opts are kkt_options fields by name (``fp32`` is
        accepted for ``factor_fp32``, ``refine_mode`` by its name, ``device``
        as for the constructor).  Ordering options are fixed by the image;
        an unknown or fixed option raises TypeError."""
        obj = cls.__new__(cls)
        obj._lib = _capi.load()
        obj._rp, obj._ci = _i32(indptr), _i32(indices)
        obj.n = int(obj._rp.size - 1)
        obj.nnz = int(obj._ci.size)
        opt = _capi.Options()
        obj._lib.kkt_default_options(C.byref(opt))
        fields = {name for name, _ in _capi.Options._fields_}
        fixed = {"ordering", "user_perm", "user_row_perm", "device"}   # set by the image / below
        for k, v in opts.items():
            if k == "device":
                continue
            k = {"fp32": "factor_fp32"}.get(k, k)     # the constructor's name for it
            if k not in fields or k in fixed:
                raise TypeError(f"from_analysis: unsupported option {k!r}")
            if k == "refine_mode":
                v = _REFINE[v]
            setattr(opt, k, int(v) if isinstance(v, bool) else v)
        dev = opts.get("device", 0)
        obj.device = None if dev is None else torch.device("cuda", int(dev))
        opt.device = -1 if dev is None else int(dev)
        obj.fp32 = bool(opt.factor_fp32)
        obj._perm = obj._row_perm = None
        obj._opt = opt
        h = C.c_void_p()
        check(obj._lib.kkt_load_analysis(image, len(image), C.byref(opt), C.byref(h)), "kkt_load_analysis")
        obj._h = h
        obj._values = None
        obj.version = 0
        return obj

    def reanalyze(self, values):
        """Analyze again with the given host values (kkt_analyze_values: a new
        max-product matching and ordering), replacing this context; the other
        options are kept, except that a caller-given ordering (meaningful for
        A, not for the new Q A) is replaced by the minimum-degree one.  The
        paper's policy when refinement fails with the fixed pivot sequence
        (Sec. 5.1)."""
        vals = np.ascontiguousarray(np.asarray(values), dtype=np.float64)
        h = C.c_void_p()
        self._opt.user_row_perm = C.POINTER(C.c_int)()
        if self._opt.ordering == _capi.ORDER_USER:
            self._opt.ordering = _capi.ORDER_AMD
            self._opt.user_perm = C.POINTER(C.c_int)()
        check(self._lib.kkt_analyze_values(self.n, self._rp.ctypes.data_as(C.POINTER(C.c_int)),
                                           self._ci.ctypes.data_as(C.POINTER(C.c_int)),
                                           vals.ctypes.data_as(C.POINTER(C.c_double)), C.byref(self._opt),
                                           C.byref(h)), "kkt_analyze_values")
        self._lib.kkt_destroy(self._h)
        self._h = h
        self._values = None

    def solve_robust(self, values: torch.Tensor, b: torch.Tensor, tol=1e-14, max_it=20, stream=None) -> dict:
        """Refactor, solve and refine; if refinement misses tol (or meets a
        non-finite value), analyze again on these values (value-aware) and
        repeat once.  Returns the refinement record with "x" and "reanalyzed"."""
        self.refactor(values, stream)
        x = self.solve(b, stream=stream)
        info = self.refine(b, x, tol, max_it, stream)
        info["reanalyzed"] = False
        if not info["converged"]:
            self.reanalyze(values.detach().cpu().numpy())
            self.refactor(values, stream)
            x = self.solve(b, stream=stream)
            info = self.refine(b, x, tol, max_it, stream)
            info["reanalyzed"] = True
        info["x"] = x
        return info

    def export_factors(self, stream=None) -> torch.Tensor:
        out = torch.empty(self.stats()["nnz_lu"], dtype=torch.float64, device=self.device)
        check(self._lib.kkt_export_factors(self._h, _ptr(out), _stream(stream)), "kkt_export_factors")
        return out

    def export_trace(self, phase: int) -> np.ndarray:
        """(items, 2) array of device claim / completion times in ns of the
        most recent launch of a phase (0 refactor, 1 forward, 2 backward,
        3 transposed forward, 4 transposed backward, 5 dense-block tile tasks)."""
        st = self.stats()
        nt = (st["dense_rows"] + 31) // 32
        m = max(self.n, st["n_tasks"], nt * (nt + 1) * (2 * nt + 1) // 6)
        buf = np.zeros(2 * m, dtype=np.uint64)
        k = C.c_longlong(0)
        check(self._lib.kkt_export_trace(self._h, int(phase), buf.ctypes.data_as(C.POINTER(C.c_ulonglong)),
                                         m, C.byref(k)), "kkt_export_trace")
        return buf[: 2 * k.value].reshape(-1, 2)

    def export_scaling(self, stream=None) -> torch.Tensor:
        out = torch.empty(self.n, dtype=torch.float64, device=self.device)
        check(self._lib.kkt_export_scaling(self._h, _ptr(out), _stream(stream)), "kkt_export_scaling")
        return out

    def inertia(self, stream=None):
        """(n_pos, n_neg, n_perturbed) of the last refactorization of a context
        created with symmetric=True (kkt_inertia); synchronises the stream."""
        p, m, z = C.c_int(0), C.c_int(0), C.c_int(0)
        check(self._lib.kkt_inertia(self._h, _stream(stream), C.byref(p), C.byref(m), C.byref(z)),
              "kkt_inertia")
        return p.value, m.value, z.value

    def status(self, stream=None):
        """(status code, perturbed-pivot count); synchronises the stream."""
        k = C.c_int(0)
        st = self._lib.kkt_status_sync(self._h, _stream(stream), C.byref(k))
        return st, k.value

    # ------------------------------------------------------------- compute
    def _vec(self, t, name):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
                and t.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
        return t

    def refactor(self, values: torch.Tensor, stream=None):
        self._vec(values, "values")
        if values.numel() != self.nnz:
            raise ValueError("values has the wrong length")
        check(self._lib.kkt_refactor(self._h, _ptr(values), _stream(stream)), "kkt_refactor")
        self._values = values      # the library reads it again in refine
        self.version += 1

    def solve(self, b: torch.Tensor, out=None, stream=None) -> torch.Tensor:
        self._vec(b, "b")
        x = torch.empty_like(b) if out is None else out
        check(self._lib.kkt_solve(self._h, _ptr(b), _ptr(x), _stream(stream)), "kkt_solve")
        return x

    def solve_jacobi(self, b: torch.Tensor, sweeps: int, transpose=False, out=None, stream=None) -> torch.Tensor:
        """Approximate solve by ``sweeps`` Jacobi sweeps per triangular factor
        (kkt_solve_jacobi)."""
        self._vec(b, "b")
        x = torch.empty_like(b) if out is None else out
        check(self._lib.kkt_solve_jacobi(self._h, _ptr(b), _ptr(x), int(sweeps), int(bool(transpose)),
                                         _stream(stream)), "kkt_solve_jacobi")
        return x

    def solve_transpose(self, g: torch.Tensor, out=None, stream=None) -> torch.Tensor:
        self._vec(g, "g")
        lam = torch.empty_like(g) if out is None else out
        check(self._lib.kkt_solve_transpose(self._h, _ptr(g), _ptr(lam), _stream(stream)),
              "kkt_solve_transpose")
        return lam

    def _refine(self, fn, b, x, tol, max_it, stream, raise_on_fail):
        info = _capi.RefineInfo()
        st = fn(self._h, _ptr(b), _ptr(x), float(tol), int(max_it), C.byref(info), _stream(stream))
        if raise_on_fail:
            check(st, "kkt_refine")
        elif st not in (_capi.KKT_OK, _capi.KKT_ERR_NOT_CONVERGED, _capi.KKT_ERR_NONFINITE):
            check(st, "kkt_refine")
        return dict(status=st, iters=info.iters, converged=bool(info.converged), omega=info.omega,
                    history=list(info.omega_hist[: info.n_hist]))

    def refine(self, b, x, tol=0.0, max_it=-1, stream=None, raise_on_fail=False) -> dict:
        self._vec(b, "b"); self._vec(x, "x")
        return self._refine(self._lib.kkt_refine, b, x, tol, max_it, stream, raise_on_fail)

    def refine_transpose(self, g, lam, tol=0.0, max_it=-1, stream=None, raise_on_fail=False) -> dict:
        self._vec(g, "g"); self._vec(lam, "lam")
        return self._refine(self._lib.kkt_refine_transpose, g, lam, tol, max_it, stream, raise_on_fail)

    def adjoint_gather(self, lam, x, out=None, stream=None) -> torch.Tensor:
        self._vec(lam, "lam"); self._vec(x, "x")
        dA = torch.empty(self.nnz, dtype=torch.float64, device=lam.device) if out is None else out
        check(self._lib.kkt_adjoint_gather(self._h, _ptr(lam), _ptr(x), _ptr(dA), _stream(stream)),
              "kkt_adjoint_gather")
        return dA


    # ------------------------------------------------------- batched systems
    def _bvec(self, t, rows, name):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
                and t.is_contiguous() and t.dim() == 2 and t.shape[0] == rows):
            raise TypeError(f"{name} must be a contiguous float64 CUDA tensor of shape ({rows}, B)")
        return t.shape[1]

    def batch_refactor(self, values: torch.Tensor, stream=None):
        """values: (nnz, B), batch innermost."""
        B = self._bvec(values, self.nnz, "values")
        check(self._lib.kkt_batch_refactor(self._h, B, _ptr(values), _stream(stream)), "kkt_batch_refactor")
        self._bvalues = values
        self.batch = B

    def batch_solve(self, b: torch.Tensor, out=None, stream=None) -> torch.Tensor:
        B = self._bvec(b, self.n, "b")
        x = torch.empty_like(b) if out is None else out
        check(self._lib.kkt_batch_solve(self._h, B, _ptr(b), _ptr(x), _stream(stream)), "kkt_batch_solve")
        return x

    def batch_solve_transpose(self, g: torch.Tensor, out=None, stream=None) -> torch.Tensor:
        B = self._bvec(g, self.n, "g")
        lam = torch.empty_like(g) if out is None else out
        check(self._lib.kkt_batch_solve_transpose(self._h, B, _ptr(g), _ptr(lam), _stream(stream)),
              "kkt_batch_solve_transpose")
        return lam

    def _brefine(self, fn, b, x, tol, max_it, stream):
        B = self._bvec(b, self.n, "b")
        om = np.zeros(B)
        it = C.c_int(0)
        st = fn(self._h, B, _ptr(b), _ptr(x), float(tol), int(max_it),
                om.ctypes.data_as(C.POINTER(C.c_double)), C.byref(it), _stream(stream))
        if st not in (_capi.KKT_OK, _capi.KKT_ERR_NOT_CONVERGED, _capi.KKT_ERR_NONFINITE):
            check(st, "kkt_batch_refine")
        return dict(status=st, iters=it.value, omega=om, converged=bool(np.all(om <= (tol or 1e-14))))

    def batch_refine(self, b, x, tol=0.0, max_it=-1, stream=None) -> dict:
        return self._brefine(self._lib.kkt_batch_refine, b, x, tol, max_it, stream)

    def batch_refine_transpose(self, g, lam, tol=0.0, max_it=-1, stream=None) -> dict:
        return self._brefine(self._lib.kkt_batch_refine_transpose, g, lam, tol, max_it, stream)

    def batch_export_factors(self, sys: int, stream=None) -> torch.Tensor:
        out = torch.empty(self.stats()["nnz_lu"], dtype=torch.float64, device=self.device)
        check(self._lib.kkt_batch_export_factors(self._h, int(sys), _ptr(out), _stream(stream)),
              "kkt_batch_export_factors")
        return out


class _KKTSolveFn(torch.autograd.Function):
    """x = A(values)^-1 b.  Backward reuses the factors of A for the
    transposed solve lam = A^-T g (refined in FP64) and returns
    dvalues_k = -lam[row_k] x[col_k] and db = lam."""

    @staticmethod
    def forward(ctx, solver: KKTSolver, values, b, tol, max_it):
        solver.refactor(values)
        x = solver.solve(b)
        # a missed target or a non-finite solution raises (KKTError) instead of
        # returning an x that does not solve the system
        info = solver.refine(b, x, tol, max_it, raise_on_fail=True)
        ctx.solver = solver
        ctx.version = solver.version
        ctx.tol, ctx.max_it = tol, max_it
        ctx.info = info
        ctx.save_for_backward(values, x)
        return x

    @staticmethod
    def backward(ctx, g):
        solver = ctx.solver
        values, x = ctx.saved_tensors
        if solver.version != ctx.version:    # factors were replaced since forward
            solver.refactor(values)
        g = g.contiguous()
        lam = solver.solve_transpose(g)
        solver.refine_transpose(g, lam, ctx.tol, ctx.max_it, raise_on_fail=True)
        dA = solver.adjoint_gather(lam, x)
        return None, dA, lam, None, None


def kkt_solve(solver: KKTSolver, values: torch.Tensor, b: torch.Tensor, tol: float = 1e-14,
              max_it: int = 20) -> torch.Tensor:
    """Differentiable x = A^-1 b for A given by ``values`` on the solver's pattern."""
    return _KKTSolveFn.apply(solver, values, b, tol, max_it)


class KKTQueue:
    """Several analysed patterns processed together: one persistent launch
    per phase over all systems, recorded into a CUDA graph (kkt_queue_*)."""

    def __init__(self, solvers):
        self._lib = _capi.load()
        self.solvers = list(solvers)
        self.m = len(self.solvers)
        arr = (C.c_void_p * self.m)(*[s_._h.value for s_ in self.solvers])
        h = C.c_void_p()
        check(self._lib.kkt_queue_create(arr, self.m, C.byref(h)), "kkt_queue_create")
        self._h = h
        self._keep = None
        self.launch = (0, 0)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.kkt_queue_destroy(h)
            self._h = None

    def set_launch(self, cta_warps=0, ctas=0):
        check(self._lib.kkt_queue_set_launch(self._h, int(cta_warps), int(ctas)), "kkt_queue_set_launch")
        self.launch = (int(cta_warps), int(ctas))

    def set_tiles(self, cta_tasks=-1):
        """How many of the longest solve tasks run on a CTA each (-1: all candidates)."""
        check(self._lib.kkt_queue_set_tiles(self._h, int(cta_tasks)), "kkt_queue_set_tiles")
        self.tiles = int(cta_tasks)

    @staticmethod
    def _ptrs(ts):
        return (C.c_void_p * len(ts))(*[t.data_ptr() for t in ts])

    def run(self, values, bs, xs, n_refine=2, omega=None, stream=None):
        """values[k], bs[k], xs[k]: float64 CUDA tensors of system k."""
        if not (len(values) == len(bs) == len(xs) == self.m):
            raise ValueError("one tensor per system")
        for k, sv in enumerate(self.solvers):
            sv._vec(values[k], "values"); sv._vec(bs[k], "b"); sv._vec(xs[k], "x")
        self._keep = (values, bs, xs, omega)
        om = C.c_void_p(omega.data_ptr()) if omega is not None else C.c_void_p(0)
        check(self._lib.kkt_queue_run(self._h, self._ptrs(values), self._ptrs(bs), self._ptrs(xs),
                                      int(n_refine), om, _stream(stream)), "kkt_queue_run")
        for k, sv in enumerate(self.solvers):
            sv._values = values[k]

    def solve_transpose(self, gs, lams, stream=None):
        check(self._lib.kkt_queue_solve_transpose(self._h, self._ptrs(gs), self._ptrs(lams), _stream(stream)),
              "kkt_queue_solve_transpose")

    def status(self, stream=None):
        k = C.c_int(0)
        st = self._lib.kkt_queue_status_sync(self._h, _stream(stream), C.byref(k))
        return st, k.value

