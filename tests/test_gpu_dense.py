"""GPU parity of the dense root block (kkt_options.dense_block): the last rows
of the elimination order factored as one dense block by k_dense_lu after the
sparse rows, against the oracle's LU of the same ordering.

Tolerances as in test_gpu_parity: FP64 entries |gpu - ref| <= max(1e-11 |ref|,
4 E), FP32 entries max(1e-5 |ref|, 4 E 2^29), E the oracle's first-order
running error bound of the entry (any summation order); the block's slots
outside the fill pattern exactly zero; perturbed-pivot counts equal; refined
solutions omega <= 1e-14, recomputed by the oracle.  Block sizes span one
panel, a ragged last panel, several tiles of the trailing update, the whole
height of the elimination tree, and a single row.
"""
import numpy as np
import pytest
import torch

import oracle
from fill_split import on_fill
from kktgen import config_sequence, random_dd_values, random_sparse_pattern
from paper_2306_14337_gb300 import KKTSolver, _capi

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
_PERM = {}


def _t(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device=DEV)


def _perm(key, n, rp, ci):
    if key not in _PERM:
        _PERM[key] = oracle.min_degree(n, rp, ci)
    return _PERM[key]


def _check(S, o, fp32):
    rp, ci, ref, E = o.F.lu_csr()
    got = on_fill(S, rp, ci, S.export_factors().cpu().numpy())
    d = np.abs(got - ref)
    tol = np.maximum(1e-5 * np.abs(ref), 4 * E * 2.0 ** 29) if fp32 else np.maximum(1e-11 * np.abs(ref), 4 * E)
    bad = np.nonzero(~(d <= tol))[0]
    assert bad.size == 0, f"{bad.size} entries off; worst {np.max(d[bad] / tol[bad]):.3g} x tol"


def _refined_omega(S, n, rp, ci, v, b, max_it=20):
    x = S.solve(_t(b))
    info = S.refine(_t(b), x, 1e-14, max_it)
    assert info["converged"], info
    w = oracle.omega(n, rp, ci, v, b, x.cpu().numpy())
    assert w <= 1e-14, w


@pytest.mark.parametrize("rows", [1, 31, 32, 33, 100, 300])
@pytest.mark.parametrize("fp32", [False, True])
def test_dense_block_200bus(rows, fp32):
    s = config_sequence(0, asym=0.1)
    p = _perm("cfg0", s.n, s.indptr, s.indices)
    v, b = s.values(9), s.rhs(9)
    tau = 2.0 ** -24 if fp32 else 1e-14
    S = KKTSolver(s.n, s.indptr, s.indices, perm=p, fp32=fp32, dense_block=rows, refine_mode="auto")
    S.refactor(_t(v))
    o = oracle.Oracle(s.n, s.indptr, s.indices, v, p, tau_rel=tau)
    # one elimination tree: the block is capped at its height (117 levels here)
    assert S.stats()["dense_rows"] == min(rows, int(o.F.levels()[0].max()) + 1)
    st, npert = S.status()
    assert st in (_capi.KKT_OK, _capi.KKT_WARN_PERTURBED)
    assert npert == o.F.n_perturbed
    _check(S, o, fp32)
    _refined_omega(S, s.n, s.indptr, s.indices, v, b)


@pytest.mark.parametrize("budget", [0, 1])
@pytest.mark.parametrize("step", [0, 29])
@pytest.mark.parametrize("fp32", [False, True])
def test_dense_block_2000bus(budget, step, fp32):
    """The 2,000-bus KKT with the automatic block (FP32 factors) or a
    requested one of 200 rows (FP64), with the update maps and without them
    (the binary-search path of the sparse rows)."""
    s = config_sequence(1)
    p = _perm("cfg1", s.n, s.indptr, s.indices)
    v, b = s.values(step), s.rhs(step)
    S = KKTSolver(s.n, s.indptr, s.indices, perm=p, update_map_budget=budget, fp32=fp32,
                  dense_block=0 if fp32 else 200, refine_mode="auto")
    assert S.stats()["dense_rows"] >= 96 if fp32 else S.stats()["dense_rows"] == 200
    S.refactor(_t(v))
    o = oracle.Oracle(s.n, s.indptr, s.indices, v, p, tau_rel=2.0 ** -24 if fp32 else 1e-14)
    assert S.status()[1] == o.F.n_perturbed
    _check(S, o, fp32)
    # FP32 factors of these systems (D over 16 decades) need many more solves
    _refined_omega(S, s.n, s.indptr, s.indices, v, b, 60 if fp32 else 20)


@pytest.mark.parametrize("n,density,seed,rows", [(60, 0.08, 7, 60), (200, 0.01, 4, 200), (200, 0.01, 4, 77)])
def test_dense_block_random_patterns(n, density, seed, rows):
    """Random patterns with heavy fill; rows = n asks for the whole matrix,
    which the analysis caps at the path of the elimination tree that ends its
    order (at most the tree's height)."""
    rp, ci = random_sparse_pattern(n, density, seed)
    v = random_dd_values(rp, ci, seed)
    p = np.random.default_rng(seed).permutation(n).astype(np.int32)
    S = KKTSolver(n, rp, ci, perm=p, dense_block=rows)
    S.refactor(_t(v))
    o = oracle.Oracle(n, rp, ci, v, p)
    assert 1 <= S.stats()["dense_rows"] <= min(rows, int(o.F.levels()[0].max()) + 1)
    assert S.status()[1] == o.F.n_perturbed
    _check(S, o, False)
    b = np.random.default_rng(seed + 1).standard_normal(n)
    _refined_omega(S, n, rp, ci, v, b)


def test_dense_block_perturbed_pivot_closed_form():
    """A zero leading pivot inside the block: the 3 x 3 closed form of the
    perturbation reading (tau = tau_rel max|A'|, pivot sign(a_11) tau, + for
    a_11 = 0), with the whole matrix as the dense block."""
    A = np.array([[0.0, 2.0, -1.0], [3.0, 5.0, 1.0], [-2.0, 4.0, 7.0]])
    rp = np.array([0, 3, 6, 9], np.int32)
    ci = np.array([0, 1, 2] * 3, np.int32)
    tau_rel = 1e-3
    S = KKTSolver(3, rp, ci, ordering="natural", equilibrate=False, pivot_tau_rel=tau_rel, dense_block=3)
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


@pytest.mark.parametrize("cfg,step,rows", [(0, 9, 100), (1, 29, 230)])
@pytest.mark.parametrize("fp32", [False, True])
def test_dense_block_symmetric_ldlt(cfg, step, rows, fp32):
    """LDL^T rows reduce only their upper part and write it to both triangles of the block;
    and counts the inertia of its pivots with the sparse rows'."""
    s = config_sequence(cfg)
    p = _perm(f"cfg{cfg}", s.n, s.indptr, s.indices)
    v = s.values(step)
    S = KKTSolver(s.n, s.indptr, s.indices, perm=p, symmetric=True, fp32=fp32, dense_block=rows)
    assert S.stats()["dense_rows"] > 0
    S.refactor(_t(v))
    o = oracle.Oracle(s.n, s.indptr, s.indices, v, p, tau_rel=2.0 ** -24 if fp32 else 1e-14)
    pos, neg, pert = S.inertia()
    assert pert == o.F.n_perturbed
    assert (pos, neg) == o.inertia()
    _check(S, o, fp32)


def test_dense_block_matches_sparse_rows():
    """The same system with and without the block: factors within the
    rounding tolerance of each other (both against the oracle), solutions
    equal to refinement accuracy, and repeated refactorizations reproduce the
    block's factors bit for bit (no state carried between launches)."""
    s = config_sequence(1)
    v, b = s.values(14), s.rhs(14)
    A = KKTSolver(s.n, s.indptr, s.indices, dense_block=-1)
    B = KKTSolver(s.n, s.indptr, s.indices, dense_block=400)
    xs = []
    for S in (A, B):
        S.refactor(_t(v))
        x = S.solve(_t(b))
        S.refine(_t(b), x, 1e-14, 20)
        xs.append(x.cpu().numpy())
    np.testing.assert_allclose(xs[1], xs[0], rtol=1e-6, atol=1e-9 * np.abs(xs[0]).max())
    f1 = B.export_factors()
    B.refactor(_t(v))
    assert torch.equal(B.export_factors(), f1)


@pytest.mark.parametrize("fp32", [False, True])
def test_dense_block_rows_in_batched_and_queued_refactorizations(fp32):
    """The batched and queued refactorizations take the dense root block's
    rows as sparse rows (its own pivot steps have no update map: their
    targets are found by binary search); their factors must still match the
    oracle, and the single-system path of the same context (k_dense_lu) too."""
    from paper_2306_14337_gb300 import KKTQueue
    s = config_sequence(0, asym=0.05)
    p = _perm("cfg0", s.n, s.indptr, s.indices)
    tau = 2.0 ** -24 if fp32 else 1e-14
    B = 6
    vals = np.stack([s.values(4, sc) for sc in range(1, B + 1)], axis=1)
    S = KKTSolver(s.n, s.indptr, s.indices, perm=p, fp32=fp32, dense_block=100, max_batch=B)
    assert S.stats()["dense_rows"] == 100
    S.batch_refactor(torch.tensor(vals, device=DEV))
    for sc in (0, 3, 5):
        o = oracle.Oracle(s.n, s.indptr, s.indices, vals[:, sc], p, tau_rel=tau)
        rp, ci, ref, E = o.F.lu_csr()
        got = on_fill(S, rp, ci, S.batch_export_factors(sc).cpu().numpy())
        tol = np.maximum(1e-5 * np.abs(ref), 4 * E * 2.0 ** 29) if fp32 else np.maximum(1e-11 * np.abs(ref), 4 * E)
        assert np.all(np.abs(got - ref) <= tol)
    # a queue of two contexts with dense blocks
    sols = [KKTSolver(s.n, s.indptr, s.indices, perm=p, fp32=fp32, dense_block=100) for _ in range(2)]
    Q = KKTQueue(sols)
    qv = [torch.tensor(vals[:, j], device=DEV) for j in range(2)]
    qb = [torch.tensor(s.csr(4, j + 1) @ s.x_true(4, j + 1), device=DEV) for j in range(2)]
    qx = [torch.zeros_like(b) for b in qb]
    Q.run(qv, qb, qx, n_refine=1)
    torch.cuda.synchronize()
    for j in range(2):
        o = oracle.Oracle(s.n, s.indptr, s.indices, vals[:, j], p, tau_rel=tau)
        rp, ci, ref, E = o.F.lu_csr()
        got = on_fill(sols[j], rp, ci, sols[j].export_factors().cpu().numpy())
        tol = np.maximum(1e-5 * np.abs(ref), 4 * E * 2.0 ** 29) if fp32 else np.maximum(1e-11 * np.abs(ref), 4 * E)
        assert np.all(np.abs(got - ref) <= tol)
    # the single-system refactorization of one of the queue's contexts
    sols[0].refactor(qv[0])
    o = oracle.Oracle(s.n, s.indptr, s.indices, vals[:, 0], p, tau_rel=tau)
    _check(sols[0], o, fp32)


def test_dense_block_with_value_aware_row_permutation():
    """A value-aware context (row permutation from the matching) with a dense
    root block: factors of Q A against the oracle with the same Q and ordering."""
    from kktgen import kkt_sequence
    s = kkt_sequence(200, 260, 40, seed=77, steps=3, reg=0.0, asym=0.05)
    v = s.values(1)
    q = oracle.max_product_matching(s.n, s.indptr, s.indices, v)
    qrp, qci, qv = oracle.row_permuted(s.n, s.indptr, s.indices, v, q)
    p = oracle.min_degree(s.n, qrp, qci)
    S = KKTSolver(s.n, s.indptr, s.indices, row_perm=q, perm=p, dense_block=64)
    assert 0 < S.stats()["dense_rows"] <= 64
    S.refactor(_t(v))
    o = oracle.Oracle(s.n, qrp, qci, qv, p)
    assert S.status()[1] == o.F.n_perturbed
    _check(S, o, False)
    b = s.rhs(1)
    x = S.solve(_t(b))
    info = S.refine(_t(b), x, 1e-14, 20)
    assert info["converged"], info
    assert oracle.omega(s.n, s.indptr, s.indices, v, b, x.cpu().numpy()) <= 1e-14


def test_dense_blocks_of_different_sizes_coexist():
    """k_dense_lu's shared-memory limit belongs to the kernel: a context with a
    smaller block created after one with a larger block must not break the
    larger one's launches."""
    s = config_sequence(1)
    p = _perm("cfg1", s.n, s.indptr, s.indices)
    v = s.values(3)
    big = KKTSolver(s.n, s.indptr, s.indices, perm=p, fp32=True, dense_block=400)
    small = KKTSolver(s.n, s.indptr, s.indices, perm=p, fp32=True, dense_block=40)
    assert big.stats()["dense_rows"] == 400 and small.stats()["dense_rows"] == 40
    o = oracle.Oracle(s.n, s.indptr, s.indices, v, p, tau_rel=2.0 ** -24)
    for S in (small, big):
        S.refactor(_t(v))
        _check(S, o, True)
