"""Host-side checks of the C library (no GPU): it loads, exports every entry
point declared in include/kkt.h, rejects malformed input, and its host-only
analysis reproduces the oracle's fill pattern and level schedules exactly
when both use the same ordering."""
import ctypes as C
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from kktgen import config_sequence, random_sparse_pattern, kkt_sequence
from paper_2306_14337_gb300 import KKTSolver, KKTError, _capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "kkt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kkt_[a-z_]+)\s*\(", src)))


def test_library_loads_and_exports_every_declared_symbol():
    L = _capi.load()
    declared = _declared_functions()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(L, name), name
    assert set(declared) == set(_capi.SIGNATURES), "binding and header disagree"


def test_default_options_and_status_strings():
    L = _capi.load()
    o = _capi.Options()
    L.kkt_default_options(C.byref(o))
    assert o.tol == 1e-14 and o.max_refine == 20 and o.fgmres_restart == 20
    assert o.equilibrate == 1 and o.factor_fp32 == 0
    for s in (0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 100):
        assert L.kkt_status_string(s).decode() not in ("", "unknown status")


@pytest.mark.parametrize("rp,ci,why", [
    ([0, 2, 3], [1, 0, 1], "unsorted"),
    ([0, 2, 3], [0, 0, 1], "duplicate"),
    ([0, 1, 2], [0, 2], "out of range"),
    ([0, 1, 2], [0, -1], "negative"),
    ([1, 1, 2], [0, 1], "row_ptr[0] != 0"),
    ([0, 2, 1], [0, 1], "decreasing row_ptr"),
])
def test_malformed_pattern_rejected(rp, ci, why):
    with pytest.raises(KKTError) as ei:
        KKTSolver(2, rp, ci, device=None)
    assert ei.value.status == _capi.KKT_ERR_PATTERN, why


def test_bad_user_permutation_rejected():
    s = kkt_sequence(20, 26, 4, seed=5)
    with pytest.raises(KKTError) as ei:
        KKTSolver(s.n, s.indptr, s.indices, perm=np.zeros(s.n, np.int32), device=None)
    assert ei.value.status == _capi.KKT_ERR_ARG


def _parity(n, rp, ci, perm):
    S = KKTSolver(n, rp, ci, perm=perm, dense_block=-1, device=None)
    sym = S.export_symbolic()
    vals = np.random.default_rng(0).standard_normal(len(ci))
    o = oracle.Oracle(n, rp, ci, vals, perm, equil=False)
    orp, oci = o.F.lu_pattern_csr()
    lev, levu = o.F.levels()
    assert np.array_equal(sym["perm"], perm)
    assert np.array_equal(sym["lu_rp"], orp)
    assert np.array_equal(sym["lu_ci"], oci)
    assert np.array_equal(sym["level"], lev)
    assert np.array_equal(sym["level_u"], levu)
    st = S.stats()
    assert st["nnz_lu"] == o.F.nnz
    assert st["n_levels"] == lev.max() + 1 and st["n_levels_u"] == levu.max() + 1
    return S


@pytest.mark.parametrize("n,density,seed,drop", [(1, 1.0, 1, 0.0), (7, 0.3, 2, 0.5),
                                                 (60, 0.05, 3, 0.3), (200, 0.01, 4, 0.1)])
def test_analysis_matches_oracle_random(n, density, seed, drop):
    rp, ci = random_sparse_pattern(n, density, seed, drop_diag=drop)
    perm = np.random.default_rng(seed).permutation(n).astype(np.int32)
    _parity(n, rp, ci, perm)


@pytest.mark.parametrize("cfg", [0, 1])
def test_analysis_matches_oracle_kkt(cfg):
    s = config_sequence(cfg)
    perm = oracle.min_degree(s.n, s.indptr, s.indices)
    _parity(s.n, s.indptr, s.indices, perm)


def test_analysis_natural_ordering_matches_oracle():
    s = kkt_sequence(50, 65, 10, seed=9)
    S = KKTSolver(s.n, s.indptr, s.indices, ordering="natural", device=None)
    assert np.array_equal(S.export_symbolic()["perm"], np.arange(s.n))
    _parity(s.n, s.indptr, s.indices, np.arange(s.n, dtype=np.int32))


@pytest.mark.parametrize("cfg", [0, 1, 2])
def test_amd_ordering_is_a_fill_reducing_permutation(cfg):
    """The library's own ordering: a permutation, deterministic, and its fill
    is comparable to the oracle's textbook minimum degree (within 1.5x), far
    below the natural order's, and a small multiple of the pattern."""
    s = config_sequence(cfg)
    S = KKTSolver(s.n, s.indptr, s.indices, device=None)
    perm = S.export_symbolic()["perm"]
    assert np.array_equal(np.sort(perm), np.arange(s.n))
    S2 = KKTSolver(s.n, s.indptr, s.indices, device=None)
    assert np.array_equal(S2.export_symbolic()["perm"], perm)
    st = S.stats()
    nnz_amd = st["nnz_lu"]
    if cfg <= 1:
        p_md = oracle.min_degree(s.n, s.indptr, s.indices)
        nnz_md = KKTSolver(s.n, s.indptr, s.indices, perm=p_md, device=None).stats()["nnz_lu"]
        assert nnz_amd <= 1.5 * nnz_md
    if cfg == 0:
        nat = KKTSolver(s.n, s.indptr, s.indices, ordering="natural", device=None).stats()["nnz_lu"]
        assert nnz_amd < 0.5 * nat
    assert nnz_amd < 8 * st["nnz_sym"]


def test_amd_fill_closed_under_path_theorem():
    """Fill of the library's own ordering satisfies the Rose-Tarjan
    characterisation (checked by brute force on a small KKT pattern)."""
    s = kkt_sequence(8, 10, 2, seed=3)
    n = s.n
    S = KKTSolver(n, s.indptr, s.indices, device=None)
    sym = S.export_symbolic()
    perm = sym["perm"]
    srp, sci = oracle.symmetrized_pattern(n, s.indptr, s.indices)
    G = sp.csr_matrix((np.ones(len(sci)), sci, srp), shape=(n, n)).toarray() != 0
    G = G[np.ix_(perm, perm)]
    F = np.eye(n, dtype=bool)
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            lim = min(i, j)
            seen, stack, found = {i}, [i], False
            while stack and not found:
                u = stack.pop()
                for w in np.nonzero(G[u])[0]:
                    if w == j:
                        found = True
                        break
                    if w < lim and w not in seen:
                        seen.add(w)
                        stack.append(w)
            F[i, j] = found
    P = sp.csr_matrix((np.ones(len(sym["lu_ci"])), sym["lu_ci"], sym["lu_rp"]), shape=(n, n)).toarray() != 0
    assert np.array_equal(P, F)


def test_host_only_context_refuses_device_calls():
    s = kkt_sequence(10, 13, 2, seed=1)
    S = KKTSolver(s.n, s.indptr, s.indices, device=None)
    L = _capi.load()
    assert L.kkt_refactor(None, C.c_void_p(8), C.c_void_p(0)) == _capi.KKT_ERR_ARG
    assert L.kkt_refactor(S._h, C.c_void_p(8), C.c_void_p(0)) == _capi.KKT_ERR_STATE
    assert L.kkt_solve(S._h, C.c_void_p(8), C.c_void_p(16), C.c_void_p(0)) == _capi.KKT_ERR_STATE


def test_stats_byte_and_flop_counts():
    s = config_sequence(0)
    S = KKTSolver(s.n, s.indptr, s.indices, device=None)
    st = S.stats()
    sym = S.export_symbolic()
    rp, ci = sym["lu_rp"], sym["lu_ci"]
    n = s.n
    # flops: every pivot d costs |L(:,d)| divisions and 2 |L(:,d)| |U(d,:)| flops
    rows = np.repeat(np.arange(n), np.diff(rp))
    lower = ci < rows
    lcount = np.bincount(ci[lower], minlength=n)
    assert st["flops_refactor"] == float(np.sum(lcount * (1 + 2 * lcount)))
    assert st["bytes_refactor"] == 12.0 * s.nnz + 12.0 * st["nnz_lu"] + 4.0 * (n + 1) + 4.0 * st["nnz_lu"]


def test_analysis_checkpoint_round_trip_and_corruption():
    """kkt_save_analysis / kkt_load_analysis on host-only contexts: the loaded
    context exports the same ordering, pattern, levels and statistics; a
    flipped byte or a truncated image is refused."""
    from kktgen import config_sequence
    from paper_2306_14337_gb300 import KKTSolver, _capi
    s = config_sequence(0)
    A = KKTSolver(s.n, s.indptr, s.indices, device=None)
    img = A.save_analysis()
    B = KKTSolver.from_analysis(img, s.indptr, s.indices, device=None)
    ea, eb = A.export_symbolic(), B.export_symbolic()
    for k in ea:
        assert np.array_equal(ea[k], eb[k]), k
    sa, sb = A.stats(), B.stats()
    for k in ("n", "nnz_lu", "n_levels", "n_levels_u", "max_row", "flops_refactor", "n_tasks", "max_task"):
        assert sa[k] == sb[k], k
    bad = bytearray(img)
    bad[len(bad) // 2] ^= 0x40
    for broken in (bytes(bad), img[:-9]):
        with pytest.raises(_capi.KKTError) as e:
            KKTSolver.from_analysis(broken, s.indptr, s.indices, device=None)
        assert e.value.status == _capi.KKT_ERR_ARG


def _brute_levels(n, rp, ci):
    """Longest dependency chains of a filled pattern, by definition: the
    forward level of row i is 0 without L entries, else 1 + the largest level
    of its L columns; the backward level of row i is 0 without U entries right
    of the diagonal, else 1 + the largest backward level of those columns."""
    lev = np.zeros(n, np.int64)
    levu = np.zeros(n, np.int64)
    for i in range(n):
        row = ci[rp[i]:rp[i + 1]]
        low = row[row < i]
        if low.size:
            lev[i] = 1 + lev[low].max()
    for i in range(n - 1, -1, -1):
        row = ci[rp[i]:rp[i + 1]]
        up = row[row > i]
        if up.size:
            levu[i] = 1 + levu[up].max()
    return lev, levu


@pytest.mark.parametrize("case,req", [("cfg1", 0), ("cfg0", 1), ("cfg0", 33), ("cfg0", 100),
                                      ("rand200", 200), ("rand200", 500)])
def test_dense_root_block_pattern(case, req):
    """A dense root block of req rows at most (0: the automatic choice): the
    exported pattern is the oracle's fill plus every pair of the block's
    rows, every block row depends on the one before it (forward levels
    strictly increase along the block), and the level schedules are those of
    the enlarged pattern."""
    from fill_split import fill_slots
    if case.startswith("cfg"):
        s = config_sequence(int(case[3:]))
        n, rp, ci = s.n, s.indptr, s.indices
    else:
        n = 200
        rp, ci = random_sparse_pattern(n, 0.01, 4, drop_diag=0.1)
    perm = oracle.min_degree(n, rp, ci)
    # the automatic choice is made for FP32 factors only
    S = KKTSolver(n, rp, ci, perm=perm, dense_block=req, fp32=True, device=None)
    st = S.stats()
    vals = np.random.default_rng(0).standard_normal(len(ci))
    o = oracle.Oracle(n, rp, ci, vals, perm, equil=False)
    orp, oci = o.F.lu_pattern_csr()
    V = S.export_dense_rows()
    if req == 0:
        assert 96 <= st["dense_rows"] <= 2048
        # the automatic block is at least 80 % full in the oracle's fill
        inV = np.zeros(n, bool)
        inV[V] = True
        rows = np.repeat(np.arange(n), np.diff(orp))
        assert np.sum(inV[rows] & inV[oci]) >= 0.8 * V.size ** 2
    elif case.startswith("cfg"):   # one tree: capped at its height
        assert st["dense_rows"] == min(req, int(o.F.levels()[0].max()) + 1)
    else:                          # maybe a forest: capped at the path ending the order
        assert 1 <= st["dense_rows"] <= min(req, int(o.F.levels()[0].max()) + 1)
    assert V.size == st["dense_rows"] and np.unique(V).size == V.size
    fill_slots(S, orp, oci)
    sym = S.export_symbolic()
    lev, levu = _brute_levels(n, sym["lu_rp"], sym["lu_ci"])
    assert np.array_equal(sym["level"], lev) and np.array_equal(sym["level_u"], levu)
    assert np.all(np.diff(sym["level"][V]) >= 1)
    assert st["nnz_lu"] == len(sym["lu_ci"])
    # the checkpoint keeps the block
    B = KKTSolver.from_analysis(S.save_analysis(), rp, ci, fp32=True, device=None)
    assert B.stats()["dense_rows"] == st["dense_rows"]
    assert np.array_equal(B.export_dense_rows(), V)


def test_dense_root_block_off_and_bad_option():
    s = config_sequence(1)
    S = KKTSolver(s.n, s.indptr, s.indices, dense_block=-1, fp32=True, device=None)
    assert S.stats()["dense_rows"] == 0 and S.export_dense_rows().size == 0
    # FP64 factors take no automatic block (not faster on this GPU), only a requested one
    assert KKTSolver(s.n, s.indptr, s.indices, device=None).stats()["dense_rows"] == 0
    assert KKTSolver(s.n, s.indptr, s.indices, dense_block=150, device=None).stats()["dense_rows"] == 150
    with pytest.raises(KKTError) as ei:
        KKTSolver(s.n, s.indptr, s.indices, dense_block=-2, device=None)
    assert ei.value.status == _capi.KKT_ERR_ARG


def test_far_source_options_validated():
    """solve_far_blocks / solve_far_ctas accept -1 (off), 0 (default) and
    positive values; anything below -1 is refused.  A host-only context runs
    no solve, so it reports no partner CTAs."""
    s = config_sequence(0)
    S = KKTSolver(s.n, s.indptr, s.indices, solve_far_blocks=2, solve_far_ctas=3, device=None)
    st = S.stats()
    assert st["solve_far_ctas"] == 0 and st["solve_far_rows"] == 0
    for kw in (dict(solve_far_blocks=-2), dict(solve_far_ctas=-2)):
        with pytest.raises(KKTError) as ei:
            KKTSolver(s.n, s.indptr, s.indices, device=None, **kw)
        assert ei.value.status == _capi.KKT_ERR_ARG


def test_loaded_analysis_validates_options_like_analyze():
    """kkt_load_analysis applies the same option ranges as kkt_analyze."""
    s = config_sequence(0)
    img = KKTSolver(s.n, s.indptr, s.indices, device=None).save_analysis()
    ok = KKTSolver.from_analysis(img, s.indptr, s.indices, device=None, solve_far_blocks=-1)
    assert ok.stats()["n"] == s.n
    for kw in (dict(solve_far_blocks=-2), dict(solve_far_ctas=-3), dict(fgmres_restart=0),
               dict(max_batch=0), dict(refine_auto_ratio=1.5), dict(dense_block=-2)):
        with pytest.raises(KKTError) as ei:
            KKTSolver.from_analysis(img, s.indptr, s.indices, device=None, **kw)
        assert ei.value.status == _capi.KKT_ERR_ARG, kw


def test_from_analysis_option_names():
    """from_analysis takes the constructor's fp32 for factor_fp32 and refuses
    names it cannot honour instead of ignoring them."""
    s = config_sequence(0)
    img = KKTSolver(s.n, s.indptr, s.indices, device=None).save_analysis()
    B = KKTSolver.from_analysis(img, s.indptr, s.indices, device=None, fp32=True, refine_mode="fgmres")
    assert B.fp32 and B.stats()["factor_fp32"] == 1
    for kw in (dict(fp23=True), dict(ordering=1)):
        with pytest.raises(TypeError):
            KKTSolver.from_analysis(img, s.indptr, s.indices, device=None, **kw)
