"""Factor entries of a context on the oracle's fill pattern.

With a dense root block (kkt_options.dense_block) the exported pattern is the
fill pattern of the ordering plus every pair of the block's rows; the added
slots hold structural zeros, which the factorization must leave exactly zero
(every product that reaches them has a structurally zero factor).
"""
import numpy as np


def fill_slots(S, rp, ci):
    """Check (bit-exact, on the integer structure) that the exported pattern
    of S is (rp, ci) plus V x V, V = the dense block's rows; return the
    exported slots of (rp, ci)'s entries in their order and the added slots."""
    sym = S.export_symbolic()
    V = S.export_dense_rows().astype(np.int64)
    n = len(rp) - 1
    erp, eci = np.asarray(sym["lu_rp"]), np.asarray(sym["lu_ci"])
    ke = np.repeat(np.arange(n, dtype=np.int64), np.diff(erp)) * n + eci
    ko = np.repeat(np.arange(n, dtype=np.int64), np.diff(np.asarray(rp))) * n + np.asarray(ci)
    want = np.union1d(ko, (V[:, None] * n + V[None, :]).ravel())
    assert np.array_equal(ke, want), "exported pattern is not the fill pattern plus the dense block"
    pos = np.searchsorted(ke, ko)
    extra = np.setdiff1d(np.arange(ke.size), pos)
    return pos, extra


def on_fill(S, rp, ci, got):
    """got (exported factor values) restricted to the fill pattern (rp, ci);
    the dense block's added slots must hold exact zeros."""
    pos, extra = fill_slots(S, rp, ci)
    got = np.asarray(got)
    assert got.shape == (len(pos) + len(extra),)
    nz = extra[got[extra] != 0.0]
    assert nz.size == 0, f"{nz.size} added dense-block slots are not zero"
    return got[pos]
