"""Uneven batch: systems with different patterns in one work queue (one
persistent launch per phase, recorded in a CUDA graph), against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from kktgen import kkt_sequence
from paper_2306_14337_gb300 import KKTQueue, KKTSolver, _capi
from fill_split import on_fill

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def _systems():
    sizes = [(30, 39, 6), (60, 78, 12), (30, 39, 6), (120, 156, 24), (60, 78, 12), (200, 260, 40)]
    return [kkt_sequence(nb, nl, ng, seed=500 + j, steps=3, W=4.0, widen=False, asym=0.05)
            for j, (nb, nl, ng) in enumerate(sizes)]


@pytest.mark.parametrize("fp32", [False, True])
def test_queue_refactor_solve_refine_and_replay(fp32):
    seqs = _systems()
    sols = [KKTSolver(s.n, s.indptr, s.indices, fp32=fp32, refine_mode="auto") for s in seqs]
    Q = KKTQueue(sols)
    vals = [torch.tensor(s.values(0), device=DEV) for s in seqs]
    bs = [torch.tensor(s.rhs(0), device=DEV) for s in seqs]
    xs = [torch.zeros_like(b) for b in bs]
    om = torch.zeros(len(seqs), dtype=torch.float64, device=DEV)
    for step in (0, 1, 2):                     # replay: values and b updated in place
        for k, s in enumerate(seqs):
            vals[k].copy_(torch.tensor(s.values(step), device=DEV))
            bs[k].copy_(torch.tensor(s.rhs(step), device=DEV))
        Q.run(vals, bs, xs, n_refine=3, omega=om)
        torch.cuda.synchronize()
        st, _ = Q.status()
        assert st in (_capi.KKT_OK, _capi.KKT_WARN_PERTURBED)
        for k, s in enumerate(seqs):
            # a system that the fixed in-graph refinement left short finishes on its context
            if om[k].item() > 1e-14:
                sols[k].refine(bs[k], xs[k], 1e-14, 40)
            v, b = s.values(step), s.rhs(step)
            w = oracle.omega(s.n, s.indptr, s.indices, v, b, xs[k].cpu().numpy())
            assert w <= 1e-14, (k, step, w, om[k].item())
    # transposed solves with the queue's factors, refined on each context
    gs = [torch.tensor(np.random.default_rng(k).standard_normal(s.n), device=DEV) for k, s in enumerate(seqs)]
    lams = [torch.zeros_like(g) for g in gs]
    Q.solve_transpose(gs, lams)
    for k, s in enumerate(seqs):
        sols[k].refine_transpose(gs[k], lams[k], 1e-14, 40)
        At = s.csr(2).T.tocsr()
        assert oracle.omega(s.n, At.indptr, At.indices, At.data, gs[k].cpu().numpy(),
                            lams[k].cpu().numpy()) <= 1e-14


def test_queue_factors_match_single_context():
    seqs = _systems()[:3]
    p = [oracle.min_degree(s.n, s.indptr, s.indices) for s in seqs]
    sols = [KKTSolver(s.n, s.indptr, s.indices, perm=p[k]) for k, s in enumerate(seqs)]
    Q = KKTQueue(sols)
    vals = [torch.tensor(s.values(1), device=DEV) for s in seqs]
    bs = [torch.tensor(s.rhs(1), device=DEV) for s in seqs]
    xs = [torch.zeros_like(b) for b in bs]
    Q.set_launch(4, 0)
    Q.run(vals, bs, xs, n_refine=1)
    torch.cuda.synchronize()
    for k, s in enumerate(seqs):
        o = oracle.Oracle(s.n, s.indptr, s.indices, s.values(1), p[k])
        rp, ci, ref, E = o.F.lu_csr()
        got = on_fill(sols[k], rp, ci, sols[k].export_factors().cpu().numpy())
        assert np.all(np.abs(got - ref) <= np.maximum(1e-11 * np.abs(ref), 4 * E))


@pytest.mark.parametrize("tiles", [0, 1, -1])
def test_queue_tile_choice_keeps_results(tiles):
    """kkt_queue_set_tiles moves tasks between CTA tasks and warp items; the
    refined solutions stay within the target either way."""
    seqs = _systems()
    sols = [KKTSolver(s.n, s.indptr, s.indices, refine_mode="auto") for s in seqs]
    Q = KKTQueue(sols)
    Q.set_launch(8, 0)
    Q.set_tiles(tiles)
    vals = [torch.tensor(s.values(1), device=DEV) for s in seqs]
    bs = [torch.tensor(s.rhs(1), device=DEV) for s in seqs]
    xs = [torch.zeros_like(b) for b in bs]
    om = torch.zeros(len(seqs), dtype=torch.float64, device=DEV)
    Q.run(vals, bs, xs, n_refine=3, omega=om)
    torch.cuda.synchronize()
    for k, s in enumerate(seqs):
        w = oracle.omega(s.n, s.indptr, s.indices, s.values(1), s.rhs(1), xs[k].cpu().numpy())
        assert w <= 1e-14 or sols[k].refine(bs[k], xs[k], 1e-14, 20)["converged"], (k, w)
