"""Multi-rank host logic on CPU (gloo, world size 2): sharding of independent
systems, per-rank work, gather, and the benchmark's max-over-ranks timing."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2306_14337_gb300.shard import contiguous_slice, lpt_assign


def test_contiguous_slice_covers_everything_once():
    for n in (0, 1, 7, 64, 65):
        for w in (1, 2, 3, 8):
            seen = []
            for r in range(w):
                a, b = contiguous_slice(n, r, w)
                seen.extend(range(a, b))
                assert b - a in (n // w, n // w + 1)
            assert seen == list(range(n))


def test_lpt_assign_balances_and_partitions():
    costs = [16, 16, 12, 12, 12, 5, 5, 5, 5, 1, 1, 1]
    parts = lpt_assign(costs, 3)
    assert sorted(i for p in parts for i in p) == list(range(len(costs)))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(costs)
    assert lpt_assign(costs, 3) == parts          # deterministic


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import oracle
    from kktgen import config_sequence
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = config_sequence(0)
    perm = oracle.min_degree(s.n, s.indptr, s.indices)
    n_sys = 5
    a, b = contiguous_slice(n_sys, rank, world)
    mine = {}
    for sc in range(a, b):
        v, rhs = s.values(1, sc + 1), s.csr(1, sc + 1) @ s.x_true(1, sc + 1)
        o = oracle.Oracle(s.n, s.indptr, s.indices, v, perm)
        x, *_ = o.refine(rhs)
        mine[sc] = (float(o.omega(rhs, x)), x[:5].tolist())
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    slowest = bench.reduce_max(float(rank + 1), world)     # the bench's timing reduction
    bench.barrier(world)
    if rank == 0:
        merged = {}
        for g in gathered:
            merged.update(g)
        q.put((merged, slowest))
    dist.destroy_process_group()


def test_two_rank_sharded_solve_matches_single_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged, slowest = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(merged) == list(range(5))
    assert slowest == 2.0
    import oracle
    from kktgen import config_sequence
    s = config_sequence(0)
    perm = oracle.min_degree(s.n, s.indptr, s.indices)
    for sc, (w, head) in merged.items():
        v, rhs = s.values(1, sc + 1), s.csr(1, sc + 1) @ s.x_true(1, sc + 1)
        o = oracle.Oracle(s.n, s.indptr, s.indices, v, perm)
        x, *_ = o.refine(rhs)
        assert w <= 1e-14
        np.testing.assert_array_equal(np.array(head), x[:5])


def _leaving_worker(rank, world, port, q):
    import datetime
    import torch.distributed as dist
    from paper_2306_14337_gb300.shard import RankLost, step_barrier
    store = dist.TCPStore("127.0.0.1", port, world, rank == 0, timeout=datetime.timedelta(seconds=30))
    try:
        for step in range(3):
            if rank == 1 and step == 1:
                q.put(("left", rank, step))    # leaves between steps: nothing of it is in flight
                return
            step_barrier(store, rank, world, step, timeout_s=3.0)
            q.put(("done", rank, step))
    except RankLost as e:
        q.put(("lost", rank, e.step, e.ranks))


def test_rank_that_leaves_between_steps_is_reported():
    """A rank that exits between steps: the survivor's next step barrier (on
    the host, before any launch of that step) names it instead of hanging."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_leaving_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    events = [q.get(timeout=120) for _ in range(4)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert ("done", 0, 0) in events and ("done", 1, 0) in events
    assert ("left", 1, 1) in events
    assert ("lost", 0, 1, [1]) in events
