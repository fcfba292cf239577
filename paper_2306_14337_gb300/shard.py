"""Sharding of independent KKT systems across ranks (one process per GPU).

A single system does not shard (its elimination is one dependency chain), so
multi-GPU runs only distribute whole systems: scenarios of a batch by
contiguous slices, systems of different sizes by longest-processing-time
first on their refactorization flops.  No collective touches the data path.
"""
from __future__ import annotations

import heapq


def contiguous_slice(n_items: int, rank: int, world: int):
    """[start, stop) of rank's share, sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world or n_items < 0:
        raise ValueError("bad rank/world")
    q, r = divmod(n_items, world)
    start = rank * q + min(rank, r)
    return start, start + q + (1 if rank < r else 0)


def lpt_assign(costs, world: int):
    """Indices per rank, greedily giving the next most expensive item to the
    least-loaded rank (ties: lowest rank); deterministic."""
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0.0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(v) for v in out]


class RankLost(RuntimeError):
    """Ranks that did not reach a step of a multi-rank run in time."""

    def __init__(self, step, ranks):
        super().__init__(f"ranks {ranks} did not reach step {step}")
        self.step = step
        self.ranks = list(ranks)


def step_barrier(store, rank: int, world: int, step: int, timeout_s: float = 10.0):
    """Announce that this rank reached ``step`` and wait, on the host, until
    every rank has announced it; raise RankLost naming the ranks that did not
    within ``timeout_s``.  Called between steps (no kernel or collective of
    this rank in flight), so a rank that failed or left is detected before
    the survivors launch the next step.  ``store`` is a torch.distributed
    Store shared by the ranks (e.g. the one of the rendezvous)."""
    from datetime import timedelta
    store.set(f"kkt/step/{step}/{rank}", "1")
    missing = []
    for r in range(world):
        try:
            store.wait([f"kkt/step/{step}/{r}"], timedelta(seconds=timeout_s))
        except Exception:                      # the store reports a timeout as an exception
            missing.append(r)
    if missing:
        raise RankLost(step, missing)
