"""Autotuner for the launch shape and tiles of the uneven-pattern queue.

Candidates are (warps per CTA, CTA count[, CTA tasks]) tuples: the persistent
kernels' CTA shape (0 CTAs = as many as fit) and, optionally, how many of the
longest solve tasks run on a whole CTA each (-1 = all candidates; CTA tasks
need 8-warp CTAs).  Each candidate is applied, run a few times and timed; the
fastest is kept.  Results are cached per set of patterns (a fingerprint of
their sizes and index arrays), in memory and optionally in a JSON file, so a
pattern set is tuned once.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics

DEFAULT_CANDIDATES = ((8, 0, -1), (8, 0, 16), (8, 0, 4), (8, 0, 0), (4, 0), (2, 0), (8, 152, -1),
                      (4, 304), (2, 608), (1, 1216))


def apply_candidate(queue, cand):
    """Set a candidate's launch shape and, when it has one, its tile choice."""
    queue.set_launch(cand[0], cand[1])
    if len(cand) > 2:
        queue.set_tiles(cand[2])
    elif hasattr(queue, "set_tiles"):
        queue.set_tiles(-1)

_memo: dict = {}


def fingerprint(patterns) -> str:
    """Stable key of a list of (n, indptr, indices) patterns."""
    h = hashlib.sha1()
    for n, rp, ci in patterns:
        h.update(str(int(n)).encode())
        h.update(memoryview(bytes(bytearray(rp))))
        h.update(memoryview(bytes(bytearray(ci))))
    return h.hexdigest()


def pick(apply, time_once, candidates=DEFAULT_CANDIDATES, reps=3):
    """Apply each candidate, time it ``reps`` times (seconds, lower is
    better) and return (best candidate, {candidate: median time})."""
    table = {}
    for cand in candidates:
        apply(cand)
        ts = [time_once() for _ in range(reps)]
        table[tuple(cand)] = statistics.median(ts)
    best = min(table, key=lambda c: (table[c], c))
    apply(best)
    return best, table


def autotune_queue(queue, run_once, patterns, candidates=DEFAULT_CANDIDATES, reps=3, cache_path=None):
    """Choose and apply the queue's launch shape.  ``run_once`` runs the
    workload once and returns its duration in seconds."""
    key = fingerprint(patterns)
    cached = _memo.get(key)
    if cached is None and cache_path and os.path.exists(cache_path):
        try:
            cached = json.load(open(cache_path)).get(key)
        except (OSError, ValueError):
            cached = None
    if cached is not None:
        apply_candidate(queue, cached)
        return tuple(cached), None
    best, table = pick(lambda c: apply_candidate(queue, c), run_once, candidates, reps)
    _memo[key] = list(best)
    if cache_path:
        data = {}
        if os.path.exists(cache_path):
            try:
                data = json.load(open(cache_path))
            except (OSError, ValueError):
                data = {}
        data[key] = list(best)
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(data, f)
        os.replace(tmp, cache_path)
    return best, table
