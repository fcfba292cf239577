"""Autotuner logic on CPU with a fake queue and timer."""
import json

from paper_2306_14337_gb300 import tune


class FakeQueue:
    def __init__(self):
        self.launch = None
        self.calls = 0

    def set_launch(self, w, c):
        self.launch = (w, c)
        self.calls += 1


def test_pick_chooses_fastest_and_applies_it():
    q = FakeQueue()
    cost = {(8, 0): 3.0, (4, 0): 1.0, (2, 0): 2.0}
    best, table = tune.pick(lambda c: q.set_launch(*c), lambda: cost[q.launch], candidates=list(cost), reps=2)
    assert best == (4, 0) and q.launch == (4, 0)
    assert table == cost


def test_autotune_caches_per_pattern_set(tmp_path):
    pats = [(3, [0, 1, 2, 3], [0, 1, 2])]
    q = FakeQueue()
    cost = {(8, 0): 2.0, (2, 608): 0.5}
    path = str(tmp_path / "tune.json")
    best, table = tune.autotune_queue(q, lambda: cost[q.launch], pats, candidates=list(cost), reps=1,
                                      cache_path=path)
    assert best == (2, 608) and table is not None
    key = tune.fingerprint(pats)
    assert json.load(open(path))[key] == [2, 608]
    tune._memo.clear()
    q2 = FakeQueue()
    best2, table2 = tune.autotune_queue(q2, lambda: 1 / 0, pats, candidates=list(cost), cache_path=path)
    assert best2 == (2, 608) and table2 is None and q2.launch == (2, 608) and q2.calls == 1
    assert tune.fingerprint(pats) != tune.fingerprint([(3, [0, 1, 2, 3], [0, 2, 1])])


def test_candidates_with_a_tile_choice_set_it():
    class TiledQueue(FakeQueue):
        def __init__(self):
            super().__init__()
            self.tiles = None

        def set_tiles(self, k):
            self.tiles = k

    q = TiledQueue()
    cost = {(8, 0, -1): 2.0, (8, 0, 4): 1.0, (4, 0): 3.0}
    best, table = tune.pick(lambda c: tune.apply_candidate(q, c),
                            lambda: cost[q.launch + ((q.tiles,) if q.launch[0] == 8 else ())],
                            candidates=list(cost), reps=1)
    assert best == (8, 0, 4) and q.launch == (8, 0) and q.tiles == 4
    tune.apply_candidate(q, (4, 0))            # no tile choice: all candidates again
    assert q.tiles == -1
