"""The device-trace summary (host logic only; the traces are synthetic)."""
import numpy as np

from paper_2306_14337_gb300.trace_tool import PHASES, summarize


def test_summary_of_a_synthetic_trace():
    base = 1_700_000_000_000_000_000                  # a global-timer value in ns
    tr = np.zeros((6, 2), dtype=np.uint64)
    #            claim (ns after base)   done
    rows = [(0, 5_000), (1_000, 3_000), (2_000, 40_000), (0, 0), (4_000, 10_000), (500, 30_500)]
    for i, (c, d) in enumerate(rows):
        if d:
            tr[i] = (base + c, base + d)
    s = summarize(tr, top=3)
    assert s["items"] == 5                            # item 3 recorded nothing
    assert s["span_us"] == 40.0 and s["last_done_item"] == 2
    assert [e["item"] for e in s["longest"]] == [2, 5, 4]
    assert s["longest"][0] == {"item": 2, "claim_us": 2.0, "done_us": 40.0, "us": 38.0}
    assert s["done_us_percentiles"]["100"] == 40.0
    assert s["done_us_percentiles"]["50"] == 10.0     # done times 3, 5, 10, 30.5, 40


def test_empty_trace_and_phase_names():
    assert summarize(np.zeros((4, 2), dtype=np.uint64)) == {"items": 0}
    assert summarize(np.zeros(0, dtype=np.uint64)) == {"items": 0}
    assert PHASES[0] == "refactor" and PHASES[5] == "dense" and len(PHASES) == 6
