"""Host logic of the warm start's fallback gate (no GPU)."""
import numpy as np

from paper_2211_05009_gb300.warmstart import choose_gate


def test_gate_minimises_the_total_of_the_policy():
    re = [150.0, 300.0, 500.0, 650.0, 720.0, 900.0]
    rest = [60, 100, 150, 180, 230, 260]
    warm = [50, 90, 145, 200, 400, 400]
    g, total = choose_gate(re, rest, warm, 1001.0)
    assert g == 650.0 and total == 50 + 90 + 145 + 180 + 230 + 260
    # brute force over every threshold between the draws
    best = min(sum(w if r < t else s for r, s, w in zip(re, rest, warm)) for t in np.linspace(0, 1100, 2201))
    assert total == best


def test_gate_extremes():
    re = [200.0, 400.0, 600.0]
    assert choose_gate(re, [10, 10, 10], [5, 5, 5], 1001.0) == (1001.0, 15.0)  # warm start everywhere
    assert choose_gate(re, [5, 5, 5], [10, 10, 10], 1001.0) == (200.0, 15.0)   # always from rest
    assert choose_gate(re, [5, 5, 5], [5, 5, 5], 1001.0)[0] == 200.0           # ties: from rest
