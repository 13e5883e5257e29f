"""Host logic of the benchmark's serving stream (config 5): the seeded Poisson
arrivals and the 60/30/10 shape mix, and the percentile used for latencies."""
import math
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_arrivals_are_seeded_poisson_with_the_mix():
    window, rate, mix, pools = 60.0, 200.0, [0.6, 0.3, 0.1], [64, 8, 32]
    a = bench._serve_arrivals(rate, window, mix, pools, seed=23)
    assert a == bench._serve_arrivals(rate, window, mix, pools, seed=23)  # reproducible
    t = np.array([x[0] for x in a])
    assert np.all(np.diff(t) > 0) and t[-1] < window
    # count ~ Poisson(rate * window): within 5 standard deviations
    assert abs(len(a) - rate * window) < 5 * math.sqrt(rate * window)
    # exponential gaps: mean 1 / rate within 5 standard errors
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / rate) < 5 * (1 / rate) / math.sqrt(len(gaps))
    shapes = np.array([x[1] for x in a])
    for s, p in enumerate(mix):
        frac = np.mean(shapes == s)
        assert abs(frac - p) < 5 * math.sqrt(p * (1 - p) / len(a))
        ks = [x[2] for x in a if x[1] == s]
        assert min(ks) >= 0 and max(ks) < pools[s]


def test_percentile_is_an_order_statistic():
    v = list(range(1, 101))
    assert bench._pct(v, 0.5) == 50 and bench._pct(v, 0.99) == 99 and bench._pct(v, 1.0) == 100
    assert bench._pct([3.0], 0.99) == 3.0 and bench._pct([], 0.5) is None
