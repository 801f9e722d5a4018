"""The Jensen-Shannon divergence helper used to compare output distributions: its closed-form values."""
import math

import numpy as np

from paper_2508_07610_gb300 import mpdo as G


def test_jsd_closed_forms():
    p = np.array([0.5, 0.25, 0.25, 0.0])
    assert abs(G.jsd(p, p)) < 1e-15
    assert abs(G.jsd([1, 0], [0, 1]) - math.log(2)) < 1e-15          # disjoint supports
    assert abs(G.jsd([1, 0], [0.5, 0.5]) - (1.5 * math.log(2) - 0.75 * math.log(3))) < 1e-15
    q = np.array([0.1, 0.2, 0.3, 0.4])
    assert abs(G.jsd(p, q) - G.jsd(q, p)) < 1e-15                      # symmetric
    assert abs(G.jsd(2 * p, 5 * q) - G.jsd(p, q)) < 1e-15              # normalises its inputs
    assert 0 < G.jsd(p, q) < math.log(2)
