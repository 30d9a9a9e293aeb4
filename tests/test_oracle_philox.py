"""Pins the oracle's Philox4x32-10 and director-noise definition.

The paper rotates directors with an unnamed GPU generator (Sussman, arXiv
1702.02939, Sec. 2.C.3); both paths use Philox4x32-10 (Salmon et al., SC'11),
pinned here by the published known-answer vectors, and Box-Muller normals,
pinned by their distribution.
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def load_kat():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    rows = load_kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert oracle.philox(ctr, key) == out


def test_director_noise_is_standard_normal():
    scipy_stats = pytest.importorskip("scipy.stats")
    xi = np.array([oracle.director_noise(1234, tag, step) for tag in range(200) for step in range(100)])
    assert abs(xi.mean()) < 4.0 / np.sqrt(len(xi))
    assert abs(xi.var() - 1.0) < 4.0 * np.sqrt(2.0 / len(xi))
    assert scipy_stats.kstest(xi, "norm").pvalue > 1e-3


def test_director_noise_depends_on_all_counter_fields():
    a = oracle.director_noise(1, 5, 7)
    assert a == oracle.director_noise(1, 5, 7)
    assert a != oracle.director_noise(2, 5, 7)
    assert a != oracle.director_noise(1, 6, 7)
    assert a != oracle.director_noise(1, 5, 8)
    assert a != oracle.director_noise(1, 5, 7 + (1 << 32))
