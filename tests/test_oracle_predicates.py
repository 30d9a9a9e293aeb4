"""Pins the oracle's exact predicates against Python's exact integer arithmetic.

The Delaunay validity test of the SPV model is the empty-circumcircle property
(Sussman, arXiv 1702.02939, Sec. 2.C.3).  Python ints are arbitrary precision,
so the determinants below are the exact definition evaluated independently of
the oracle's 128/256-bit code and of its floating-point filter.
"""
import random

import pytest

import oracle


def py_orient(a, b, c):
    v = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
    return (v > 0) - (v < 0)


def py_incircle(a, b, c, d):
    rows = []
    for p in (a, b, c):
        dx, dy = p[0] - d[0], p[1] - d[1]
        rows.append((dx, dy, dx * dx + dy * dy))
    (a0, a1, a2), (b0, b1, b2), (c0, c1, c2) = rows
    v = a0 * (b1 * c2 - b2 * c1) - a1 * (b0 * c2 - b2 * c0) + a2 * (b0 * c1 - b1 * c0)
    return (v > 0) - (v < 0)


def rand_pt(rng, bits):
    m = 1 << bits
    return (rng.randrange(-m, m), rng.randrange(-m, m))


@pytest.mark.parametrize("bits", [3, 20, 50, 55])
def test_orient_incircle_random(bits):
    rng = random.Random(bits)
    for _ in range(3000):
        a, b, c, d = (rand_pt(rng, bits) for _ in range(4))
        assert oracle.orient2d(a, b, c) == py_orient(a, b, c)
        assert oracle.incircle(a, b, c, d) == py_incircle(a, b, c, d)


def test_incircle_near_degenerate():
    """Points on a large circle, one of them nudged by a single grid unit:
    the floating-point filter must defer to the exact path."""
    rng = random.Random(7)
    R = 1 << 45
    # Pythagorean-like exactly cocircular points: (R,0), (0,R), (-R,0), (0,-R)
    base = [(R, 0), (0, R), (-R, 0), (0, -R)]
    for nudge in (-1, 0, 1):
        for axis in (0, 1):
            pts = [list(p) for p in base]
            pts[3][axis] += nudge
            a, b, c, d = (tuple(p) for p in pts)
            assert oracle.incircle(a, b, c, d) == py_incircle(a, b, c, d)
    # random exactly cocircular quadruples from integer points on x^2+y^2 = r^2
    circle_pts = [(x, y) for x in range(-65, 66) for y in range(-65, 66) if x * x + y * y == 65 * 65]
    assert len(circle_pts) >= 12
    for _ in range(500):
        a, b, c, d = rng.sample(circle_pts, 4)
        s = 1 << 40
        off = rand_pt(rng, 30)
        A, B, Cc, D = ((p[0] * s + off[0], p[1] * s + off[1]) for p in (a, b, c, d))
        assert py_incircle(A, B, Cc, D) == 0
        assert oracle.incircle(A, B, Cc, D) == 0
        D2 = (D[0] + rng.choice((-1, 1)), D[1])
        assert oracle.incircle(A, B, Cc, D2) == py_incircle(A, B, Cc, D2)


def test_sos_tie_break_is_consistent():
    """On exactly cocircular input the perturbed predicate is never 0, is
    antisymmetric under swapping two of a,b,c (orientation flips) and agrees
    with a tiny explicit lift of the highest-key point."""
    rng = random.Random(3)
    circle_pts = [(x, y) for x in range(-25, 26) for y in range(-25, 26) if x * x + y * y == 625]
    for _ in range(400):
        pts = rng.sample(circle_pts, 4)
        keys = rng.sample(range(100), 4)
        s = oracle.incircle_sos(*pts, keys)
        assert s in (-1, 1)
        a, b, c, d = pts
        ka, kb, kc, kd = keys
        assert oracle.incircle_sos(b, a, c, d, [kb, ka, kc, kd]) == -s
        # explicit perturbation: lift of the top-key point raised by delta
        top = max(range(4), key=lambda k: keys[k])
        # lifted 4x4 determinant sign, with |p|^2 + delta on the top point
        rows = []
        for k, p in enumerate(pts):
            rows.append([p[0], p[1], p[0] ** 2 + p[1] ** 2 + (1 if k == top else 0), 1])
        det4 = _det4(rows)
        # the 4x4 lifted determinant has the sign of incircle for (a,b,c,d)
        assert (det4 > 0) - (det4 < 0) == s


def _det4(m):
    def det3(a):
        return (a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1])
                - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0])
                + a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]))
    total = 0
    for col in range(4):
        minor = [[m[r][c] for c in range(4) if c != col] for r in range(1, 4)]
        total += (-1) ** col * m[0][col] * det3(minor)
    return total


def test_lifted_det_matches_incircle_sign():
    rng = random.Random(11)
    for _ in range(500):
        a, b, c, d = (rand_pt(rng, 10) for _ in range(4))
        rows = [[p[0], p[1], p[0] ** 2 + p[1] ** 2, 1] for p in (a, b, c, d)]
        det4 = _det4(rows)
        assert (det4 > 0) - (det4 < 0) == py_incircle(a, b, c, d)
