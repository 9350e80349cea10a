"""CPU check of the error bound behind the projection's second-stage recheck.

The recheck computes a flagged dot product a.x with Dot2 (Ogita, Rump and
Oishi: TwoProduct by FMA, TwoSum, error terms summed separately) split over
eight lanes, each over its coordinates 4s..4s+3, 4s+32, ... in order, the
eight (sum, error) pairs merged by a tree of TwoSums.  The interval it
tests is sh + sc +- (2.2 (2d)(d+1) u^2 |a||x| + 2^-50 |sh + sc|).  Here the
same arithmetic is emulated in IEEE float32 (numpy) and compared with the
correctly rounded sum of the exact products (math.fsum), on random and on
cancelling inputs (a.x forced near zero).
"""
import math

import numpy as np

F32 = np.float32
U = 2.0 ** -24


def _two_sum(a, b):
    s = F32(a + b)
    z = F32(s - a)
    return s, F32(F32(a - F32(s - z)) + F32(b - z))


def _two_prod(a, b):
    p = F32(a * b)
    # a*b is exact in float64 (24 + 24 bits); its difference to p fits a float32
    return p, F32(np.float64(a) * np.float64(b) - np.float64(p))


def _dot2_lanes(a, x, lanes=8):
    d = len(a)
    parts = []
    for s in range(lanes):
        sh, sc = F32(0), F32(0)
        for b in range(4 * s, d, 4 * lanes):
            for j in range(b, min(b + 4, d)):
                p, h = _two_prod(a[j], x[j])
                sh, er = _two_sum(sh, p)
                sc = F32(sc + F32(er + h))
        parts.append((sh, sc))
    o = 1
    while o < lanes:
        merged = []
        for l in range(lanes):
            (sh, sc), (sh2, sc2) = parts[l], parts[l ^ o]
            t, er = _two_sum(sh, sh2)
            merged.append((t, F32(F32(sc + sc2) + er)))
        parts = merged
        o <<= 1
    assert all(p == parts[0] for p in parts)  # every lane ends with the same pair
    return float(parts[0][0]) + float(parts[0][1])


def test_lane_tree_dot2_within_the_recheck_bound():
    rng = np.random.default_rng(20210618)
    worst = 0.0
    for it in range(600):
        d = int(rng.choice([1, 3, 8, 37, 64, 128]))
        a = rng.standard_normal(d).astype(F32)
        x = (rng.standard_normal(d) * 10.0 ** rng.uniform(-3, 3)).astype(F32)
        if it % 3 == 0 and d > 1:  # cancellation: the last term nearly undoes the rest
            x[-1] = F32(-math.fsum(float(a[j]) * float(x[j]) for j in range(d - 1)) / float(a[-1]))
        S = _dot2_lanes(a, x)
        exact = math.fsum(float(a[j]) * float(x[j]) for j in range(d))
        an = math.sqrt(math.fsum(float(v) ** 2 for v in a))
        xn = math.sqrt(math.fsum(float(v) ** 2 for v in x))
        bound = 2.2 * (2 * d) * (d + 1) * U * U * an * xn + abs(S) * 2.0 ** -50
        assert abs(S - exact) <= bound, (it, d, S, exact, bound)
        if bound > 0:
            worst = max(worst, abs(S - exact) / bound)
    assert worst < 0.5
