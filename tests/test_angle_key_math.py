"""The exactness argument of the device's angle key, checked on the CPU with
Python integers: two sector bits and floor(t 2^61) of the sector-reduced
slope t, by two 64-bit divisions.  Two distinct slopes of integers up to
2^30 differ by at least 2^-60, so the keys of distinct directions differ and
keep the angular order; equal directions give equal keys.  The hardest
cases are Farey neighbours with the largest denominators (consecutive
Fibonacci ratios, whose cross product is +-1)."""
from fractions import Fraction

import numpy as np
import pytest

ONE = 1 << 61


def slope_bits(num, den):
    hi = num << 31
    q1, r1 = divmod(hi, den)
    assert hi < 1 << 64 and (r1 << 30) < 1 << 64            # both divisions fit 64 bits
    return (q1 << 30) + ((r1 << 30) // den)


def angle_key(dx, dy):
    if dx > 0 and dy <= dx:
        return slope_bits(dy, dx)
    if dx >= 0:
        return (1 << 62) | (ONE - slope_bits(dx, dy))
    if dy >= -dx:
        return (2 << 62) | slope_bits(-dx, dy)
    return (3 << 62) | (ONE - slope_bits(dy, -dx))


def exact_angle(dx, dy):
    # the angle as an exact sortable value, independent of the key's sectors
    if dx > 0:
        return (0, Fraction(dy, dx))
    if dx == 0:
        return (1, Fraction(0))
    return (2, Fraction(dy, dx))


def fib(k):
    a, b = 0, 1
    for _ in range(k):
        a, b = b, a + b
    return a


def _directions():
    F = [fib(k) for k in range(46)]
    assert F[44] < 1 << 30 < F[45]
    out = []
    for k in (40, 41, 42, 43):                     # consecutive ratios: Farey neighbours
        a, b, c = F[k - 1], F[k], F[k + 1]
        out += [(c, b), (b, a), (b, c), (a, b), (-b, c), (-a, b), (-c, b), (-b, a)]
    m = (1 << 30)
    out += [(m, m - 1), (m - 1, m - 2), (m, 1), (m - 1, 1), (1, m), (1, m - 1), (-1, m), (-m, 1), (-m + 1, 1),
            (m, m), (7, 7), (0, m), (0, 1), (-m, m), (-3, 3), (m, 0), (1, 0)]
    rng = np.random.default_rng(90)
    for _ in range(3000):
        dy = int(rng.integers(0, m + 1))
        dx = int(rng.integers(-m, m + 1))
        if dy == 0 and dx <= 0:
            continue
        out.append((dx, dy))
    return out


def test_key_order_is_the_angle_order():
    d = _directions()
    by_key = sorted(range(len(d)), key=lambda i: (angle_key(*d[i]), i))
    by_angle = sorted(range(len(d)), key=lambda i: (exact_angle(*d[i]), i))
    assert by_key == by_angle
    for i in range(len(d)):
        for j in (i + 1, i + 2):
            if j < len(d):
                same = exact_angle(*d[i]) == exact_angle(*d[j])
                assert (angle_key(*d[i]) == angle_key(*d[j])) == same


def test_farey_neighbours_get_distinct_keys():
    F = [fib(k) for k in range(46)]
    a, b, c = F[42], F[43], F[44]
    assert abs(c * a - b * b) == 1                  # Cassini: the slopes differ by 1 / (b c)
    k1, k2 = angle_key(b, a), angle_key(c, b)
    assert k1 != k2 and (k1 < k2) == (Fraction(a, b) < Fraction(b, c))
    assert abs(k1 - k2) >= 1


@pytest.mark.parametrize("s", [1, 2, 3, 5, 1000, (1 << 29) - 1])
def test_equal_directions_equal_keys(s):
    for dx, dy in [(3, 2), (2, 3), (-2, 3), (-3, 2), (1, 1), (0, 1), (-1, 1), (1, 0)]:
        if max(abs(dx * s), abs(dy * s)) <= 1 << 30:
            assert angle_key(dx * s, dy * s) == angle_key(dx, dy)
