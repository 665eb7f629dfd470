"""Pins for the lower bounds of Sec. 3.2 (Eq. (9), Thms 3.2-3.5, Table 1, Eq. (13), Table 4)."""
import itertools
from fractions import Fraction as F

import pytest

from conftest import read_golden
from oracle.bounds import ball_size, clique_C, clique_odd, clique_size, lower_bound, lower_bound_p0


def table1(d, a, b):
    """Table 1 closed forms for |C(d, a, b)|."""
    a, b = F(a), F(b)
    if d == 1:
        return 2 * a + 1
    if d == 2:
        return -2 * b ** 2 + 4 * a * b + 2 * a + 1
    if d == 3:
        return F(-8, 3) * b ** 3 + (4 * a - 2) * b ** 2 + (4 * a + F(2, 3)) * b + 2 * a + 1
    return F(1, 3) * (2 * (4 * b ** 3 + 6 * b ** 2 + 8 * b + 3) * a
                      - 6 * b ** 4 - 8 * b ** 3 - 6 * b ** 2 + 2 * b + 3)


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_table1_closed_forms(d):
    for a in range(0, 7):
        for b in range(0, a + 1):
            assert clique_size(d, a, b) == table1(d, a, b)


def test_ball_sizes():
    # |B_r| in 2D is 2r^2 + 2r + 1; in 4D: 1, 9, 41, 129, 321
    for r in range(6):
        assert ball_size(2, r) == 2 * r * r + 2 * r + 1
    assert [ball_size(4, r) for r in range(5)] == [1, 9, 41, 129, 321]


def test_eq4_is_eq13_at_p0():
    for d in (2, 3, 4):
        for k in range(1, 9):
            assert lower_bound_p0(d, k) == lower_bound(d, 0, k)


def test_theorems_3_2_3_3():
    for k in range(1, 8):
        assert lower_bound(4, k, k) == 2 * k + 1
        for p in range(k + 1, k + 9):
            # the two forms printed in Thm 3.3 agree
            assert lower_bound(4, p, k) == -(-2 * k // (p - k)) + 2


def _in_N(x, y, p, k):
    """x in N(y, p, k) on the infinite lattice (Eq. (8)), displacement along dim 0."""
    up = sum(abs(x[i] - y[i] - (p if i == 0 else 0)) for i in range(len(x)))
    dn = sum(abs(x[i] - y[i] + (p if i == 0 else 0)) for i in range(len(x)))
    return up <= k or dn <= k


@pytest.mark.parametrize("d,p,k", [(d, p, k) for d in (1, 2, 3) for k in range(1, 7)
                                   for p in range(0, k) if (k + p) % 2 == 0])
def test_theorem_3_4_clique(d, p, k):
    """Thm 3.4: C(d, a, b) is a distance-k clique for displacement p."""
    C = clique_C(d, (k + p) // 2, (k - p) // 2)
    for x, y in itertools.combinations(C, 2):
        assert _in_N(x, y, p, k)


@pytest.mark.parametrize("d,p,k", [(d, p, k) for d in (2, 3) for k in range(1, 7)
                                   for p in range(0, k) if (k + p) % 2 == 1])
def test_theorem_3_5_clique(d, p, k):
    """Thm 3.5: C' = C u T u S is a distance-k clique (checked on the literal sets)."""
    C = clique_odd(d, p, k)
    for x, y in itertools.combinations(C, 2):
        assert _in_N(x, y, p, k)


def test_table4_lower_bounds():
    """Table 4 second numbers.  Eq. (13) reproduces all but two printed values:
    (p, k) = (6, 1) prints 4 where Thm 3.3 gives ceil(12/5) = 3, and (3, 7)
    prints 192 where Table 1 gives |C(4, 5, 2)| = 191.  The formula is taken as
    authoritative for both."""
    rows = [(int(r[0]), int(r[1]), int(r[7])) for r in read_golden("table4_colours.txt")]
    rows += [(int(r[0]), int(r[1]), int(r[2])) for r in read_golden("table4_lower_bounds_k8_10.txt")]
    assert len(rows) == 90
    mismatches = {(p, k): (lb, lower_bound(4, p, k)) for p, k, lb in rows if lower_bound(4, p, k) != lb}
    assert mismatches == {(6, 1): (4, 3), (3, 7): (192, 191)}
