"""Lower bounds on the number of colours of a displaced distance-k colouring.

Sec. 3.2.  All bounds are for the infinite lattice Z^d_inf with the
displacement p along one dimension (taken as the first in the paper).

* p = 0, Eq. (9): an L1 ball of radius floor(k/2), plus a (d-1)-dimensional
  ball of the same radius when k is odd.
* Thm 3.2: p = k  ->  2k + 1.
* Thm 3.3: p > k  ->  ceil(2p / (p - k)).
* Thms 3.4, 3.5 and Eq. (13): p < k  ->  |C(d, a, b)|, plus |C(d-1, a, b)|
  when k + p is odd, with a = floor((k+p)/2), b = floor((k-p)/2) and
  C(d, a, b) = {x : ||x||_1 <= a and sum_{i>=2} |x_i| <= b}  (Eq. (10)).

Algorithm 3 (the recursive counter) is not used: as printed it never uses a
and returns the size of an L1 ball of radius b.  |C| is counted here by direct
enumeration of the set definition instead.
"""
import itertools
import math


def ball_size(d, r):
    """|N^d(0, 0, r)|: integer points of Z^d with L1 norm <= r (counted)."""
    if r < 0:
        return 0
    if d == 0:
        return 1
    rng = range(-r, r + 1)
    return sum(1 for x in itertools.product(rng, repeat=d) if sum(abs(c) for c in x) <= r)


def clique_C(d, a, b):
    """Points of C(d, a, b) (Eq. (10)), the first coordinate being the
    displaced one.  d = 0 gives the single empty point."""
    if d == 0:
        return [()]
    rng = range(-a, a + 1)
    return [x for x in itertools.product(rng, repeat=d)
            if sum(abs(c) for c in x) <= a and sum(abs(c) for c in x[1:]) <= b]


def clique_size(d, a, b):
    return len(clique_C(d, a, b))


def lower_bound_p0(d, k):
    """Eq. (9)."""
    h = k // 2
    if k % 2 == 0:
        return ball_size(d, h)
    return ball_size(d, h) + ball_size(d - 1, h)


def lower_bound(d, p, k):
    """Eq. (13): col(Z^d_inf, p, k)."""
    if k == p:
        return 2 * k + 1
    if k < p:
        return math.ceil(2 * p / (p - k))
    a = (k + p) // 2
    b = (k - p) // 2
    if (k + p) % 2 == 0:
        return clique_size(d, a, b)
    return clique_size(d, a, b) + clique_size(d - 1, a, b)


def clique_odd(d, p, k):
    """The set C' = C(d,a,b) U T U S of Thm 3.5 (Eqs. (11), (12)), literally."""
    a = (k + p) // 2
    b = (k - p) // 2
    pts = set(clique_C(d, a, b))
    R = a + 2
    rng = range(-R, R + 1)
    for x in itertools.product(rng, repeat=d):
        tail = sum(abs(c) for c in x[1:])
        if d >= 2 and -(p - 1) <= x[0] <= p and 1 <= x[1] < b + 1 and tail == b + 1:
            pts.add(x)                                    # T
        x2 = abs(x[1]) if d >= 2 else 0
        if p + 1 <= x[0] <= a + 1 and x2 <= b and sum(abs(c) for c in x) == a + 1:
            pts.add(x)                                    # S
    return sorted(pts)
