"""The binomial (revolve) checkpoint schedule behind hydro_forward_revolve, checked on the CPU.

Reversing n steps from a stored state with s free state slots: store the state at m, reverse [m, n) with
s - 1 free slots, then [0, m) with s; with no free slot, recompute every step from the start. The library
takes, at every level, the m that minimises m + P(n - m, s - 1) + P(m, s) with the closed form
P(n, s) = t n - C(c + t, t - 1), c = s + 1, t the least integer with C(c + t, t) >= n (Griewank's bound on
forward steps). Here P is checked against the optimum over ALL split sequences (a brute-force dynamic
program), and the argmin rule against P, so the schedule the library runs is optimal."""
from functools import lru_cache
from math import comb

import pytest


def P(n, s):
    if n <= 1:
        return 0
    if s == 0:
        return n * (n - 1) // 2
    c, t = s + 1, 0
    while comb(c + t, t) < n:
        t += 1
    return t * n - comb(c + t, t - 1)


@lru_cache(None)
def optimum(n, s):
    if n <= 1:
        return 0
    if s == 0:
        return n * (n - 1) // 2
    return min(m + optimum(n - m, s - 1) + optimum(m, s) for m in range(1, n))


def schedule_cost(n, s):
    """Forward steps of the library's rule (argmin split at every level)."""
    if n <= 1:
        return 0
    if s == 0:
        return n * (n - 1) // 2
    m = min(range(1, n), key=lambda k: (k + P(n - k, s - 1) + P(k, s), k))
    return m + schedule_cost(n - m, s - 1) + schedule_cost(m, s)


@pytest.mark.parametrize("s", range(0, 7))
def test_closed_form_is_the_optimum_and_the_rule_attains_it(s):
    for n in range(1, 81):
        assert P(n, s) == optimum(n, s), (n, s)
        assert schedule_cost(n, s) == P(n, s), (n, s)


def test_known_values():
    # with at least n - 1 free slots every step is recomputed once at most: n - 1 forward steps
    assert [P(30, s) for s in (29, 40)] == [29, 29]
    # the 30-step gradient case of the GPU test and the 200-step configuration with 10 slots
    assert [P(30, s) for s in range(7)] == [435, 126, 85, 69, 62, 54, 51]
    assert P(200, 10) == 509
