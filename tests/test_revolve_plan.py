"""The binomial checkpoint schedule (rt_revolve_plan, host arithmetic in the
CUDA library, no device needed): the forward steps it recomputes equal
Griewank & Walther's minimum t n - beta(s + 2, t - 1) for every step count
up to 2000 and every slot count up to 64, and a brute-force dynamic program
over all split points on small cases confirms that minimum."""
from functools import lru_cache
from math import comb

import pytest


def _rt():
    from paper_2608_04085_b300 import build
    build.build()
    import paper_2608_04085_b300 as rt
    return rt


@lru_cache(None)
def _best(n, s):
    """Fewest recomputed steps to reverse n steps from a held start state
    with s free slots: advance m steps, store, reverse the right part with
    s - 1 slots, then the left part with s slots; with no slot every step is
    recomputed from the start."""
    if n <= 1:
        return 0
    if s == 0:
        return n * (n - 1) // 2
    return min(m + _best(n - m, s - 1) + _best(m, s) for m in range(1, n))


def test_schedule_matches_brute_force_on_small_cases():
    rt = _rt()
    for s in range(0, 7):
        for n in range(0, 90):
            got, opt = rt.revolve_plan(n, s)
            assert got == _best(n, s), (n, s, got)
            assert opt == got


def test_schedule_reaches_the_griewank_walther_optimum():
    rt = _rt()
    for s in range(0, 65):
        c = s + 1
        for n in range(2, 2001):
            t = 0
            while comb(c + t, c) < n:
                t += 1
            want = t * n - comb(c + t, c + 1)  # beta(c + 1, t - 1) = C(c + t, c + 1)
            got, opt = rt.revolve_plan(n, s)
            assert got == want == opt, (n, s, got, want)


def test_large_configuration_and_bad_arguments():
    """58,300 steps with 791 free slots (the 1024x3072, T = 6 case under a
    40 GB cap): two advances per step, t n - beta(793, 1)."""
    rt = _rt()
    got, opt = rt.revolve_plan(58300, 791)
    assert got == opt == 2 * 58300 - 794
    with pytest.raises(rt.RtError):
        rt.revolve_plan(-1, 3)
