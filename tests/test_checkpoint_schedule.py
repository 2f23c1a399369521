"""Binomial checkpointing: the dynamic-programming schedule's cost (extra forward steps to reverse n
steps with s free snapshots) obeys the known limits and the Griewank-Walther binomial bound."""
import functools
import math


@functools.lru_cache(None)
def cost(n, s):
    if n == 1:
        return 0
    if s == 0:
        return n * (n - 1) // 2
    return min(m + cost(n - m, s - 1) + cost(m, s) for m in range(1, n))


def test_limits():
    for n in range(1, 30):
        assert cost(n, 0) == n * (n - 1) // 2
        assert cost(n, max(n - 1, 0)) == max(n - 1, 0)


def test_binomial_bound():
    # With s snapshots and r repetitions at most C(s + r, s) steps can be reversed while every step is
    # recomputed at most r times: the extra forward steps are at most r * n (Griewank and Walther).
    for s in range(1, 5):
        for r in range(1, 4):
            n = math.comb(s + r, s)
            if n > 40:
                continue
            assert cost(n, s) <= r * n
            assert cost(n + 1, s) > cost(n, s)
