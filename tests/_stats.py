"""Small statistics helpers of the tests (no BP arithmetic)."""
import math


def mcnemar_exact(b: int, c: int) -> float:
    """Two-sided exact McNemar p-value of b against c discordant pairs: under
    equal proportions each discordant pair leans either way with probability
    1/2, so min(b, c) is the lower tail of Binomial(b + c, 1/2)."""
    n = b + c
    if n == 0:
        return 1.0
    tail = sum(math.comb(n, i) for i in range(min(b, c) + 1)) / 2.0 ** n
    return min(1.0, 2.0 * tail)
