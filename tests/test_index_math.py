"""Quotients by multiply-high, as the CUDA kernels take them (CPU check).

The tile kernels map a flat work index to (row group, column quad) and the
adjoint kernel maps a flat index to (box, row, column) by
q = floor(x * m / 2^32) with m = floor((2^32 - 1) / n) + 1 instead of a
division.  The claim is exactness whenever n >= 2 and x * n <= 2^32; this
checks it with exact integer arithmetic at the edges of that range and on
random operands, and checks that the bound is needed (outside it the
quotient can be one too large).
"""
import numpy as np

TWO32 = 1 << 32


def mulhi_quotient(x, n):
    m = (TWO32 - 1) // n + 1
    return (x * m) >> 32


def test_small_divisors_exhaustive_prefix():
    for n in range(2, 520):
        x = np.arange(0, 1 << 14, dtype=np.uint64)
        m = np.uint64((TWO32 - 1) // n + 1)
        q = (x * m) >> np.uint64(32)
        assert np.array_equal(q, x // np.uint64(n)), n


def test_edges_of_the_exact_range():
    rng = np.random.default_rng(0)
    divisors = list(range(2, 2000)) + [int(v) for v in rng.integers(2000, 1 << 20, 400)] + [3 * 785, 256 * 785, 65535]
    for n in divisors:
        x_end = TWO32 // n
        xs = {x_end, x_end - 1, x_end - n, max(0, x_end - 2 * n + 1)}
        xs |= {k * n - 1 for k in (1, 2, 3) if k * n - 1 >= 0}
        xs |= {(x_end // n) * n + r for r in (0, n - 1) if (x_end // n) * n + r <= x_end}
        xs |= {int(v) for v in rng.integers(0, x_end + 1, 64)}
        for x in (v for v in xs if 0 <= v <= x_end):
            assert x * n <= TWO32
            assert mulhi_quotient(x, n) == x // n, (x, n)


def test_powers_of_two_exact_everywhere():
    for s in range(1, 31):
        n = 1 << s
        for x in (0, 1, n - 1, n, TWO32 - 1, TWO32 // 3):
            assert mulhi_quotient(x, n) == x // n


def test_bound_is_needed():
    # n = 7: m = ceil(2^32 / 7) = (2^32 + 3) / 7, so x * 3 / 2^32 is added to
    # x / 7; near x = 2^32 that is almost 3, which carries x = 7k + 6 over
    n = 7
    x = (TWO32 - 1) - ((TWO32 - 1) % n) - 1
    assert x % n == n - 1 and x * n > TWO32
    assert mulhi_quotient(x, n) == x // n + 1
