"""Quotients by multiply-high, as the CUDA kernels take them (CPU check).

The tile kernels map a flat work index to (row group, column quad) and the
adjoint kernel maps a flat index to (box, row, column) by
q = floor(x * m / 2^32) with m = floor((2^32 - 1) / n) + 1 instead of a
division.  The claim is exactness whenever n >= 2 and x * n <= 2^32; this
checks it with exact integer arithmetic at the edges of that range and on
random operands, and checks that the bound is needed (outside it the
quotient can be one too large).  It also checks, on a restatement of the
float64 cluster tile's dealing of a layer's work over the CTAs of a cluster,
that every product tile and every constant item of every admitted shape is
computed exactly once, within the CTA's threads.
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


def _deal(total, n_const, n_in, CL=4, NT=256):
    """The float64 cluster tile's dealing of one layer's work, restated: rank
    r takes product tiles r, r + CL, ... (each on `parts` neighbouring lanes)
    and constant items r, r + CL, ... on the lanes past the products."""
    most = (total + CL - 1) // CL
    parts = 1
    while parts < 8 and 2 * parts * most <= NT and n_in >= 8 * parts:
        parts *= 2
    busy = parts * most
    tiles, consts = [], []
    for rank in range(CL):
        my_const = (n_const - rank + CL - 1) // CL
        for tid in range(NT):
            li, part = divmod(tid, parts)
            item = rank + CL * li
            if tid < busy and item < total and part == 0:
                tiles.append(item)
            t = tid - busy
            while t < my_const:
                if t >= 0:
                    consts.append(rank + CL * t)
                t += NT
    return busy, parts, tiles, consts


def test_cluster_dealing_covers_each_item_once():
    # every shape the host admits: (2d + 4) T / 4 column quads x n_max_pad / 8
    # row groups <= 4 x 256 product tiles; T in {2 (odd d), 4}
    for d in range(1, 65):
        for T in ((2, 4) if d % 2 else (4,)):
            for width in (1, 3, 8, 16, 50, 64, 100, 128, 256, 512, 1024):
                G = (width + 7) // 8
                total = G * (2 * d + 4) * T // 4
                if total > 4 * 256:
                    continue
                n_const = ((width + 1) // 2) * T
                busy, parts, tiles, consts = _deal(total, n_const, width)
                assert busy <= 256 and 32 % parts == 0
                assert sorted(tiles) == list(range(total)), (d, T, width)
                assert sorted(consts) == list(range(n_const)), (d, T, width)
