"""The kernels' remainder by a 64-bit reciprocal (q = floor(y mul / 2^64) with
mul = floor(2^64 / d), then one conditional subtraction) restated in Python
integers: it equals y mod d for every divisor kind the filter uses (block
counts up to 2^40 and the ranges 481..511 of distinct bit selection) and for
dividends at the edges of the 64-bit range."""
import random

M64 = (1 << 64) - 1


def mod_mul_for(d):
    return M64 // d + (1 if M64 % d == d - 1 else 0)


def mod_fast(y, d, mul):
    q = (y * mul) >> 64
    r = (y - q * d) & M64
    return r - d if r >= d else r


def test_reciprocal_is_floor():
    for d in list(range(2, 2000)) + [3 << 30, (1 << 32) + 1, (1 << 40) - 3, M64]:
        assert mod_mul_for(d) == (1 << 64) // d


def test_remainder_is_exact():
    rng = random.Random(7)
    divisors = list(range(2, 600)) + [481 + i for i in range(31)] + \
        [rng.randrange(3, 1 << 40) for _ in range(400)] + [(1 << 32) - 1, (1 << 32) + 1, 6250, 2075, 9022]
    edges = [0, 1, M64, M64 - 1, 1 << 63, (1 << 63) - 1, 1 << 32]
    for d in divisors:
        mul = mod_mul_for(d)
        ys = edges + [rng.getrandbits(64) for _ in range(200)] + [d - 1, d, d + 1, (M64 // d) * d,
                                                                   (M64 // d) * d - 1]
        for y in ys:
            y &= M64
            assert mod_fast(y, d, mul) == y % d, (y, d)
