"""Reading C18 (generated costs): the quotient C_ij = a / divisor is formed
without a division instruction by Markstein's correction step for division
by a rounded reciprocal,

    inv = RN(1 / divisor)            (on the host, IEEE single precision)
    q   = RN(a * inv)
    r   = RN(a - q * divisor)        (one fused multiply-add)
    c   = RN(q + r * inv)            (another),

and is claimed to equal the correctly rounded quotient RN(a / divisor) for
every squared distance of a pixel grid divided by its maximum.  This test
restates the method in exact rational arithmetic (each RN applied once to
the exact value, as an FMA does) and checks the claim on CPU, exhaustively
for several grid sizes and on random single-precision pairs."""
from fractions import Fraction

import numpy as np

f32 = np.float32


def rn32(x: Fraction) -> np.float32:
    """Round-to-nearest-even of an exact rational to single precision."""
    a = f32(float(x))
    best = None
    for c in (a, np.nextafter(a, f32(np.inf)), np.nextafter(a, f32(-np.inf))):
        d = abs(Fraction(float(c)) - x)
        if best is None or d < best[0] or (d == best[0] and int(np.float32(c).view(np.uint32)) % 2 == 0):
            best = (d, c)
    return f32(best[1])


def markstein_quotient(a: np.float32, div: np.float32) -> np.float32:
    inv = f32(1.0) / div                        # IEEE single-precision division
    q = rn32(Fraction(float(a)) * Fraction(float(inv)))
    r = rn32(Fraction(float(a)) - Fraction(float(q)) * Fraction(float(div)))
    return rn32(Fraction(float(q)) + Fraction(float(r)) * Fraction(float(inv)))


def correctly_rounded(a: np.float32, div: np.float32) -> np.float32:
    return rn32(Fraction(float(a)) / Fraction(float(div)))


def test_rn32_is_round_to_nearest_even():
    one = Fraction(1)
    ulp = Fraction(2) ** -23
    assert rn32(one + ulp / 2) == f32(1.0)                     # tie to even
    assert rn32(one + 3 * ulp / 2) == f32(1.0) + f32(2.0 ** -22)   # tie to even (upwards)
    assert rn32(one + ulp / 2 + Fraction(1, 2 ** 60)) == f32(1.0) + f32(2.0 ** -23)
    assert rn32(Fraction(1, 3)) == f32(1.0) / f32(3.0)


def test_grid_squared_distances_over_their_maximum_are_correctly_rounded():
    for G in (8, 16, 64, 128):
        div = f32(2 * (G - 1) ** 2)
        sums = sorted({dx * dx + dy * dy for dx in range(G) for dy in range(G)})
        for a in sums:
            a = f32(a)
            assert markstein_quotient(a, div) == correctly_rounded(a, div), (G, a)


def test_random_single_precision_pairs():
    rng = np.random.default_rng(20240727)
    worst = 0
    for _ in range(3000):
        a = f32(rng.random() * 3.0)
        div = f32(rng.uniform(0.5, 8000.0))
        got, want = markstein_quotient(a, div), correctly_rounded(a, div)
        ulps = abs(int(got.view(np.int32)) - int(want.view(np.int32)))
        worst = max(worst, ulps)
    assert worst <= 1          # in general within one unit in the last place
