"""Host check of the error bounds behind the mixed path's tiers (CPU only).

The emulated-FP64 tile product slices every operand row x (K = 128 entries, scaled by 2^e with
2^(e-1) <= max|x| < 2^e) into the integer F = floor(|x| 2^(55-e)) < 2^55, written as 7 balanced
8-bit digits F = sum_p d_p 2^(48-8p) (chunks from the least significant up; a chunk of 128 or
more becomes chunk - 256 with a carry, so |d_p| <= 128), with the sign of x on every digit:
x ~ 2^e sum_p d_p 2^(-7-8p).  A product over K keeps the digit products with p + q <= np - 1 for
np = 7, 3 or 1 planes.  The mixed path picks np per task from e = ea + eb (the largest row
exponents of its A and B tiles) and tau = tol sigma^2, l2 = floor(log2 tau):
    skipped  when e < l2 - 7    (every entry is below 128 2^e <= tau / 2),
    1 plane  when e < l2 - 1    (error at most 2^e),
    3 planes when e < l2 + 13   (error at most 2^(e-16)),
    7 planes otherwise          (error at most K 2^-54 2^e: FP64-class),
so every task's product stays within tau / 2.  This test restates the slicing from that
definition, forms the tiered products in exact integer arithmetic, and checks each bound against
the exact product of the FP64 inputs (Python fractions), on random rows of mixed magnitudes and
on rows built to maximise the dropped digits."""
import math
from fractions import Fraction

import numpy as np
import pytest

K = 128
S = 7


def row_exponent(x):
    m = float(np.max(np.abs(x)))
    if m == 0.0:
        return 0
    return math.frexp(m)[1]            # 2^(e-1) <= m < 2^e


def slice_row(x):
    """Digits d[p][k] (Python ints) and the row exponent e, from the definition."""
    e = row_exponent(x)
    digits = [[0] * len(x) for _ in range(S)]
    for k, v in enumerate(x):
        F = math.floor(Fraction(abs(float(v))) * Fraction(2) ** (55 - e))
        assert 0 <= F < 2 ** 55
        carry = 0
        for p in range(S - 1, -1, -1):
            d = ((F >> (48 - 8 * p)) & 255) + carry
            carry = 1 if (p > 0 and d >= 128) else 0
            d -= 256 * carry
            assert -128 <= d <= 128
            digits[p][k] = -d if v < 0 else d
    return digits, e


def tiered_product(da, ea, db, eb, planes):
    """sum over p + q <= planes - 1 of the digit products, exactly, as a Fraction."""
    total = 0
    for p in range(S):
        for q in range(S):
            if p + q > planes - 1:
                continue
            dot = sum(a * b for a, b in zip(da[p], db[q]))
            total += Fraction(dot) * Fraction(2) ** (ea + eb - 14 - 8 * (p + q))
    return total


def exact_product(a, b):
    return sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))


BOUND = {1: lambda e: Fraction(2) ** e,
         3: lambda e: Fraction(2) ** (e - 16),
         7: lambda e: K * Fraction(2) ** (e - 54)}


def rows(seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(6):
        scale = 2.0 ** rng.integers(-30, 30)
        x = rng.standard_normal(K) * scale * np.exp(rng.uniform(-8, 0, K))   # mixed magnitudes
        out.append(x)
    # adversarial: every entry just below the row scale with all lower digits large
    e = 3
    base = (2.0 ** e) * (1 - 2.0 ** -9)
    out.append(np.array([base * (1 if k % 2 else -1) for k in range(K)]))
    out.append(np.full(K, (2.0 ** e) * (0.5 + 127.0 / 256.0 + 127.0 / 65536.0)))
    return out


@pytest.mark.parametrize("planes", [1, 3, 7])
def test_tier_error_bounds(planes):
    A = rows(1)
    B = rows(2)
    sliced_a = [slice_row(a) for a in A]
    sliced_b = [slice_row(b) for b in B]
    for a, (da, ea) in zip(A, sliced_a):
        for b, (db, eb) in zip(B, sliced_b):
            err = abs(tiered_product(da, ea, db, eb, planes) - exact_product(a, b))
            assert err <= BOUND[planes](ea + eb), (planes, float(err), float(BOUND[planes](ea + eb)))


def test_skip_bound_and_thresholds_keep_tau_over_two():
    # every entry of a skipped product is below 128 2^e
    A, B = rows(3), rows(4)
    for a in A:
        for b in B:
            e = row_exponent(a) + row_exponent(b)
            assert abs(exact_product(a, b)) < K * Fraction(2) ** e
    # the thresholds: the largest e of each tier keeps its error (or the skipped product) within
    # tau / 2 for every tau with floor(log2 tau) = l2
    for l2 in (-60, -30, -1, 0, 7):
        tau_min = Fraction(2) ** l2
        assert K * Fraction(2) ** (l2 - 8) <= tau_min / 2          # skipped: e <= l2 - 8
        assert BOUND[1](l2 - 2) <= tau_min / 2                      # 1 plane: e <= l2 - 2
        assert BOUND[3](l2 + 12) <= tau_min / 2                     # 3 planes: e <= l2 + 12
