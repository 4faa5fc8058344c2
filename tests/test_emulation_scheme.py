"""Host model of the digit scheme behind the emulated-FP64 products (not part of the paper's
method): each row of op(A) and column of op(B) is scaled by 2^-e (e: the frexp exponent of its
largest magnitude), rounded to a 53-bit integer X, and written as nine balanced base-64 digits
D_1..D_9, X = sum_s D_s 64^(9 - s); the product keeps the digit pairs with s + t <= 12.

Checked here in exact integer arithmetic, with no GPU:
* every digit lies in [-32, 32] (exact in bfloat16), including carry chains that reach the top
  digit, and the digits reconstruct X exactly;
* a digit product is at most 2^10, so 2^14 of them stay within 2^24 (exact in FP32);
* the scheme's own error (53-bit rounding plus the dropped pairs, before any FP64 summation)
  stays within the bound tests/test_gpu_emulated.py holds the kernel to."""

import math
from fractions import Fraction

import numpy as np
import pytest

S, T, BITS = 9, 12, 6


def split_row(x):
    """Exponent e and the (9, len(x)) integer digits of one row, most significant first."""
    amax = float(np.max(np.abs(x))) if len(x) else 0.0
    if amax == 0.0:
        return None, np.zeros((S, len(x)), dtype=np.int64)
    e = math.frexp(amax)[1]
    X = np.array([int(np.rint(math.ldexp(float(v), 53 - e))) for v in x], dtype=np.int64)
    U, sgn = np.abs(X), np.where(X < 0, -1, 1)
    D = np.zeros((S, len(x)), dtype=np.int64)
    carry = np.zeros(len(x), dtype=np.int64)
    for s in range(S - 1, 0, -1):                       # 0-based s: weight 64^(8 - s)
        d = ((U >> (BITS * (S - 1 - s))) & 63) + carry
        carry = (d >= 32).astype(np.int64)
        D[s] = sgn * (d - 64 * carry)
    D[0] = sgn * ((U >> (BITS * (S - 1))) + carry)
    return e, D


def reconstruct(D):
    return sum(int(D[s]) * 64 ** (S - 1 - s) for s in range(S))


def adversarial_values(rng, n):
    """Magnitudes whose 6-bit groups are all 63 or all 32, powers of two, and random values."""
    pool = [1 - 2.0 ** -53, 0.5 + 2.0 ** -53, 2.0 ** -1, 1 - 2.0 ** -30, float(0b100000_100000_100000) / 2 ** 18,
            (2 ** 53 - 1) / 2.0 ** 53, 2.0 ** -40 * (1 - 2.0 ** -53)]
    v = np.array([rng.choice(pool) if rng.random() < 0.5 else rng.standard_normal() for _ in range(n)])
    return v * rng.choice([-1.0, 1.0], n) * 2.0 ** rng.integers(-6, 7, n)


@pytest.mark.parametrize("seed", range(6))
def test_digits_bounded_and_exact(seed):
    rng = np.random.default_rng(seed)
    x = adversarial_values(rng, 400)
    x[0] = (1 - 2.0 ** -53) * 2.0 ** 10         # the row maximum: X = 2^53 - 1, every group 63
    e, D = split_row(x)
    assert np.abs(D).max() <= 32
    assert np.abs(D[0]).max() == 32                # the carry reached the top digit
    for j in range(len(x)):
        X = int(np.rint(math.ldexp(float(x[j]), 53 - e)))
        assert abs(X) < 2 ** 53
        assert reconstruct(D[:, j]) == X
        # the digits stand for the entry to within half a unit of 2^(e - 53)
        assert abs(Fraction(X) * Fraction(2) ** (e - 53) - Fraction(float(x[j]))) <= Fraction(2) ** (e - 54)
    assert (32 * 32) * 2 ** 14 <= 2 ** 24            # the FP32 budget of one accumulator


def emulated_entry(Da, ea, Db, eb):
    """Exact value of the kept digit pairs for one output entry (Fractions)."""
    acc = Fraction(0)
    for s in range(S):
        for t in range(S):
            if (s + 1) + (t + 1) > T:
                continue
            acc += Fraction(int(np.dot(Da[s], Db[t]))) * Fraction(2) ** (-BITS * (s + t + 2))
    return acc * Fraction(2) ** (ea + eb + 2)


@pytest.mark.parametrize("seed,k", [(1, 64), (2, 300), (3, 1000)])
def test_scheme_error_within_the_gpu_test_bound(seed, k):
    """Rounding to 53 bits plus the dropped pairs, in exact arithmetic, against the trunc +
    dropped part of tests/test_gpu_emulated.py's bound: 2^-52 (rowmax sum|b| + colmax sum|a|)
    + 1e-16 k rowmax colmax."""
    rng = np.random.default_rng(seed)
    A = adversarial_values(rng, 3 * k).reshape(3, k)
    B = adversarial_values(rng, 3 * k).reshape(k, 3)
    A[1] *= 1e-7                                     # rows and columns of very different size
    B[:, 2] *= 1e5
    rows = [split_row(A[i]) for i in range(3)]
    cols = [split_row(B[:, j]) for j in range(3)]
    for i in range(3):
        for j in range(3):
            (ea, Da), (eb, Db) = rows[i], cols[j]
            got = emulated_entry(Da, ea, Db, eb)
            exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(A[i], B[:, j]))
            rowmax, colmax = float(np.abs(A[i]).max()), float(np.abs(B[:, j]).max())
            bound = 2.0 ** -52 * (rowmax * float(np.abs(B[:, j]).sum()) + colmax * float(np.abs(A[i]).sum())) \
                + 1e-16 * k * rowmax * colmax
            assert abs(float(got - exact)) <= bound, (i, j, float(got - exact), bound)
