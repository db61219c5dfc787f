"""Pins of the ordered-reduction oracle (oracle/ordered.py): the composition of
affine maps in iteration order against a second formulation (suffix
products), exact rationals, closed forms of constant recurrences,
associativity over any split and non-commutativity; planted mistakes (a
swapped combine, a reversed fold, a dropped term) each fail a pin."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import ordered as oo


def _ab(n, seed, lo=0.5, hi=1.0):
    g = np.random.Generator(np.random.PCG64(seed))
    return g.uniform(lo, hi, n), g.standard_normal(n)


@pytest.mark.parametrize("n", [0, 1, 2, 7, 100, 4096])
def test_fold_equals_suffix_products(n):
    a, b = _ab(n, n + 1, -1.2, 1.2)
    A1, B1 = oo.compose(a, b)
    A2, B2 = oo.closed(a, b)
    assert A1 == pytest.approx(A2, rel=1e-12, abs=1e-300)
    assert B1 == pytest.approx(B2, rel=1e-10, abs=1e-12 * oo.abs_bound(a, b)[1] + 1e-300)


def test_rows_equal_single_folds():
    a, b = _ab(6 * 50, 3)
    a, b = a.reshape(6, 50), b.reshape(6, 50)
    A, B = oo.compose_rows(a, b)
    for o in range(6):
        assert (A[o], B[o]) == oo.compose(a[o], b[o])


def test_exact_rationals_on_dyadic_inputs():
    g = np.random.Generator(np.random.PCG64(5))
    a = g.integers(-4, 5, 40) / 4.0           # dyadic: FP64 products and sums are exact at this size
    b = g.integers(-8, 9, 40) / 8.0
    A, B = oo.compose_exact(a.tolist(), b.tolist())
    assert oo.compose(a, b) == (float(A), float(B))


@pytest.mark.parametrize("c,d,n", [(0.5, 3.0, 10), (0.9, -1.0, 37), (1.0, 2.5, 64), (-0.75, 1.0, 9)])
def test_constant_recurrence_closed_form(c, d, n):
    A, B = oo.compose(np.full(n, c), np.full(n, d))
    assert A == pytest.approx(c ** n, rel=1e-13)
    ref = n * d if c == 1.0 else d * (1.0 - c ** n) / (1.0 - c)
    assert B == pytest.approx(ref, rel=1e-12)


def test_associative_over_every_split_and_not_commutative():
    g = np.random.Generator(np.random.PCG64(6))
    a = [Fraction(int(v), 7) for v in g.integers(-9, 10, 24)]
    b = [Fraction(int(v), 5) for v in g.integers(-9, 10, 24)]
    whole = oo.compose_exact(a, b)
    for cut in range(25):
        left, right = oo.compose_exact(a[:cut], b[:cut]), oo.compose_exact(a[cut:], b[cut:])
        assert oo.combine(left, right) == whole
    left, right = oo.compose_exact(a[:11], b[:11]), oo.compose_exact(a[11:], b[11:])
    assert oo.combine(right, left) != whole         # order matters


def test_abs_bound_dominates():
    a, b = _ab(500, 8, -1.1, 1.1)
    A, B = oo.compose(a, b)
    Aa, Ba = oo.abs_bound(a, b)
    assert abs(A) <= Aa * (1 + 1e-12) and abs(B) <= Ba * (1 + 1e-12)
    assert oo.error_bound(10) == pytest.approx(20 * 2.0 ** -24, rel=1e-5)


def test_fp32_tree_within_the_bound():
    # an FP32 evaluation by blocks of 16 and a pairwise tree stays within gamma_{2k}
    a, b = _ab(1024, 9, 0.9, 1.1)
    a32, b32 = a.astype(np.float32), b.astype(np.float32)
    parts = []
    for s in range(0, 1024, 16):
        A, B = np.float32(1), np.float32(0)
        for x in range(s, s + 16):
            A = np.float32(a32[x] * A)
            B = np.float32(np.float64(a32[x]) * np.float64(B) + np.float64(b32[x]))   # one rounding: an FMA
        parts.append((A, B))
    while len(parts) > 1:
        parts = [(np.float32(p2[0] * p1[0]), np.float32(np.float64(p2[0]) * np.float64(p1[1]) + np.float64(p2[1])))
                 for p1, p2 in zip(parts[0::2], parts[1::2])]
    A, B = oo.compose(a32.astype(np.float64), b32.astype(np.float64))
    Aa, Ba = oo.abs_bound(a32.astype(np.float64), b32.astype(np.float64))
    k = 16 + int(math.log2(64))
    assert abs(float(parts[0][0]) - A) <= oo.error_bound(k) * Aa
    assert abs(float(parts[0][1]) - B) <= oo.error_bound(k) * Ba


# ---- planted mistakes
def _mut_swapped_combine(a, b):
    n = len(a) // 2
    return oo.combine(oo.compose(a[n:], b[n:]), oo.compose(a[:n], b[:n]))


def _mut_reversed(a, b):
    return oo.compose(a[::-1], b[::-1])


def _mut_dropped(a, b):
    return oo.compose(a[:-1], b[:-1])


@pytest.mark.parametrize("mut", [_mut_swapped_combine, _mut_reversed, _mut_dropped])
def test_planted_mistakes_fail_a_pin(mut):
    a, b = _ab(33, 10, -1.5, 1.5)
    A, B = oo.closed(a, b)
    Am, Bm = mut(a, b)
    assert not (Am == pytest.approx(A, rel=1e-9) and Bm == pytest.approx(B, rel=1e-9))
