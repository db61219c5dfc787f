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
    k = 1023   # combines in all: the relative errors of every combine add
    assert abs(float(parts[0][0]) - A) <= oo.error_bound(k) * Aa
    assert abs(float(parts[0][1]) - B) <= oo.error_bound(k) * Ba
    assert abs(float(parts[0][0]) - A) <= oo.prob_bound(k) * Aa
    assert abs(float(parts[0][1]) - B) <= oo.prob_bound(k) * Ba


def test_product_errors_add_over_every_combine():
    # R equal factors multiplied in a balanced FP32 tree of depth log2 R: every
    # level squares the partial products and doubles the relative error they
    # carry, so the error grows with the number of combines (R - 1), far beyond
    # what a bound on the depth of the tree would allow
    a32 = np.float32(1.0 + 2.0 ** -12 + 3 * 2.0 ** -23)
    R = 1 << 14
    v = [a32] * R
    while len(v) > 1:
        v = [np.float32(v[i] * v[i + 1]) for i in range(0, len(v), 2)]
    exact = math.exp(R * math.log1p(float(a32) - 1.0))
    rel = abs(float(v[0]) - exact) / exact
    assert rel <= oo.error_bound(R - 1)
    assert rel > 100 * oo.error_bound(14)


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


# ---------------------------------------------------------------- 2x2 matrix products

def _fib(n):
    sympy = pytest.importorskip("sympy")
    return int(sympy.fibonacci(n))


@pytest.mark.parametrize("n", [1, 2, 10, 40, 70])
def test_mat2_fibonacci_powers(n):
    # [[1, 1], [1, 0]]^n = [[F(n+1), F(n)], [F(n), F(n-1)]] (exact integers)
    M = oo.mat2_exact([(1, 1, 1, 0)] * n)
    assert M == (_fib(n + 1), _fib(n), _fib(n), _fib(n - 1))
    if n <= 70:   # F(71) < 2^53: the FP64 fold is exact
        assert oo.mat2_product(np.tile([1.0, 1.0, 1.0, 0.0], (n, 1))) == tuple(float(v) for v in M)


def test_mat2_of_affine_maps_equals_their_composition():
    # f(y) = a y + b is the matrix [[a, b], [0, 1]] acting on (y, 1)
    g = np.random.Generator(np.random.PCG64(21))
    a, b = g.uniform(-1.5, 1.5, 300), g.standard_normal(300)
    m = np.stack([a, b, np.zeros(300), np.ones(300)], axis=1)
    M = oo.mat2_product(m)
    A, B = oo.compose(a, b)
    assert M[2] == 0.0 and M[3] == 1.0
    assert M[0] == pytest.approx(A, rel=1e-13) and M[1] == pytest.approx(B, rel=1e-10, abs=1e-12)


def test_mat2_rotations_and_shears():
    g = np.random.Generator(np.random.PCG64(22))
    th = g.uniform(-0.3, 0.3, 500)
    rot = np.stack([np.cos(th), -np.sin(th), np.sin(th), np.cos(th)], axis=1)
    t = th.sum()
    assert np.allclose(oo.mat2_product(rot), [np.cos(t), -np.sin(t), np.sin(t), np.cos(t)], atol=1e-12)
    s = g.integers(-16, 17, 200) / 8.0
    shear = np.stack([np.ones(200), s, np.zeros(200), np.ones(200)], axis=1)
    assert oo.mat2_product(shear) == (1.0, s.sum(), 0.0, 1.0)


def test_mat2_second_order_recurrence():
    # y_x = p_x y_{x-1} + q_x y_{x-2}: the step matrix [[p, q], [1, 0]] maps
    # (y_{x-1}, y_{x-2}) to (y_x, y_{x-1}); run the recurrence directly
    g = np.random.Generator(np.random.PCG64(23))
    p, q = g.integers(-3, 4, 30), g.integers(-3, 4, 30)
    y1, y2 = 2, -1                    # y_{-1}, y_{-2}
    ym1, ym2 = y1, y2
    for x in range(30):
        ym1, ym2 = p[x] * ym1 + q[x] * ym2, ym1
    M = oo.mat2_exact([(int(p[x]), int(q[x]), 1, 0) for x in range(30)])
    assert (M[0] * y1 + M[1] * y2, M[2] * y1 + M[3] * y2) == (ym1, ym2)


def test_mat2_associative_not_commutative():
    g = np.random.Generator(np.random.PCG64(24))
    m = [tuple(int(v) for v in g.integers(-3, 4, 4)) for _ in range(12)]
    whole = oo.mat2_exact(m)
    for k in range(13):
        assert oo.mat2_combine(oo.mat2_exact(m[:k]), oo.mat2_exact(m[k:])) == whole
    assert oo.mat2_exact(m[::-1]) != whole
    assert oo.mat2_exact([]) == (1, 0, 0, 1)


def test_mat2_rows_equal_single_folds():
    g = np.random.Generator(np.random.PCG64(25))
    m = g.standard_normal((5, 40, 4))
    rows = oo.mat2_rows(m)
    for o in range(5):
        assert tuple(rows[o]) == oo.mat2_product(m[o])
    assert np.array_equal(oo.mat2_abs_rows(m), oo.mat2_rows(np.abs(m)))


@pytest.mark.parametrize("mistake", ["swapped", "transposed", "dropped"])
def test_mat2_planted_mistakes_fail_a_pin(mistake, monkeypatch):
    def swapped(e, l):
        (e00, e01, e10, e11), (l00, l01, l10, l11) = e, l
        return (e00 * l00 + e01 * l10, e00 * l01 + e01 * l11, e10 * l00 + e11 * l10, e10 * l01 + e11 * l11)

    def transposed(e, l):
        (e00, e01, e10, e11), (l00, l01, l10, l11) = e, l
        return (l00 * e00 + l10 * e10, l00 * e01 + l10 * e11, l01 * e00 + l11 * e10, l01 * e01 + l11 * e11)

    def dropped(e, l):
        (e00, e01, e10, e11), (l00, l01, l10, l11) = e, l
        return (l00 * e00 + l01 * e10, l00 * e01, l10 * e00 + l11 * e10, l10 * e01 + l11 * e11)

    monkeypatch.setattr(oo, "mat2_combine", {"swapped": swapped, "transposed": transposed, "dropped": dropped}[mistake])
    with pytest.raises(AssertionError):
        test_mat2_second_order_recurrence()
        test_mat2_of_affine_maps_equals_their_composition()


# ---------------------------------------------------------------- last valid value

def _gaps(n, seed, p_nan):
    g = np.random.Generator(np.random.PCG64(seed))
    v = g.standard_normal(n).astype(np.float32)
    v[g.random(n) < p_nan] = np.nan
    return v


@pytest.mark.parametrize("n,p_nan", [(0, 0.5), (1, 0.0), (1, 1.0), (50, 0.5), (1000, 0.99), (1000, 1.0)])
def test_last_valid_is_the_value_at_the_last_non_nan_index(n, p_nan):
    v = _gaps(n, n + 7, p_nan)
    idx = np.nonzero(~np.isnan(v))[0]
    got = oo.last_valid(v)
    if idx.size == 0:
        assert np.isnan(got)
    else:
        assert got == v[idx[-1]]


def test_last_valid_associative_not_commutative():
    v = _gaps(64, 3, 0.6)

    def comb(e, l):
        return e if np.isnan(l) else l

    whole = oo.last_valid(v)
    for k in range(65):
        r = comb(oo.last_valid(v[:k]), oo.last_valid(v[k:]))
        assert r == whole or (np.isnan(r) and np.isnan(whole))
    w = np.array([1.0, np.nan, 2.0], np.float32)
    assert oo.last_valid(w) == 2.0 and oo.last_valid(w[::-1]) == 1.0


def test_last_valid_rows_equal_single_scans():
    v = _gaps(7 * 300, 4, 0.97).reshape(7, 300)
    v[3] = np.nan
    rows = oo.last_valid_rows(v)
    for o in range(7):
        want = oo.last_valid(v[o])
        assert (np.isnan(rows[o]) and np.isnan(want)) or rows[o] == want
