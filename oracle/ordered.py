"""Ordered reductions with a non-commutative operator: sequential CPU oracle.

TEST INFRASTRUCTURE ONLY.  The product path never imports this module: only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of
``bench.py`` may use it.  It shares no code with the CUDA library.

What is computed (Sec. 2: a reduction combines on each level the results of
all sibling tasks; OpenMP's reduction clause does not allow non-commutative
user-defined operators, which a hierarchy that combines siblings in order
can).  The operator composes affine maps: iteration x of an output contributes
f_x(y) = a_x * y + b_x, and the output is the composition in iteration order

    F = f_{R-1} o ... o f_1 o f_0,      F(y) = A * y + B,

with A = prod_x a_x and B = sum_x b_x * prod_{z > x} a_z, i.e. B is the last
value of the linear recurrence y_x = a_x * y_{x-1} + b_x started from 0.
Combining two adjacent ranges, the earlier (A1, B1) and the later (A2, B2):
(A2 * A1, A2 * B1 + B2): associative, not commutative; identity (1, 0).

``compose`` folds the maps one by one in FP64 (the definition); ``closed``
evaluates the two sums/products with numpy's cumulative products (a second
formulation); ``compose_exact`` works in exact rationals; ``abs_bound`` gives
|A| and sum |b_x| prod_{z > x} |a_z| (the scale of rounding errors).

Two more non-commutative operators of the same kind:

* 2x2 matrix products in iteration order, M = M_{R-1} ... M_1 M_0 (the later
  matrix on the left), each iteration's matrix stored row-major as 4 values;
  combining adjacent ranges: (earlier E, later L) -> L E; identity I.  The
  affine maps are the special case [[a, b], [0, 1]].  ``mat2_product`` folds
  in FP64, ``mat2_exact`` in rationals, ``mat2_abs`` gives prod |M_x|
  (entrywise absolute values), the scale of rounding errors.
* the last valid value: the value of the last iteration that is not NaN
  (NaN marks "no value"), NaN if there is none; combining: the later range's
  value unless it is NaN.  Exact (values are copied, never computed).
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def combine(earlier, later):
    """Composition of two adjacent ranges: apply `earlier` first."""
    a1, b1 = earlier
    a2, b2 = later
    return (a2 * a1, a2 * b1 + b2)


def compose(a, b):
    """(A, B) of one output: the maps folded one by one in order, FP64."""
    A, B = 1.0, 0.0
    for ax, bx in zip(np.asarray(a, np.float64).tolist(), np.asarray(b, np.float64).tolist()):
        A, B = ax * A, ax * B + bx
    return A, B


def compose_rows(a2d, b2d):
    """Every row of (O, R) arrays: arrays A[O], B[O] in FP64 (vectorised over rows)."""
    a = np.asarray(a2d, np.float64)
    b = np.asarray(b2d, np.float64)
    A = np.ones(a.shape[0])
    B = np.zeros(a.shape[0])
    for x in range(a.shape[1]):
        A = a[:, x] * A
        B = a[:, x] * B + b[:, x]
    return A, B


def closed(a, b):
    """The same (A, B) from A = prod a, B = sum_x b_x prod_{z > x} a_z (suffix products)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if a.size == 0:
        return 1.0, 0.0
    suffix = np.concatenate([np.cumprod(a[::-1])[::-1][1:], [1.0]])   # prod_{z > x} a_z
    return float(np.prod(a)), float(np.sum(b * suffix))


def compose_exact(a, b):
    """Exact rational composition (for small integer or dyadic inputs)."""
    A, B = Fraction(1), Fraction(0)
    for ax, bx in zip(a, b):
        ax, bx = Fraction(ax), Fraction(bx)
        A, B = ax * A, ax * B + bx
    return A, B


def abs_bound(a, b):
    """(|A|, sum |b_x| prod_{z > x} |a_z|) of one output."""
    return closed(np.abs(np.asarray(a, np.float64)), np.abs(np.asarray(b, np.float64)))


def abs_bound_rows(a2d, b2d):
    return compose_rows(np.abs(np.asarray(a2d, np.float64)), np.abs(np.asarray(b2d, np.float64)))


def error_bound(k: int) -> float:
    """gamma_{2k} = 2k u / (1 - 2k u), u = 2^-24: the worst-case relative bound (on the
    scales of ``abs_bound`` / ``mat2_abs_rows``) of an FP32 evaluation that makes k
    combines in all (R maps in any tree: k = R - 1), each rounding twice (a product
    and a fused multiply-add).  For products the relative errors of every combine
    add, whatever the tree's shape (a product of R numbers carries R - 1
    roundings), so k counts all combines, not the depth of the tree."""
    u = 2.0 ** -24
    return 2 * k * u / (1.0 - 2 * k * u)


def prob_bound(k: int, lam: float = 10.0) -> float:
    """lam sqrt(2k) u: the probabilistic bound for the same evaluation, modelling the
    2k rounding errors as independent, mean zero and bounded by u (a Hoeffding bound
    on their weighted sum: it fails with probability below 2 exp(-lam^2 / 2))."""
    return lam * math.sqrt(2 * max(k, 0)) * 2.0 ** -24


# ---------------------------------------------------------------- 2x2 matrix products

def mat2_combine(earlier, later):
    """Adjacent ranges: `earlier` applied first, so the product is later @ earlier."""
    (e00, e01, e10, e11), (l00, l01, l10, l11) = earlier, later
    return (l00 * e00 + l01 * e10, l00 * e01 + l01 * e11, l10 * e00 + l11 * e10, l10 * e01 + l11 * e11)


def mat2_product(m):
    """M_{R-1} ... M_0 of one output, m of shape (R, 4) (row-major entries), FP64,
    folded one iteration at a time in order."""
    M = (1.0, 0.0, 0.0, 1.0)
    for row in np.asarray(m, np.float64).reshape(-1, 4).tolist():
        M = mat2_combine(M, tuple(row))
    return M


def mat2_rows(m3d):
    """Every output of an (O, R, 4) array: (O, 4) in FP64 (vectorised over outputs)."""
    m = np.asarray(m3d, np.float64)
    O = m.shape[0]
    M = np.tile(np.array([1.0, 0.0, 0.0, 1.0]), (O, 1))
    for x in range(m.shape[1]):
        l00, l01, l10, l11 = (m[:, x, i] for i in range(4))
        e00, e01, e10, e11 = (M[:, i].copy() for i in range(4))
        M[:, 0] = l00 * e00 + l01 * e10
        M[:, 1] = l00 * e01 + l01 * e11
        M[:, 2] = l10 * e00 + l11 * e10
        M[:, 3] = l10 * e01 + l11 * e11
    return M


def mat2_exact(m):
    """Exact rational product (small integer or dyadic entries)."""
    M = (Fraction(1), Fraction(0), Fraction(0), Fraction(1))
    for row in m:
        M = mat2_combine(M, tuple(Fraction(v) for v in row))
    return M


def mat2_abs_rows(m3d):
    """prod |M_x| per output: the entrywise scale of the rounding error bound."""
    return mat2_rows(np.abs(np.asarray(m3d, np.float64)))


# ---------------------------------------------------------------- last valid value

def last_valid(v):
    """The last value of v that is not NaN, NaN if there is none (scanning in order)."""
    out = float("nan")
    for x in np.asarray(v, np.float32).tolist():
        if not np.isnan(x):
            out = x
    return out


def last_valid_rows(v2d):
    """Every row of an (O, R) array (float32 results, NaN where a row has no value)."""
    v = np.asarray(v2d, np.float32)
    out = np.full(v.shape[0], np.nan, np.float32)
    for x in range(v.shape[1]):
        col = v[:, x]
        keep = ~np.isnan(col)
        out[keep] = col[keep]
    return out
