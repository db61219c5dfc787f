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
"""
from __future__ import annotations

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
    """gamma_{2k} = 2k u / (1 - 2k u), u = 2^-24: the first-order relative bound (on the
    scales of ``abs_bound``) of an FP32 evaluation in which every element passes
    through at most k folds or combines, each rounding its product once and its
    fused multiply-add once."""
    u = 2.0 ** -24
    return 2 * k * u / (1.0 - 2 * k * u)
