"""Pure-Python brute force of the nest semantics, for tiny nests only.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  A third formulation,
written with ``itertools.product`` over the levels and exactly rounded sums
(``math.fsum``) / Python integers, used to pin the C oracle on small inputs.
"""
from __future__ import annotations

import itertools
import math


def _body(body, flat, rflat, A, w, params, is_int):
    if body == "load":
        return int(A[flat]) if is_int else float(A[flat])
    if body == "dot_bcast":
        if is_int:
            return int(A[flat]) * int(w[rflat])
        return float(A[flat]) * float(w[rflat])
    if body == "affine":
        a, b, m = (int(p) for p in params[:3])
        v = a + b * (flat % m)
        return v if is_int else float(v)
    q, m = float(params[0]), int(params[1])
    k = flat % m
    import numpy as np
    return float(np.float32(q ** k))


def rect(extents, red_level, op, prec, body, A=None, w=None, params=None):
    """Return a list with one exact (int) or exactly rounded (float) value per output."""
    is_int = prec in ("i32", "i64")
    d = len(extents)
    out_ext = extents[:red_level]
    red_ext = extents[red_level:]
    results = []
    for oi in itertools.product(*[range(n) for n in out_ext]):
        terms = []
        for ri in itertools.product(*[range(n) for n in red_ext]):
            idx = tuple(oi) + tuple(ri)
            flat = 0
            for l in range(d):
                flat = flat * extents[l] + idx[l]
            rflat = 0
            for l, i in enumerate(ri):
                rflat = rflat * red_ext[l] + i
            t = _body(body, flat, rflat, A, w, params, is_int)
            if prec == "i32":
                t = ((t + 2**31) % 2**32) - 2**31   # 32-bit nests: values modulo 2^32
            terms.append(t)
        if op == "sum":
            v = sum(terms) if is_int else math.fsum(terms)
            if prec == "i32":
                v = ((v + 2**31) % 2**32) - 2**31
        elif op == "max":
            ident = (-(2**31) if prec == "i32" else -(2**63)) if is_int else -math.inf
            v = max(terms, default=ident)
        else:
            ident = ((2**31 - 1) if prec == "i32" else (2**63 - 1)) if is_int else math.inf
            v = min(terms, default=ident)
        results.append(v)
    return results


def rect_conditioning(extents, red_level, body, A=None, w=None, params=None):
    """Per output, the exactly rounded sum|t| and sum t^2 of its FP body values.

    The conditioning of a sum (Sec. 2's recursive reduction reaches the exact
    sum only up to rounding; its error scales with these two quantities).  Each
    t is formed in FP64 as in the C oracle (a product of two FP32 numbers is
    exact there); the sums use ``math.fsum``.
    """
    d = len(extents)
    out_ext = extents[:red_level]
    red_ext = extents[red_level:]
    abs_sums, sq_sums = [], []
    for oi in itertools.product(*[range(n) for n in out_ext]):
        ts = []
        for ri in itertools.product(*[range(n) for n in red_ext]):
            idx = tuple(oi) + tuple(ri)
            flat = 0
            for l in range(d):
                flat = flat * extents[l] + idx[l]
            rflat = 0
            for l, i in enumerate(ri):
                rflat = rflat * red_ext[l] + i
            ts.append(_body(body, flat, rflat, A, w, params, False))
        abs_sums.append(math.fsum(abs(t) for t in ts))
        sq_sums.append(math.fsum(t * t for t in ts))
    return abs_sums, sq_sums
