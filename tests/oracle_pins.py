"""Pins of the CPU oracle against things other than itself.

Each pin takes an oracle library handle (so the mutation checks can run the
same battery against deliberately broken builds) and raises AssertionError on a
mismatch.  What pins what:

* closed forms: sums of arithmetic sequences (AFFINE body) and of geometric
  sequences (GEOMETRIC body) over every reduction level, maxima / minima of
  arithmetic sequences, iteration counts of rectangular, triangular and ragged
  spaces;
* library special cases: GEMV and a 4-index contraction (numpy FP64),
  CSR SpMV (scipy.sparse FP64), row max / min (numpy), histogram (np.bincount);
* exactness: FP sums against math.fsum (exactly rounded) on ill-conditioned
  data, integer sums modulo 2^32 against Python integers;
* brute force: every nest of depth <= 3 with extents <= 3 against pure-Python
  loops (oracle/brute.py), both oracle formulations;
* the paper's worked examples (tests/golden/paper_examples.json): structure only,
  since the paper prints no result values;
* the conditioning sums sum|t| and sum t^2 that every FP result carries (they
  set the scale of every FP tolerance): closed forms of integer-valued and
  geometric bodies, numpy / scipy reductions of the FP64 body values, and the
  pure-Python formulation.
"""
from __future__ import annotations

import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np

import oracle
import oracle.brute as brute

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _affine_prefix(N: int, a: int, b: int, m: int) -> int:
    q, s = divmod(N, m)
    return N * a + b * (q * m * (m - 1) // 2 + s * (s - 1) // 2)


def _geom_prefix(N: int, q: Fraction, m: int) -> Fraction:
    def S(k):
        return (1 - q ** k) / (1 - q)
    cnt, s = divmod(N, m)
    return cnt * S(m) + S(s)


def _max_residue(lo: int, hi: int, m: int) -> int:
    if hi - lo >= m or lo % m + (hi - lo - 1) >= m:
        return m - 1
    return (hi - 1) % m


def _min_residue(lo: int, hi: int, m: int) -> int:
    if hi - lo >= m or lo % m + (hi - lo - 1) >= m:
        return 0
    return lo % m


SHAPES = [(7,), (3, 5), (4, 1, 6), (2, 3, 4, 5), (3, 2, 1, 4, 3), (5, 0, 3), (1, 1, 1)]


def pin_affine_sum_every_level(lib):
    a, b, m = -7, 3, 11
    for ext in SHAPES:
        d = len(ext)
        for r in range(d + 1):
            O = int(np.prod(ext[:r])) if r else 1
            R = int(np.prod(ext[r:])) if r < d else 1
            want = [_affine_prefix((o + 1) * R, a, b, m) - _affine_prefix(o * R, a, b, m) for o in range(O)]
            for prec in ("i64", "f32"):
                got = oracle.rect(ext, r, "sum", prec, "affine", params=[a, b, m], lib=lib).values
                assert got.size == O, (ext, r)
                assert [int(v) for v in got] == want, ("affine sum", ext, r, prec)


def pin_affine_max_min_every_level(lib):
    a, b, m = 5, 4, 9
    for ext in SHAPES:
        d = len(ext)
        for r in range(d):
            O = int(np.prod(ext[:r])) if r else 1
            R = int(np.prod(ext[r:]))
            if R == 0:
                continue
            mx = [a + b * _max_residue(o * R, (o + 1) * R, m) for o in range(O)]
            mn = [a + b * _min_residue(o * R, (o + 1) * R, m) for o in range(O)]
            for prec in ("i32", "f32"):
                got = oracle.rect(ext, r, "max", prec, "affine", params=[a, b, m], lib=lib).values
                assert [int(v) for v in got] == mx, ("affine max", ext, r)
                got = oracle.rect(ext, r, "min", prec, "affine", params=[a, b, m], lib=lib).values
                assert [int(v) for v in got] == mn, ("affine min", ext, r)


def pin_geometric_sum_every_level(lib):
    for q, m in ((Fraction(1, 2), 24), (Fraction(3, 4), 13)):
        for ext in SHAPES:
            d = len(ext)
            for r in range(d + 1):
                O = int(np.prod(ext[:r])) if r else 1
                R = int(np.prod(ext[r:])) if r < d else 1
                got = oracle.rect(ext, r, "sum", "f32_comp", "geometric", params=[float(q), m], lib=lib).values
                for o in range(O):
                    want = float(_geom_prefix((o + 1) * R, q, m) - _geom_prefix(o * R, q, m))
                    assert abs(got[o] - want) <= 1e-14 * max(1.0, abs(want)), ("geometric", ext, r, o)


def pin_iteration_counts(lib):
    for ext in SHAPES:
        d = len(ext)
        total = int(np.prod(ext))
        ones = np.ones(max(total, 1), dtype=np.int32)
        for r in range(d + 1):
            R = int(np.prod(ext[r:])) if r < d else 1
            got = oracle.rect(ext, r, "sum", "i64", "load", A=ones, lib=lib).values
            assert all(int(v) == R for v in got), ("count", ext, r)
            assert int(got.sum()) == total
    # triangular ragged space: row i has i + 1 entries -> nnz n(n+1)/2
    n = 300
    lens = np.arange(1, n + 1, dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(lens)])
    nnz = int(off[-1])
    assert nnz == n * (n + 1) // 2
    res = oracle.csr(off, np.zeros(nnz, np.int32), np.ones(nnz, np.float32), np.ones(1, np.float32), lib=lib)
    assert [int(v) for v in res.values] == list(range(1, n + 1))
    h = oracle.hist(np.arange(nnz, dtype=np.int32) % 97, 0, 97, lib=lib)
    assert int(h.values.sum()) == nnz and h.overflow == 0


def pin_library_gemv_and_contraction(lib):
    g = np.random.Generator(np.random.PCG64(101))
    A = g.standard_normal((37, 129)).astype(np.float32)
    x = g.uniform(-1, 1, 129).astype(np.float32)
    got = oracle.rect([37, 129], 1, "sum", "f32", "dot_bcast", A=A, w=x, lib=lib)
    want = A.astype(np.float64) @ x.astype(np.float64)
    tol = 4 * 129 * 2.0 ** -53 * got.abs_sum
    assert np.all(np.abs(got.values - want) <= tol), "gemv"
    B = g.standard_normal((3, 5, 4, 33)).astype(np.float32)
    w = g.uniform(-1, 1, (4, 33)).astype(np.float32)
    got = oracle.rect([3, 5, 4, 33], 2, "sum", "f32_comp", "dot_bcast", A=B, w=w, lib=lib)
    want = np.einsum("bijk,jk->bi", B.astype(np.float64), w.astype(np.float64)).ravel()
    tol = 4 * 132 * 2.0 ** -53 * got.abs_sum
    assert np.all(np.abs(got.values - want) <= tol), "einsum"
    # reduction over levels j only of a 3-level nest: w indexed by (j, k) pairs again
    got = oracle.rect([3, 5, 4, 33], 1, "sum", "f32", "dot_bcast", A=B, w=g.uniform(-1, 1, 5 * 4 * 33).astype(np.float32), lib=lib)
    assert got.values.size == 3
    # int GEMV exact
    Ai = g.integers(-100, 101, (16, 64)).astype(np.int32)
    xi = g.integers(-100, 101, 64).astype(np.int32)
    got = oracle.rect([16, 64], 1, "sum", "i32", "dot_bcast", A=Ai, w=xi, lib=lib).values
    assert np.array_equal(got, Ai.astype(np.int64) @ xi.astype(np.int64)), "int gemv"


def pin_library_rowwise_load(lib):
    g = np.random.Generator(np.random.PCG64(102))
    ext = (4, 3, 5, 7)
    A = g.standard_normal(int(np.prod(ext))).astype(np.float32)
    for r in range(len(ext)):
        O = int(np.prod(ext[:r])) if r else 1
        M = A.astype(np.float64).reshape(O, -1)
        s = oracle.rect(ext, r, "sum", "f32", "load", A=A, lib=lib)
        assert np.all(np.abs(s.values - M.sum(axis=1)) <= 1e-13 * s.abs_sum), ("rowsum", r)
        mx = oracle.rect(ext, r, "max", "f32", "load", A=A, lib=lib).values
        mn = oracle.rect(ext, r, "min", "f32", "load", A=A, lib=lib).values
        assert np.array_equal(mx, M.max(axis=1)) and np.array_equal(mn, M.min(axis=1)), ("max/min", r)
    Ai = g.integers(-1000, 1001, int(np.prod(ext))).astype(np.int32)
    for r in range(len(ext)):
        O = int(np.prod(ext[:r])) if r else 1
        M = Ai.astype(np.int64).reshape(O, -1)
        assert np.array_equal(oracle.rect(ext, r, "sum", "i64", "load", A=Ai, lib=lib).values, M.sum(axis=1))
        assert np.array_equal(oracle.rect(ext, r, "max", "i32", "load", A=Ai, lib=lib).values, M.max(axis=1))


def pin_library_spmv_and_hist(lib):
    import scipy.sparse as sp
    g = np.random.Generator(np.random.PCG64(103))
    n_rows, n_cols = 500, 700
    lens = np.minimum(g.zipf(1.5, n_rows), 300)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    nnz = int(off[-1])
    col = g.integers(0, n_cols, nnz).astype(np.int32)
    val = g.standard_normal(nnz).astype(np.float32)
    x = g.standard_normal(n_cols).astype(np.float32)
    got = oracle.csr(off, col, val, x, lib=lib)
    M = sp.csr_matrix((val.astype(np.float64), col, off), shape=(n_rows, n_cols))
    want = M @ x.astype(np.float64)
    assert np.all(np.abs(got.values - want) <= 4 * 300 * 2.0 ** -53 * got.abs_sum), "spmv"
    rows = g.integers(0, n_rows, 50)
    sub = oracle.csr(off, col, val, x, rows=rows, lib=lib)
    assert np.array_equal(sub.values, got.values[rows]), "csr rows"
    h = oracle.hist(col, 4, (n_cols >> 4) + 1, lib=lib)
    assert np.array_equal(h.values, np.bincount(col >> 4, minlength=(n_cols >> 4) + 1)), "hist"
    h = oracle.hist(col, 4, 10, lib=lib)
    assert h.overflow == int(np.sum((col >> 4) >= 10)), "hist outside count"


def pin_exact_sums(lib):
    # ill-conditioned FP sums: exactly rounded reference from math.fsum
    big = np.float32(2.0 ** 60)
    A = np.array([big, 1, -big, 1, 3, big, -1, -big] * 4, dtype=np.float32)
    got = oracle.rect([A.size], 0, "sum", "f32_comp", "load", A=A, lib=lib).values[0]
    assert got == math.fsum(float(v) for v in A), "cancellation"
    g = np.random.Generator(np.random.PCG64(104))
    for n in (1, 2, 17, 1000, 4099):
        a = (g.standard_normal(n) * np.exp2(g.integers(-30, 30, n))).astype(np.float32)
        b = g.standard_normal(n).astype(np.float32)
        got = oracle.rect([n], 0, "sum", "f32", "dot_bcast", A=a, w=b, lib=lib).values[0]
        want = math.fsum(float(x) * float(y) for x, y in zip(a, b))
        assert abs(got - want) <= 2.0 ** -52 * abs(want) + 1e-300, ("fsum", n)
    # 32-bit sums modulo 2^32, 64-bit sums exact
    Ai = np.full(8, 2 ** 30, dtype=np.int32)
    assert int(oracle.rect([8], 0, "sum", "i32", "load", A=Ai, lib=lib).values[0]) == 0
    assert int(oracle.rect([8], 0, "sum", "i64", "load", A=Ai, lib=lib).values[0]) == 2 ** 33
    Ai = g.integers(-2 ** 31, 2 ** 31, 1000).astype(np.int32)
    exact = int(sum(int(v) for v in Ai))
    assert int(oracle.rect([1000], 0, "sum", "i64", "load", A=Ai, lib=lib).values[0]) == exact
    wrapped = ((exact + 2 ** 31) % 2 ** 32) - 2 ** 31
    assert int(oracle.rect([1000], 0, "sum", "i32", "load", A=Ai, lib=lib).values[0]) == wrapped


def pin_empty_levels(lib):
    ident = {("sum", "f32"): 0.0, ("max", "f32"): -math.inf, ("min", "f32"): math.inf,
             ("sum", "i32"): 0, ("max", "i32"): -(2 ** 31), ("min", "i32"): 2 ** 31 - 1,
             ("sum", "i64"): 0, ("max", "i64"): -(2 ** 63), ("min", "i64"): 2 ** 63 - 1}
    for (op, prec), v in ident.items():
        got = oracle.rect([3, 0], 1, op, prec, "affine", params=[1, 1, 5], lib=lib).values
        assert got.size == 3 and all(x == v for x in got), (op, prec)
        got = oracle.rect([0, 4], 1, op, prec, "affine", params=[1, 1, 5], lib=lib).values
        assert got.size == 0


def pin_brute_force_tiny(lib):
    g = np.random.Generator(np.random.PCG64(105))
    for d in (1, 2, 3):
        for ext in itertools.product(range(4), repeat=d):
            total = int(np.prod(ext))
            Af = g.standard_normal(max(total, 1)).astype(np.float32)
            Ai = g.integers(-50, 51, max(total, 1)).astype(np.int32)
            for r in range(d + 1):
                R = int(np.prod(ext[r:])) if r < d else 1
                wf = g.uniform(-1, 1, max(R, 1)).astype(np.float32)
                wi = g.integers(-50, 51, max(R, 1)).astype(np.int32)
                for op in ("sum", "max", "min"):
                    for prec, A, w in (("f32", Af, wf), ("i32", Ai, wi), ("i64", Ai, wi)):
                        want = brute.rect(ext, r, op, prec, "dot_bcast", A=A, w=w)
                        for fn in (oracle.rect, oracle.rect_flat):
                            got = fn(ext, r, op, prec, "dot_bcast", A=A, w=w, lib=lib).values
                            if prec == "f32":
                                ok = all(gv == wv for gv, wv in zip(got, want))
                            else:
                                ok = [int(v) for v in got] == want
                            assert ok and len(got) == len(want), ("brute", ext, r, op, prec, fn.__name__)


def pin_formulations_agree(lib):
    g = np.random.Generator(np.random.PCG64(106))
    for _ in range(12):
        d = int(g.integers(1, 6))
        ext = tuple(int(v) for v in g.integers(1, 7, d))
        total = int(np.prod(ext))
        A = g.standard_normal(total).astype(np.float32)
        r = int(g.integers(0, d + 1))
        R = int(np.prod(ext[r:])) if r < d else 1
        w = g.uniform(-1, 1, R).astype(np.float32)
        a = oracle.rect(ext, r, "sum", "f32", "dot_bcast", A=A, w=w, lib=lib)
        b = oracle.rect_flat(ext, r, "sum", "f32", "dot_bcast", A=A, w=w, lib=lib)
        assert np.array_equal(a.values, b.values) and np.array_equal(a.abs_sum, b.abs_sum), ext
        O = a.values.size
        idx = g.integers(0, O, min(O, 5))
        s = oracle.rect_sampled(ext, r, "sum", "f32", "dot_bcast", idx, A=A, w=w, lib=lib)
        assert np.array_equal(s.values, a.values[idx]), ("sampled", ext, r)


def pin_paper_examples(lib):
    with open(os.path.join(GOLDEN, "paper_examples.json")) as f:
        ex = json.load(f)
    # Sec. 3.6: 32 values over simd(8) lanes, 4 per lane; lane partials sum to the total
    s = ex["simd8_partial_sums"]
    n, lanes = s["elements"], s["lanes"]
    assert n // lanes == s["values_per_lane"]
    A = np.arange(1, n + 1, dtype=np.int32)
    # lane l owns A[l], A[l + lanes], ... (consecutive lanes read consecutive values)
    lane_major = A.reshape(n // lanes, lanes).T.copy()
    lane_sums = oracle.rect([lanes, n // lanes], 1, "sum", "i64", "load", A=lane_major, lib=lib).values
    total = oracle.rect([n], 0, "sum", "i64", "load", A=A, lib=lib).values[0]
    assert lane_sums.size == lanes
    assert [int(v) for v in lane_sums] == [sum(range(l + 1, n + 1, lanes)) for l in range(lanes)]
    assert int(lane_sums.sum()) == int(total) == n * (n + 1) // 2
    # Sec. 3.4: the 128 x 64 nest bound to two parallel levels has 8192 iterations
    b = ex["bind_ancestor_nest"]
    ones = np.ones(b["extents"][0] * b["extents"][1], dtype=np.int32)
    cnt = oracle.rect(b["extents"], 0, "sum", "i64", "load", A=ones, lib=lib).values[0]
    assert int(cnt) == b["iterations"]
    per_row = oracle.rect(b["extents"], 1, "sum", "i64", "load", A=ones, lib=lib).values
    assert per_row.size == b["extents"][0] and all(int(v) == b["extents"][1] for v in per_row)
    # Sec. 4: 1024^2 array over 4 devices; 'to' sections 513 x 513 overlap, 'from' sections partition
    m = ex["ghost_map"]
    N, D = m["array"][0], m["devices"]
    cover = np.zeros((N, N), dtype=np.int32)
    for dev in range(D):
        r0, c0 = (dev // 2) * m["from_offset_step"], (dev % 2) * m["from_offset_step"]
        cover[r0:r0 + m["from_size"], c0:c0 + m["from_size"]] += 1
        t0, u0 = (dev // 2) * m["to_offset_step"], (dev % 2) * m["to_offset_step"]
        assert t0 + m["to_size"] <= N and u0 + m["to_size"] <= N
    assert np.all(cover == 1)


def _affine_power_sums(lo: int, hi: int, a: int, b: int, m: int):
    """Exact sum|t| and sum t^2 of t = a + b (f mod m) over f in [lo, hi), by residue counts."""
    s1 = s2 = 0
    for k in range(m):
        # number of f in [lo, hi) with f mod m == k
        cnt = (hi - 1 - k) // m - (lo - 1 - k) // m if hi > lo else 0
        t = a + b * k
        s1 += cnt * abs(t)
        s2 += cnt * t * t
    return s1, s2


def pin_conditioning_closed_forms(lib):
    """sum|t| and sum t^2 of integer-valued AFFINE bodies are exact integers below
    2^53, so every FP64 partial is exact: compare bit for bit with the closed
    form from residue counts, for every op and every reduction level."""
    for a, b, m in ((-7, 3, 11), (2, 5, 7), (-40, 9, 9)):
        for ext in SHAPES:
            d = len(ext)
            for r in range(d + 1):
                O = int(np.prod(ext[:r])) if r else 1
                R = int(np.prod(ext[r:])) if r < d else 1
                want = [_affine_power_sums(o * R, (o + 1) * R, a, b, m) for o in range(O)]
                for op in ("sum", "max"):
                    for fn in (oracle.rect, oracle.rect_flat):
                        res = fn(ext, r, op, "f32", "affine", params=[a, b, m], lib=lib)
                        assert [int(v) for v in res.abs_sum] == [w[0] for w in want], ("abs_sum", fn.__name__, ext, r, op)
                        assert [int(v) for v in res.sq_sum] == [w[1] for w in want], ("sq_sum", fn.__name__, ext, r, op)
                        assert np.all(res.abs_sum == np.rint(res.abs_sum)) and np.all(res.sq_sum == np.rint(res.sq_sum))
    # geometric q^k with 0 < q < 1: every term positive, so sum|t| equals the
    # geometric closed form and sum t^2 the closed form of the ratio q^2
    q, m = Fraction(1, 2), 24
    for ext in SHAPES:
        d = len(ext)
        for r in range(d + 1):
            O = int(np.prod(ext[:r])) if r else 1
            R = int(np.prod(ext[r:])) if r < d else 1
            res = oracle.rect(ext, r, "sum", "f32_comp", "geometric", params=[float(q), m], lib=lib)
            for o in range(O):
                w1 = float(_geom_prefix((o + 1) * R, q, m) - _geom_prefix(o * R, q, m))
                w2 = float(_geom_prefix((o + 1) * R, q * q, m) - _geom_prefix(o * R, q * q, m))
                assert abs(res.abs_sum[o] - w1) <= 1e-14 * max(w1, 1e-300), ("geom abs_sum", ext, r, o)
                assert abs(res.sq_sum[o] - w2) <= 1e-14 * max(w2, 1e-300), ("geom sq_sum", ext, r, o)


def pin_conditioning_library(lib):
    """sum|t| and sum t^2 against numpy reductions of the FP64 body values (each
    t = A x w is exact in FP64), for every oracle entry that returns them:
    rect, rect_flat and rect_sampled (LOAD and DOT_BCAST, sum and max), and the
    CSR rows against scipy-built per-row values.  A sequential FP64 sum of n
    non-negative terms errs by at most (n-1) u64 relative."""
    g = np.random.Generator(np.random.PCG64(107))
    u = 2.0 ** -53
    for ext, r in (((6, 5, 33), 1), ((4, 3, 7, 9), 2), ((2, 300), 1), ((513,), 0), ((3, 4, 5), 3)):
        d = len(ext)
        O = int(np.prod(ext[:r])) if r else 1
        R = int(np.prod(ext[r:])) if r < d else 1
        A = (g.standard_normal(int(np.prod(ext))) * np.exp2(g.integers(-8, 9, int(np.prod(ext))))).astype(np.float32)
        w = g.uniform(-3, 3, R).astype(np.float32)
        for body in ("load", "dot_bcast"):
            T = A.astype(np.float64).reshape(O, R)
            if body == "dot_bcast":
                T = T * w.astype(np.float64)[None, :]
            want1 = np.abs(T).sum(axis=1)
            want2 = (T * T).sum(axis=1)
            tol = (R + 2) * u
            for op in ("sum", "max"):
                for res in (oracle.rect(ext, r, op, "f32", body, A=A, w=w, lib=lib),
                            oracle.rect_flat(ext, r, op, "f32", body, A=A, w=w, lib=lib)):
                    assert np.all(np.abs(res.abs_sum - want1) <= tol * want1), ("abs_sum", ext, r, body, op)
                    assert np.all(np.abs(res.sq_sum - want2) <= tol * want2), ("sq_sum", ext, r, body, op)
                idx = g.integers(0, O, min(O, 7))
                res = oracle.rect_sampled(ext, r, op, "f32", body, idx, A=A, w=w, lib=lib)
                assert np.all(np.abs(res.abs_sum - want1[idx]) <= tol * want1[idx]), ("sampled abs_sum", ext, r)
                assert np.all(np.abs(res.sq_sum - want2[idx]) <= tol * want2[idx]), ("sampled sq_sum", ext, r)
    # CSR rows: per-row |val x| and (val x)^2 summed by numpy
    n_rows, n_cols = 400, 500
    lens = np.minimum(g.zipf(1.5, n_rows), 200)
    lens[::37] = 0
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    nnz = int(off[-1])
    col = g.integers(0, n_cols, nnz).astype(np.int32)
    val = g.standard_normal(nnz).astype(np.float32)
    x = g.standard_normal(n_cols).astype(np.float32)
    t = val.astype(np.float64) * x.astype(np.float64)[col]
    want1 = np.array([np.abs(t[off[i]:off[i + 1]]).sum() for i in range(n_rows)])
    want2 = np.array([(t[off[i]:off[i + 1]] ** 2).sum() for i in range(n_rows)])
    for op in ("sum", "max"):
        res = oracle.csr(off, col, val, x, op=op, lib=lib)
        assert np.all(np.abs(res.abs_sum - want1) <= 202 * u * want1), ("csr abs_sum", op)
        assert np.all(np.abs(res.sq_sum - want2) <= 202 * u * want2), ("csr sq_sum", op)
        assert np.all(res.abs_sum[lens == 0] == 0) and np.all(res.sq_sum[lens == 0] == 0)
    rows = g.integers(0, n_rows, 40)
    res = oracle.csr(off, col, val, x, rows=rows, lib=lib)
    assert np.array_equal(res.abs_sum, oracle.csr(off, col, val, x, lib=lib).abs_sum[rows]), "csr rows abs_sum"


def pin_conditioning_brute(lib):
    """sum|t| and sum t^2 against the pure-Python formulation (exactly rounded
    sums) on every nest of depth <= 3 with extents <= 3."""
    g = np.random.Generator(np.random.PCG64(108))
    for d in (1, 2, 3):
        for ext in itertools.product(range(4), repeat=d):
            total = int(np.prod(ext))
            A = g.standard_normal(max(total, 1)).astype(np.float32)
            for r in range(d + 1):
                R = int(np.prod(ext[r:])) if r < d else 1
                w = g.uniform(-2, 2, max(R, 1)).astype(np.float32)
                want1, want2 = brute.rect_conditioning(ext, r, "dot_bcast", A=A, w=w)
                for fn in (oracle.rect, oracle.rect_flat):
                    res = fn(ext, r, "sum", "f32", "dot_bcast", A=A, w=w, lib=lib)
                    assert len(res.abs_sum) == len(want1)
                    for got, want in ((res.abs_sum, want1), (res.sq_sum, want2)):
                        assert all(abs(gv - wv) <= 32 * 2.0 ** -53 * wv for gv, wv in zip(got, want)), \
                            ("brute conditioning", ext, r, fn.__name__)


ALL_PINS = [
    pin_affine_sum_every_level,
    pin_affine_max_min_every_level,
    pin_geometric_sum_every_level,
    pin_iteration_counts,
    pin_library_gemv_and_contraction,
    pin_library_rowwise_load,
    pin_library_spmv_and_hist,
    pin_exact_sums,
    pin_empty_levels,
    pin_brute_force_tiny,
    pin_formulations_agree,
    pin_paper_examples,
    pin_conditioning_closed_forms,
    pin_conditioning_library,
    pin_conditioning_brute,
]
