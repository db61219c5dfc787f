"""Sequential CPU oracle of the hierarchical loop-nest semantics.

TEST INFRASTRUCTURE ONLY.  The product path never imports this package: only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of
``bench.py`` may use it.  It shares no code with the CUDA library; its C file
(``hp_oracle.c``) defines its own codes and is built with gcc by :func:`build`.

Semantics (Sec. 2 recursive reduction over the levels of a nest; Sec. 3.4 loops
bound to parallel levels):

    out[i_0..i_{r-1}] = OP_{i_r} ... OP_{i_{d-1}} body(i_0..i_{d-1})

evaluated in lexicographic order, FP32 inputs widened to FP64 (products exact),
Neumaier-compensated FP64 sums, exact int64 integers (32-bit sums reported
modulo 2^32).  Every FP result comes with ``abs_sum`` = sum|t| and
``sq_sum`` = sum t^2 for per-result error statements.

Names used by the tests: op in {"sum", "max", "min"}; prec in {"f32",
"f32_comp", "i32", "i64"}; body in {"load", "dot_bcast", "affine",
"geometric"}.  Body definitions (flat = row-major index over all levels,
rflat = row-major index over the reduced levels r..d-1):

    load       A[flat]
    dot_bcast  A[flat] * w[rflat]
    affine     a + b * (flat mod m)        params (a, b, m), integers
    geometric  fl32(q ** (flat mod m))     params (q, m), q**k formed in FP64

Stencil nests with ghost zones (Sec. 2 stencils, Sec. 4 map sections) have
their own oracle in ``oracle/stencil.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_OPS = {"sum": 0, "max": 1, "min": 2}
_BODIES = {"load": 0, "dot_bcast": 1, "affine": 3, "geometric": 4}
_INT_BITS = {"f32": 0, "f32_comp": 0, "i32": 32, "i64": 64}

GCC_FLAGS = ["-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def build(out_path: str = _LIB, extra_flags=()) -> str:
    """Compile hp_oracle.c with gcc into a shared library (no GPU needed)."""
    cmd = ["gcc", *GCC_FLAGS, *extra_flags, _SRC, "-o", out_path, "-lm"]
    subprocess.run(cmd, check=True)
    return out_path


_lib_cache: dict = {}


def load(path: str = _LIB) -> ctypes.CDLL:
    """Load (building first if needed) an oracle library; cached per path."""
    if path in _lib_cache:
        return _lib_cache[path]
    if path == _LIB and (not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)):
        build()
    lib = ctypes.CDLL(path)
    p = ctypes.c_void_p
    i64 = ctypes.c_int64
    i32 = ctypes.c_int
    lib.oracle_rect.restype = i64
    lib.oracle_rect.argtypes = [i32, p, i32, i32, i32, i32, p, p, p, p, p, p, p, p, p]
    lib.oracle_rect_sampled.restype = i64
    lib.oracle_rect_sampled.argtypes = [i32, p, i32, i32, i32, i32, p, p, p, p, p, p, i64, p, p, p, p]
    lib.oracle_rect_flat.restype = i64
    lib.oracle_rect_flat.argtypes = [i32, p, i32, i32, i32, i32, p, p, p, p, p, p, p, p, p, p]
    lib.oracle_flat_scratch_per_output.restype = i64
    lib.oracle_csr.restype = i32
    lib.oracle_csr.argtypes = [i64, p, p, p, p, i64, i32, p, i64, p, p, p]
    lib.oracle_hist.restype = i64
    lib.oracle_hist.argtypes = [i64, p, i32, i64, p]
    _lib_cache[path] = lib
    return lib


@dataclass
class Result:
    """Oracle output: values (float64 or int64) and, for FP, conditioning sums."""
    values: np.ndarray
    abs_sum: np.ndarray | None = None
    sq_sum: np.ndarray | None = None
    overflow: int = 0


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _prep(extents, prec, body, A, w, params):
    ext = np.ascontiguousarray(np.asarray(extents, dtype=np.int64))
    int_bits = _INT_BITS[prec]
    Af = wf = Ai = wi = None
    if body in ("load", "dot_bcast"):
        if int_bits:
            Ai = np.ascontiguousarray(A, dtype=np.int32).reshape(-1)
            if body == "dot_bcast":
                wi = np.ascontiguousarray(w, dtype=np.int32).reshape(-1)
        else:
            Af = np.ascontiguousarray(A, dtype=np.float32).reshape(-1)
            if body == "dot_bcast":
                wf = np.ascontiguousarray(w, dtype=np.float32).reshape(-1)
    prm = np.zeros(4, dtype=np.float64)
    if params is not None:
        prm[: len(params)] = np.asarray(params, dtype=np.float64)
    return ext, int_bits, Af, wf, Ai, wi, prm


def _check_sizes(ext, r, body, Af, wf, Ai, wi):
    total = int(np.prod(ext)) if len(ext) else 1
    red = int(np.prod(ext[r:])) if r < len(ext) else 1
    A = Af if Af is not None else Ai
    w = wf if wf is not None else wi
    if body in ("load", "dot_bcast") and (A is None or A.size < total):
        raise ValueError("A is smaller than the iteration space")
    if body == "dot_bcast" and (w is None or w.size < red):
        raise ValueError("w is smaller than the reduced space")


def rect(extents, red_level, op, prec, body, A=None, w=None, params=None, lib=None) -> Result:
    """Evaluate a rectangular nest completely (recursive formulation)."""
    lib = lib or load()
    ext, int_bits, Af, wf, Ai, wi, prm = _prep(extents, prec, body, A, w, params)
    _check_sizes(ext, red_level, body, Af, wf, Ai, wi)
    n_out = int(np.prod(ext[:red_level])) if red_level else 1
    if int_bits:
        out = np.zeros(n_out, dtype=np.int64)
        ov = lib.oracle_rect(len(ext), _ptr(ext), red_level, _OPS[op], _BODIES[body], int_bits,
                             None, None, _ptr(Ai), _ptr(wi), _ptr(prm), None, _ptr(out), None, None)
        if ov < 0:
            raise ValueError("oracle rejected the arguments")
        return Result(out, overflow=int(ov))
    out = np.zeros(n_out, dtype=np.float64)
    ab = np.zeros(n_out, dtype=np.float64)
    sq = np.zeros(n_out, dtype=np.float64)
    ov = lib.oracle_rect(len(ext), _ptr(ext), red_level, _OPS[op], _BODIES[body], 0,
                         _ptr(Af), _ptr(wf), None, None, _ptr(prm), _ptr(out), None, _ptr(ab), _ptr(sq))
    if ov < 0:
        raise ValueError("oracle rejected the arguments")
    return Result(out, ab, sq)


def rect_sampled(extents, red_level, op, prec, body, out_idx, A=None, w=None, params=None, lib=None) -> Result:
    """Evaluate only the outputs listed in out_idx (row-major output indices)."""
    lib = lib or load()
    ext, int_bits, Af, wf, Ai, wi, prm = _prep(extents, prec, body, A, w, params)
    _check_sizes(ext, red_level, body, Af, wf, Ai, wi)
    idx = np.ascontiguousarray(np.asarray(out_idx, dtype=np.int64))
    n = idx.size
    if int_bits:
        out = np.zeros(n, dtype=np.int64)
        ov = lib.oracle_rect_sampled(len(ext), _ptr(ext), red_level, _OPS[op], _BODIES[body], int_bits,
                                     None, None, _ptr(Ai), _ptr(wi), _ptr(prm), _ptr(idx), n,
                                     None, _ptr(out), None, None)
        if ov < 0:
            raise ValueError("oracle rejected the arguments")
        return Result(out, overflow=int(ov))
    out = np.zeros(n, dtype=np.float64)
    ab = np.zeros(n, dtype=np.float64)
    sq = np.zeros(n, dtype=np.float64)
    ov = lib.oracle_rect_sampled(len(ext), _ptr(ext), red_level, _OPS[op], _BODIES[body], 0,
                                 _ptr(Af), _ptr(wf), None, None, _ptr(prm), _ptr(idx), n,
                                 _ptr(out), None, _ptr(ab), _ptr(sq))
    if ov < 0:
        raise ValueError("oracle rejected the arguments")
    return Result(out, ab, sq)


def rect_flat(extents, red_level, op, prec, body, A=None, w=None, params=None, lib=None) -> Result:
    """Evaluate a rectangular nest with the flat mixed-radix formulation."""
    lib = lib or load()
    ext, int_bits, Af, wf, Ai, wi, prm = _prep(extents, prec, body, A, w, params)
    _check_sizes(ext, red_level, body, Af, wf, Ai, wi)
    n_out = int(np.prod(ext[:red_level])) if red_level else 1
    scratch = np.zeros(max(1, n_out) * lib.oracle_flat_scratch_per_output(), dtype=np.uint8)
    if int_bits:
        out = np.zeros(n_out, dtype=np.int64)
        ov = lib.oracle_rect_flat(len(ext), _ptr(ext), red_level, _OPS[op], _BODIES[body], int_bits,
                                  None, None, _ptr(Ai), _ptr(wi), _ptr(prm), None, _ptr(out), None, None,
                                  _ptr(scratch))
        return Result(out, overflow=int(ov))
    out = np.zeros(n_out, dtype=np.float64)
    ab = np.zeros(n_out, dtype=np.float64)
    sq = np.zeros(n_out, dtype=np.float64)
    lib.oracle_rect_flat(len(ext), _ptr(ext), red_level, _OPS[op], _BODIES[body], 0,
                         _ptr(Af), _ptr(wf), None, None, _ptr(prm), _ptr(out), None, _ptr(ab), _ptr(sq),
                         _ptr(scratch))
    return Result(out, ab, sq)


def csr(offsets, col, val, x, op="sum", rows=None, lib=None) -> Result:
    """Ragged CSR nest out[i] = OP_e val[e] * x[col[e]] (all rows or the listed rows)."""
    lib = lib or load()
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    c = np.ascontiguousarray(col, dtype=np.int32)
    v = np.ascontiguousarray(val, dtype=np.float32)
    xx = np.ascontiguousarray(x, dtype=np.float32)
    n_rows = off.size - 1
    rr = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    n = n_rows if rr is None else rr.size
    out = np.zeros(n, dtype=np.float64)
    ab = np.zeros(n, dtype=np.float64)
    sq = np.zeros(n, dtype=np.float64)
    rc = lib.oracle_csr(n_rows, _ptr(off), _ptr(c), _ptr(v), _ptr(xx), xx.size, _OPS[op],
                        _ptr(rr), 0 if rr is None else rr.size, _ptr(out), _ptr(ab), _ptr(sq))
    if rc != 0:
        raise ValueError("oracle rejected the CSR arguments")
    return Result(out, ab, sq)


def hist(col, shift, n_bins, lib=None) -> Result:
    """Count histogram hist[b] = #{e : col[e] >> shift == b}; overflow = entries outside."""
    lib = lib or load()
    c = np.ascontiguousarray(col, dtype=np.int32)
    h = np.zeros(n_bins, dtype=np.int64)
    outside = lib.oracle_hist(c.size, _ptr(c), shift, n_bins, _ptr(h))
    return Result(h, overflow=int(outside))


def batch(nests, lib=None):
    """Evaluate a list of independent nests; each item is a dict of rect() kwargs."""
    return [rect(lib=lib, **n) for n in nests]
