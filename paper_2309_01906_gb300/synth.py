"""Seeded synthetic inputs for the loop-nest workloads.

This module only draws random numbers: it holds none of the method's
arithmetic, and both the CUDA path and the oracle receive its arrays.  Every
draw is reproducible from (seed, stream) alone and independent of the number of
host threads used: the index space is cut into fixed chunks of ``CHUNK``
elements and chunk c draws from ``PCG64(SeedSequence(seed, spawn_key=(stream, c)))``.

Workload recipes (sizes are parameters so the tests can shrink them):

* GEMV-shaped 2-level nest: A[n][m], x[m] FP32 uniform[-1, 1] (seed 1), or int32
  uniform in [-100, 100] (seed 2).
* 4-level nest b x i x j x k: A FP32 normal(0, 1) (seed 3), w[j][k] FP32
  uniform[-1, 1] (seed 4).
* Ragged CSR nest: row lengths Zipf(1.5) drawn then clipped to [1, 65536]
  (seed 5), col uniform in [0, n_cols) (seed 6), val FP32 normal(0, 1)
  (seed 7), x FP32 normal(0, 1) (seed 8).
* Batched uneven nests (seed 9): depth uniform in {2..5}; total size T
  lognormal(ln 2^16, 2) clipped to [2^8, 2^24]; level weights Dirichlet(1..1)
  and n_l = max(1, round(T ** w_l)); op sum (FP32 normal inputs) or int32 max
  (int32 uniform inputs in [-2^20, 2^20]) with probability 1/2 each; reduction
  level uniform in {0..d-1}.
* Serving arrivals: Poisson process (exponential gaps) at a given rate
  (seed 10).
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

CHUNK = 1 << 22
_THREADS = max(1, min(32, os.cpu_count() or 1))


def _gen(seed: int, stream: int, chunk: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed, spawn_key=(stream, chunk))))


def _fill(n: int, dtype, seed: int, stream: int, draw) -> np.ndarray:
    out = np.empty(n, dtype=dtype)
    n_chunks = (n + CHUNK - 1) // CHUNK

    def work(c):
        lo = c * CHUNK
        hi = min(n, lo + CHUNK)
        draw(_gen(seed, stream, c), out[lo:hi])

    if n_chunks <= 1:
        for c in range(n_chunks):
            work(c)
    else:
        with ThreadPoolExecutor(min(_THREADS, n_chunks)) as ex:
            list(ex.map(work, range(n_chunks)))
    return out


def uniform_f32(n: int, lo: float, hi: float, seed: int, stream: int = 0) -> np.ndarray:
    def draw(g, o):
        g.random(out=o, dtype=np.float32)
        o *= np.float32(hi - lo)
        o += np.float32(lo)
    return _fill(n, np.float32, seed, stream, draw)


def normal_f32(n: int, seed: int, stream: int = 0) -> np.ndarray:
    def draw(g, o):
        g.standard_normal(out=o, dtype=np.float32)
    return _fill(n, np.float32, seed, stream, draw)


def uniform_i32(n: int, lo: int, hi: int, seed: int, stream: int = 0) -> np.ndarray:
    """Integers uniform in [lo, hi] (both ends included)."""
    def draw(g, o):
        o[:] = g.integers(lo, hi, size=o.size, dtype=np.int32, endpoint=True)
    return _fill(n, np.int32, seed, stream, draw)


# ----------------------------------------------------------------------------
# workload recipes

def gemv_f32(n: int = 1024, m: int = 1024, seed: int = 1):
    """A[n][m], x[m] FP32 uniform[-1, 1]."""
    A = uniform_f32(n * m, -1.0, 1.0, seed, 0).reshape(n, m)
    x = uniform_f32(m, -1.0, 1.0, seed, 1)
    return A, x


def gemv_i32(n: int = 1024, m: int = 1024, seed: int = 2):
    """A[n][m], x[m] int32 uniform in [-100, 100]."""
    A = uniform_i32(n * m, -100, 100, seed, 0).reshape(n, m)
    x = uniform_i32(m, -100, 100, seed, 1)
    return A, x


def nest4_f32(b: int = 64, i: int = 512, j: int = 16, k: int = 1024, seed_a: int = 3, seed_w: int = 4):
    """A[b][i][j][k] FP32 normal(0, 1); w[j][k] FP32 uniform[-1, 1]."""
    A = normal_f32(b * i * j * k, seed_a, 0).reshape(b, i, j, k)
    w = uniform_f32(j * k, -1.0, 1.0, seed_w, 0).reshape(j, k)
    return A, w


def stencil_f32(ny: int = 16384, nx: int = 16384, seed: int = 11) -> np.ndarray:
    """The stencil workload's array: FP32 uniform[-1, 1], row-major ny x nx."""
    return uniform_f32(ny * nx, -1.0, 1.0, seed).reshape(ny, nx)


# 9-point diffusion stencil (weights sum to 1): the stencil workload's coefficients
DIFFUSION9 = [0.025, 0.1, 0.025, 0.1, 0.5, 0.1, 0.025, 0.1, 0.025]


def zipf_lengths(n_rows: int, alpha: float = 1.5, max_len: int = 65536, seed: int = 5) -> np.ndarray:
    """Row lengths Zipf(alpha) drawn, then clipped to [1, max_len]."""
    def draw(g, o):
        o[:] = np.minimum(g.zipf(alpha, size=o.size), max_len)
    return _fill(n_rows, np.int64, seed, 0, draw)


@dataclass
class CSRInputs:
    offsets: np.ndarray   # int64[n_rows + 1]
    col: np.ndarray       # int32[nnz]
    val: np.ndarray       # float32[nnz]
    x: np.ndarray         # float32[n_cols]

    @property
    def n_rows(self) -> int:
        return self.offsets.size - 1

    @property
    def nnz(self) -> int:
        return int(self.offsets[-1])


def csr_zipf(n_rows: int = 1 << 22, n_cols: int = 1 << 22, alpha: float = 1.5, max_len: int = 65536,
             seeds=(5, 6, 7, 8)) -> CSRInputs:
    lens = zipf_lengths(n_rows, alpha, max_len, seeds[0])
    off = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    nnz = int(off[-1])
    col = uniform_i32(nnz, 0, n_cols - 1, seeds[1], 0)
    val = normal_f32(nnz, seeds[2], 0)
    x = normal_f32(n_cols, seeds[3], 0)
    return CSRInputs(off, col, val, x)


def csr_from_lengths(lens, n_cols: int, seeds=(6, 7, 8)) -> CSRInputs:
    """CSR with the given row lengths and random col / val / x."""
    lens = np.asarray(lens, dtype=np.int64)
    off = np.zeros(lens.size + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    nnz = int(off[-1])
    return CSRInputs(off, uniform_i32(nnz, 0, n_cols - 1, seeds[0], 0), normal_f32(nnz, seeds[1], 0),
                     normal_f32(n_cols, seeds[2], 0))


@dataclass
class NestShape:
    extents: tuple
    red_level: int
    op: str          # "sum" (FP32) or "max" (int32)
    prec: str        # "f32_comp" / "f32" for sums, "i32" for max

    @property
    def size(self) -> int:
        return int(np.prod(self.extents))

    @property
    def n_out(self) -> int:
        return int(np.prod(self.extents[: self.red_level])) if self.red_level else 1


def uneven_shapes(n_nests: int = 10000, seed: int = 9, mu: float = float(np.log(2.0 ** 16)),
                  sigma: float = 2.0, t_min: int = 1 << 8, t_max: int = 1 << 24,
                  sum_prec: str = "f32_comp"):
    """Shapes of the batched / served workloads (see the module docstring)."""
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))
    shapes = []
    for _ in range(n_nests):
        d = int(g.integers(2, 6))
        T = float(np.clip(g.lognormal(mu, sigma), t_min, t_max))
        wts = g.dirichlet(np.ones(d))
        ext = tuple(max(1, int(round(T ** float(wl)))) for wl in wts)
        is_sum = bool(g.random() < 0.5)
        r = int(g.integers(0, d))
        shapes.append(NestShape(ext, r, "sum" if is_sum else "max", sum_prec if is_sum else "i32"))
    return shapes


def nest_input(shape: NestShape, index: int, seed: int = 9) -> np.ndarray:
    """The contiguous input of nest `index` (FP32 normal for sums, int32 for max)."""
    if shape.op == "sum":
        return normal_f32(shape.size, seed, 1 + index)
    return uniform_i32(shape.size, -(1 << 20), 1 << 20, seed, 1 + index)


def poisson_arrivals(rate: float = 20000.0, duration: float = 60.0, seed: int = 10) -> np.ndarray:
    """Arrival times (seconds) of a Poisson stream at `rate` requests/s over `duration` s."""
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))
    n_est = int(rate * duration * 1.2 + 100)
    t = np.cumsum(g.exponential(1.0 / rate, size=n_est))
    while t[-1] < duration:
        t = np.concatenate([t, t[-1] + np.cumsum(g.exponential(1.0 / rate, size=n_est))])
    return t[t < duration]
