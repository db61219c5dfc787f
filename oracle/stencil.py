"""Stencil nests with ghost zones: sequential CPU oracle.

TEST INFRASTRUCTURE ONLY.  The product path never imports this module: only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of
``bench.py`` may use it.  It shares no code with the CUDA library.

What is computed (Sec. 2: stencils, tiled to any level that has local memory;
Sec. 4: mapped array sections that overlap by a ghost surface).  One step of a
2-D stencil of radius r with coefficients c[(2r+1)][(2r+1)] is the
cross-correlation

    (S v)[y][x] = sum_{dy=-r..r} sum_{dx=-r..r} c[dy+r][dx+r] * v[y+dy][x+dx]

with v = 0 outside the array (a zero ghost surface at the array's edge).  A
nest of T steps computes S^T(A): every step reads the previous step's values,
and values outside the array stay 0 at every step.

``steps`` evaluates it in FP64 with numpy slices; ``brute`` is a pure-Python
restatement for tiny arrays; ``abs_steps`` gives |C|^T |A| (the scale of the
rounding error); ``error_bound`` gives the a-priori relative bound of an FP32
evaluation that rounds every step's values to FP32 and sums the (2r+1)^2 terms
of a point with one rounding each (K roundings):

    |got - exact| <= T * gamma_K * (|C|^T |A|)   (first order; gamma_K = K u / (1 - K u), u = 2^-24)

``sections`` lists the tiles of a tiling with their overlapping ``to`` boxes
(tile + ghost border of width h, clipped to the array) and unique ``from``
boxes (the tile, clipped): the map sections of Sec. 4.
"""
from __future__ import annotations

import numpy as np

U32 = 2.0 ** -24


def _coeffs(coeffs, radius):
    c = np.asarray(coeffs, dtype=np.float64).reshape(2 * radius + 1, 2 * radius + 1)
    return c


def step(v: np.ndarray, coeffs, radius: int) -> np.ndarray:
    """One stencil step in FP64 (zero outside the array)."""
    r = radius
    c = _coeffs(coeffs, r)
    ny, nx = v.shape
    p = np.zeros((ny + 2 * r, nx + 2 * r), dtype=np.float64)
    p[r:r + ny, r:r + nx] = v
    out = np.zeros((ny, nx), dtype=np.float64)
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            out += c[dy + r, dx + r] * p[r + dy:r + dy + ny, r + dx:r + dx + nx]
    return out


def steps(A: np.ndarray, coeffs, radius: int, n_steps: int) -> np.ndarray:
    """S^T(A) in FP64."""
    v = np.asarray(A, dtype=np.float64)
    for _ in range(n_steps):
        v = step(v, coeffs, radius)
    return v


def abs_steps(A: np.ndarray, coeffs, radius: int, n_steps: int) -> np.ndarray:
    """|C|^T |A|: the same steps with absolute coefficients and inputs."""
    return steps(np.abs(np.asarray(A, dtype=np.float64)), np.abs(_coeffs(coeffs, radius)), radius, n_steps)


def point(A: np.ndarray, coeffs, radius: int, n_steps: int, y: int, x: int) -> float:
    """S^T(A)[y][x] from the window of half-width h = r*T around (y, x): a
    point after T steps depends only on inputs within h (Sec. 2's tiling
    argument).  Window points outside the array are 0 at every step, as in
    ``steps``; window points inside it are updated, their own values being
    exact wherever the centre can still see them."""
    r, h = radius, radius * n_steps
    ny, nx = A.shape
    c = _coeffs(coeffs, r)
    ys, xs = np.arange(y - h, y + h + 1), np.arange(x - h, x + h + 1)
    inside = ((ys >= 0) & (ys < ny))[:, None] & ((xs >= 0) & (xs < nx))[None, :]
    v = np.zeros((2 * h + 1, 2 * h + 1))
    v[inside] = np.asarray(A, np.float64)[np.clip(ys, 0, ny - 1)][:, np.clip(xs, 0, nx - 1)][inside]
    for _ in range(n_steps):
        v = step(v, c, r) * inside
    return float(v[h, h])


def brute(A, coeffs, radius: int, n_steps: int):
    """Pure-Python loops (tiny arrays only)."""
    ny, nx = len(A), len(A[0])
    r = radius
    c = [[float(x) for x in row] for row in _coeffs(coeffs, r)]
    v = [[float(A[y][x]) for x in range(nx)] for y in range(ny)]
    for _ in range(n_steps):
        w = [[0.0] * nx for _ in range(ny)]
        for y in range(ny):
            for x in range(nx):
                s = 0.0
                for dy in range(-r, r + 1):
                    for dx in range(-r, r + 1):
                        yy, xx = y + dy, x + dx
                        if 0 <= yy < ny and 0 <= xx < nx:
                            s += c[dy + r][dx + r] * v[yy][xx]
                w[y][x] = s
        v = w
    return v


def error_bound(radius: int, n_steps: int) -> float:
    """T * gamma_K for K = (2r+1)^2 roundings per point and step."""
    K = (2 * radius + 1) ** 2
    return n_steps * K * U32 / (1.0 - K * U32)


def sections(ny: int, nx: int, tile_y: int, tile_x: int, halo_y: int, halo_x: int):
    """Tiles in row-major order: ((y0, y1), (x0, x1)) boxes of the ``to``
    section (tile plus ghost border, clipped to the array) and of the ``from``
    section (the tile, clipped)."""
    out = []
    for ty in range(0, ny, tile_y):
        for tx in range(0, nx, tile_x):
            to = ((max(0, ty - halo_y), min(ny, ty + tile_y + halo_y)),
                  (max(0, tx - halo_x), min(nx, tx + tile_x + halo_x)))
            fr = ((ty, min(ny, ty + tile_y)), (tx, min(nx, tx + tile_x)))
            out.append({"to": to, "from": fr})
    return out
