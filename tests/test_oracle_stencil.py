"""Pins of the stencil oracle (oracle/stencil.py) against what the mathematics
and the paper fix, on the CPU: a library routine (scipy's correlate with a
zero boundary), pure-Python brute force, the identity and shift stencils,
linearity, conservation away from the edges, the first-order error bound on a
simulated FP32 evaluation, and the map sections of the paper's example (Sec. 4).
Plausible mistakes planted in a copy of the oracle (transposed coefficients, a
sign, a wrapping boundary, a stale step) each fail one of these pins."""
import json
import os

import numpy as np
import pytest

from oracle import stencil as so

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_examples.json")


def _rand(shape, seed):
    return np.random.Generator(np.random.PCG64(seed)).uniform(-1.0, 1.0, shape)


def _coeffs(r, seed):
    return np.random.Generator(np.random.PCG64(seed)).uniform(-1.0, 1.0, (2 * r + 1, 2 * r + 1))


@pytest.mark.parametrize("r", [0, 1, 2, 4])
def test_one_step_is_scipy_correlate_with_zero_boundary(r):
    ndimage = pytest.importorskip("scipy.ndimage")
    A, c = _rand((37, 53), 1 + r), _coeffs(r, 2 + r)
    ref = ndimage.correlate(A, c, mode="constant", cval=0.0)
    assert np.allclose(so.step(A, c, r), ref, rtol=0, atol=1e-12)


def test_steps_compose_scipy_correlate():
    ndimage = pytest.importorskip("scipy.ndimage")
    A, c = _rand((20, 31), 3), _coeffs(1, 4)
    ref = A
    for _ in range(4):
        ref = ndimage.correlate(ref, c, mode="constant", cval=0.0)
    assert np.allclose(so.steps(A, c, 1, 4), ref, rtol=0, atol=1e-11)


@pytest.mark.parametrize("ny,nx,r,T", [(1, 1, 1, 1), (3, 4, 1, 2), (5, 2, 2, 1), (6, 6, 2, 3), (4, 7, 0, 2)])
def test_brute_force_tiny(ny, nx, r, T):
    A, c = _rand((ny, nx), ny * 10 + nx), _coeffs(r, r + 7)
    got = so.steps(A, c, r, T)
    ref = np.array(so.brute(A.tolist(), c, r, T))
    assert np.allclose(got, ref, rtol=0, atol=1e-12)


def test_identity_and_shift_stencils_are_exact():
    A = _rand((9, 12), 5)
    ident = np.zeros((3, 3))
    ident[1, 1] = 1.0
    assert np.array_equal(so.steps(A, ident, 1, 3), A)
    # c[dy+r][dx+r] = 1 at (dy, dx) = (1, -1): out[y][x] = A[y+1][x-1], zero where that falls outside
    shift = np.zeros((3, 3))
    shift[2, 0] = 1.0
    ref = np.zeros_like(A)
    ref[:-1, 1:] = A[1:, :-1]
    assert np.array_equal(so.steps(A, shift, 1, 1), ref)
    # two steps shift twice
    ref2 = np.zeros_like(A)
    ref2[:-2, 2:] = A[2:, :-2]
    assert np.array_equal(so.steps(A, shift, 1, 2), ref2)


def test_linearity():
    A, B, c = _rand((15, 16), 6), _rand((15, 16), 7), _coeffs(2, 8)
    lhs = so.steps(2.5 * A - 0.5 * B, c, 2, 3)
    rhs = 2.5 * so.steps(A, c, 2, 3) - 0.5 * so.steps(B, c, 2, 3)
    assert np.allclose(lhs, rhs, rtol=0, atol=1e-10)


def test_constant_field_is_conserved_away_from_the_edges():
    # coefficients summing to 1 keep a constant field constant wherever the
    # T-step domain of dependence stays inside the array
    c = np.array([[0.05, 0.1, 0.05], [0.1, 0.4, 0.1], [0.05, 0.1, 0.05]])
    A = np.full((20, 24), 3.0)
    T = 3
    out = so.steps(A, c, 1, T)
    assert np.allclose(out[T:-T, T:-T], 3.0, rtol=0, atol=1e-13)
    assert out[0, 0] < 3.0 - 0.5      # the zero ghost surface pulls the corner down


@pytest.mark.parametrize("r,T", [(1, 1), (1, 3), (2, 2), (0, 2)])
def test_point_equals_the_full_evaluation(r, T):
    A, c = _rand((13, 17), 30 + r), _coeffs(r, 31 + T)
    full = so.steps(A, c, r, T)
    for y in range(13):
        for x in range(17):
            assert so.point(A, c, r, T, y, x) == pytest.approx(full[y, x], abs=1e-12)


def test_abs_steps_bounds_the_result():
    A, c = _rand((18, 21), 9), _coeffs(1, 10)
    assert np.all(np.abs(so.steps(A, c, 1, 3)) <= so.abs_steps(A, c, 1, 3) + 1e-15)


def _fp32_steps(A, c, r, T):
    """An FP32 evaluation that rounds after every multiply-add (twice per term:
    a stricter rounding than one FMA) and stores every step in FP32."""
    v = A.astype(np.float32)
    c32 = c.astype(np.float32)
    ny, nx = v.shape
    for _ in range(T):
        p = np.zeros((ny + 2 * r, nx + 2 * r), np.float32)
        p[r:r + ny, r:r + nx] = v
        acc = np.zeros((ny, nx), np.float32)
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                acc = (acc + (c32[dy + r, dx + r] * p[r + dy:r + dy + ny, r + dx:r + dx + nx]).astype(np.float32)
                       ).astype(np.float32)
        v = acc
    return v


@pytest.mark.parametrize("r,T", [(1, 1), (1, 4), (2, 3)])
def test_error_bound_holds_for_an_fp32_evaluation(r, T):
    # rounding twice per term gives at most 2K roundings per point: the bound with 2K must hold
    A = _rand((40, 40), 11 + r).astype(np.float32).astype(np.float64)
    c = _coeffs(r, 12 + T).astype(np.float32).astype(np.float64)
    got = _fp32_steps(A, c, r, T).astype(np.float64)
    ref = so.steps(A, c, r, T)
    scale = so.abs_steps(A, c, r, T)
    assert np.all(np.abs(got - ref) <= 2 * so.error_bound(r, T) * 1.01 * scale + 1e-30)
    assert so.error_bound(r, T) == pytest.approx(T * (2 * r + 1) ** 2 * 2.0 ** -24, rel=1e-5)


def test_paper_map_sections():
    # Sec. 4: A[1024][1024] over 4 devices; 'to' sections A[(d/2)*511:513][(d%2)*511:513]
    # (overlapping by the ghost surface), 'from' sections A[(d/2)*512:512][(d%2)*512:512]
    ex = json.load(open(GOLDEN))["ghost_map"]
    n = ex["array"][0]
    secs = so.sections(n, n, ex["from_size"], ex["from_size"], 1, 1)
    assert len(secs) == ex["devices"]
    for d, s in enumerate(secs):
        (ty0, ty1), (tx0, tx1) = s["to"]
        (fy0, fy1), (fx0, fx1) = s["from"]
        assert (ty0, ty1 - ty0) == ((d // 2) * ex["to_offset_step"], ex["to_size"])
        assert (tx0, tx1 - tx0) == ((d % 2) * ex["to_offset_step"], ex["to_size"])
        assert (fy0, fy1 - fy0) == ((d // 2) * ex["from_offset_step"], ex["from_size"])
        assert (fx0, fx1 - fx0) == ((d % 2) * ex["from_offset_step"], ex["from_size"])
    # 'from' sections partition the array; 'to' sections cover each tile's domain of dependence
    cover = np.zeros((n, n), np.int32)
    for s in secs:
        (fy0, fy1), (fx0, fx1) = s["from"]
        cover[fy0:fy1, fx0:fx1] += 1
    assert np.all(cover == 1)


# ---- planted mistakes: each variant must fail one of the pins above
def _mut_transposed(A, c, r, T):
    return so.steps(A, np.asarray(c).reshape(2 * r + 1, -1).T, r, T)


def _mut_sign(A, c, r, T):
    cc = np.asarray(c, dtype=np.float64).reshape(2 * r + 1, -1).copy()
    cc[0, 0] = -cc[0, 0]
    return so.steps(A, cc, r, T)


def _mut_wrap(A, c, r, T):
    v = np.asarray(A, np.float64)
    cc = np.asarray(c, dtype=np.float64).reshape(2 * r + 1, -1)
    for _ in range(T):
        out = np.zeros_like(v)
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                out += cc[dy + r, dx + r] * np.roll(np.roll(v, -dy, 0), -dx, 1)
        v = out
    return v


def _mut_stale(A, c, r, T):
    # every step reads the input instead of the previous step
    v = np.asarray(A, np.float64)
    out = v
    for _ in range(T):
        out = so.step(v, c, r)
    return out


@pytest.mark.parametrize("mut", [_mut_transposed, _mut_sign, _mut_wrap, _mut_stale])
def test_planted_mistakes_fail_a_pin(mut):
    A = _rand((6, 7), 21)
    c = _coeffs(1, 22)
    ref = np.array(so.brute(A.tolist(), c, 1, 2))
    assert not np.allclose(mut(A, c, 1, 2), ref, rtol=0, atol=1e-9)
