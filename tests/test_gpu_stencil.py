"""GPU tests of stencil nests with ghost zones (hp_stencil_*): parity with the
oracle within the FP32 bound T * gamma_K * (|C|^T |A|), and bit-identical
results across the things that must not matter (steps fused in shared memory
or run one by one, tensor copies or plain loads, tile and section sizes)."""
import numpy as np
import pytest

from oracle import stencil as so
from paper_2309_01906_gb300 import binding as hb

pytestmark = pytest.mark.gpu


def _data(ny, nx, r, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    A = g.uniform(-1.0, 1.0, (ny, nx)).astype(np.float32)
    c = g.uniform(-0.5, 0.5, (2 * r + 1) ** 2).astype(np.float32)
    return A, c


def _run(A, c, r, T, tile=(0, 0), section=(0, 0), offset=0):
    """Run on device; `offset` floats of padding before the input (misaligns it)."""
    import torch
    ny, nx = A.shape
    buf = torch.zeros(ny * nx + offset + 4, dtype=torch.float32, device="cuda")
    buf[offset:offset + ny * nx] = torch.from_numpy(A.reshape(-1)).cuda()
    out = torch.full((ny * nx + 1,), float("nan"), dtype=torch.float32, device="cuda")
    st = hb.Stencil(ny, nx, r, c.tolist(), T, section=section, tile=tile)
    s = torch.cuda.current_stream().cuda_stream
    st.run(buf.data_ptr() + 4 * offset, out.data_ptr(), s)
    assert st.check(s) == 0
    st.close()
    assert torch.isnan(out[ny * nx]).item()       # nothing written past the array
    return out[:ny * nx].reshape(ny, nx)


def _assert_parity(got, A, c, r, T, what):
    A64, c64 = A.astype(np.float64), c.astype(np.float64)
    ref = so.steps(A64, c64, r, T)
    tol = 1.01 * so.error_bound(r, T) * so.abs_steps(A64, c64, r, T) + 1e-30
    err = np.abs(got.astype(np.float64) - ref)
    assert np.all(err <= tol), f"{what}: max err {err.max():.3e}, worst ratio {(err / tol).max():.3f}"


CASES = [(1, 1, 1, 1), (3, 5, 1, 2), (64, 128, 1, 1), (130, 260, 1, 1), (130, 261, 1, 3), (200, 300, 2, 2),
         (97, 512, 0, 1), (150, 388, 3, 2), (120, 200, 4, 2), (257, 1024, 1, 8), (61, 64, 2, 5), (33, 100, 4, 8)]


@pytest.mark.parametrize("ny,nx,r,T", CASES)
def test_parity_with_the_oracle(ny, nx, r, T):
    A, c = _data(ny, nx, r, ny * 1000 + nx)
    got = _run(A, c, r, T).cpu().numpy()
    _assert_parity(got, A, c, r, T, f"{ny}x{nx} r={r} T={T}")


@pytest.mark.parametrize("ny,nx,r,T", [(130, 260, 1, 4), (200, 300, 2, 3), (70, 72, 4, 2), (3, 5, 1, 8)])
def test_fused_steps_equal_single_steps(ny, nx, r, T):
    import torch
    A, c = _data(ny, nx, r, 7 + T)
    fused = _run(A, c, r, T)
    v = A
    for _ in range(T):
        v = _run(v, c, r, 1).cpu().numpy()
    assert torch.equal(fused.cpu(), torch.from_numpy(v))


@pytest.mark.parametrize("ny,nx,r,T", [(130, 260, 1, 1), (200, 300, 2, 3), (64, 512, 0, 2)])
def test_tensor_copies_equal_plain_loads(ny, nx, r, T):
    import torch
    A, c = _data(ny, nx, r, 11)
    tma = _run(A, c, r, T)                 # nx % 4 == 0 and an aligned base: tensor copies
    plain = _run(A, c, r, T, offset=1)     # base misaligned by 4 bytes: plain loads
    assert torch.equal(tma, plain)


def test_tiles_and_sections_do_not_change_results():
    import torch
    A, c = _data(300, 520, 2, 13)
    ref = _run(A, c, 2, 3)
    for tile, section in [((16, 64), (0, 0)), ((64, 128), (128, 256)), ((8, 4), (16, 8)), ((100, 200), (0, 0))]:
        assert torch.equal(_run(A, c, 2, 3, tile=tile, section=section), ref), (tile, section)


def test_identity_and_shift_are_exact():
    import torch
    A, _ = _data(90, 130, 1, 17)
    ident = np.zeros(9, np.float32)
    ident[4] = 1.0
    assert torch.equal(_run(A, ident, 1, 5).cpu(), torch.from_numpy(A))
    shift = np.zeros(9, np.float32)
    shift[6] = 1.0           # (dy, dx) = (1, -1): out[y][x] = A[y+1][x-1]
    ref = np.zeros_like(A)
    ref[:-1, 1:] = A[1:, :-1]
    assert torch.equal(_run(A, shift, 1, 1).cpu(), torch.from_numpy(ref))


def test_full_size_sampled():
    # the measured configuration: 16384^2, 9-point stencil, 4 steps fused; sampled points
    import torch
    ny = nx = 16384
    r, T = 1, 4
    g = np.random.Generator(np.random.PCG64(19))
    c = g.uniform(-0.5, 0.5, 9).astype(np.float32)
    dA = torch.empty((ny, nx), dtype=torch.float32, device="cuda").uniform_(-1.0, 1.0,
                                                                          generator=torch.Generator("cuda").manual_seed(5))
    out = torch.empty_like(dA)
    st = hb.Stencil(ny, nx, r, c.tolist(), T)
    s = torch.cuda.current_stream().cuda_stream
    st.run(dA.data_ptr(), out.data_ptr(), s)
    assert st.check(s) == 0
    st.close()
    pts = [(0, 0), (0, nx - 1), (ny - 1, 0), (ny - 1, nx - 1), (1, 2), (63, 127), (64, 128), (8191, 8192)]
    pts += [tuple(int(v) for v in g.integers(0, ny, 2)) for _ in range(120)]
    c64 = c.astype(np.float64)
    h = r * T
    for (y, x) in pts:
        y0, y1, x0, x1 = max(0, y - h), min(ny, y + h + 1), max(0, x - h), min(nx, x + h + 1)
        win = dA[y0:y1, x0:x1].cpu().numpy().astype(np.float64)
        # place the window in a zero frame so that `point` sees the true array edges
        full = np.zeros((2 * h + 1, 2 * h + 1))
        full[y0 - (y - h):y1 - (y - h), x0 - (x - h):x1 - (x - h)] = win
        inside_y = (np.arange(y - h, y + h + 1) >= 0) & (np.arange(y - h, y + h + 1) < ny)
        inside_x = (np.arange(x - h, x + h + 1) >= 0) & (np.arange(x - h, x + h + 1) < nx)
        # evaluate on an array that is exactly the in-bounds part of the window
        sub = full[np.ix_(inside_y, inside_x)]
        ref = so.point(sub, c64, r, T, y - y0, x - x0) if sub.size else 0.0
        scale = so.point(np.abs(sub), np.abs(c64), r, T, y - y0, x - x0)
        got = float(out[y, x])
        assert abs(got - ref) <= 1.01 * so.error_bound(r, T) * scale + 1e-30, (y, x, got, ref)
