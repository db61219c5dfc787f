"""GPU parity of ragged (CSR) nests against the oracle, through the C ABI:
SpMV over rows of every length class, the fused and standalone int64
histograms (bit-exact), fixed-class maps, reproducibility, full size."""
import numpy as np
import pytest

import oracle
from paper_2309_01906_gb300 import binding as hb
from paper_2309_01906_gb300 import synth
from tests.hp_testutil import assert_close

pytestmark = pytest.mark.gpu


def gpu_csr(csr, op="sum", prec="f32_comp", fuse=False, shift=10, n_bins=None, level_map=None, repeat=1):
    import torch
    n_cols = csr.x.size
    n_bins = n_bins if n_bins is not None else (n_cols >> shift) + 1
    p = hb.hp_csr_params(csr.nnz, n_cols, shift, 1 if fuse else 0, n_bins)
    n = hb.Nest(csr_rows=csr.n_rows, red_level=1, op=op, prec=prec, body="csr_gather", params=p,
                level_map=level_map)
    d_off = torch.from_numpy(csr.offsets).cuda()
    d_col = torch.from_numpy(csr.col).cuda()
    d_val = torch.from_numpy(csr.val).cuda()
    d_x = torch.from_numpy(csr.x).cuda()
    y = torch.empty(max(csr.n_rows, 1), dtype=torch.float32, device="cuda")
    h = torch.empty(n_bins, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    ins = [d_off.data_ptr(), d_col.data_ptr(), d_val.data_ptr(), d_x.data_ptr(), h.data_ptr()]
    outs = []
    for _ in range(repeat):
        y.fill_(7.0)
        h.fill_(-1)
        n.run(ins, y.data_ptr(), s)
        assert n.check(s) == 0
        torch.cuda.synchronize()
        outs.append((y[:csr.n_rows].cpu().numpy().copy(), h.cpu().numpy().copy() if fuse else None))
    n.close()
    return outs if repeat > 1 else outs[0]


def gpu_hist(col, shift, n_bins):
    import torch
    p = hb.hp_csr_params(col.size, int(col.max()) + 1 if col.size else 1, shift, 0, n_bins)
    n = hb.Nest(csr_rows=1, red_level=0, op="hist", prec="i64", body="csr_gather", params=p)
    d_col = torch.from_numpy(col).cuda()
    h = torch.full((n_bins,), -1, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    n.run([0, d_col.data_ptr(), 0, 0], h.data_ptr(), s)
    assert n.check(s) == 0
    torch.cuda.synchronize()
    n.close()
    return h.cpu().numpy()


BOUNDARY_LENGTHS = [0, 1, 2, 4, 5, 31, 32, 33, 100, 1023, 1024, 1025, 5000, 16383, 16384, 16385, 40000, 65536, 3, 7]


@pytest.mark.parametrize("prec", ["f32_comp", "f32"])
def test_every_length_class(prec):
    csr = synth.csr_from_lengths(BOUNDARY_LENGTHS * 3, n_cols=5000)
    y, h = gpu_csr(csr, prec=prec, fuse=True, shift=4)
    ref = oracle.csr(csr.offsets, csr.col, csr.val, csr.x)
    assert_close(y, ref, prec, "sum", what=f"csr classes {prec}")
    href = oracle.hist(csr.col, 4, (5000 >> 4) + 1)
    assert np.array_equal(h, href.values) and int(h.sum()) == csr.nnz


@pytest.mark.parametrize("op", ["max", "min"])
def test_max_min(op):
    csr = synth.csr_from_lengths(BOUNDARY_LENGTHS, n_cols=3000, seeds=(16, 17, 18))
    y, _ = gpu_csr(csr, op=op, prec="f32")
    ref = oracle.csr(csr.offsets, csr.col, csr.val, csr.x, op=op)
    nonempty = np.diff(csr.offsets) > 0
    got = y[nonempty].astype(np.float64)
    want = ref.values[nonempty].astype(np.float32).astype(np.float64)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("level_map", [["grid", "seq"], ["grid", ("subwarp", 8, 0)], ["grid", "warp"],
                                       ["grid", "cta"], ["grid", "grid"]], ids=str)
def test_fixed_classes(level_map):
    csr = synth.csr_from_lengths([0, 1, 3, 9, 40, 700, 2000, 20000, 5], n_cols=4000, seeds=(26, 27, 28))
    y, h = gpu_csr(csr, prec="f32_comp", fuse=True, shift=3, level_map=level_map)
    ref = oracle.csr(csr.offsets, csr.col, csr.val, csr.x)
    assert_close(y, ref, "f32_comp", "sum", what=f"csr fixed {level_map}")
    assert np.array_equal(h, oracle.hist(csr.col, 3, (4000 >> 3) + 1).values)


def test_zipf_rows_reproducible_and_hist_paths():
    csr = synth.csr_zipf(n_rows=20000, n_cols=1 << 16, seeds=(35, 36, 37, 38))
    runs = gpu_csr(csr, prec="f32_comp", fuse=True, shift=2, repeat=3)
    for y, h in runs[1:]:
        assert np.array_equal(y, runs[0][0]) and np.array_equal(h, runs[0][1])
    ref = oracle.csr(csr.offsets, csr.col, csr.val, csr.x)
    assert_close(runs[0][0], ref, "f32_comp", "sum", what="zipf 20000 rows")
    # 16385 bins: counted straight into global memory (beyond the shared-memory budget)
    assert np.array_equal(runs[0][1], oracle.hist(csr.col, 2, (1 << 14) + 1).values)
    # standalone histogram, shared-memory and global paths
    for shift, bins in ((10, 64), (0, 1 << 16)):
        assert np.array_equal(gpu_hist(csr.col, shift, bins), oracle.hist(csr.col, shift, bins).values)
    # a ragged tail that is not a multiple of the 4-wide loads
    col = csr.col[:1003]
    assert np.array_equal(gpu_hist(col, 4, 5000), oracle.hist(col, 4, 5000).values)


def test_triangular_closed_form():
    n = 3000
    lens = np.arange(1, n + 1)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    nnz = int(off[-1])
    csr = synth.CSRInputs(off, np.zeros(nnz, np.int32), np.ones(nnz, np.float32), np.ones(1, np.float32))
    y, h = gpu_csr(csr, prec="f32_comp", fuse=True, shift=0, n_bins=1)
    assert np.array_equal(y, np.arange(1, n + 1, dtype=np.float32))
    assert int(h[0]) == n * (n + 1) // 2


@pytest.mark.slow
@pytest.mark.parametrize("n_rows", [1 << 20, 1 << 22])
def test_full_size_zipf(n_rows):
    # 2^22 rows, lengths Zipf(1.5) clipped to [1, 65536] (about 1.6e9 entries), col uniform in [0, 2^22)
    csr = synth.csr_zipf(n_rows=n_rows, n_cols=1 << 22)
    assert csr.nnz > 300 * n_rows   # Zipf(1.5) draw-then-clip: about 376 entries per row
    y, h = gpu_csr(csr, prec="f32_comp", fuse=True, shift=10, n_bins=(1 << 22) >> 10)
    g = np.random.Generator(np.random.PCG64(77))
    lens = np.diff(csr.offsets)
    rows = np.concatenate([g.integers(0, n_rows, 3000), np.argsort(lens)[-100:]])
    ref = oracle.csr(csr.offsets, csr.col, csr.val, csr.x, rows=rows)
    assert_close(y[rows], ref, "f32_comp", "sum", what=f"full-size zipf {n_rows} sampled rows")
    href = oracle.hist(csr.col, 10, (1 << 22) >> 10)
    assert np.array_equal(h, href.values) and int(h.sum()) == csr.nnz


def test_gather_probe_reads_what_its_hash_names():
    # the gather-rate probe reads x at murmur3-finalizer indices of (i, seed),
    # scaled to [0, n_x); with small integer values every FP32 sum is exact, so
    # the device sum must equal the host sum of the same reads
    import torch
    from paper_2309_01906_gb300 import binding as hb

    def idx(i, seed, n_x):
        i = np.asarray(i, dtype=np.uint64)
        h = (i & np.uint64(0xffffffff)) ^ (((i >> np.uint64(32)) * np.uint64(0x9e3779b9)) & np.uint64(0xffffffff))
        h = (h ^ np.uint64(seed)) & np.uint64(0xffffffff)
        for sh, mul in ((16, 0x85ebca6b), (13, 0xc2b2ae35)):
            h ^= h >> np.uint64(sh)
            h = (h * np.uint64(mul)) & np.uint64(0xffffffff)
        h ^= h >> np.uint64(16)
        return (h * np.uint64(n_x)) >> np.uint64(32)

    for n_x, n in ((1 << 22, 123457), (1000, 5000), (7, 3)):
        x = (np.arange(n_x) % 8).astype(np.float32)
        dx = torch.from_numpy(x).cuda()
        s = torch.full((1,), 123.0, dtype=torch.float32, device="cuda")
        hb.hp_probe_gather(dx.data_ptr(), n_x, n, 42, s.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        ii = idx(np.arange(n), 42, n_x)
        assert ii.max() < n_x
        assert float(s.item()) == float(x[ii.astype(np.int64)].astype(np.float64).sum())
