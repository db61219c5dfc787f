"""Shared helpers of the test suite: run a nest through the C ABI on the GPU and
compare with the oracle.

Tolerances (the paper fixes none; these are the readings the design states):
  * integer precisions and MAX / MIN: bit-exact (FP max / min against the
    oracle's exact value rounded to FP32, which rounding's monotonicity makes
    the max / min of the FP32 body values);
  * compensated FP32 sums: |got - ref| <= 1e-6 * max(|ref|, 2^-20 * sum|t|);
  * plain FP32 sums:       |got - ref| <= 1e-5 * max(|ref|, sqrt(sum t^2));
  * both also within the library's own a-priori bound:
        |got - ref| <= bound * sum|t| + 2^-24 * |ref|.
ref, sum|t| and sum t^2 come from the oracle (FP64, Neumaier).
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2309_01906_gb300 import binding as hb

TOL_COMP = 1e-6
TOL_PLAIN = 1e-5


def torch_mod():
    import torch
    return torch


def to_dev(a: np.ndarray):
    torch = torch_mod()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def out_dtype(prec):
    torch = torch_mod()
    return {"f32": torch.float32, "f32_comp": torch.float32, "i32": torch.int32, "i64": torch.int64}[prec]


def make_params(body, params):
    if body == "affine":
        a, b, m = params
        return hb.hp_affine_params(int(a), int(b), int(m))
    if body == "geometric":
        q, m = params
        return hb.hp_geometric_params(float(q), int(m))
    return None


def gpu_rect(extents, red_level, op, prec, body, level_map=None, A=None, w=None, params=None, repeat=1):
    """Run a rectangular nest on cuda:0 through the C ABI; returns (outputs, nest dict)."""
    torch = torch_mod()
    n = hb.Nest(extents, red_level, op, prec, body, level_map=level_map, params=make_params(body, params))
    try:
        ins = []
        if body in ("load", "dot_bcast"):
            ins.append(to_dev(A.reshape(-1)))
            if body == "dot_bcast":
                ins.append(to_dev(w.reshape(-1)))
        O = int(np.prod(extents[:red_level])) if red_level else 1
        out = torch.empty(max(O, 1), dtype=out_dtype(prec), device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        outs = []
        for _ in range(repeat):
            out.fill_(7)
            n.run([t.data_ptr() for t in ins], out.data_ptr(), stream)
            assert n.check(stream) == 0
            torch.cuda.synchronize()
            outs.append(out[:O].cpu().numpy().copy())
        return outs if repeat > 1 else outs[0], n.describe(), n.error_bound()
    finally:
        n.close()


def oracle_rect(extents, red_level, op, prec, body, A=None, w=None, params=None):
    return oracle.rect(extents, red_level, op, prec, body, A=A, w=w, params=params)


def assert_close(got, ref: "oracle.Result", prec: str, op: str, bound: float | None = None, what=""):
    """Element-wise parity of GPU outputs against the oracle (see module docstring)."""
    got = np.asarray(got)
    assert got.shape[0] == ref.values.shape[0], (what, got.shape, ref.values.shape)
    if prec in ("i32", "i64"):
        g = got.astype(np.int64)
        bad = np.nonzero(g != ref.values)[0]
        assert bad.size == 0, f"{what}: {bad.size} integer mismatches, first at {bad[:5]}: got {g[bad[:5]]} want {ref.values[bad[:5]]}"
        return 0.0
    g = got.astype(np.float64)
    r = ref.values
    if op in ("max", "min"):
        # the body value is an FP32 number; rounding to FP32 is monotonic, so the
        # max / min of the rounded values is the oracle's exact max / min rounded
        r = r.astype(np.float32).astype(np.float64)
        bad = np.nonzero(g != r)[0]
        assert bad.size == 0, f"{what}: {bad.size} max/min mismatches at {bad[:5]}: got {g[bad[:5]]} want {r[bad[:5]]}"
        return 0.0
    err = np.abs(g - r)
    if prec == "f32_comp":
        scale = np.maximum(np.abs(r), 2.0 ** -20 * ref.abs_sum)
        tol = TOL_COMP
    else:
        scale = np.maximum(np.abs(r), np.sqrt(ref.sq_sum))
        tol = TOL_PLAIN
    zero = scale == 0
    assert np.all(err[zero] == 0), f"{what}: empty/zero results not exact"
    norm = np.where(zero, 0.0, err / np.where(zero, 1.0, scale))
    worst = int(np.argmax(norm)) if norm.size else 0
    assert norm.size == 0 or norm[worst] <= tol, (
        f"{what}: normalized error {norm[worst]:.3e} > {tol} at {worst}: got {g[worst]!r} ref {r[worst]!r} "
        f"sum|t| {ref.abs_sum[worst]!r}")
    if bound is not None:
        lim = bound * ref.abs_sum + 2.0 ** -24 * np.abs(r)
        over = np.nonzero(err > lim * (1 + 1e-12) + 1e-300)[0]
        assert over.size == 0, f"{what}: {over.size} results exceed the library's a-priori bound"
    return float(norm.max()) if norm.size else 0.0
