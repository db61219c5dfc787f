"""CPU model of the batched executor's streamed tiles (no GPU).

For plans the planner actually produces, the model replays what the producer
warp copies (16-byte-widened byte range of a tile, cut into ring stages) and
what every consumer thread reads, phase by phase, with the phase rules of the
kernel (block teams: whole steps of about two stages, a short remainder joins
the last phase; lanes teams: as many items as fit half the ring).  It checks
that every read lies in a stage the thread has waited for and its warp has not
released, inside the copied bytes and inside one stage; that each thread folds
exactly fold_item's iterations in fold_item's order; that every stage of a tile
is waited for and released; and that no phase needs more stages than the ring
holds when the other warps are one phase behind (no deadlock).  The ring
constants are read from the kernel header."""
import os
import random
import re

import numpy as np
import pytest

from paper_2309_01906_gb300 import binding as hb
from paper_2309_01906_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _ring_constants():
    src = open(os.path.join(ROOT, "paper_2309_01906_gb300", "csrc", "batch_kernels.cuh")).read()
    sb = int(re.search(r"#define HP_BATCH_STAGE_BYTES (\d+)", src).group(1))
    ns = int(re.search(r"#define HP_BATCH_STAGES (\d+)", src).group(1))
    assert "kLanesWindowBytes = kRingBytes / 2 - 16" in src
    assert "kBlockPhaseBytes = 2 * kStageBytes" in src
    return sb, ns


SB, NS = _ring_constants()
CAP = SB * NS
LANES_WIN = CAP // 2 - 16
BLOCK_PHASE = 2 * SB
WARPS = 8


def _span(d, item):
    G, R, vn0 = d["grid_parts"], d["reduced"], d["levels"][0]["n"]
    o, g = divmod(item, G)
    if G == 1:
        return o * R, 0, vn0
    lo = g * d["tile"]
    return o * R, lo, min(lo + d["tile"], vn0)


def _check_tile(d, gA, item0, count, k0):
    lv = d["levels"][0]
    R, P, V = d["reduced"], lv["slots"], d["vec"]
    b0, l0, _ = _span(d, item0)
    b1, _, h1 = _span(d, item0 + count - 1)
    a0 = (gA + 4 * (b0 + l0)) & ~15
    a1 = (gA + 4 * (b1 + h1) + 15) & ~15
    nst = (a1 - a0 + SB - 1) // SB
    copied = {k0 + i: (a0 + i * SB, min(SB, a1 - a0 - i * SB)) for i in range(nst)}
    for src, n in copied.values():
        assert src % 16 == 0 and n % 16 == 0 and 0 < n <= SB
    stage = lambda e: k0 + (4 * e + gA - a0) // SB
    ready, rel = [k0] * WARPS, [k0] * WARPS

    def wait(e_hi):
        last = stage(e_hi - 1)
        assert last < k0 + nst
        assert last - min(rel) < NS, "a phase needs more stages than the ring holds"
        for w in range(WARPS):
            ready[w] = max(ready[w], last + 1)

    def release(e_end):
        lim = stage(e_end)
        assert lim <= k0 + nst
        for w in range(WARPS):
            rel[w] = max(rel[w], lim)

    def read(w, e):
        st = stage(e)
        assert rel[w] <= st < ready[w], "read outside the live stages"
        src, n = copied[st]
        assert src <= gA + 4 * e and gA + 4 * e + 4 * V <= src + n, "element outside its stage"
        if V == 4:
            assert (4 * e + gA - a0 + (k0 % NS) * SB) % 16 == 0

    if d["team"] == "block":
        W, gl = d["warps"], d["group_lanes"]
        KP = P * max(1, (BLOCK_PHASE // 4) // P)
        for m in range(count):
            base, lo, hi = _span(d, item0 + m)
            seqs = {}
            w0 = lo
            while w0 < hi:
                w1 = min(w0 + KP, hi)
                if hi - w1 < KP // 2:
                    w1 = hi
                wait(base + w1)
                for w in range(W):
                    for lane in range(32):
                        s0 = w * lv["c_warp"] + (lane // gl) * lv["c_group"] + (lane % gl) * lv["c_lane"]
                        for x in range(w0 + s0, w1, P):
                            read(w, base + x)
                            seqs.setdefault((w, lane), []).append(x)
                release(base + w1)
                w0 = w1
            cover = []
            for w in range(W):
                for lane in range(32):
                    s0 = w * lv["c_warp"] + (lane // gl) * lv["c_group"] + (lane % gl) * lv["c_lane"]
                    ref = list(range(lo + s0, hi, P))            # fold_item's sequence
                    assert seqs.get((w, lane), []) == ref
                    for x in ref:
                        cover.extend(range(x, x + V))
            assert sorted(cover) == list(range(lo, hi))
    else:
        L, gl = d["team_lanes"], d["group_lanes"]
        teams = WARPS * (32 // L)
        fit = LANES_WIN // (4 * R)
        per = (fit // teams) * teams if fit >= teams else max(fit, 1)
        for b in range(0, count, per):
            n = min(per, count - b)
            base, _, hi = _span(d, item0 + b + n - 1)
            wait(base + hi)
            for j in range(n):
                t = j % teams
                base_j, lo, hi_j = _span(d, item0 + b + j)
                cover = []
                for lt in range(L):
                    w = (t * L + lt) // 32
                    s0 = (lt // gl) * lv["c_group"] + (lt % gl) * lv["c_lane"]
                    for x in range(lo + s0, hi_j, P):
                        read(w, base_j + x)
                        cover.extend(range(x, x + V))
                assert sorted(cover) == list(range(lo, hi_j))
            release(base + hi)
    assert all(r == k0 + nst for r in ready), "a stage of the tile was never waited for"
    return nst


def _streams(d):
    if d["team"] == "map" or len(d["levels"]) != 1 or d["levels"][0]["stride"] != 1 or d["reduced"] < 1:
        return False
    return not (d["team"] == "lanes" and 4 * d["reduced"] > LANES_WIN)


def _run(descs, seed):
    rng = random.Random(seed)
    k0, kinds = 0, set()
    for d in descs:
        if not _streams(d):
            continue
        kinds.add((d["team"], d["vec"], d["grid_parts"] > 1, d["team_lanes"]))
        gA = (1 << 20) + (16 * rng.randrange(1000) if d["vec"] == 4 else 4 * rng.randrange(4000))
        i0 = 0
        while i0 < d["items"]:
            c = min(d["items"] - i0, rng.choice([1, 2, 3, 7, 33, 300]))
            k0 += _check_tile(d, gA, i0, c, k0)
            i0 += c
    return kinds


def _describe(ext, r, lm=None):
    n = hb.Nest(list(ext), r, "sum", "f32_comp", "load", level_map=lm)
    d = n.describe()
    n.close()
    return d


def test_planner_maps_of_uneven_nests():
    shapes = synth.uneven_shapes(n_nests=60, seed=11, mu=float(np.log(2.0 ** 12)), sigma=2.0, t_max=1 << 19)
    kinds = _run([_describe(sh.extents, sh.red_level) for sh in shapes], 1)
    assert {k[0] for k in kinds} == {"block", "lanes"}


@pytest.mark.parametrize("O,R", [(3, 5), (40, 64), (7, 256), (100, 200), (9, 1028), (5, 4096), (3, 70000),
                                 (2, 300001), (13, 8188)])
def test_tuner_candidate_maps(O, R):
    descs = []
    for lm in (["grid", "seq"], ["grid", "lane"], ["grid", ("subwarp", 2, 0)], ["grid", ("subwarp", 8, 0)],
               ["grid", "warp"], ["grid", ("cta", 4, 0)], ["grid", ("cta", 8, 0)], ["grid", ("grid", 0, 4096)],
               ["grid", ("grid", 0, 1000)]):
        try:
            descs.append(_describe([O, R], 1, lm))
        except hb.HPError:
            continue
    assert descs
    _run(descs, O * R)
