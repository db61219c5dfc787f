"""GPU tests of the serving loop: continuous batching under a memory budget.

A request's result must be the same alone and in a mix of other requests
(bit for bit: same plan, same reduction tree) and equal hp_nest_run's; the
budget and slot limits must hold at every moment; the plain per-request mode
must give the same results.  The resident mode (a persistent kernel fed
through mapped host memory) is held to the same: bit-identical to hp_nest_run
alone and in a mix, for FP32 and int32, across instance turnovers and idle
restarts, with grid-split and thousand-tile requests, within budget and
slots."""
import time

import numpy as np
import pytest

from paper_2309_01906_gb300 import binding as hb
from paper_2309_01906_gb300 import synth
from tests.hp_testutil import assert_close, oracle_rect

pytestmark = pytest.mark.gpu


def _pool(n_shapes, seed=501, t_max=1 << 18):
    """Nests of the batched-workload distribution with device inputs (FP32 compensated sums)."""
    import torch
    shapes = synth.uneven_shapes(n_nests=n_shapes, seed=seed, mu=float(np.log(2.0 ** 12)), sigma=1.5,
                                 t_max=t_max, sum_prec="f32_comp")
    pool = []
    for i, sh in enumerate(shapes):
        op, prec = ("sum", "f32_comp") if sh.op == "sum" else ("max", "i32")
        A = synth.nest_input(sh, i, seed)
        nest = hb.Nest(list(sh.extents), sh.red_level, op, prec, "load")
        pool.append(dict(nest=nest, A=A, dA=torch.from_numpy(A).cuda(), shape=sh, op=op, prec=prec,
                         O=max(sh.n_out, 1), dt=torch.float32 if prec == "f32_comp" else torch.int32))
    return pool


def _serve(server, items):
    """Submit (pool item, output tensor) pairs, wait for all; returns tickets.
    The outputs' fills on torch's stream finish before submission (the server
    orders its work after nothing on the caller's streams)."""
    import torch
    torch.cuda.current_stream().synchronize()
    tickets = [hb.hp_serve_submit(server, it["nest"].handle, [it["dA"].data_ptr()], out.data_ptr())
               for it, out in items]
    for t in tickets:
        assert hb.hp_serve_poll(server, t, -1) == hb.HP_OK
    return tickets


def test_same_result_alone_and_in_the_mix():
    import torch
    pool = _pool(64)
    server = hb.hp_serve_create(8 << 30, 256, 4)
    try:
        s = torch.cuda.current_stream().cuda_stream
        for probe in (pool[0], pool[7], pool[21], pool[40]):
            alone = torch.full((probe["O"],), 3, dtype=probe["dt"], device="cuda")
            _serve(server, [(probe, alone)])
            mixed = torch.full((probe["O"],), 5, dtype=probe["dt"], device="cuda")
            items = [(it, torch.empty(it["O"], dtype=it["dt"], device="cuda")) for it in pool]
            items.insert(len(items) // 2, (probe, mixed))
            _serve(server, items)
            single = torch.empty(probe["O"], dtype=probe["dt"], device="cuda")
            probe["nest"].run([probe["dA"].data_ptr()], single.data_ptr(), s)
            torch.cuda.synchronize()
            assert torch.equal(alone, mixed) and torch.equal(alone, single)
            sh = probe["shape"]
            ref = oracle_rect(list(sh.extents), sh.red_level, probe["op"], probe["prec"], "load", A=probe["A"])
            assert_close(alone.cpu().numpy(), ref, probe["prec"], probe["op"], what=f"served {sh.extents}")
        c = hb.hp_serve_counters(server)
        assert c["completed"] >= 4 * (len(pool) + 2) and c["steps"] >= 8
        p50, p99 = hb.hp_serve_stats(server)["p50_us"], hb.hp_serve_stats(server)["p99_us"]
        assert 0 < p50 <= p99
    finally:
        hb.hp_serve_destroy(server)
        for it in pool:
            it["nest"].close()


def test_budget_and_slots_bound_admission():
    import torch
    pool = _pool(48, seed=502)
    need = [4 * it["shape"].size + 4 * it["O"] for it in pool]
    budget = 3 * max(need)          # a few requests at a time
    server = hb.hp_serve_create(budget, 5, 3)
    try:
        items = [(it, torch.empty(it["O"], dtype=it["dt"], device="cuda")) for it in pool for _ in range(3)]
        _serve(server, items)
        c = hb.hp_serve_counters(server)
        assert c["completed"] == len(items)
        assert 0 < c["peak_bytes"] <= budget and 1 <= c["peak_slots"] <= 5
        s = torch.cuda.current_stream().cuda_stream
        for it, out in items[:20]:
            single = torch.empty(it["O"], dtype=it["dt"], device="cuda")
            it["nest"].run([it["dA"].data_ptr()], single.data_ptr(), s)
            torch.cuda.synchronize()
            assert torch.equal(out, single)
        # a request that can never fit the budget is refused at submission
        big = max(pool, key=lambda it: it["shape"].size)
        small_server = hb.hp_serve_create(1024, 4, 1)
        try:
            with pytest.raises(hb.HPError) as e:
                hb.hp_serve_submit(small_server, big["nest"].handle, [big["dA"].data_ptr()], 0x1000)
            assert e.value.status == hb.HP_ENOMEM
        finally:
            hb.hp_serve_destroy(small_server)
    finally:
        hb.hp_serve_destroy(server)
        for it in pool:
            it["nest"].close()


def test_plain_mode_and_poll_semantics():
    import torch
    pool = _pool(24, seed=503)
    hb.hp_set_option("serve_batching", 0)
    try:
        plain = hb.hp_serve_create(8 << 30, 64, 4)
    finally:
        hb.hp_set_option("serve_batching", 1)
    batched = hb.hp_serve_create(8 << 30, 64, 4)
    try:
        outs_p = [(it, torch.empty(it["O"], dtype=it["dt"], device="cuda")) for it in pool]
        outs_b = [(it, torch.empty(it["O"], dtype=it["dt"], device="cuda")) for it in pool]
        _serve(plain, outs_p)
        tickets = [hb.hp_serve_submit(batched, it["nest"].handle, [it["dA"].data_ptr()], o.data_ptr())
                   for it, o in outs_b]
        st = hb.hp_serve_poll(batched, tickets[-1], 0)
        assert st in (hb.HP_OK, hb.HP_EAGAIN)
        for t in tickets:
            deadline = time.time() + 60
            while hb.hp_serve_poll(batched, t, 1000) != hb.HP_OK:
                assert time.time() < deadline
        for (it, a), (_, b) in zip(outs_p, outs_b):
            assert torch.equal(a, b), it["shape"].extents
        with pytest.raises(hb.HPError):
            hb.hp_serve_poll(batched, 10 ** 9, 0)
    finally:
        hb.hp_serve_destroy(plain)
        hb.hp_serve_destroy(batched)
        for it in pool:
            it["nest"].close()


def test_latency_counts_from_scheduled_arrival():
    # a request whose arrival was scheduled 50 ms before its submission carries
    # those 50 ms in its latency; an arrival in the future is refused
    import torch
    pool = _pool(4, seed=504)
    server = hb.hp_serve_create(8 << 30, 64, 2)
    try:
        it = pool[0]
        out = torch.empty(it["O"], dtype=it["dt"], device="cuda")
        due = hb.hp_serve_clock_us() - 50_000.0
        t = hb.hp_serve_submit_at(server, it["nest"].handle, [it["dA"].data_ptr()], out.data_ptr(), due)
        assert hb.hp_serve_poll(server, t, -1) == hb.HP_OK
        assert hb.hp_serve_stats(server)["p50_us"] >= 50_000.0
        with pytest.raises(hb.HPError) as e:
            hb.hp_serve_submit_at(server, it["nest"].handle, [it["dA"].data_ptr()], out.data_ptr(),
                                  hb.hp_serve_clock_us() + 1e6)
        assert e.value.status == hb.HP_EINVAL
        single = torch.empty(it["O"], dtype=it["dt"], device="cuda")
        it["nest"].run([it["dA"].data_ptr()], single.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert torch.equal(out, single)
    finally:
        hb.hp_serve_destroy(server)
        for p in pool:
            p["nest"].close()


# ---------------------------------------------------------------- resident mode
def _resident_server(budget=8 << 30, slots=256, streams=2):
    hb.hp_set_option("serve_batching", 2)
    try:
        return hb.hp_serve_create(budget, slots, streams)
    finally:
        hb.hp_set_option("serve_batching", 1)


def _sum_pool(n, seed, t_max=1 << 18):
    """FP32 compensated sums only (a resident server runs one arithmetic)."""
    return [it for it in _pool(n, seed=seed, t_max=t_max) if it["op"] == "sum"]


def _single(it):
    import torch
    out = torch.empty(it["O"], dtype=it["dt"], device="cuda")
    it["nest"].run([it["dA"].data_ptr()], out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.current_stream().synchronize()
    return out


def test_resident_same_result_alone_mixed_and_single():
    import torch
    pool = _sum_pool(96, seed=511)
    server = _resident_server()
    try:
        for probe in (pool[0], pool[5], pool[17], pool[-1]):
            alone = torch.full((probe["O"],), 3, dtype=probe["dt"], device="cuda")
            _serve(server, [(probe, alone)])
            mixed = torch.full((probe["O"],), 5, dtype=probe["dt"], device="cuda")
            items = [(it, torch.empty(it["O"], dtype=it["dt"], device="cuda")) for it in pool]
            items.insert(len(items) // 3, (probe, mixed))
            _serve(server, items)
            single = _single(probe)
            assert torch.equal(alone, mixed) and torch.equal(alone, single)
            sh = probe["shape"]
            ref = oracle_rect(list(sh.extents), sh.red_level, probe["op"], probe["prec"], "load", A=probe["A"])
            assert_close(alone.cpu().numpy(), ref, probe["prec"], probe["op"], what=f"resident {sh.extents}")
            for it, out in items[:: max(1, len(items) // 12)]:
                assert torch.equal(out, _single(it)), it["shape"].extents
        c = hb.hp_serve_counters(server)
        assert c["completed"] == 4 * (len(pool) + 2)
        st = hb.hp_serve_stats(server)
        assert 0 < st["p50_us"] <= st["p99_us"]
    finally:
        hb.hp_serve_destroy(server)
        for it in pool:
            it["nest"].close()


def test_resident_grid_split_and_large_requests():
    # one output reduced over 2^24 elements (a grid-split plan: partials and
    # tickets from the server's pools) and a 2^24-element request with many
    # outputs (about a thousand tiles), beside small requests
    import torch
    from paper_2309_01906_gb300 import synth as sy
    shapes = [([1 << 24], 0), ([4, 1 << 22], 1), ([4096, 4096], 1), ([1 << 12, 16, 256], 1), ([300, 7], 1)]
    items = []
    for i, (ext, red) in enumerate(shapes):
        size = int(np.prod(ext))
        A = sy.normal_f32(size, 512, i)
        nest = hb.Nest(ext, red, "sum", "f32_comp", "load")
        O = max(int(np.prod(ext[:red])) if red else 1, 1)
        items.append(dict(nest=nest, A=A, dA=torch.from_numpy(A).cuda(), O=O, ext=ext, red=red,
                          dt=torch.float32, op="sum", prec="f32_comp"))
    assert any(it["nest"].describe()["grid_parts"] > 1 for it in items)
    server = _resident_server(slots=16)
    try:
        for rep in range(3):
            outs = [(it, torch.full((it["O"],), float("nan"), dtype=torch.float32, device="cuda"))
                    for it in items for _ in range(2)]
            _serve(server, outs)
            for it, out in outs:
                assert torch.equal(out, _single(it)), it["ext"]
        for it in items:
            ref = oracle_rect(it["ext"], it["red"], "sum", "f32_comp", "load", A=it["A"])
            assert_close(_single(it).cpu().numpy(), ref, "f32_comp", "sum", what=f"{it['ext']}")
    finally:
        hb.hp_serve_destroy(server)
        for it in items:
            it["nest"].close()


def test_resident_runs_one_arithmetic():
    import torch
    pool = _pool(40, seed=513)
    sums = [it for it in pool if it["op"] == "sum"]
    maxes = [it for it in pool if it["op"] == "max"]
    assert sums and maxes
    server = _resident_server()
    try:
        out = torch.empty(sums[0]["O"], dtype=torch.float32, device="cuda")
        _serve(server, [(sums[0], out)])
        o2 = torch.empty(maxes[0]["O"], dtype=torch.int32, device="cuda")
        with pytest.raises(hb.HPError) as e:
            hb.hp_serve_submit(server, maxes[0]["nest"].handle, [maxes[0]["dA"].data_ptr()], o2.data_ptr())
        assert e.value.status == hb.HP_EUNSUPPORTED
    finally:
        hb.hp_serve_destroy(server)
    # int64 nests are not served resident at all
    n64 = hb.Nest([64, 64], 1, "sum", "i64", "load")
    server = _resident_server()
    try:
        A = torch.ones(64 * 64, dtype=torch.int64, device="cuda")
        o = torch.empty(64, dtype=torch.int64, device="cuda")
        with pytest.raises(hb.HPError) as e:
            hb.hp_serve_submit(server, n64.handle, [A.data_ptr()], o.data_ptr())
        assert e.value.status == hb.HP_EUNSUPPORTED
    finally:
        hb.hp_serve_destroy(server)
        n64.close()
        for it in pool:
            it["nest"].close()


def test_resident_int32_max_server():
    import torch
    pool = [it for it in _pool(60, seed=514) if it["op"] == "max"]
    server = _resident_server()
    try:
        outs = [(it, torch.empty(it["O"], dtype=torch.int32, device="cuda")) for it in pool]
        _serve(server, outs)
        for it, out in outs:
            assert torch.equal(out, _single(it)), it["shape"].extents
        sh = pool[0]["shape"]
        ref = oracle_rect(list(sh.extents), sh.red_level, "max", "i32", "load", A=pool[0]["A"])
        assert_close(outs[0][1].cpu().numpy(), ref, "i32", "max", what=f"resident {sh.extents}")
    finally:
        hb.hp_serve_destroy(server)
        for it in pool:
            it["nest"].close()


def test_resident_instances_turn_over_and_restart_after_idle():
    # a stream longer than one instance's epoch (100 ms) runs on several
    # instances in turn; after an idle pause (the instance stops) the next
    # request starts a new one
    import torch
    pool = _sum_pool(32, seed=515, t_max=1 << 16)
    server = _resident_server()
    try:
        outs = []
        t_end = time.time() + 0.45
        while time.time() < t_end:
            it = pool[len(outs) % len(pool)]
            out = torch.empty(it["O"], dtype=torch.float32, device="cuda")
            outs.append((it, out, hb.hp_serve_submit(server, it["nest"].handle, [it["dA"].data_ptr()],
                                                     out.data_ptr())))
            time.sleep(0.0005)
        for _, _, t in outs:
            assert hb.hp_serve_poll(server, t, -1) == hb.HP_OK
        launches = hb.hp_serve_counters(server)["steps"]
        assert launches >= 3, launches
        time.sleep(0.05)
        it = pool[3]
        late = torch.empty(it["O"], dtype=torch.float32, device="cuda")
        t = hb.hp_serve_submit(server, it["nest"].handle, [it["dA"].data_ptr()], late.data_ptr())
        assert hb.hp_serve_poll(server, t, -1) == hb.HP_OK
        assert hb.hp_serve_counters(server)["steps"] == launches + 1
        for it, out, _ in outs[::7] + [(it, late, 0)]:
            assert torch.equal(out, _single(it))
    finally:
        hb.hp_serve_destroy(server)
        for it in pool:
            it["nest"].close()


def test_resident_budget_and_slots_bound_admission():
    import torch
    pool = _sum_pool(48, seed=516)
    need = [4 * it["shape"].size + 4 * it["O"] for it in pool]
    budget = 3 * max(need)
    server = _resident_server(budget=budget, slots=5)
    try:
        items = [(it, torch.empty(it["O"], dtype=it["dt"], device="cuda")) for it in pool for _ in range(3)]
        _serve(server, items)
        c = hb.hp_serve_counters(server)
        assert c["completed"] == len(items)
        assert 0 < c["peak_bytes"] <= budget and 1 <= c["peak_slots"] <= 5
        for it, out in items[:20]:
            assert torch.equal(out, _single(it))
    finally:
        hb.hp_serve_destroy(server)
        for it in pool:
            it["nest"].close()
