"""GPU tests of the serving loop: continuous batching under a memory budget.

A request's result must be the same alone and in a mix of other requests
(bit for bit: same plan, same reduction tree) and equal hp_nest_run's; the
budget and slot limits must hold at every moment; the plain per-request mode
must give the same results."""
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
    """Submit (pool item, output tensor) pairs, wait for all; returns tickets."""
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
