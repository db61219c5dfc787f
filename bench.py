"""Benchmark of the hierarchical loop-nest executor on GB300.

Workload: the 4-level rectangular nest b=64 x i=512 x j=16 x k=1024,
out[b][i] = sum_j sum_k A[b][i][j][k] * w[j][k], A FP32 normal(0, 1) (2 GiB),
w FP32 uniform[-1, 1]; levels bound grid / grid / cluster (4 CTAs) / CTA
(4 warps): k reduced by lanes (xor-shuffle) and warps (shared memory), j by the
CTAs of a cluster (distributed shared memory), each CTA folding 4 of the 16 j
rows.  Compensated FP32 accumulation.

One step = one run of the nest (all its launches) over the resident inputs.
Metric: nest iterations per second (2^29 iterations per step).  The line also
carries the per-result error of every output the CPU-baseline leg evaluated
against the FP64 oracle (`parity`), and, after the headline's timed region,
the GEMV-shaped nest, 10 s of Poisson serving (resident, batched-launch and
plain servers), the ragged CSR nest and the 10,000-nest batch (`workloads`;
--extras none leaves them out).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hp|reference]

--impl reference times the sequential CPU oracle on the host cores instead
(each step a bounded sample of the same workload).  With N > 1 (torchrun) each
rank runs an independent replica (no data exchange); value = all ranks'
iterations / max over ranks of the timed region.

Other workloads (--workload; one JSON line each, with rooflines; not the
headline):  gemv (1024 x 1024, cold and warm), csr (Zipf(1.5) ragged rows with
the fused histogram), batch (10,000 uneven nests in one persistent launch),
serve (Poisson arrivals through the serving loop), stencil (16384^2 with ghost
zones, 1 and 4 fused steps), ordered (non-commutative reductions:
--ordered-op compose | mat2 | last), narrow (int8 / int16 nests with
SIMD-in-register sub-lanes).
"""
from __future__ import annotations

import argparse
import ctypes
import gc
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

EXTENTS = [64, 512, 16, 1024]
RED_LEVEL = 2
LEVEL_MAP = [("grid", 0, 0), ("grid", 0, 0), ("cluster", 4, 0), ("cta", 4, 0)]
ITERS = int(np.prod(EXTENTS))
N_OUT = EXTENTS[0] * EXTENTS[1]
R = EXTENTS[2] * EXTENTS[3]
# algorithmic bytes of one launch: A once, w once, outputs once
ALG_BYTES = ITERS * 4 + R * 4 + N_OUT * 4
WORKLOAD = "4-level nest b=64 i=512 j=16 k=1024, out[b][i]=sum_j sum_k A[b][i][j][k]*w[j][k]"
# DRAM traffic of one launch (dram__bytes_read.sum + dram__bytes_write.sum) taken from
# an ncu capture of this workload, not measured by this script; reported only while
# the kernel sources still hash to the fingerprint the capture was taken at
TRAFFIC = {"sources": ["paper_2309_01906_gb300/csrc/rect_kernels.cuh", "paper_2309_01906_gb300/csrc/accum.cuh"],
           "sha256_16": "ee144f98346f8f5a", "bytes_per_launch": 2191.61e6,
           "how": "ncu capture of one launch of the same kernel and map at b=8 (268.55 MB read + 5.40 MB "
                  "written), scaled by 8 to b=64; null once the kernel sources changed since"}


def traffic_per_launch():
    import hashlib
    h = hashlib.sha256()
    try:
        for f in TRAFFIC["sources"]:
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
    except OSError:
        return None
    return TRAFFIC["bytes_per_launch"] if h.hexdigest()[:16] == TRAFFIC["sha256_16"] else None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def host_cores():
    """Host cores this process may run on (affinity) and online in the machine."""
    try:
        aff = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        aff = os.cpu_count() or 1
    return {"affinity": aff, "online": os.cpu_count() or aff}


def threaded(fn, items, threads):
    """fn over items on `threads` host threads, results in order.  The oracle's
    C entry points run outside the interpreter lock (ctypes releases it), so
    its calls on disjoint outputs run in parallel."""
    from concurrent.futures import ThreadPoolExecutor
    if threads <= 1:
        return [fn(x) for x in items]
    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(fn, items))


def fp_parity(got, ref, prec, bound, tol):
    """Per-result error of GPU FP32 sums against the FP64 oracle, summarised.

    For each result: err = |got - ref|; the relative error err / |ref| where
    |ref| >= 2^-20 sum|t| (the relative clause), else the normalized error
    err / (2^-20 sum|t|) (cond = sum|t| / |ref| above 2^20); the plain relative
    error err / |ref| of every nonzero ref; cond = sum|t| / |ref|; and the
    a-priori bound check err <= bound sum|t| + 2^-24 |ref|.  Plain FP32 sums
    are also scaled by sqrt(sum t^2) (a random-sign sum's natural scale)."""
    g = np.asarray(got, np.float64)
    r, ab, sq = ref.values, ref.abs_sum, ref.sq_sum
    err = np.abs(g - r)
    floor = 2.0 ** -20 * ab
    rel_clause = np.abs(r) >= floor
    scale = np.maximum(np.abs(r), floor)
    safe = np.where(scale > 0, scale, 1.0)
    # a nonzero result where every term is zero has no scale: its error counts as 1e300
    norm = np.where(scale > 0, err / safe, np.where(err > 0, 1e300, 0.0))
    nz = r != 0
    rel = err[nz] / np.abs(r[nz])
    cond = np.where(nz, ab / np.where(nz, np.abs(r), 1.0), np.inf)
    lim = bound * ab + 2.0 ** -24 * np.abs(r)
    worst = int(np.argmax(norm)) if norm.size else 0
    d = {
        "n_checked": int(g.size), "prec": prec, "tolerance": tol,
        "clause": "|got-ref| / max(|ref|, 2^-20 sum|t|)",
        "n_relative_clause": int(rel_clause.sum()), "n_normalized_clause": int((~rel_clause).sum()),
        "max_norm_err": float(norm.max()) if norm.size else 0.0,
        "p50_norm_err": float(np.median(norm)) if norm.size else 0.0,
        "p99_norm_err": float(np.quantile(norm, 0.99)) if norm.size else 0.0,
        "worst": {"index": worst, "got": float(g[worst]), "ref": float(r[worst]), "sum_abs": float(ab[worst]),
                  "cond": float(cond[worst]) if np.isfinite(cond[worst]) else None} if norm.size else None,
        "max_plain_rel_err": float(rel.max()) if rel.size else 0.0,
        "max_cond": float(cond[np.isfinite(cond)].max()) if np.isfinite(cond).any() else None,
        "median_cond": float(np.median(cond)) if cond.size else None,
        "n_exact_zero_ref": int((~nz).sum()),
        "a_priori_bound": bound, "max_err_over_sum_abs": float((err / np.where(ab > 0, ab, 1.0)).max()) if err.size else 0.0,
        "within_a_priori_bound": bool(np.all(err <= lim * (1 + 1e-12) + 1e-300)),
    }
    if prec == "f32":
        l2 = np.sqrt(sq)
        s2 = np.maximum(np.abs(r), l2)
        n2 = np.where(s2 > 0, err / np.where(s2 > 0, s2, 1.0), 0.0)
        d["max_norm_err_l2_scale"] = float(n2.max()) if n2.size else 0.0
        d["pass"] = bool(d["max_norm_err_l2_scale"] <= tol and d["within_a_priori_bound"])
        d["pass_sum_abs_clause"] = bool(d["max_norm_err"] <= tol)
    else:
        d["pass"] = bool(d["max_norm_err"] <= tol and d["within_a_priori_bound"])
    return d


def write_parity_table(path, idx, got, ref):
    """Per-result error table (one line per checked output) for --parity-out."""
    g = np.asarray(got, np.float64)
    r = ref.values
    with open(path, "w") as f:
        f.write("output,got,ref_fp64,sum_abs,cond,abs_err,rel_err,norm_err,clause\n")
        for k in range(g.size):
            gk, rk, ak = float(g[k]), float(r[k]), float(ref.abs_sum[k])
            e = abs(gk - rk)
            fl = 2.0 ** -20 * ak
            clause = "relative" if abs(rk) >= fl else "normalized"
            sc = max(abs(rk), fl)
            cond = ak / abs(rk) if rk else float("inf")
            rel = e / abs(rk) if rk else float("inf")
            norm = e / sc if sc else 0.0
            f.write(f"{int(idx[k])},{gk!r},{rk!r},{ak!r},{cond!r},{e!r},{rel!r},{norm!r},{clause}\n")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def run_hp(args):
    import torch
    import torch.distributed as dist

    from paper_2309_01906_gb300 import binding as hb
    from paper_2309_01906_gb300 import synth

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    A, w = synth.nest4_f32(*EXTENTS)
    dA = torch.from_numpy(A.reshape(-1)).cuda()
    dw = torch.from_numpy(w.reshape(-1)).cuda()
    out = torch.empty(N_OUT, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    nests = {p: hb.Nest(EXTENTS, RED_LEVEL, "sum", p, "dot_bcast", level_map=LEVEL_MAP) for p in ("f32_comp", "f32")}
    plan = nests["f32_comp"].describe()
    launches_per_step = 1 + (1 if plan["grid_parts"] > 1 else 0)

    from paper_2309_01906_gb300 import replicas

    def barrier():
        torch.cuda.synchronize()
        replicas.barrier()
        torch.cuda.synchronize()

    def timed(nest, steps, warmup):
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                nest.run([dA.data_ptr(), dw.data_ptr()], out.data_ptr(), sp)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            barrier()
            t_all0 = torch.cuda.Event(enable_timing=True)
            t_all1 = torch.cuda.Event(enable_timing=True)
            t_all0.record(stream)
            for i in range(steps):
                ev[i][0].record(stream)
                nest.run([dA.data_ptr(), dw.data_ptr()], out.data_ptr(), sp)
                ev[i][1].record(stream)
            t_all1.record(stream)
            barrier()
        total_ms = t_all0.elapsed_time(t_all1)
        per = [a.elapsed_time(b) for a, b in ev]
        return total_ms, per

    # plain FP32 variant (context), then the headline compensated run with clock sampling
    plain_ms, plain_per = timed(nests["f32"], max(3, args.steps), args.warmup)
    got_plain = out.cpu().numpy().copy()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    total_ms, per = timed(nests["f32_comp"], args.steps, args.warmup)
    clocks = sampler.stop()
    assert nests["f32_comp"].check(sp) == 0
    got_comp = out.cpu().numpy().copy()

    max_ms = replicas.max_over_ranks(total_ms, device="cuda")   # the slowest replica times the job

    # end to end through the C ABI with host buffers: H2D of A and w, run, D2H of out
    hA = torch.from_numpy(A.reshape(-1)).pin_memory()
    hw = torch.from_numpy(w.reshape(-1)).pin_memory()
    hout = torch.empty(N_OUT, dtype=torch.float32).pin_memory()
    e2e_steps = max(2, min(args.steps, 5))
    ne = nests["f32_comp"]

    def e2e_time():
        ne.run_host([hA.data_ptr(), hw.data_ptr()], hout.data_ptr(), sp)   # warm-up (allocates staging once)
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            ne.run_host([hA.data_ptr(), hw.data_ptr()], hout.data_ptr(), sp)
        barrier()
        return replicas.max_over_ranks((time.perf_counter() - t0) / e2e_steps, device="cuda")

    # the library's default: the kernel reads the page-locked A in place over
    # the host link; then, for comparison, A copied to device staging first
    e2e_s = e2e_time()
    e2e_same = bool(torch.equal(hout, out.cpu()))
    hb.hp_set_option("host_zero_copy", 0)
    try:
        e2e_staged_s = e2e_time()
    finally:
        hb.hp_set_option("host_zero_copy", 1)

    cpu, parity = None, None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, sel, ref = cpu_baseline(A, w, seconds=args.cpu_seconds)
        # the oracle's outputs of the CPU-baseline leg are the parity reference:
        # every output it evaluated, compensated and plain FP32 against FP64
        parity = {"f32_comp": fp_parity(got_comp[sel], ref, "f32_comp", nests["f32_comp"].error_bound(), 1e-6),
                  "f32": fp_parity(got_plain[sel], ref, "f32", nests["f32"].error_bound(), 1e-5),
                  "oracle": "FP64 Neumaier sums of the FP64 products (exact) in loop order"}
        if args.parity_out:
            write_parity_table(args.parity_out, sel, got_comp[sel], ref)
    workloads = {}
    if rank == 0 and ws == 1:   # replicas runs (N > 1) time the headline alone
        for name in [x for x in args.extras.split(",") if x and x != "none"]:
            # each workload starts from a collected heap and an emptied device cache,
            # so that host memory freed by the previous one is not reclaimed under it
            gc.collect()
            torch.cuda.empty_cache()
            t_w = time.perf_counter()
            workloads[name] = EXTRAS[name](args)
            workloads[name]["wall_s"] = time.perf_counter() - t_w

    if rank == 0:
        peak, peak_kind = measured_peaks()
        avg_launch_ms = float(np.mean(per))
        achieved = ALG_BYTES / (avg_launch_ms * 1e-3) / 1e9
        value = ITERS * args.steps * ws / (max_ms * 1e-3)
        line = {
            "metric": "nest iterations/s",
            "value": value,
            "unit": "iterations/s",
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": max_ms / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic (seeded): A normal(0,1) seed 3, w uniform[-1,1] seed 4",
            "config": {
                "workload": WORKLOAD,
                "map": "b,i->grid; j->cluster(4 CTAs, DSMEM); k->CTA(4 warps x 32 lanes x 4 vector slots)",
                "precision": "compensated FP32 (Dot2) at every level",
                "l2": "inputs (2 GiB) larger than L2 (129 MB); no flush",
                "plan": {k: plan[k] for k in ("team", "cluster", "warps", "vec", "grid_parts", "kernel")},
                "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
            },
            "roofline": {
                "bound": "hbm",
                "achieved": achieved,
                "peak": peak,
                "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": traffic_per_launch(),
                "traffic_source": TRAFFIC["how"],
                "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": ALG_BYTES,
                "kernel": plan["kernel"],
            },
            "variants": {
                "f32_plain": {"value": ITERS * len(plain_per) / (plain_ms * 1e-3), "unit": "iterations/s",
                              "ms_per_step": plain_ms / len(plain_per)},
            },
            "e2e": {
                "value": ITERS * ws / e2e_s,
                "unit": "iterations/s",
                "h2d_bytes_per_step": int(A.nbytes + w.nbytes),
                "d2h_bytes_per_step": int(N_OUT * 4),
                "ms_per_step": e2e_s * 1e3,
                "how": "hp_nest_run_host on pinned host buffers: A read in place by the kernel over the host link, "
                       "w staged, outputs copied back, stream synchronized",
                "same_bits_as_device_run": e2e_same,
                "staged_copy_variant": {"value": ITERS * ws / e2e_staged_s, "ms_per_step": e2e_staged_s * 1e3},
            },
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
            "cpu_baseline": cpu,
            "parity": parity,
            "host_cores": host_cores(),
            "workloads": workloads,
        }
        print(json.dumps(line))
    for n in nests.values():
        n.close()
    if ws > 1:
        dist.destroy_process_group()


def cpu_baseline(A, w, seconds=15.0):
    """The oracle as it stands (sequential, one host core) on a bounded sample:
    whole outputs of the same workload, as many as fit in about `seconds`.
    Then, as context, the same outputs evaluated with the outermost level
    spread over every host core (one oracle call per block of outputs).
    Returns (baseline dict, evaluated output indices, oracle result)."""
    import oracle
    oracle.load()
    t0 = time.perf_counter()
    n_done = 0
    chunk = 256
    idx = np.arange(N_OUT, dtype=np.int64)
    parts = []
    while n_done < N_OUT and time.perf_counter() - t0 < seconds:
        sel = idx[n_done:n_done + chunk]
        parts.append(oracle.rect_sampled(EXTENTS, RED_LEVEL, "sum", "f32_comp", "dot_bcast", sel, A=A, w=w))
        n_done += sel.size
        chunk = min(chunk * 2, 4096)
    dt = time.perf_counter() - t0
    ref = oracle.Result(np.concatenate([p.values for p in parts]), np.concatenate([p.abs_sum for p in parts]),
                        np.concatenate([p.sq_sum for p in parts]))
    cores = host_cores()
    threads = cores["affinity"]
    blocks = np.array_split(idx[:n_done], max(1, threads * 4))
    t1 = time.perf_counter()
    par = threaded(lambda b: oracle.rect_sampled(EXTENTS, RED_LEVEL, "sum", "f32_comp", "dot_bcast", b, A=A, w=w),
                   blocks, threads)
    dt_all = time.perf_counter() - t1
    same = bool(np.array_equal(np.concatenate([p.values for p in par]), ref.values))
    return ({"value": n_done * R / dt, "unit": "iterations/s", "cores": 1, "kind": "oracle",
             "sample": f"{n_done} of {N_OUT} outputs ({n_done * R} iterations) of the same workload, {dt:.1f} s",
             "host_cores": cores,
             "all_cores_context": {"value": n_done * R / dt_all, "unit": "iterations/s", "cores": threads,
                                   "seconds": dt_all, "same_values": same,
                                   "how": "the same oracle calls, outermost level split over host threads"}},
            idx[:n_done], ref)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2309_01906_gb300 import synth
    A, w = synth.nest4_f32(*EXTENTS)
    import oracle
    oracle.load()
    # each step: a bounded sample of the workload (a block of whole outputs)
    per_step_outputs = args.ref_outputs
    idx = np.arange(N_OUT, dtype=np.int64)
    for s in range(args.warmup):
        oracle.rect_sampled(EXTENTS, RED_LEVEL, "sum", "f32_comp", "dot_bcast", idx[:per_step_outputs], A=A, w=w)
    t0 = time.perf_counter()
    for s in range(args.steps):
        lo = (s * per_step_outputs) % N_OUT
        oracle.rect_sampled(EXTENTS, RED_LEVEL, "sum", "f32_comp", "dot_bcast", idx[lo:lo + per_step_outputs],
                            A=A, w=w)
    dt = time.perf_counter() - t0
    value = args.steps * per_step_outputs * R / dt
    sample = f"{per_step_outputs} whole outputs ({per_step_outputs * R} iterations) of the same workload per step"
    line = {
        "impl": "reference",
        "metric": "nest iterations/s",
        "value": value,
        "unit": "iterations/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded): A normal(0,1) seed 3, w uniform[-1,1] seed 4",
        "config": {"workload": WORKLOAD, "l2": "host run"},
        "cpu_baseline": {"value": value, "unit": "iterations/s", "cores": 1, "kind": "oracle", "sample": sample,
                         "host_cores": host_cores()},
        "e2e": {"value": value, "unit": "iterations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_profile_case(args):
    """Reduced case for profiler captures: the headline nest with b = args.profile_b
    (same map, same kernel), warm-up then `steps` runs, one timing line."""
    import torch

    from paper_2309_01906_gb300 import binding as hb
    from paper_2309_01906_gb300 import synth
    ext = [args.profile_b] + EXTENTS[1:]
    A, w = synth.nest4_f32(*ext)
    dA = torch.from_numpy(A.reshape(-1)).cuda()
    dw = torch.from_numpy(w.reshape(-1)).cuda()
    out = torch.empty(ext[0] * ext[1], dtype=torch.float32, device="cuda")
    n = hb.Nest(ext, RED_LEVEL, "sum", args.prec, "dot_bcast", level_map=LEVEL_MAP)
    sp = torch.cuda.current_stream().cuda_stream
    for _ in range(args.warmup):
        n.run([dA.data_ptr(), dw.data_ptr()], out.data_ptr(), sp)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        n.run([dA.data_ptr(), dw.data_ptr()], out.data_ptr(), sp)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"profile_case": ext, "prec": args.prec, "ms_per_launch": ms,
                      "algorithmic_gbs": (A.nbytes + w.nbytes + out.numel() * 4) / ms / 1e6,
                      "kernel": n.describe()["kernel"]}))
    n.close()


def _event_time(fn, steps, warmup, stream, flush=None):
    """Mean ms per call of fn() on `stream`, CUDA events; optional L2 flush between calls."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        per = []
        for _ in range(steps):
            if flush is not None:
                flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            per.append((e0, e1))
        torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in per]))


def csr_measure(args):
    """Ragged CSR nest: 2^22 rows (or --csr-rows), Zipf(1.5) lengths clipped to
    [1, 65536], col uniform in [0, 2^22), FP32 normal val / x, compensated SpMV
    with the int64 histogram of col >> 10 fused into the same sweep.

    Two rooflines: HBM (the algorithmic bytes) and the x gathers, whose random
    4-byte reads each take one 32-byte L2 sector: their rate is measured on
    this GPU by a gather-only kernel (hp_probe_gather, the same loads, as many
    reads as the nest has entries, on the same x).  The CPU-baseline leg runs
    the oracle on 1024 seeded rows and the whole histogram; parity compares the
    rows within tolerance and the histogram bit for bit."""
    import torch

    from paper_2309_01906_gb300 import binding as hb
    from paper_2309_01906_gb300 import synth
    n_rows = args.csr_rows
    n_cols = 1 << 22
    t0 = time.perf_counter()
    csr = synth.csr_zipf(n_rows=n_rows, n_cols=n_cols)
    setup_s = time.perf_counter() - t0
    n_bins = n_cols >> 10
    d = [torch.from_numpy(a).cuda() for a in (csr.offsets, csr.col, csr.val, csr.x)]
    y = torch.empty(n_rows, dtype=torch.float32, device="cuda")
    h = torch.empty(n_bins, dtype=torch.int64, device="cuda")
    p = hb.hp_csr_params(csr.nnz, n_cols, 10, 0 if args.no_hist else 1, n_bins)
    n = hb.Nest(csr_rows=n_rows, red_level=1, op="sum", prec=args.prec, body="csr_gather", params=p)
    stream = torch.cuda.Stream()
    ins = [t.data_ptr() for t in d] + [h.data_ptr()]
    steps = max(3, min(args.steps, 20))
    ms = _event_time(lambda: n.run(ins, y.data_ptr(), stream.cuda_stream), steps, args.warmup, stream)
    assert n.check(stream.cuda_stream) == 0
    # gather-only probe: as many random reads of the same x as the nest has entries
    psum = torch.zeros(1, dtype=torch.float32, device="cuda")
    ms_probe = _event_time(lambda: hb.hp_probe_gather(d[3].data_ptr(), n_cols, csr.nnz, 7, psum.data_ptr(),
                                                      stream.cuda_stream), steps, args.warmup, stream)
    alg = 8 * csr.nnz + 8 * (n_rows + 1) + 4 * n_cols + 4 * n_rows + 8 * n_bins
    peak, kind = measured_peaks()
    lens = np.diff(csr.offsets)
    limits = n.describe()["class_limits"]
    gather_rate = csr.nnz / (ms_probe * 1e-3)
    parity, cpu = None, None
    if not args.no_cpu_baseline:
        import oracle
        g = np.random.Generator(np.random.PCG64(23))
        rows = np.sort(g.choice(n_rows, size=min(n_rows, 1024), replace=False))
        # the longest rows too: they take the split (grid-part) path
        rows = np.unique(np.concatenate([rows, np.argsort(lens)[-16:]]))
        t1 = time.perf_counter()
        ref = oracle.csr(csr.offsets, csr.col, csr.val, csr.x, rows=rows)
        dt = time.perf_counter() - t1
        got = y.cpu().numpy()[rows]
        parity = {"rows": fp_parity(got, ref, args.prec, n.error_bound(), 1e-6 if args.prec == "f32_comp" else 1e-5)}
        cpu = {"value": float(lens[rows].sum()) / dt, "unit": "entries/s", "cores": 1, "kind": "oracle",
               "sample": f"{rows.size} rows ({int(lens[rows].sum())} entries): 1024 seeded + the 16 longest"}
        if not args.no_hist:
            hr = oracle.hist(csr.col, 10, n_bins)
            parity["histogram_bit_exact"] = bool(np.array_equal(h.cpu().numpy(), hr.values) and hr.overflow == 0)
            parity["histogram_total"] = int(hr.values.sum())
    res = {
        "workload": f"CSR {n_rows} rows, Zipf(1.5) clipped [1,65536], nnz {csr.nnz}, SpMV"
                    + ("" if args.no_hist else " + fused int64 histogram"),
        "metric": "nest iterations/s", "value": csr.nnz / (ms * 1e-3), "unit": "iterations/s",
        "ms_per_step": ms, "prec": args.prec, "steps": steps, "warmup": args.warmup,
        "roofline": {"bound": "hbm", "achieved": alg / (ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": alg / (ms * 1e-3) / 1e9 / peak, "peak_kind": kind, "algorithmic_bytes": alg},
        "roofline_gather": {"bound": "l2_sectors", "achieved": csr.nnz / (ms * 1e-3), "peak": gather_rate,
                            "unit": "gathers/s (one 32-byte L2 sector each)", "frac": (csr.nnz / (ms * 1e-3)) / gather_rate,
                            "peak_kind": "measured by hp_probe_gather on this GPU (same x, nnz random reads)",
                            "probe_ms": ms_probe, "sector_bytes": 32 * csr.nnz,
                            "sector_gbs": 32 * csr.nnz / (ms * 1e-3) / 1e9,
                            "probe_sector_gbs": 32 * gather_rate / 1e9},
        "rows_by_class": [int(np.sum((lens > lo) & (lens <= hi))) for lo, hi in
                          zip([-1] + limits, limits + [1 << 62])],
        "class_limits": limits,
        "parity": parity, "cpu_baseline": cpu, "setup_s": setup_s,
        "l2": "inputs larger than L2; no flush (x, 16 MiB, stays in L2 by design)"}
    n.close()
    return res


def run_csr_workload(args):
    print(json.dumps(csr_measure(args)))


def gemv_measure(args):
    """2-level nest 1024 x 1024 (GEMV-shaped), compensated FP32, plain FP32 and
    int32, one launch per step; timed cold (L2 flushed between launches by a
    256 MiB write), warm, and warm as a one-launch CUDA graph replay.  Its
    CPU-baseline leg evaluates every output in the oracle; parity compares them
    (FP within tolerance, int32 bit for bit)."""
    import torch

    from paper_2309_01906_gb300 import binding as hb
    from paper_2309_01906_gb300 import synth
    stream = torch.cuda.Stream()
    scrub = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    peak, kind = measured_peaks()
    alg = 4 * (1 << 20) + 2 * 4096
    steps = max(args.steps, 20)
    res, cpu = {}, None
    for prec, (A, x) in (("f32_comp", synth.gemv_f32()), ("f32", synth.gemv_f32()), ("i32", synth.gemv_i32())):
        dA = torch.from_numpy(A.reshape(-1)).cuda()
        dx = torch.from_numpy(x).cuda()
        out = torch.empty(1024, dtype=torch.int32 if prec == "i32" else torch.float32, device="cuda")
        n = hb.Nest([1024, 1024], 1, "sum", prec, "dot_bcast", level_map=args.gemv_map)
        sp = stream.cuda_stream
        if args.gemv_map is None:
            # the autotuner picks the binding (single-run timing), untimed here
            n.tune([dA.data_ptr(), dx.data_ptr()], out.data_ptr(), sp, retime=True)
        run = hb.PreparedRun(n.handle, [dA.data_ptr(), dx.data_ptr()], out.data_ptr())
        cold = _event_time(lambda: run(sp), steps, args.warmup, stream, flush=lambda: scrub.fill_(1.0))
        warm = _event_time(lambda: run(sp), steps, args.warmup, stream)
        # the same launch captured once in a CUDA graph and replayed
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            run(torch.cuda.current_stream().cuda_stream)
        warm_graph = _event_time(g.replay, steps, args.warmup, stream)
        cold_graph = _event_time(g.replay, steps, args.warmup, stream, flush=lambda: scrub.fill_(1.0))
        # device time per launch: 20 launches back to back in one graph (the GPU, not the host, sets the pace)
        g20 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g20, stream=stream):
            for _ in range(20):
                run(torch.cuda.current_stream().cuda_stream)
        b2b = _event_time(g20.replay, max(3, steps // 4), args.warmup, stream) / 20
        got = out.cpu().numpy()
        plan = n.describe()
        # CPU-baseline leg: the oracle on all 1024 outputs, timed; its outputs are the parity reference
        import oracle
        t0 = time.perf_counter()
        ref = oracle.rect([1024, 1024], 1, "sum", prec, "dot_bcast", A=A, w=x)
        dt = time.perf_counter() - t0
        if prec == "i32":
            par = {"n_checked": 1024, "bit_exact": bool(np.array_equal(got.astype(np.int64), ref.values))}
        else:
            par = fp_parity(got, ref, prec, n.error_bound(), 1e-6 if prec == "f32_comp" else 1e-5)
        if prec == "f32_comp":
            cpu = {"value": (1 << 20) / dt, "unit": "iterations/s", "cores": 1, "kind": "oracle",
                   "sample": "all 1024 outputs of the compensated FP32 nest"}
        res[prec] = {"cold_us": cold * 1e3, "warm_us": warm * 1e3, "graph_warm_us": warm_graph * 1e3,
                     "graph_cold_us": cold_graph * 1e3, "device_us_per_launch_warm": b2b * 1e3,
                     "iterations_per_s_cold": (1 << 20) / (cold * 1e-3),
                     "roofline_cold": {"bound": "hbm", "achieved": alg / (cold * 1e-3) / 1e9, "peak": peak,
                                       "unit": "GB/s", "frac": alg / (cold * 1e-3) / 1e9 / peak, "peak_kind": kind},
                     "plan": {k: plan[k] for k in ("team", "warps", "team_lanes", "vec", "grid_parts", "kernel", "tuned")},
                     "parity": par}
        del g, g20
        n.close()
    return {"workload": "2-level nest 1024 x 1024, out[i] = sum_j A[i][j] * x[j], one launch (FP32 uniform[-1,1] "
                        "seed 1; int32 uniform [-100,100] seed 2)",
            "map": str(args.gemv_map) if args.gemv_map else "autotuned (single-run timing)", "results": res,
            "algorithmic_bytes": alg, "cpu_baseline": cpu, "steps": steps,
            "timing": "cold / warm: CUDA events around one launch from the host; graph_*: around a one-launch "
                      "CUDA graph replay (both include the host's submission); device_us_per_launch_warm: "
                      "20 launches back to back in one graph",
            "l2": "cold: 256 MiB write between launches; warm: inputs resident in L2"}


def run_gemv_workload(args):
    print(json.dumps(gemv_measure(args)))


# FP32 FMA peak derived from unit counts and clocks: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz
FP32_FMA_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def run_stencil_workload(args):
    """Stencil nest with ghost zones: 16384 x 16384 FP32 (seed 11), 9-point
    diffusion stencil, zero ghost surface; steps 1 (HBM-bound) and 4 (steps fused
    in shared memory, ghost border 4).  Inputs (1 GiB) are larger than L2."""
    import torch

    from paper_2309_01906_gb300 import binding as hb
    from paper_2309_01906_gb300 import synth
    ny = nx = args.stencil_n
    r = 1
    c = synth.DIFFUSION9
    A = synth.stencil_f32(ny, nx)
    dA = torch.from_numpy(A).cuda()
    out = torch.empty_like(dA)
    stream = torch.cuda.Stream()
    peak, kind = measured_peaks()
    res = {}
    for T in [int(t) for t in args.stencil_steps.split(",")]:
        st = hb.Stencil(ny, nx, r, c, T)
        plan = st.describe()
        plan.pop("sections", None)
        ms = _event_time(lambda: st.run(dA.data_ptr(), out.data_ptr(), stream.cuda_stream), args.steps, args.warmup,
                         stream)
        assert st.check(stream.cuda_stream) == 0
        st.close()
        pts = ny * nx
        gbs = 8 * pts / (ms * 1e-3) / 1e9
        tflops = 2 * 9 * T * pts / (ms * 1e-3) / 1e12
        res[f"steps_{T}"] = {
            "ms": ms, "point_updates_per_s": pts * T / (ms * 1e-3), "plan": plan,
            "roofline_hbm": {"achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak, "peak_kind": kind,
                             "algorithmic_bytes": 8 * pts},
            "roofline_alu": {"achieved": tflops, "peak": FP32_FMA_TFLOPS, "unit": "TFLOP/s",
                             "frac": tflops / FP32_FMA_TFLOPS, "flops": 2 * 9 * T * pts,
                             "peak_kind": "derived (152 SMs x 128 FP32 lanes x 2 x 2.07 GHz)"}}
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import stencil as so
        sub = A[:1024, :1024].astype(np.float64)
        t0 = time.perf_counter()
        so.steps(sub, c, r, 1)
        dt = time.perf_counter() - t0
        cpu = {"value": sub.size / dt, "unit": "point updates/s", "cores": 1, "kind": "oracle",
               "sample": "one step of the 9-point stencil on the 1024 x 1024 corner (FP64 numpy slices)"}
    print(json.dumps({"workload": f"stencil nest {ny} x {nx} FP32, 9-point diffusion stencil, zero ghost surface",
                      "metric": "stencil point updates/s", "steps": args.steps, "warmup": args.warmup,
                      "results": res, "cpu_baseline": cpu, "l2": "inputs (1 GiB) larger than L2; no flush"}))


def run_ordered_workload(args):
    """Ordered reductions with a non-commutative operator (--ordered-op), 64 rows:
    compose: 2^22 affine maps per row (a uniform [0.9, 1) seed 12, b normal seed
    13), composed in iteration order (the last value of y = a y + b from 0, and
    the product of a); 2 GiB.  mat2: 2^21 two-state Markov matrices per row
    [[1-p, p], [q, 1-q]] (p seed 12, q seed 13, uniform [0, 1)) multiplied in
    order; 2 GiB.  last: 2^22 values per row (normal seed 13), 90% of them
    missing (NaN where a uniform seed-12 draw < 0.9), the last value present;
    1 GiB.  Inputs are larger than L2."""
    import torch

    from paper_2309_01906_gb300 import binding as hb
    from paper_2309_01906_gb300 import synth
    op = args.ordered_op
    O, R = args.ordered_rows, args.ordered_len // (2 if op == "mat2" else 1)
    u = torch.from_numpy(synth.uniform_f32(O * R, 0.9 if op == "compose" else 0.0, 1.0, 12)).cuda()
    w = torch.from_numpy(synth.uniform_f32(O * R, 0.0, 1.0, 13) if op == "mat2" else synth.normal_f32(O * R, 13)).cuda()
    if op == "compose":
        ins, nout, ib = [u, w], 2, 8
        what = "composition of affine maps in iteration order"
    elif op == "mat2":
        ins, nout, ib = [torch.stack([1 - u, u, w, 1 - w], dim=-1).contiguous()], 4, 16
        what = "product of 2x2 Markov matrices in iteration order"
    else:
        ins, nout, ib = [torch.where(u < 0.9, torch.full_like(w, float("nan")), w)], 1, 4
        what = "last value present (90% missing)"
    del u, w
    out = torch.empty(nout * O, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    n = hb.Nest([O, R], 1, {"compose": "compose", "mat2": "mat2", "last": "last"}[op], "f32", "load")
    plan = n.describe()
    ptrs = [t.data_ptr() for t in ins]
    ms = _event_time(lambda: n.run(ptrs, out.data_ptr(), stream.cuda_stream), args.steps, args.warmup, stream)
    n.close()
    peak, kind = measured_peaks()
    nbytes = ib * O * R + 4 * nout * O
    gbs = nbytes / (ms * 1e-3) / 1e9
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import ordered as oo
        m = min(R, 1 << 20)
        row = [t[:m].cpu().numpy() for t in ins]
        t0 = time.perf_counter()
        if op == "compose":
            oo.compose(row[0].astype(np.float64), row[1].astype(np.float64))
        elif op == "mat2":
            oo.mat2_product(row[0])
        else:
            oo.last_valid(row[0])
        dt = time.perf_counter() - t0
        cpu = {"value": m / dt, "unit": "iterations/s", "cores": 1, "kind": "oracle",
               "sample": f"the first {m} iterations of row 0, in order"}
    print(json.dumps({"workload": f"ordered reduction {O} x {R}: {what}", "op": op,
                      "metric": "nest iterations/s", "value": O * R / (ms * 1e-3), "unit": "iterations/s",
                      "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup, "plan": plan,
                      "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                                   "peak_kind": kind, "algorithmic_bytes": nbytes},
                      "cpu_baseline": cpu, "l2": f"inputs ({nbytes / 2**30:.1f} GiB) larger than L2; no flush"}))

def run_narrow_workload(args):
    """Nests on 8- / 16-bit integers with SIMD-in-register sub-lanes: 1 GiB of
    uniform values (seed 14) as 16384 (--narrow-rows) x 65536 int8 (dot with an
    int8 vector, seed 15; sum; max) and 16384 x 32768 int16 (sum; max).
    Inputs > L2."""
    import torch

    from paper_2309_01906_gb300 import binding as hb
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence(14)))
    O = args.narrow_rows
    stream = torch.cuda.Stream()
    peak, kind = measured_peaks()
    res = {}
    cases = [("i8_dot", "i8", "sum", "dot_bcast", 65536), ("i8_sum", "i8", "sum", "load", 65536),
             ("i8_max", "i8", "max", "load", 65536), ("i16_sum", "i16", "sum", "load", 32768),
             ("i16_max", "i16", "max", "load", 32768)]
    if args.narrow_cases:
        cases = [c for c in cases if c[0] in args.narrow_cases.split(",")]
    cpu = None
    for name, prec, op, body, R in cases:
        tdt = torch.int8 if prec == "i8" else torch.int16
        dA = torch.randint(-128 if prec == "i8" else -32768, 128 if prec == "i8" else 32768, (O * R,), dtype=tdt,
                           device="cuda", generator=torch.Generator("cuda").manual_seed(int(g.integers(1 << 30))))
        ins = [dA.data_ptr()]
        if body == "dot_bcast":
            dw = torch.randint(-128, 128, (R,), dtype=torch.int8, device="cuda",
                               generator=torch.Generator("cuda").manual_seed(15))
            ins.append(dw.data_ptr())
        out = torch.empty(O, dtype=torch.int32, device="cuda")
        n = hb.Nest([O, R], 1, op, prec, body)
        ms = _event_time(lambda: n.run(ins, out.data_ptr(), stream.cuda_stream), args.steps, args.warmup, stream)
        plan = n.describe()
        n.close()
        nbytes = dA.numel() * dA.element_size() + 4 * O
        gbs = nbytes / (ms * 1e-3) / 1e9
        if name == "i8_dot" and not args.no_cpu_baseline:
            import oracle
            rows, dt = 1, 0.0
            Ah = dA[: 1024 * R].cpu().numpy().astype(np.int32)
            wh = dw.cpu().numpy().astype(np.int32)
            while rows <= 1024:   # grow the sample until it takes about 2 s
                t0 = time.perf_counter()
                oracle.rect([rows, R], 1, "sum", "i32", "dot_bcast", A=Ah[: rows * R], w=wh)
                dt = time.perf_counter() - t0
                if dt > 2.0 or rows == 1024:
                    break
                rows *= 2
            cpu = {"value": rows * R / dt, "unit": "iterations/s", "cores": 1, "kind": "oracle",
                   "sample": f"i8_dot: {rows} rows of {R} (int32 definition on the widened inputs)"}
        res[name] = {"ms": ms, "iterations_per_s": O * R / (ms * 1e-3), "plan": {k: plan[k] for k in
                     ("team", "warps", "grid_parts", "vec", "simd", "kernel")},
                     "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                                  "peak_kind": kind, "algorithmic_bytes": nbytes}}
        del dA
    print(json.dumps({"workload": f"nests on 8- / 16-bit integers, {O} x 64 KiB each, SIMD-in-register sub-lanes",
                      "metric": "nest iterations/s", "steps": args.steps, "warmup": args.warmup, "results": res,
                      "cpu_baseline": cpu, "data": "synthetic (seeded on the device)", "l2": "inputs (64 KiB per row) larger than L2 from 2048 rows on; no flush"}))


def make_uneven_batch(n_nests, seed=9, tune=False, stream=None):
    """The batched workload: n_nests shapes drawn as in synth.uneven_shapes, their
    inputs packed into two device buffers (FP32 for sums, int32 for max), 16-byte
    aligned per nest; outputs likewise.  Returns a dict of nests, pointers, sizes."""
    import torch

    from paper_2309_01906_gb300 import binding as hb
    from paper_2309_01906_gb300 import synth
    shapes = synth.uneven_shapes(n_nests=n_nests, seed=seed)
    off_in = {"f": 0, "i": 0}
    off_out = {"f": 0, "i": 0}
    place = []
    for sh in shapes:
        k = "f" if sh.op == "sum" else "i"
        place.append((k, off_in[k], off_out[k]))
        off_in[k] += (sh.size + 3) // 4 * 4
        off_out[k] += (max(sh.n_out, 1) + 3) // 4 * 4
    host = {"f": np.empty(max(off_in["f"], 4), np.float32), "i": np.empty(max(off_in["i"], 4), np.int32)}
    from concurrent.futures import ThreadPoolExecutor

    def fill(i):
        k, oi, _ = place[i]
        host[k][oi:oi + shapes[i].size] = synth.nest_input(shapes[i], i, seed)
    with ThreadPoolExecutor(max(1, min(32, os.cpu_count() or 1))) as ex:
        list(ex.map(fill, range(len(shapes))))
    dev_in = {"f": torch.from_numpy(host["f"]).cuda(), "i": torch.from_numpy(host["i"]).cuda()}
    dev_out = {"f": torch.zeros(max(off_out["f"], 4), dtype=torch.float32, device="cuda"),
               "i": torch.zeros(max(off_out["i"], 4), dtype=torch.int32, device="cuda")}
    ins = [[dev_in[place[i][0]].data_ptr() + 4 * place[i][1]] for i in range(len(shapes))]
    outs = [dev_out[place[i][0]].data_ptr() + 4 * place[i][2] for i in range(len(shapes))]
    tuned_classes = 0
    if tune:
        # one representative per shape class is timed; the rest take the cached binding
        def clog2(v):
            return 0 if v <= 1 else (v - 1).bit_length()
        seen = set()
        sp = stream.cuda_stream if stream is not None else 0
        for i, sh in enumerate(shapes):
            R = sh.size // max(sh.n_out, 1) if sh.n_out else 0
            key = (clog2(sh.n_out), clog2(R), R % 4 == 0, sh.op, sh.prec)
            if key in seen:
                continue
            seen.add(key)
            n = hb.Nest(list(sh.extents), sh.red_level, sh.op, sh.prec, "load")
            n.tune(ins[i], outs[i], sp, batched=True)   # timed in the executor the nests run in
            n.close()
        tuned_classes = len(seen)
    nests = [hb.Nest(list(sh.extents), sh.red_level, sh.op, sh.prec, "load") for sh in shapes]
    return {"shapes": shapes, "nests": nests, "ins": ins, "outs": outs, "dev_in": dev_in, "dev_out": dev_out,
            "tuned_classes": tuned_classes,
            "host": host, "place": place, "bytes": int(sum(sh.size for sh in shapes)) * 4,
            "iters": int(sum(sh.size for sh in shapes))}


def _plan_class(d):
    """Plan class of a described nest: team / lanes or warps [/ split]."""
    return f"{d['team']}/{d['team_lanes'] if d['team'] == 'lanes' else d['warps']}" + \
        ("/split" if d["grid_parts"] > 1 else "")


def batch_parity(wl, idxs, threads):
    """CPU-baseline leg of the batched workload: the oracle evaluates the listed
    nests (all their outputs) on `threads` host threads; the batched outputs are
    compared with it (FP32 compensated sums within 1e-6 of the normalized
    error, int32 max bit for bit).  Returns (parity dict, oracle seconds)."""
    import oracle
    import torch
    from paper_2309_01906_gb300 import synth

    def one(i):
        sh = wl["shapes"][i]
        A = synth.nest_input(sh, i, 9)
        return oracle.rect(list(sh.extents), sh.red_level, sh.op, sh.prec, "load", A=A)

    t0 = time.perf_counter()
    refs = threaded(one, idxs, threads)
    dt = time.perf_counter() - t0
    worst, n_fp, n_int, int_ok, bound_ok, n_out = 0.0, 0, 0, True, True, 0
    for i, ref in zip(idxs, refs):
        sh = wl["shapes"][i]
        k, _, oo = wl["place"][i]
        got = wl["dev_out"][k][oo:oo + sh.n_out].cpu().numpy() if sh.n_out else np.zeros(0)
        n_out += sh.n_out
        if sh.op == "sum":
            n_fp += 1
            p = fp_parity(got, ref, "f32_comp", wl["nests"][i].error_bound(), 1e-6)
            worst = max(worst, p["max_norm_err"])
            bound_ok &= p["within_a_priori_bound"]
        else:
            n_int += 1
            int_ok &= bool(np.array_equal(got.astype(np.int64), ref.values))
    torch.cuda.synchronize()
    return ({"nests_checked": len(idxs), "outputs_checked": n_out, "fp32_comp_sum_nests": n_fp,
             "int32_max_nests": n_int, "max_norm_err": worst, "tolerance": 1e-6,
             "within_a_priori_bound": bool(bound_ok), "int32_bit_exact": bool(int_ok),
             "pass": bool(worst <= 1e-6 and bound_ok and int_ok),
             "sample": f"{len(idxs)} nests drawn with seed 19 from the same 10,000 (sigma 2, T up to 2^24)"}, dt)


def batch_measure(args):
    """Batched uneven nests: one persistent launch per arithmetic under a CUDA graph
    vs one hp_nest_run per nest (same plans, same stream, no graph).  Batched
    outputs must equal the per-nest ones bit for bit; a seeded sample of nests
    is checked against the oracle."""
    import torch

    from paper_2309_01906_gb300 import binding as hb
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    wl = make_uneven_batch(args.batch_nests, tune=args.tune, stream=stream)
    setup_s = time.perf_counter() - t0
    if args.batch_class:
        # keep only the nests of one plan class (to time or profile it alone)
        keep = [i for i, nest in enumerate(wl["nests"]) if _plan_class(nest.describe()) == args.batch_class]
        if not keep:
            raise SystemExit(f"no nest of plan class {args.batch_class!r}")
        for i, nest in enumerate(wl["nests"]):
            if i not in set(keep):
                nest.close()
        for k in ("shapes", "nests", "ins", "outs", "place"):
            wl[k] = [wl[k][i] for i in keep]
        wl["bytes"] = int(sum(sh.size for sh in wl["shapes"])) * 4
        wl["iters"] = int(sum(sh.size for sh in wl["shapes"]))
    sp = stream.cuda_stream
    handles = [n.handle for n in wl["nests"]]
    # arguments marshalled once for both forms: the timed region holds only the
    # library calls (one per nest, or one per batch)
    runs = [hb.PreparedRun(n.handle, i, o) for n, i, o in zip(wl["nests"], wl["ins"], wl["outs"])]
    prepared = hb.PreparedBatch(handles, wl["ins"], wl["outs"])

    def plain():
        for r in runs:
            r(sp)

    def batched():
        hb.hp_nest_run_batch(prepared, stream=sp)

    steps = max(1, min(args.steps, 20))
    breakdown = {}
    if args.batch_breakdown:
        # each plan class batched alone: where the batched time goes
        classes = {}
        for idx, nest in enumerate(wl["nests"]):
            classes.setdefault(_plan_class(nest.describe()), []).append(idx)
        for key, idxs in classes.items():
            pb = hb.PreparedBatch([handles[i] for i in idxs], [wl["ins"][i] for i in idxs],
                                  [wl["outs"][i] for i in idxs])
            ms = _event_time(lambda: hb.hp_nest_run_batch(pb, stream=sp), steps, args.warmup, stream)
            nbytes = sum(wl["shapes"][i].size for i in idxs) * 4
            breakdown[key] = {"nests": len(idxs), "bytes": nbytes, "ms": ms, "gbs": nbytes / (ms * 1e-3) / 1e9}
    plain_steps = max(1, min(steps, args.batch_plain_steps))
    ms_plain = _event_time(plain, plain_steps, min(args.warmup, 3), stream)
    ref = {k: v.clone() for k, v in wl["dev_out"].items()}
    ms_batch = _event_time(batched, steps, args.warmup, stream)
    same = all(torch.equal(ref[k], wl["dev_out"][k]) for k in ref)
    peak, kind = measured_peaks()
    n = len(wl["nests"])
    teams = {}
    for nest in wl["nests"]:
        key = _plan_class(nest.describe())
        teams[key] = teams.get(key, 0) + 1
    parity, cpu = None, None
    if args.batch_check > 0 and not args.no_cpu_baseline:
        g = np.random.Generator(np.random.PCG64(19))
        idxs = sorted(int(i) for i in g.choice(n, size=min(n, args.batch_check), replace=False))
        threads = host_cores()["affinity"]
        parity, dt = batch_parity(wl, idxs, threads)
        it = int(sum(wl["shapes"][i].size for i in idxs))
        cpu = {"value": len(idxs) / dt, "unit": "nests/s", "iterations_per_s": it / dt, "cores": threads,
               "kind": "oracle", "sample": f"{len(idxs)} of the {n} nests ({it} iterations), whole nests"}
    gbs = wl["bytes"] / (ms_batch * 1e-3) / 1e9
    res = {
        "workload": f"{n} uneven nests (depth 2-5, lognormal sizes), FP32 compensated sums and int32 max",
        "metric": "nests/s", "iterations": wl["iters"], "input_bytes": wl["bytes"],
        "batched": {"ms": ms_batch, "nests_per_s": n / (ms_batch * 1e-3),
                    "iterations_per_s": wl["iters"] / (ms_batch * 1e-3)},
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                     "peak_kind": kind, "algorithmic_bytes": wl["bytes"], "kernel": "batch_kernel"},
        "plain_one_launch_per_nest": {"ms": ms_plain, "nests_per_s": n / (ms_plain * 1e-3),
                                      "achieved_gbs": wl["bytes"] / (ms_plain * 1e-3) / 1e9, "steps": plain_steps},
        "speedup": ms_plain / ms_batch, "bit_identical_to_per_nest_runs": bool(same),
        "plans": teams, "breakdown": breakdown, "tuned_classes": wl["tuned_classes"], "setup_s": setup_s,
        "parity": parity, "cpu_baseline": cpu, "steps": steps, "warmup": args.warmup,
        "l2": "inputs (16 GB) larger than L2; no flush"}
    for nest in wl["nests"]:
        nest.close()
    return res


def run_batch_workload(args):
    print(json.dumps(batch_measure(args)))


def serve_measure(args):
    """Serving: a Poisson stream of nest requests (seed 10) at --serve-rate for
    --serve-seconds; shapes drawn as in the batched workload (seed 9), all FP32
    compensated sums over pre-generated device inputs; 40 GiB admission budget.
    The same arrival sequence is served, one after the other, by the resident
    server (a persistent kernel fed through mapped host memory), the server
    that launches batched steps and the plain per-request server
    (--serve-modes).  Latency runs from each request's scheduled arrival to
    the server observing its completion (hp_serve_submit_at), so a client that
    falls behind its schedule counts its lag.  A seeded 1% of the requests
    write to outputs of their own; each is compared bit for bit with a single
    hp_nest_run of its nest and, in the CPU-baseline leg, with the oracle."""
    import torch

    from paper_2309_01906_gb300 import binding as hb
    from paper_2309_01906_gb300 import synth
    n_pool = args.serve_pool
    shapes = synth.uneven_shapes(n_nests=n_pool, seed=9, sum_prec="f32_comp")
    t_setup = time.perf_counter()
    hosts = threaded(lambda i: synth.normal_f32(shapes[i].size, 9, 1 + i), range(n_pool), 4)
    pool = []
    for i, sh in enumerate(shapes):
        n = hb.Nest(list(sh.extents), sh.red_level, "sum", "f32_comp", "load")
        outs = [torch.empty(max(sh.n_out, 1), dtype=torch.float32, device="cuda") for _ in range(4)]
        pool.append((n, torch.from_numpy(hosts[i]).cuda(), outs, sh))
    arrivals = synth.poisson_arrivals(rate=args.serve_rate, duration=args.serve_seconds, seed=10)
    pick = np.random.Generator(np.random.PCG64(np.random.SeedSequence(10, spawn_key=(1,)))).integers(
        0, n_pool, arrivals.size)
    g_s = np.random.Generator(np.random.PCG64(np.random.SeedSequence(10, spawn_key=(2,))))
    sampled = np.sort(g_s.choice(arrivals.size, size=max(1, int(arrivals.size * args.serve_check)), replace=False))
    sampled_set = set(int(j) for j in sampled)
    # single-run results of every sampled nest (the same plan: the served bits must equal them)
    stream = torch.cuda.current_stream().cuda_stream
    single = {}
    for k in sorted(set(int(pick[j]) for j in sampled)):
        n, dA, _, sh = pool[k]
        o = torch.empty(max(sh.n_out, 1), dtype=torch.float32, device="cuda")
        n.run([dA.data_ptr()], o.data_ptr(), stream)
        single[k] = o
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    iters = float(np.mean([pool[k][3].size for k in pick]))

    def serve(mode):
        hb.hp_set_option("serve_batching", mode)
        try:
            server = hb.hp_serve_create(40 << 30, 4096, 4)
        finally:
            hb.hp_set_option("serve_batching", 1)
        use = [0] * n_pool
        lags = np.zeros(arrivals.size)
        own = {}
        for j in sampled:
            sh = pool[int(pick[j])][3]
            own[int(j)] = torch.full((max(sh.n_out, 1),), float("nan"), dtype=torch.float32, device="cuda")
        # every argument of every submission marshalled before the stream starts,
        # so that the client's own call overhead stays small (it is inside the
        # latency: the clock starts at the scheduled arrival)
        in_arrs = [hb._ptr_array([dA.data_ptr()]) for (_, dA, _, _) in pool]
        handles = [n.handle for (n, _, _, _) in pool]
        out_ptrs = []
        for j in range(arrivals.size):
            k = int(pick[j])
            if j in sampled_set:
                out_ptrs.append(own[j].data_ptr())
            else:
                out_ptrs.append(pool[k][2][use[k] % 4].data_ptr())
                use[k] += 1
        submit_at = hb.lib().hp_serve_submit_at
        ticket = ctypes.c_uint64()
        ticket_ref = ctypes.byref(ticket)
        ks = [int(k) for k in pick]
        t_arrs = (arrivals * 1e6).tolist()
        lag = np.full(arrivals.size, 1.0)   # written (so its pages are mapped) before the stream
        torch.cuda.synchronize()
        clock = hb.lib().hp_serve_clock_us
        # the garbage collector stays off while the stream runs: its full passes
        # over the process's objects stalled this client thread for up to 143 ms;
        # the loop keeps no object per request alive (the lags go to a float
        # array), so it allocates no new memory while the stream runs
        gc.collect()
        gc.disable()
        try:
            t0 = clock()
            for j in range(arrivals.size):
                due = t0 + t_arrs[j]
                now = clock()
                while now < due:
                    now = clock()
                lag[j] = now - due
                k = ks[j]
                if submit_at(server, handles[k], in_arrs[k], out_ptrs[j], due, ticket_ref) != 0:
                    raise RuntimeError("hp_serve_submit_at: " + hb.hp_last_error())
        finally:
            gc.enable()
        lags[:] = lag
        hb.hp_serve_poll(server, ticket.value, -1)
        deadline = time.perf_counter() + 120
        while hb.hp_serve_counters(server)["completed"] < arrivals.size and time.perf_counter() < deadline:
            time.sleep(0.01)
        st = hb.hp_serve_stats(server)
        c = hb.hp_serve_counters(server)
        hb.hp_serve_destroy(server)
        torch.cuda.synchronize()
        same = all(torch.equal(own[int(j)], single[int(pick[j])]) for j in sampled)
        st.update({"completed": c["completed"], "steps": c["steps"], "peak_bytes": c["peak_bytes"],
                   "peak_slots": c["peak_slots"], "submit_lag_us_p50": float(np.median(lags)),
                   "submit_lag_us_p99": float(np.quantile(lags, 0.99)), "submit_lag_us_max": float(lags.max()),
                   "sampled_bit_identical_to_single_runs": bool(same)})
        return st, own

    modes = [int(m) for m in args.serve_modes.split(",")]
    skipped = {"skipped": "not in --serve-modes", "p50_us": 0.0, "p99_us": 0.0, "p999_us": 0.0,
               "sampled_bit_identical_to_single_runs": True}
    resident, own_r = serve(2) if 2 in modes else (dict(skipped), None)
    batched, own_b = serve(1) if 1 in modes else (dict(skipped), None)
    plain, own_p = serve(0) if 0 in modes else (dict(skipped), None)
    if own_r is None:
        own_r = own_b if own_b is not None else own_p
    # CPU-baseline leg: the oracle on every distinct sampled nest; the served outputs against it
    parity, cpu = None, None
    if not args.no_cpu_baseline:
        import oracle
        ks = sorted(single)
        threads = host_cores()["affinity"]
        t1 = time.perf_counter()
        refs = dict(zip(ks, threaded(lambda k: oracle.rect(list(pool[k][3].extents), pool[k][3].red_level, "sum",
                                                           "f32_comp", "load", A=hosts[k]), ks, threads)))
        dt = time.perf_counter() - t1
        worst, bound_ok = 0.0, True
        for j in sampled:
            k = int(pick[j])
            sh = pool[k][3]
            got = own_r[int(j)][:sh.n_out].cpu().numpy() if sh.n_out else np.zeros(0)
            p = fp_parity(got, refs[k], "f32_comp", pool[k][0].error_bound(), 1e-6)
            worst = max(worst, p["max_norm_err"])
            bound_ok &= p["within_a_priori_bound"]
        parity = {"requests_checked": int(sampled.size), "distinct_nests": len(ks), "max_norm_err": worst,
                  "tolerance": 1e-6, "within_a_priori_bound": bool(bound_ok),
                  "pass": bool(worst <= 1e-6 and bound_ok and resident["sampled_bit_identical_to_single_runs"]
                               and batched["sampled_bit_identical_to_single_runs"]),
                  "sample": f"seeded {100 * args.serve_check:.0f}% of the requests of the resident run (the "
                            "batched run's sample bit-identical to single runs too)"}
        it = int(sum(pool[k][3].size for k in ks))
        cpu = {"value": len(ks) / dt, "unit": "nests/s", "iterations_per_s": it / dt, "cores": threads,
               "kind": "oracle", "sample": f"{len(ks)} distinct sampled nests ({it} iterations)"}
    res = {
        "workload": f"Poisson {args.serve_rate:.0f} req/s for {args.serve_seconds:.0f} s, {arrivals.size} requests over "
                    f"{n_pool} pre-generated uneven nests (FP32 compensated sums), 40 GiB budget, 4 streams",
        "metric": "latency from scheduled arrival (us) and nests/s",
        "mean_iterations_per_request": iters, "offered_gbs": args.serve_rate * iters * 4 / 1e9,
        "resident": resident, "batched": batched, "plain_per_request": plain,
        "p99_speedup": plain["p99_us"] / resident["p99_us"] if resident["p99_us"] and plain["p99_us"] else None,
        "p99_speedup_launched_batches": plain["p99_us"] / batched["p99_us"] if batched["p99_us"] and plain["p99_us"] else None,
        "parity": parity, "cpu_baseline": cpu, "setup_s": setup_s}
    for n, _, _, _ in pool:
        n.close()
    return res


def run_serve_workload(args):
    print(json.dumps(serve_measure(args)))


EXTRAS = {"gemv": lambda a: gemv_measure(a), "csr": lambda a: csr_measure(a), "batch": lambda a: batch_measure(a),
          "serve": lambda a: serve_measure(a)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="hp", choices=["hp", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-outputs", type=int, default=512)
    ap.add_argument("--profile-b", type=int, default=0,
                    help="profiler case: run only the headline nest with this outer extent b")
    ap.add_argument("--prec", default="f32_comp", choices=["f32_comp", "f32"])
    ap.add_argument("--workload", default="nest4", choices=["nest4", "csr", "gemv", "batch", "serve", "stencil", "ordered", "narrow"],
                    help="nest4: the headline line; csr / gemv: measurement of the other workloads")
    ap.add_argument("--csr-rows", type=int, default=1 << 22)
    ap.add_argument("--stencil-n", type=int, default=16384, help="stencil: array side")
    ap.add_argument("--ordered-rows", type=int, default=64, help="ordered: rows (outputs)")
    ap.add_argument("--ordered-len", type=int, default=1 << 22, help="ordered: maps per row (half for mat2)")
    ap.add_argument("--ordered-op", default="compose", choices=["compose", "mat2", "last"],
                    help="ordered: the non-commutative operator")
    ap.add_argument("--narrow-rows", type=int, default=16384, help="narrow: rows (outputs) of 64 KiB")
    ap.add_argument("--narrow-cases", default="", help="narrow: comma list of cases to keep (e.g. i8_dot,i16_sum)")
    ap.add_argument("--stencil-steps", default="1,4", help="stencil: steps per launch to time (comma list)")
    ap.add_argument("--batch-nests", type=int, default=10000)
    ap.add_argument("--batch-breakdown", action="store_true", help="batch: also time each plan class alone")
    ap.add_argument("--batch-class", default="", help="batch: keep only the nests of this plan class (e.g. lanes/1)")
    ap.add_argument("--tune", action="store_true", help="batch: autotune one nest per shape class first")
    ap.add_argument("--serve-rate", type=float, default=20000.0)
    ap.add_argument("--serve-seconds", type=float, default=None,
                    help="serve: seconds of arrivals (60 for --workload serve, 10 inside the headline line)")
    ap.add_argument("--serve-pool", type=int, default=2000)
    ap.add_argument("--serve-modes", default="2,1,0",
                    help="serve: servers to run (2 resident kernel, 1 batched launches, 0 plain launches)")
    ap.add_argument("--no-hist", action="store_true", help="csr: SpMV without the fused histogram")
    ap.add_argument("--extras", default="gemv,serve,csr,batch",
                    help="nest4: other workloads measured after the headline and added to its line "
                         "(comma list of gemv, serve, csr, batch, in that order by default: the latency-"
                         "sensitive serving stream runs before the large CSR and batch workloads; 'none' "
                         "for the headline alone)")
    ap.add_argument("--parity-out", default="", help="nest4: write the per-result error table (CSV) here")
    ap.add_argument("--batch-check", type=int, default=256, help="batch: nests compared with the oracle")
    ap.add_argument("--batch-plain-steps", type=int, default=3, help="batch: timed passes of one launch per nest")
    ap.add_argument("--serve-check", type=float, default=0.01, help="serve: fraction of requests checked")
    ap.add_argument("--gemv-map", default="", help="gemv: level map, e.g. grid,warp (default: the planner's)")
    args = ap.parse_args()
    args.gemv_map = [x.strip() for x in args.gemv_map.split(",")] if args.gemv_map else None
    if args.serve_seconds is None:
        args.serve_seconds = 60.0 if args.workload == "serve" else 10.0
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.profile_b:
        run_profile_case(args)
    elif args.workload == "csr":
        run_csr_workload(args)
    elif args.workload == "narrow":
        run_narrow_workload(args)
    elif args.workload == "ordered":
        run_ordered_workload(args)
    elif args.workload == "stencil":
        run_stencil_workload(args)
    elif args.workload == "gemv":
        run_gemv_workload(args)
    elif args.workload == "batch":
        run_batch_workload(args)
    elif args.workload == "serve":
        run_serve_workload(args)
    else:
        run_hp(args)


if __name__ == "__main__":
    main()
