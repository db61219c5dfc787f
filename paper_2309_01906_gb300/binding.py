"""Thin ctypes binding of libhp.so (include/hp.h), same names as the C ABI.

Argument marshalling only: every step of the nest runs in the library's CUDA
kernels.  There is no CPU fallback: if libhp.so is missing the first call
raises, and on a machine without a GPU runs return HP_ECUDA.

Device buffers are passed as integer addresses (e.g. ``tensor.data_ptr()``);
streams as integer ``cudaStream_t`` handles (``torch.cuda.current_stream().cuda_stream``)
or 0 for the legacy default stream.
"""
from __future__ import annotations

import ctypes
import json
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhp.so")

# ---- enums (include/hp.h)
HP_OK, HP_EINVAL, HP_ENOMEM, HP_EBUSY, HP_EAGAIN, HP_ETIMEOUT, HP_ECUDA, HP_EUNSUPPORTED = range(8)
STATUS_NAMES = ["HP_OK", "HP_EINVAL", "HP_ENOMEM", "HP_EBUSY", "HP_EAGAIN", "HP_ETIMEOUT", "HP_ECUDA",
                "HP_EUNSUPPORTED"]
HP_HW_GRID, HP_HW_CLUSTER, HP_HW_CTA, HP_HW_WARP, HP_HW_SUBWARP, HP_HW_LANE, HP_HW_SEQ, HP_HW_AUTO = range(8)
HP_RED_SUM, HP_RED_MAX, HP_RED_MIN, HP_RED_HIST_COUNT = range(4)
HP_F32, HP_F32_COMP, HP_I32, HP_I64 = range(4)
HP_BODY_LOAD, HP_BODY_DOT_BCAST, HP_BODY_CSR_GATHER, HP_BODY_AFFINE, HP_BODY_GEOMETRIC = range(5)
HP_MAX_DEPTH = 5

HW = {"grid": HP_HW_GRID, "cluster": HP_HW_CLUSTER, "cta": HP_HW_CTA, "warp": HP_HW_WARP,
      "subwarp": HP_HW_SUBWARP, "lane": HP_HW_LANE, "seq": HP_HW_SEQ, "auto": HP_HW_AUTO}
OPS = {"sum": HP_RED_SUM, "max": HP_RED_MAX, "min": HP_RED_MIN, "hist": HP_RED_HIST_COUNT, "compose": 4,
       "mat2": 5, "last": 6}
PRECS = {"f32": HP_F32, "f32_comp": HP_F32_COMP, "i32": HP_I32, "i64": HP_I64, "i8": 4, "i16": 5}
BODIES = {"load": HP_BODY_LOAD, "dot_bcast": HP_BODY_DOT_BCAST, "csr_gather": HP_BODY_CSR_GATHER,
          "affine": HP_BODY_AFFINE, "geometric": HP_BODY_GEOMETRIC}

# every entry point include/hp.h declares
EXPORTED = ["hp_nest_create", "hp_nest_run", "hp_nest_run_comp", "hp_nest_run_host", "hp_nest_run_static", "hp_nest_run_batch",
            "hp_nest_tune", "hp_nest_tune_req", "hp_nest_error_bound",
            "hp_nest_describe", "hp_nest_check", "hp_nest_destroy", "hp_serve_create", "hp_serve_submit",
            "hp_serve_submit_at", "hp_serve_clock_us", "hp_probe_gather",
            "hp_serve_poll", "hp_serve_stats", "hp_serve_counters", "hp_serve_destroy", "hp_set_option", "hp_get_option",
            "hp_last_error", "hp_version", "hp_stencil_create", "hp_stencil_run", "hp_stencil_describe",
            "hp_stencil_check", "hp_stencil_destroy", "hp_level_properties", "hp_level_select",
            "hp_level_check"]

# level properties (Sec. 3.2)
PROPS = {"barrier": 1 << 0, "critical": 1 << 1, "atomic": 1 << 2, "shuffle": 1 << 3, "oversub": 1 << 4,
         "dynamic": 1 << 5, "lockstep": 1 << 6, "progress": 1 << 7, "globalmem": 1 << 8, "localmem": 1 << 9,
         "groupmem": 1 << 10, "cache": 1 << 11}
HW_NAMES = {v: k for k, v in HW.items()}


class hp_level_req(ctypes.Structure):
    _fields_ = [("sync", ctypes.c_uint32), ("reserve", ctypes.c_uint32), ("min_num", ctypes.c_int64)]


class hp_stencil_map(ctypes.Structure):
    _fields_ = [("section_y", ctypes.c_int64), ("section_x", ctypes.c_int64), ("tile_y", ctypes.c_int32),
                ("tile_x", ctypes.c_int32)]


class hp_level_map(ctypes.Structure):
    _fields_ = [("hw", ctypes.c_int32), ("sub_width", ctypes.c_int32), ("tile", ctypes.c_int64)]


class hp_affine_params(ctypes.Structure):
    _fields_ = [("a", ctypes.c_int64), ("b", ctypes.c_int64), ("m", ctypes.c_int64)]


class hp_geometric_params(ctypes.Structure):
    _fields_ = [("q", ctypes.c_double), ("m", ctypes.c_int64)]


class hp_csr_params(ctypes.Structure):
    _fields_ = [("nnz", ctypes.c_int64), ("n_cols", ctypes.c_int64), ("hist_shift", ctypes.c_int32),
                ("fuse_hist", ctypes.c_int32), ("n_bins", ctypes.c_int64)]


class HPError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")


_lib = None
_lock = threading.Lock()


def lib() -> ctypes.CDLL:
    """Load libhp.so (raises if it was not built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2309_01906_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        p, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
        L.hp_nest_create.restype = i32
        L.hp_nest_create.argtypes = [i32, p, p, i64, p, i32, i32, i32, i32, p, ctypes.POINTER(p)]
        L.hp_nest_run.restype = i32
        L.hp_nest_run.argtypes = [p, p, p, p]
        L.hp_nest_run_comp.restype = i32
        L.hp_nest_run_comp.argtypes = [p, p, p, p, p]
        L.hp_nest_run_host.restype = i32
        L.hp_nest_run_host.argtypes = [p, p, p, p]
        L.hp_nest_run_static.restype = i32
        L.hp_nest_run_static.argtypes = [p, p, p, p]
        L.hp_nest_run_batch.restype = i32
        L.hp_nest_run_batch.argtypes = [p, p, p, i32, p]
        L.hp_nest_tune.restype = i32
        L.hp_nest_tune.argtypes = [p, p, p, p, ctypes.c_int32]
        L.hp_nest_error_bound.restype = i32
        L.hp_nest_error_bound.argtypes = [p, ctypes.POINTER(ctypes.c_double)]
        L.hp_nest_describe.restype = i32
        L.hp_nest_describe.argtypes = [p, ctypes.c_char_p, ctypes.c_size_t]
        L.hp_nest_check.restype = i32
        L.hp_nest_check.argtypes = [p, p, ctypes.POINTER(ctypes.c_int32)]
        L.hp_nest_destroy.restype = None
        L.hp_nest_destroy.argtypes = [p]
        L.hp_probe_gather.restype = i32
        L.hp_probe_gather.argtypes = [p, i64, i64, ctypes.c_uint32, p, p]
        L.hp_serve_create.restype = i32
        L.hp_serve_create.argtypes = [ctypes.c_size_t, i32, i32, ctypes.POINTER(p)]
        L.hp_serve_submit.restype = i32
        L.hp_serve_submit.argtypes = [p, p, p, p, ctypes.POINTER(u64)]
        L.hp_serve_submit_at.restype = i32
        L.hp_serve_submit_at.argtypes = [p, p, p, p, ctypes.c_double, ctypes.POINTER(u64)]
        L.hp_serve_clock_us.restype = ctypes.c_double
        L.hp_serve_clock_us.argtypes = []
        L.hp_serve_poll.restype = i32
        L.hp_serve_poll.argtypes = [p, u64, i32]
        L.hp_serve_stats.restype = i32
        L.hp_serve_stats.argtypes = [p] + [ctypes.POINTER(ctypes.c_double)] * 4
        L.hp_serve_counters.restype = i32
        L.hp_serve_counters.argtypes = [p, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(ctypes.c_size_t),
                                        ctypes.POINTER(ctypes.c_int32)]
        L.hp_serve_destroy.restype = None
        L.hp_serve_destroy.argtypes = [p]
        L.hp_last_error.restype = ctypes.c_char_p
        L.hp_last_error.argtypes = []
        L.hp_version.restype = i32
        L.hp_version.argtypes = []
        L.hp_set_option.restype = i32
        L.hp_set_option.argtypes = [ctypes.c_char_p, i64]
        L.hp_get_option.restype = i32
        L.hp_get_option.argtypes = [ctypes.c_char_p, ctypes.POINTER(i64)]
        L.hp_level_properties.restype = i32
        L.hp_level_properties.argtypes = [i32, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(i64)]
        L.hp_level_select.restype = i32
        L.hp_level_select.argtypes = [i32, ctypes.POINTER(hp_level_req), ctypes.POINTER(hp_level_map)]
        L.hp_level_check.restype = i32
        L.hp_level_check.argtypes = [i32, ctypes.POINTER(hp_level_req), ctypes.POINTER(hp_level_map)]
        L.hp_nest_tune_req.restype = i32
        L.hp_nest_tune_req.argtypes = [p, ctypes.POINTER(hp_level_req), p, p, p, ctypes.c_int32]
        L.hp_stencil_create.restype = i32
        L.hp_stencil_create.argtypes = [i64, i64, i32, ctypes.POINTER(ctypes.c_float), i32,
                                        ctypes.POINTER(hp_stencil_map), ctypes.POINTER(p)]
        L.hp_stencil_run.restype = i32
        L.hp_stencil_run.argtypes = [p, p, p, p]
        L.hp_stencil_describe.restype = i32
        L.hp_stencil_describe.argtypes = [p, ctypes.c_char_p, ctypes.c_size_t]
        L.hp_stencil_check.restype = i32
        L.hp_stencil_check.argtypes = [p, p, ctypes.POINTER(ctypes.c_int32)]
        L.hp_stencil_destroy.restype = None
        L.hp_stencil_destroy.argtypes = [p]
        _lib = L
        return L


def hp_last_error() -> str:
    return lib().hp_last_error().decode()


def hp_version() -> int:
    return lib().hp_version()


def hp_set_option(name: str, value: int):
    _check(lib().hp_set_option(name.encode(), int(value)), "hp_set_option")


def hp_get_option(name: str) -> int:
    v = ctypes.c_int64()
    _check(lib().hp_get_option(name.encode(), ctypes.byref(v)), "hp_get_option")
    return v.value


def _check(st: int, where: str):
    if st != HP_OK:
        raise HPError(st, where, hp_last_error())


def _ptr_array(ptrs):
    arr = (ctypes.c_void_p * max(1, len(ptrs)))()
    for i, v in enumerate(ptrs):
        arr[i] = ctypes.c_void_p(int(v)) if v else None
    return arr


def make_map(levels):
    """levels: list of (hw, sub_width, tile) tuples or hw names -> hp_level_map array."""
    arr = (hp_level_map * len(levels))()
    for i, lv in enumerate(levels):
        if isinstance(lv, str):
            lv = (lv, 0, 0)
        hw, sw, tile = (tuple(lv) + (0, 0))[:3]
        arr[i].hw = HW[hw] if isinstance(hw, str) else int(hw)
        arr[i].sub_width = int(sw)
        arr[i].tile = int(tile)
    return arr


def hp_nest_create(depth, extents, csr_offsets, n_rows, level_map, op, red_level, prec, body, body_params=None):
    """Returns an opaque nest handle (int).  extents: list of ints or None; level_map:
    make_map() array or list or None; body_params: ctypes struct or None."""
    ext = (ctypes.c_int64 * max(1, depth))(*(extents or [])) if extents is not None else None
    mp = level_map if (level_map is None or isinstance(level_map, ctypes.Array)) else make_map(level_map)
    bp = ctypes.byref(body_params) if body_params is not None else None
    h = ctypes.c_void_p()
    off = ctypes.c_void_p(int(csr_offsets)) if csr_offsets else None
    st = lib().hp_nest_create(depth, ext, off, int(n_rows), mp, OPS.get(op, op), red_level, PRECS.get(prec, prec),
                              BODIES.get(body, body), bp, ctypes.byref(h))
    _check(st, "hp_nest_create")
    return h.value


def hp_nest_run(nest, in_ptrs, out_ptr, stream=0):
    st = lib().hp_nest_run(nest, _ptr_array(in_ptrs), out_ptr or None, stream or None)
    _check(st, "hp_nest_run")


def hp_nest_run_comp(nest, in_ptrs, out_ptr, comp_ptr, stream=0):
    """hp_nest_run of a compensated FP32 sum that also writes each output's residual."""
    st = lib().hp_nest_run_comp(nest, _ptr_array(in_ptrs), out_ptr or None, comp_ptr or None, stream or None)
    _check(st, "hp_nest_run_comp")


def hp_nest_run_host(nest, in_host_ptrs, out_host_ptr, stream=0):
    st = lib().hp_nest_run_host(nest, _ptr_array(in_host_ptrs), out_host_ptr or None, stream or None)
    _check(st, "hp_nest_run_host")


def hp_nest_run_static(nest, in_ptrs, out_ptr, stream=0):
    """Run without allocating: grid-part partials go to the library's fixed static array."""
    st = lib().hp_nest_run_static(nest, _ptr_array(in_ptrs), out_ptr or None, stream or None)
    _check(st, "hp_nest_run_static")


class PreparedBatch:
    """Marshalled arguments of hp_nest_run_batch, built once and reused."""

    def __init__(self, nests, in_ptr_lists, out_ptrs):
        n = len(nests)
        self.n = n
        self.harr = (ctypes.c_void_p * max(1, n))(*nests)
        self.keep = [_ptr_array(x) for x in in_ptr_lists]
        self.inarr = (ctypes.c_void_p * max(1, n))(*[ctypes.cast(k, ctypes.c_void_p) for k in self.keep])
        self.outarr = _ptr_array(out_ptrs)


def hp_nest_run_batch(nests, in_ptr_lists=None, out_ptrs=None, stream=0):
    """nests: list of handles (with in_ptr_lists, out_ptrs) or a PreparedBatch."""
    pb = nests if isinstance(nests, PreparedBatch) else PreparedBatch(nests, in_ptr_lists, out_ptrs)
    st = lib().hp_nest_run_batch(pb.harr, pb.inarr, pb.outarr, pb.n, stream or None)
    _check(st, "hp_nest_run_batch")


class PreparedRun:
    """Marshalled arguments of one hp_nest_run, built once and reused."""

    def __init__(self, nest, in_ptrs, out_ptr):
        self.nest = ctypes.c_void_p(nest)
        self.inarr = _ptr_array(in_ptrs)
        self.out = ctypes.c_void_p(out_ptr) if out_ptr else None

    def __call__(self, stream=0):
        st = lib().hp_nest_run(self.nest, self.inarr, self.out, stream or None)
        _check(st, "hp_nest_run")


def hp_nest_tune(nest, in_ptrs, out_ptr, stream=0, retime=False, batched=False, req=None):
    """Time candidate bindings on these buffers, install the fastest (synchronous);
    batched=True times them in the batched executor (flags bit 1); req: per-level
    requirements (as for hp_level_select) that every timed map must meet."""
    flags = (1 if retime else 0) | (2 if batched else 0)
    if req is None:
        st = lib().hp_nest_tune(nest, _ptr_array(in_ptrs), out_ptr or None, stream or None, flags)
        _check(st, "hp_nest_tune")
    else:
        st = lib().hp_nest_tune_req(nest, _req_array(req), _ptr_array(in_ptrs), out_ptr or None, stream or None, flags)
        _check(st, "hp_nest_tune_req")


def hp_nest_error_bound(nest) -> float:
    v = ctypes.c_double()
    _check(lib().hp_nest_error_bound(nest, ctypes.byref(v)), "hp_nest_error_bound")
    return v.value


def hp_nest_describe(nest) -> dict:
    buf = ctypes.create_string_buffer(8192)
    _check(lib().hp_nest_describe(nest, buf, len(buf)), "hp_nest_describe")
    return json.loads(buf.value.decode())


def hp_nest_check(nest, stream=0) -> int:
    v = ctypes.c_int32()
    st = lib().hp_nest_check(nest, stream or None, ctypes.byref(v))
    if st not in (HP_OK, HP_ETIMEOUT):
        _check(st, "hp_nest_check")
    return v.value


def hp_nest_destroy(nest):
    if nest:
        lib().hp_nest_destroy(nest)


def hp_probe_gather(x_ptr, n_x, n_gathers, seed, sum_ptr, stream=0):
    """Gather-rate probe: n_gathers random 4-byte reads of x (see include/hp.h)."""
    _check(lib().hp_probe_gather(x_ptr, int(n_x), int(n_gathers), int(seed) & 0xffffffff, sum_ptr, stream or None),
           "hp_probe_gather")


def hp_serve_create(mem_budget_bytes, max_slots, n_streams):
    h = ctypes.c_void_p()
    _check(lib().hp_serve_create(int(mem_budget_bytes), max_slots, n_streams, ctypes.byref(h)), "hp_serve_create")
    return h.value


def hp_serve_submit(server, nest, in_ptrs, out_ptr) -> int:
    t = ctypes.c_uint64()
    _check(lib().hp_serve_submit(server, nest, _ptr_array(in_ptrs), out_ptr or None, ctypes.byref(t)),
           "hp_serve_submit")
    return t.value


def hp_serve_submit_at(server, nest, in_ptrs, out_ptr, arrival_us) -> int:
    t = ctypes.c_uint64()
    _check(lib().hp_serve_submit_at(server, nest, _ptr_array(in_ptrs), out_ptr or None, float(arrival_us),
                                    ctypes.byref(t)), "hp_serve_submit_at")
    return t.value


def hp_serve_clock_us() -> float:
    return float(lib().hp_serve_clock_us())


def hp_serve_poll(server, ticket, timeout_us=0) -> int:
    """Returns HP_OK (done), HP_EAGAIN (pending) or HP_ETIMEOUT; raises on errors."""
    st = lib().hp_serve_poll(server, ticket, timeout_us)
    if st not in (HP_OK, HP_EAGAIN, HP_ETIMEOUT):
        _check(st, "hp_serve_poll")
    return st


def hp_serve_stats(server):
    v = [ctypes.c_double() for _ in range(4)]
    _check(lib().hp_serve_stats(server, *[ctypes.byref(x) for x in v]), "hp_serve_stats")
    return {"p50_us": v[0].value, "p99_us": v[1].value, "p999_us": v[2].value, "nests_per_s": v[3].value}


def hp_serve_counters(server):
    c, st, pb, ps = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_size_t(), ctypes.c_int32()
    _check(lib().hp_serve_counters(server, ctypes.byref(c), ctypes.byref(st), ctypes.byref(pb), ctypes.byref(ps)),
           "hp_serve_counters")
    return {"completed": c.value, "steps": st.value, "peak_bytes": pb.value, "peak_slots": ps.value}


def hp_serve_destroy(server):
    if server:
        lib().hp_serve_destroy(server)


def _props(names):
    v = 0
    for n in names or ():
        v |= PROPS[n]
    return v


def hp_level_properties(hw):
    """(set of property names, num) of a hardware level ('grid', 'cluster', ...)."""
    pr, num = ctypes.c_uint32(), ctypes.c_int64()
    _check(lib().hp_level_properties(HW[hw], ctypes.byref(pr), ctypes.byref(num)), "hp_level_properties")
    return {k for k, bit in PROPS.items() if pr.value & bit}, num.value


def _req_array(reqs):
    return (hp_level_req * len(reqs))(*[hp_level_req(_props(r.get("sync")), _props(r.get("reserve")),
                                                     r.get("min_num", 0)) for r in reqs])


def hp_level_select(reqs):
    """Level map from per-level requirements: a list of dicts with optional
    keys sync (property names), reserve (property names) and min_num.
    Returns [(hw name, sub_width, tile), ...]."""
    n = len(reqs)
    out = (hp_level_map * n)()
    _check(lib().hp_level_select(n, _req_array(reqs), out), "hp_level_select")
    return [(HW_NAMES[m.hw], m.sub_width, m.tile) for m in out]


def hp_level_check(reqs, level_map):
    """True if the level map (as for Nest's level_map) meets the requirements;
    False with the reason otherwise: returns (ok, message)."""
    n = len(reqs)
    mp = level_map if isinstance(level_map, ctypes.Array) else make_map(level_map)
    st = lib().hp_level_check(n, _req_array(reqs), mp)
    if st == HP_OK:
        return True, ""
    if st != HP_EINVAL:
        _check(st, "hp_level_check")
    return False, hp_last_error()


def hp_stencil_create(ny, nx, radius, coeffs, steps, section=(0, 0), tile=(0, 0)):
    """Plan a stencil nest (host only); coeffs: (2r+1)^2 floats, row-major over (dy, dx)."""
    cs = [float(v) for v in coeffs]
    if 0 <= radius <= 4 and len(cs) != (2 * radius + 1) ** 2:
        raise HPError(HP_EINVAL, "hp_stencil_create", f"{(2 * radius + 1) ** 2} coefficients expected, got {len(cs)}")
    arr = (ctypes.c_float * max(len(cs), 81))(*cs)   # the library reads (2r+1)^2 of them (r <= 4)
    m = hp_stencil_map(section[0], section[1], tile[0], tile[1])
    h = ctypes.c_void_p()
    _check(lib().hp_stencil_create(ny, nx, radius, arr, steps, ctypes.byref(m), ctypes.byref(h)), "hp_stencil_create")
    return h.value


def hp_stencil_run(st, in_ptr, out_ptr, stream=0):
    _check(lib().hp_stencil_run(st, in_ptr, out_ptr, stream or None), "hp_stencil_run")


def hp_stencil_describe(st) -> dict:
    buf = ctypes.create_string_buffer(16384)
    _check(lib().hp_stencil_describe(st, buf, len(buf)), "hp_stencil_describe")
    return json.loads(buf.value.decode())


def hp_stencil_check(st, stream=0) -> int:
    v = ctypes.c_int32()
    status = lib().hp_stencil_check(st, stream or None, ctypes.byref(v))
    if status not in (HP_OK, HP_ETIMEOUT):
        _check(status, "hp_stencil_check")
    return v.value


def hp_stencil_destroy(st):
    if st:
        lib().hp_stencil_destroy(st)


class Stencil:
    """Convenience owner of one stencil handle."""

    def __init__(self, ny, nx, radius, coeffs, steps=1, section=(0, 0), tile=(0, 0)):
        self.handle = None
        self.handle = hp_stencil_create(ny, nx, radius, coeffs, steps, section, tile)

    def run(self, in_ptr, out_ptr, stream=0):
        hp_stencil_run(self.handle, in_ptr, out_ptr, stream)

    def describe(self) -> dict:
        return hp_stencil_describe(self.handle)

    def check(self, stream=0) -> int:
        return hp_stencil_check(self.handle, stream)

    def close(self):
        if self.handle:
            hp_stencil_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Nest:
    """Convenience owner of one nest handle (destroyed on close / garbage collection)."""

    def __init__(self, extents=None, red_level=0, op="sum", prec="f32", body="load", level_map=None,
                 params=None, csr_rows=None):
        self.handle = None
        if csr_rows is not None:
            self.depth = 2
            self.handle = hp_nest_create(2, None, 1, csr_rows, level_map, op, red_level, prec, body, params)
        else:
            self.depth = len(extents)
            self.handle = hp_nest_create(len(extents), list(extents), None, 0, level_map, op, red_level, prec, body,
                                         params)

    def run(self, in_ptrs, out_ptr, stream=0):
        hp_nest_run(self.handle, in_ptrs, out_ptr, stream)

    def run_comp(self, in_ptrs, out_ptr, comp_ptr, stream=0):
        hp_nest_run_comp(self.handle, in_ptrs, out_ptr, comp_ptr, stream)

    def run_static(self, in_ptrs, out_ptr, stream=0):
        hp_nest_run_static(self.handle, in_ptrs, out_ptr, stream)

    def run_host(self, in_ptrs, out_ptr, stream=0):
        hp_nest_run_host(self.handle, in_ptrs, out_ptr, stream)

    def tune(self, in_ptrs, out_ptr, stream=0, retime=False, batched=False, req=None):
        hp_nest_tune(self.handle, in_ptrs, out_ptr, stream, retime, batched, req)

    def describe(self) -> dict:
        return hp_nest_describe(self.handle)

    def error_bound(self) -> float:
        return hp_nest_error_bound(self.handle)

    def check(self, stream=0) -> int:
        return hp_nest_check(self.handle, stream)

    def close(self):
        if self.handle:
            hp_nest_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
