"""Python binding of the GB300 DF / DF-P PageRank library (arXiv 2401.15870).

Argument marshalling only: every step of the update runs in the CUDA kernels of
``libdfpr.so`` behind the C ABI declared in ``include/dfpr.h``; the functions
below carry the same names as the C entry points.  Host arrays are numpy
arrays; device arrays are torch CUDA tensors (PyTorch provides device memory
and streams, nothing else).  There is no CPU fallback: if the library is not
built, loading fails with an error.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdfpr.so")

PR_STATIC, PR_NAIVE_DYNAMIC, PR_DYNAMIC_TRAVERSAL, PR_DF, PR_DFP = 0, 1, 2, 3, 4
METHODS = {"static": PR_STATIC, "nd": PR_NAIVE_DYNAMIC, "dt": PR_DYNAMIC_TRAVERSAL, "df": PR_DF, "dfp": PR_DFP}
STATUS = {0: "PR_OK", 1: "PR_EINVAL", 2: "PR_ERANGE", 3: "PR_ENOMEM", 4: "PR_ENORANKS", 5: "PR_ECUDA",
          6: "PR_ETIMEOUT"}


class PRError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        super().__init__("%s%s" % (STATUS.get(status, str(status)), (": " + msg) if msg else ""))


class pr_options(ctypes.Structure):
    _fields_ = [("tau_f", ctypes.c_double), ("tau_p", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


class pr_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32), ("delta_R", ctypes.c_double),
                ("vertices_ever_affected", ctypes.c_int64), ("edges_processed", ctypes.c_int64),
                ("vertices_processed", ctypes.c_int64), ("eff_deletions", ctypes.c_int64),
                ("eff_insertions", ctypes.c_int64), ("ms_apply", ctypes.c_double), ("ms_update", ctypes.c_double),
                ("ms_sweep", ctypes.c_double), ("sweeps", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class pr_tuning(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("quads_per_lane", ctypes.c_int32), ("hub_vertices", ctypes.c_int32),
                ("fused_epilogue", ctypes.c_int32), ("ranges", ctypes.c_int32), ("hub_min_degree", ctypes.c_int32),
                ("ms_gather", ctypes.c_float),
                ("candidates", ctypes.c_int32)]


@dataclass
class Tuning:
    threads: int
    quads_per_lane: int
    hub_vertices: int
    fused_epilogue: int
    ranges: int
    hub_min_degree: int
    ms_gather: float
    candidates: int


class pr_group_tuning(ctypes.Structure):
    _fields_ = [("quads_per_lane", ctypes.c_int32), ("steps_per_unit", ctypes.c_int32),
                ("chunks_per_unit", ctypes.c_int32), ("ms_update", ctypes.c_float), ("candidates", ctypes.c_int32)]


@dataclass
class GroupTuning:
    quads_per_lane: int
    steps_per_unit: int
    chunks_per_unit: int
    ms_update: float
    candidates: int


@dataclass
class Stats:
    iterations: int
    converged: bool
    delta_R: float
    vertices_ever_affected: int
    edges_processed: int
    vertices_processed: int
    eff_deletions: int
    eff_insertions: int
    ms_apply: float
    ms_update: float
    ms_sweep: float
    sweeps: int


_lib = None
_P = ctypes.c_void_p


def load():
    """Load libdfpr.so (built by build.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libdfpr.so is not built (run __graft_entry__.build() or "
                           "python paper_2401_15870_gb300/build.py)")
    lib = ctypes.CDLL(LIB_PATH)
    i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "pr_graph_create": ([i32, i64, _P, _P, _P, ctypes.POINTER(_P)], ctypes.c_int),
        "pr_graph_create_edges": ([i32, i64, _P, _P, i32, i32, _P, ctypes.POINTER(_P)], ctypes.c_int),
        "pr_graph_destroy": ([_P], None),
        "pr_set_stream": ([_P, _P], ctypes.c_int),
        "pr_apply_batch": ([_P, _P, _P, i64, _P, _P, i64], ctypes.c_int),
        "pr_apply_batch_device": ([_P, _P, _P, i64, _P, _P, i64], ctypes.c_int),
        "pr_update": ([_P, ctypes.c_int, f64, f64, _P, _P], ctypes.c_int),
        "pr_ranks": ([_P, _P], ctypes.c_int),
        "pr_ranks_device": ([_P, _P], ctypes.c_int),
        "pr_set_ranks": ([_P, _P], ctypes.c_int),
        "pr_set_ranks_device": ([_P, _P], ctypes.c_int),
        "pr_graph_info": ([_P, ctypes.POINTER(i32), ctypes.POINTER(i64)], ctypes.c_int),
        "pr_get_csr": ([_P, i32, _P, _P], ctypes.c_int),
        "pr_get_rows": ([_P, i32, i64, _P, _P, _P], ctypes.c_int),
        "pr_last_delta": ([_P, ctypes.POINTER(i64), ctypes.POINTER(i64), _P, _P, _P, _P], ctypes.c_int),
        "pr_affected": ([_P, i32, _P], ctypes.c_int),
        "pr_last_error": ([_P], ctypes.c_char_p),
        "pr_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "pr_kernel_launches": ([], ctypes.c_ulonglong),
        "pr_sweep_noalloc": ([i32, _P, _P, _P, _P, _P, f64, _P, _P], ctypes.c_int),
        "pr_group_create": ([i32, _P, _P, ctypes.POINTER(_P)], ctypes.c_int),
        "pr_group_update": ([_P, ctypes.c_int, f64, f64, _P, _P], ctypes.c_int),
        "pr_group_destroy": ([_P], None),
        "pr_group_update_members": ([_P, ctypes.c_int, f64, f64, _P, _P, i32, _P], ctypes.c_int),
        "pr_server_create": ([i32, _P, _P, ctypes.POINTER(_P)], ctypes.c_int),
        "pr_server_submit": ([_P, i32, _P, _P, i64, _P, _P, i64, ctypes.POINTER(i64)], ctypes.c_int),
        "pr_server_wait": ([_P, i64, f64, _P], ctypes.c_int),
        "pr_server_drain": ([_P, f64], ctypes.c_int),
        "pr_server_clock": ([], f64),
        "pr_server_destroy": ([_P], None),
        "pr_autotune": ([_P, ctypes.c_int, f64, f64, i32, _P], ctypes.c_int),
        "pr_debug_fail_alloc": ([i64], None),
        "pr_apply_batches_device": ([i32, _P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
        "pr_apply_batches": ([i32, _P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
        "pr_get_tuning": ([_P, _P], ctypes.c_int),
        "pr_set_tuning": ([_P, _P], ctypes.c_int),
        "pr_group_autotune": ([_P, ctypes.c_int, f64, f64, i32, _P], ctypes.c_int),
        "pr_group_get_tuning": ([_P, _P], ctypes.c_int),
        "pr_group_set_tuning": ([_P, _P], ctypes.c_int),
        "pr_graph_resize": ([_P, i32], ctypes.c_int),
        "pr_sweep_log": ([_P, _P, i32, ctypes.POINTER(i32)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(rc, h=None):
    if rc != 0:
        msg = load().pr_last_error(h).decode() if h else ""
        raise PRError(rc, msg)


def _host_i32(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
    return a, (a.ctypes.data if a.size else None)


def _dev_ptr(t, dtype_name):
    if t is None:
        return None, 0
    if not (hasattr(t, "is_cuda") and t.is_cuda):
        raise TypeError("expected a CUDA tensor")
    if str(t.dtype) != "torch." + dtype_name or not t.is_contiguous():
        raise TypeError("expected a contiguous %s CUDA tensor" % dtype_name)
    return t.data_ptr(), t.numel()


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------ C-ABI mirrors

def pr_graph_create(n, row_off, col, stream=None):
    lib = load()
    ro = np.ascontiguousarray(np.asarray(row_off, dtype=np.int64))
    c, cp = _host_i32(col)
    h = _P()
    rc = lib.pr_graph_create(int(n), int(c.size), ro.ctypes.data, cp, _stream_handle(stream), ctypes.byref(h))
    _check(rc)
    return h


def pr_graph_create_edges(n, src, dst, device=False, keep_order=False, stream=None):
    lib = load()
    flags = 1 if keep_order else 0
    h = _P()
    if device:
        sp, m = _dev_ptr(src, "int32")
        dp, m2 = _dev_ptr(dst, "int32")
        if m != m2:
            raise ValueError("src and dst differ in length")
        rc = lib.pr_graph_create_edges(int(n), m, sp, dp, 1, flags, _stream_handle(stream), ctypes.byref(h))
    else:
        s, sp = _host_i32(src)
        d, dp = _host_i32(dst)
        if s.size != d.size:
            raise ValueError("src and dst differ in length")
        rc = lib.pr_graph_create_edges(int(n), s.size, sp, dp, 0, flags, _stream_handle(stream), ctypes.byref(h))
    _check(rc)
    return h


def pr_graph_destroy(h):
    if h:
        load().pr_graph_destroy(h)


def pr_set_stream(h, stream):
    _check(load().pr_set_stream(h, _stream_handle(stream)), h)


def pr_apply_batch(h, del_src=(), del_dst=(), ins_src=(), ins_dst=()):
    ds, dsp = _host_i32(del_src)
    dd, ddp = _host_i32(del_dst)
    is_, isp = _host_i32(ins_src)
    id_, idp = _host_i32(ins_dst)
    if ds.size != dd.size or is_.size != id_.size:
        raise ValueError("endpoint arrays differ in length")
    _check(load().pr_apply_batch(h, dsp, ddp, ds.size, isp, idp, is_.size), h)


def pr_apply_batch_device(h, del_src=None, del_dst=None, ins_src=None, ins_dst=None):
    dsp, nd = _dev_ptr(del_src, "int32")
    ddp, nd2 = _dev_ptr(del_dst, "int32")
    isp, ni = _dev_ptr(ins_src, "int32")
    idp, ni2 = _dev_ptr(ins_dst, "int32")
    if nd != nd2 or ni != ni2:
        raise ValueError("endpoint arrays differ in length")
    _check(load().pr_apply_batch_device(h, dsp, ddp, nd, isp, idp, ni), h)


def pr_apply_batches_device(handles, batches):
    """One batch per graph (each (del_src, del_dst, ins_src, ins_dst) device
    int32 tensors or None), every graph's work queued before the host waits."""
    k = len(handles)
    if len(batches) != k:
        raise ValueError("one batch per graph")
    P = ctypes.c_void_p
    ptr = [(P * k)() for _ in range(4)]
    cnt = [(ctypes.c_int64 * k)() for _ in range(2)]
    for i, b in enumerate(batches):
        ds, dd, is_, id_ = b
        dsp, nd = _dev_ptr(ds, "int32")
        ddp, nd2 = _dev_ptr(dd, "int32")
        isp, ni = _dev_ptr(is_, "int32")
        idp, ni2 = _dev_ptr(id_, "int32")
        if nd != nd2 or ni != ni2:
            raise ValueError("endpoint arrays differ in length")
        ptr[0][i], ptr[1][i], ptr[2][i], ptr[3][i] = dsp, ddp, isp, idp
        cnt[0][i], cnt[1][i] = nd, ni
    hs = (P * k)(*handles)
    _check(load().pr_apply_batches_device(k, hs, ptr[0], ptr[1], cnt[0], ptr[2], ptr[3], cnt[1]))


def pr_apply_batches(handles, batches):
    """As pr_apply_batches_device with host arrays (anything numpy can view as
    int32; each batch (del_src, del_dst, ins_src, ins_dst))."""
    k = len(handles)
    if len(batches) != k:
        raise ValueError("one batch per graph")
    P = ctypes.c_void_p
    ptr = [(P * k)() for _ in range(4)]
    cnt = [(ctypes.c_int64 * k)() for _ in range(2)]
    keep = []
    for i, b in enumerate(batches):
        arrs = [_host_i32(x if x is not None else ()) for x in b]
        keep.append(arrs)
        if arrs[0][0].size != arrs[1][0].size or arrs[2][0].size != arrs[3][0].size:
            raise ValueError("endpoint arrays differ in length")
        for j in range(4):
            ptr[j][i] = arrs[j][1]
        cnt[0][i], cnt[1][i] = arrs[0][0].size, arrs[2][0].size
    hs = (P * k)(*handles)
    _check(load().pr_apply_batches(k, hs, ptr[0], ptr[1], cnt[0], ptr[2], ptr[3], cnt[1]))


PR_OPT_TIME_SWEEPS, PR_OPT_FORCE_PULL, PR_OPT_FORCE_PUSH = 1, 2, 4
PR_OPT_DEVICE_LOOP, PR_OPT_HOST_LOOP = 8, 16
PR_OPT_ONE_KERNEL = 256   # the device loop as one cooperative kernel
PR_ONE_KERNEL_SLOTS = 1 << 20
LOOPS = {None: 0, "device": PR_OPT_DEVICE_LOOP, "host": PR_OPT_HOST_LOOP, "one": PR_OPT_ONE_KERNEL}
PR_OPT_ASYNC = 128   # asynchronous order (Sec. 4.4): one contribution vector, updated in place
PR_DEVICE_LOOP_SLOTS = 1 << 24


MEASURES = {None: 0, "relative": 0, "absolute": 32, "contrib": 64}   # PR_OPT_MEASURE_* (Sec. 4.3)


def pr_update(h, method, alpha=0.85, tau=1e-10, tau_f=1e-6, tau_p=1e-6, max_iter=500, time_sweeps=False,
              direction=None, loop=None, measure=None, order="sync") -> Stats:
    """direction: None (chosen per iteration), "pull" or "push" (DF / DF-P and
    DT, host loop).
    loop: None (by graph size), "device" (CUDA graph), "one" (one cooperative
    kernel) or "host".  measure: the DF / DF-P
    measure compared with tau_f / tau_p: "relative" (default), "absolute" or
    "contrib".  order: "sync" (every vertex of a sweep reads the ranks of its
    start) or "async" (one contribution vector updated in place, Sec. 4.4)."""
    m = METHODS[method] if isinstance(method, str) else int(method)
    flags = (PR_OPT_TIME_SWEEPS if time_sweeps else 0) | {None: 0, "pull": PR_OPT_FORCE_PULL,
                                                          "push": PR_OPT_FORCE_PUSH}[direction]
    flags |= LOOPS[loop]
    flags |= MEASURES[measure]
    flags |= {"sync": 0, "async": PR_OPT_ASYNC}[order]
    opts = pr_options(tau_f, tau_p, int(max_iter), flags)
    st = pr_stats()
    _check(load().pr_update(h, m, float(alpha), float(tau), ctypes.byref(opts), ctypes.byref(st)), h)
    return _stats(st)


def _stats(st):
    return Stats(st.iterations, bool(st.converged), st.delta_R, st.vertices_ever_affected, st.edges_processed,
                 st.vertices_processed, st.eff_deletions, st.eff_insertions, st.ms_apply, st.ms_update, st.ms_sweep,
                 st.sweeps)


def pr_graph_info(h):
    n = ctypes.c_int32()
    m = ctypes.c_int64()
    _check(load().pr_graph_info(h, ctypes.byref(n), ctypes.byref(m)), h)
    return n.value, m.value


def pr_ranks(h, out=None):
    n, _ = pr_graph_info(h)
    if out is None:
        out = np.empty(n, np.float64)
    if out.dtype != np.float64 or out.size != n or not out.flags["C_CONTIGUOUS"]:
        raise ValueError("out must be a contiguous float64 array of n elements")
    _check(load().pr_ranks(h, out.ctypes.data), h)
    return out


def pr_ranks_device(h, out):
    p, k = _dev_ptr(out, "float64")
    n, _ = pr_graph_info(h)
    if k != n:
        raise ValueError("out must hold n elements")
    _check(load().pr_ranks_device(h, p), h)
    return out


def pr_set_ranks(h, r):
    a = np.ascontiguousarray(np.asarray(r, dtype=np.float64))
    n, _ = pr_graph_info(h)
    if a.size != n:
        raise ValueError("ranks must hold n elements")
    _check(load().pr_set_ranks(h, a.ctypes.data), h)


def pr_set_ranks_device(h, r):
    p, k = _dev_ptr(r, "float64")
    n, _ = pr_graph_info(h)
    if k != n:
        raise ValueError("ranks must hold n elements")
    _check(load().pr_set_ranks_device(h, p), h)


def pr_get_csr(h, which=0):
    n, m = pr_graph_info(h)
    off = np.empty(n + 1, np.int64)
    adj = np.empty(max(m, 1), np.int32)
    _check(load().pr_get_csr(h, int(which), off.ctypes.data, adj.ctypes.data), h)
    return off, adj[: off[-1]]


def pr_get_rows(h, which, vertices, degrees_only=False):
    """Rows of the given vertices (which 0: out, 1: in): (off, adj) with
    adj[off[k]:off[k+1]] the sorted neighbours of vertices[k]; with
    degrees_only, just off."""
    v, vp = _host_i32(vertices)
    off = np.empty(v.size + 1, np.int64)
    lib = load()
    _check(lib.pr_get_rows(h, int(which), v.size, vp, off.ctypes.data, None), h)
    if degrees_only:
        return off
    adj = np.empty(max(int(off[-1]), 1), np.int32)
    _check(lib.pr_get_rows(h, int(which), v.size, vp, off.ctypes.data, adj.ctypes.data), h)
    return off, adj[: off[-1]]


def pr_last_delta(h):
    nd, ni = ctypes.c_int64(), ctypes.c_int64()
    lib = load()
    _check(lib.pr_last_delta(h, ctypes.byref(nd), ctypes.byref(ni), None, None, None, None), h)
    arrs = [np.empty(max(k, 1), np.int32) for k in (nd.value, nd.value, ni.value, ni.value)]
    _check(lib.pr_last_delta(h, None, None, *[a.ctypes.data for a in arrs]), h)
    dm = np.stack([arrs[0][: nd.value], arrs[1][: nd.value]], 1)
    dp = np.stack([arrs[2][: ni.value], arrs[3][: ni.value]], 1)
    return dm, dp


def pr_affected(h, which):
    n, _ = pr_graph_info(h)
    f = np.empty(n, np.uint8)
    _check(load().pr_affected(h, int(which), f.ctypes.data), h)
    return f.astype(bool)


def pr_last_error(h) -> str:
    return load().pr_last_error(h).decode()


class pr_sweep_record(ctypes.Structure):
    _fields_ = [("iteration", ctypes.c_int32), ("form", ctypes.c_int32), ("ms", ctypes.c_double),
                ("edges", ctypes.c_int64), ("vertices", ctypes.c_int64)]


PR_SWEEP_LIST, PR_SWEEP_EVERY_VERTEX = 0, 1


def pr_sweep_log(h):
    """Per-sweep records of the graph's last timed host-loop update, as a list
    of (iteration, form, ms, edges, vertices); form 0 = list (push) sweep,
    1 = every-vertex (pull) sweep."""
    cnt = ctypes.c_int32(0)
    _check(load().pr_sweep_log(h, None, 0, ctypes.byref(cnt)), h)
    recs = (pr_sweep_record * max(cnt.value, 1))()
    _check(load().pr_sweep_log(h, recs, cnt.value, ctypes.byref(cnt)), h)
    return [(r.iteration, r.form, r.ms, r.edges, r.vertices) for r in recs[:cnt.value]]


def pr_graph_resize(h, n_new):
    """Vertex insertion / deletion at the end of the id range; ranks carried
    over by the closed form r * n / n_new (new vertices 1 / n_new)."""
    _check(load().pr_graph_resize(h, int(n_new)), h)


PR_NOALLOC_MAX_N = 524288


def pr_sweep_noalloc(n, in_off, in_src, out_deg, r_in, r_out, alpha, delta_out, stream=None):
    """One Eq. 1 sweep over a caller-provided device in-CSR without any device
    allocation (all arguments are CUDA tensors the caller owns)."""
    ptrs = [_dev_ptr(in_off, "int64")[0], _dev_ptr(in_src, "int32")[0], _dev_ptr(out_deg, "int32")[0],
            _dev_ptr(r_in, "float64")[0], _dev_ptr(r_out, "float64")[0]]
    dp = _dev_ptr(delta_out, "float64")[0]
    _check(load().pr_sweep_noalloc(int(n), *ptrs, float(alpha), dp, _stream_handle(stream)))


PR_GROUP_MAX = 1024


def pr_group_create(handles, stream=None):
    arr = (_P * len(handles))(*[h.value if isinstance(h, _P) else h for h in handles])
    out = _P()
    _check(load().pr_group_create(len(handles), arr, _stream_handle(stream), ctypes.byref(out)))
    _group_sizes[out.value] = len(handles)
    return out


def pr_group_update(q, method, alpha=0.85, tau=1e-10, tau_f=1e-6, tau_p=1e-6, max_iter=500, loop=None,
                    measure=None):
    """One update of every graph of the group; returns one Stats per graph.
    loop: None (by size: one kernel below PR_ONE_KERNEL_SLOTS in-CSR slots in
    all, else the CUDA graph), "device" (CUDA graph), "one" (one cooperative
    kernel) or "host" (kernels launched one by one).  measure: as in pr_update."""
    m = METHODS[method] if isinstance(method, str) else int(method)
    opts = pr_options(tau_f, tau_p, int(max_iter), LOOPS[loop] | MEASURES[measure])
    n = _group_sizes[q.value]
    st = (pr_stats * n)()
    _check(load().pr_group_update(q, m, float(alpha), float(tau), ctypes.byref(opts), st))
    return [_stats(x) for x in st]


def pr_group_update_members(q, members, method, alpha=0.85, tau=1e-10, tau_f=1e-6, tau_p=1e-6, max_iter=500):
    """Update only the graphs at the given group positions; returns {position: Stats}."""
    m = METHODS[method] if isinstance(method, str) else int(method)
    opts = pr_options(tau_f, tau_p, int(max_iter), 0)
    mem = np.ascontiguousarray(np.asarray(members, np.int32))
    st = (pr_stats * _group_sizes[q.value])()
    _check(load().pr_group_update_members(q, m, float(alpha), float(tau), ctypes.byref(opts), mem.ctypes.data,
                                          mem.size, st))
    return {int(i): _stats(st[int(i)]) for i in mem}


def pr_group_destroy(q):
    _group_sizes.pop(q.value, None)
    load().pr_group_destroy(q)


_group_sizes = {}


def _tuning(t):
    return Tuning(*(getattr(t, f) for f, _ in pr_tuning._fields_))


def pr_autotune(h, method="nd", alpha=0.85, tau=1e-10, reps=0):
    """Time the candidate sweep settings on the graph and keep the fastest:
    every-vertex sweeps (static / nd) or whole updates from the current ranks
    (df / dfp, which leaves the graph as after one update)."""
    m = METHODS[method] if isinstance(method, str) else int(method)
    t = pr_tuning()
    _check(load().pr_autotune(h, m, float(alpha), float(tau), int(reps), ctypes.byref(t)), h)
    return _tuning(t)


def pr_get_tuning(h):
    t = pr_tuning()
    _check(load().pr_get_tuning(h, ctypes.byref(t)), h)
    return _tuning(t)


def pr_set_tuning(h, threads=1024, quads_per_lane=2, hub_vertices=0, fused_epilogue=0, ranges=1):
    t = pr_tuning(int(threads), int(quads_per_lane), int(hub_vertices), int(fused_epilogue), int(ranges), 0, 0.0, 0)
    _check(load().pr_set_tuning(h, ctypes.byref(t)), h)


def _group_tuning(t):
    return GroupTuning(*(getattr(t, f) for f, _ in pr_group_tuning._fields_))


def pr_group_autotune(q, method="dfp", alpha=0.85, tau=1e-10, reps=0):
    """Time the group kernels' unit sizes on whole group updates and keep the
    fastest; every graph's ranks on entry are put back."""
    m = METHODS[method] if isinstance(method, str) else int(method)
    t = pr_group_tuning()
    _check(load().pr_group_autotune(q, m, float(alpha), float(tau), int(reps), ctypes.byref(t)))
    return _group_tuning(t)


def pr_group_get_tuning(q):
    t = pr_group_tuning()
    _check(load().pr_group_get_tuning(q, ctypes.byref(t)))
    return _group_tuning(t)


def pr_group_set_tuning(q, quads_per_lane=4, chunks_per_unit=4, steps_per_unit=1):
    t = pr_group_tuning(int(quads_per_lane), int(steps_per_unit), int(chunks_per_unit), 0.0, 0)
    _check(load().pr_group_set_tuning(q, ctypes.byref(t)))


def pr_debug_fail_alloc(k):
    """Make the k-th device allocation of the library from now fail (0: disarm)."""
    load().pr_debug_fail_alloc(int(k))


def pr_kernel_launches() -> int:
    return int(load().pr_kernel_launches())


# ------------------------------------------------------------------ convenience wrapper

class Graph:
    """Owning wrapper around a pr_graph handle."""

    def __init__(self, handle):
        self._h = handle

    @classmethod
    def from_csr(cls, n, row_off, col, stream=None):
        return cls(pr_graph_create(n, row_off, col, stream))

    @classmethod
    def from_edges(cls, n, src, dst, device=False, keep_order=False, stream=None):
        return cls(pr_graph_create_edges(n, src, dst, device, keep_order, stream))

    def close(self):
        if self._h:
            pr_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def n(self):
        return pr_graph_info(self._h)[0]

    @property
    def m(self):
        return pr_graph_info(self._h)[1]

    def apply_batch(self, del_src=(), del_dst=(), ins_src=(), ins_dst=()):
        pr_apply_batch(self._h, del_src, del_dst, ins_src, ins_dst)

    def apply_batch_device(self, del_src, del_dst, ins_src, ins_dst):
        pr_apply_batch_device(self._h, del_src, del_dst, ins_src, ins_dst)

    def update(self, method, **kw) -> Stats:
        return pr_update(self._h, method, **kw)

    def ranks(self, out=None):
        return pr_ranks(self._h, out)

    def ranks_device(self, out):
        return pr_ranks_device(self._h, out)

    def set_ranks(self, r):
        pr_set_ranks(self._h, r)

    def set_ranks_device(self, r):
        pr_set_ranks_device(self._h, r)

    def rows(self, which, vertices, degrees_only=False):
        return pr_get_rows(self._h, which, vertices, degrees_only)

    def out_csr(self):
        return pr_get_csr(self._h, 0)

    def in_csr(self):
        return pr_get_csr(self._h, 1)

    def effective_delta(self):
        return pr_last_delta(self._h)

    def resize(self, n_new):
        pr_graph_resize(self._h, n_new)

    def sweep_log(self):
        return pr_sweep_log(self._h)

    def initial_affected(self):
        return pr_affected(self._h, 0)

    def dt_affected(self):
        return pr_affected(self._h, 1)

    def save(self, path):
        """Checkpoint: the out-CSR (user ids, sorted rows, self-loops included),
        the ranks (if any) and the sweep setting, as one .npz file.  Graph.load
        rebuilds an equivalent graph: the same edge set and ranks, so every
        later update gives the same results as on this graph."""
        off, adj = self.out_csr()
        tu = self.tuning()
        extra = {}
        try:
            extra["ranks"] = self.ranks()
        except PRError:
            pass
        np.savez(path, off=off, adj=adj, tuning=np.array([tu.threads, tu.quads_per_lane, tu.hub_vertices,
                                                          tu.fused_epilogue, tu.ranges], np.int32), **extra)

    @classmethod
    def load(cls, path, stream=None):
        with np.load(path) as z:
            off, adj = z["off"], z["adj"]
            g = cls.from_csr(len(off) - 1, off, adj, stream)
            g.set_tuning(*[int(x) for x in z["tuning"]])
            if "ranks" in z:
                g.set_ranks(z["ranks"])
        return g

    def autotune(self, method="nd", alpha=0.85, tau=1e-10, reps=0) -> Tuning:
        return pr_autotune(self._h, method, alpha, tau, reps)

    def tuning(self) -> Tuning:
        return pr_get_tuning(self._h)

    def set_tuning(self, threads=1024, quads_per_lane=2, hub_vertices=0, fused_epilogue=0, ranges=1):
        pr_set_tuning(self._h, threads, quads_per_lane, hub_vertices, fused_epilogue, ranges)


class Group:
    """Owning wrapper around a pr_group handle; keeps its graphs alive."""

    def __init__(self, graphs, stream=None):
        self.graphs = list(graphs)
        self._q = pr_group_create([g.handle for g in self.graphs], stream)

    def update(self, method, **kw):
        return pr_group_update(self._q, method, **kw)

    def update_members(self, members, method, **kw):
        return pr_group_update_members(self._q, members, method, **kw)

    def apply_batches_device(self, batches):
        """One device batch per graph of the group, in group order."""
        pr_apply_batches_device([g.handle for g in self.graphs], batches)

    def apply_batches(self, batches):
        """One host batch per graph of the group, in group order."""
        pr_apply_batches([g.handle for g in self.graphs], batches)

    def autotune(self, method="dfp", alpha=0.85, tau=1e-10, reps=0) -> GroupTuning:
        return pr_group_autotune(self._q, method, alpha, tau, reps)

    def tuning(self) -> GroupTuning:
        return pr_group_get_tuning(self._q)

    def set_tuning(self, quads_per_lane=4, chunks_per_unit=4, steps_per_unit=1):
        pr_group_set_tuning(self._q, quads_per_lane, chunks_per_unit, steps_per_unit)

    def close(self):
        if self._q:
            pr_group_destroy(self._q)
            self._q = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ serving

PR_SERVE_GROUPED, PR_SERVE_PLAIN = 0, 1


class pr_server_options(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("method", ctypes.c_int32), ("alpha", ctypes.c_double),
                ("tau", ctypes.c_double), ("opts", pr_options), ("hbm_reserve", ctypes.c_int64),
                ("max_round_edges", ctypes.c_int64)]


class pr_request_info(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_int64), ("graph", ctypes.c_int32), ("status", ctypes.c_int32),
                ("round", ctypes.c_int64), ("merged", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_done", ctypes.c_double),
                ("stats", pr_stats)]


@dataclass
class RequestInfo:
    ticket: int
    graph: int
    status: int
    round: int
    merged: int
    t_submit: float
    t_start: float
    t_done: float
    stats: Stats


def pr_server_clock() -> float:
    return float(load().pr_server_clock())


class Server:
    """Request loop over resident graphs (pr_server_*); keeps its graphs alive."""

    def __init__(self, graphs, mode="grouped", method="dfp", alpha=0.85, tau=1e-10, tau_f=1e-6, tau_p=1e-6,
                 max_iter=500, hbm_reserve=0, max_round_edges=0):
        self.graphs = list(graphs)
        o = pr_server_options(PR_SERVE_GROUPED if mode == "grouped" else PR_SERVE_PLAIN,
                              METHODS[method] if isinstance(method, str) else int(method), float(alpha),
                              float(tau), pr_options(tau_f, tau_p, int(max_iter), 0), int(hbm_reserve),
                              int(max_round_edges))
        arr = (_P * len(self.graphs))(*[g.handle.value if isinstance(g.handle, _P) else g.handle
                                        for g in self.graphs])
        out = _P()
        _check(load().pr_server_create(len(self.graphs), arr, ctypes.byref(o), ctypes.byref(out)))
        self._s = out

    def submit(self, graph, del_src=(), del_dst=(), ins_src=(), ins_dst=()):
        ds, dsp = _host_i32(del_src)
        dd, ddp = _host_i32(del_dst)
        is_, isp = _host_i32(ins_src)
        id_, idp = _host_i32(ins_dst)
        if ds.size != dd.size or is_.size != id_.size:
            raise ValueError("endpoint arrays differ in length")
        t = ctypes.c_int64()
        _check(load().pr_server_submit(self._s, int(graph), dsp, ddp, ds.size, isp, idp, is_.size, ctypes.byref(t)))
        return t.value

    def wait(self, ticket, timeout=600.0) -> RequestInfo:
        info = pr_request_info()
        _check(load().pr_server_wait(self._s, int(ticket), float(timeout), ctypes.byref(info)))
        return RequestInfo(info.ticket, info.graph, info.status, info.round, info.merged, info.t_submit,
                           info.t_start, info.t_done, _stats(info.stats))

    def drain(self, timeout=600.0):
        _check(load().pr_server_drain(self._s, float(timeout)))

    def close(self):
        if self._s:
            load().pr_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
