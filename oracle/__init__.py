"""CPU oracle for the DF / DF-P PageRank update (arXiv 2401.15870).

TEST INFRASTRUCTURE ONLY: a plain, slow FP64 C implementation
(``dfpr_oracle.c``) of Static, Naive-dynamic, Dynamic Traversal, DF and DF-P
PageRank, in the synchronous order, with the batch update of Sec. 3.2.  It is
built single-threaded, and from the same source with OpenMP for the large
workloads (``Graph(..., parallel=True)``): both builds return the same bits.  Only the tests, the package smoke check and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the CUDA library and never imports it.

Every function follows a passage of the paper:
  * ``Graph``            -- edge set with one self-loop per vertex (Sec. 5.1.3)
  * ``Graph.apply_batch`` -- E_t = (E_{t-1} \\ D) u I, effective deltas (Sec. 3.2)
  * ``Graph.update``      -- Static / ND / DT / DF / DF-P (Sec. 3.1, 2.3, Alg. 1),
                             with the expansion measures of Sec. 4.3 and the
                             asynchronous order of Alg. 1 (Sec. 4.4) as options
  * ``Graph.initial_affected`` -- initial marking of Alg. 1
  * ``Graph.dt_affected`` -- reachability of Dynamic Traversal (Sec. 3.3.2)
  * ``rank_plain`` / ``rank_closed_loop`` -- Eq. 1 and Eq. 2

Parity status: Static / ND / DT ranks are pinned to the linear-system
solution, to closed forms and to mass conservation; the marking and
reachability sets to brute force and to the worked example of Sec. 4.1.3.
DF / DF-P ranks on general inputs are pinned only by their invariants and
by their limits (tau_f = tau_p = 0 gives the linear-system solution;
tau_f = inf with tau_p = 0 gives the solution of the system restricted to
the initial marking): parity unpinned beyond those.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dfpr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# the same source built with -fopenmp: synchronous sweeps, sorts and the
# adjacency rebuild on every host core, bit-identical results
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")

STATIC, NAIVE_DYNAMIC, DYNAMIC_TRAVERSAL, DF, DFP = 0, 1, 2, 3, 4
METHODS = {"static": STATIC, "nd": NAIVE_DYNAMIC, "dt": DYNAMIC_TRAVERSAL, "df": DF, "dfp": DFP}
# the DF / DF-P measures of Sec. 4.3: dr / max(r, R[v]) (Alg. 1), dr, dr / d
METRICS = {"relative": 0, "absolute": 1, "contrib": 2}
ORDERS = {"sync": 0, "async": 1, "ranges": 2}
_ERR = {1: "invalid argument", 2: "vertex id out of range", 3: "out of memory", 4: "no previous ranks"}


def _compile(lib: str, extra, force: bool) -> str:
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        tmp = lib + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", *extra, "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, lib)
    return lib


def build(force: bool = False, parallel: bool = None) -> str:
    """Compile the oracle with gcc (plain -O2, IEEE FP64): liboracle.so, and
    liboracle_omp.so from the same source with -fopenmp.  parallel=None builds
    both and returns the plain one's path."""
    if parallel is None:
        _compile(_LIB_OMP, ["-fopenmp"], force)
        return _compile(_LIB, [], force)
    return _compile(_LIB_OMP, ["-fopenmp"], force) if parallel else _compile(_LIB, [], force)


_libs = {}


def set_threads(k: int) -> None:
    """Threads of the OpenMP build (it uses every host core by default)."""
    _load(True).or_set_threads(int(k))


def threads(parallel: bool = True) -> int:
    return _load(parallel).or_threads()


def _load(parallel: bool = False):
    lib = _libs.get(parallel)
    if lib is None:
        lib = ctypes.CDLL(build(parallel=parallel))
        P = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        lib.or_graph_create.argtypes = [i32, i64, P, P, ctypes.POINTER(P)]
        lib.or_graph_create.restype = ctypes.c_int
        lib.or_graph_destroy.argtypes = [P]
        lib.or_apply_batch.argtypes = [P, P, P, i64, P, P, i64]
        lib.or_apply_batch.restype = ctypes.c_int
        lib.or_num_vertices.argtypes = [P]
        lib.or_num_vertices.restype = i32
        for f in ("or_num_edges", "or_num_eff_del", "or_num_eff_ins"):
            getattr(lib, f).argtypes = [P]
            getattr(lib, f).restype = i64
        lib.or_get_out_csr.argtypes = [P, P, P]
        lib.or_get_in_csr.argtypes = [P, P, P]
        lib.or_get_eff_delta.argtypes = [P, P, P]
        lib.or_initial_affected.argtypes = [P, P]
        lib.or_dt_affected.argtypes = [P, P]
        lib.or_dt_affected.restype = ctypes.c_int
        lib.or_rank_plain.argtypes = [f64, i32, f64]
        lib.or_rank_plain.restype = f64
        lib.or_rank_closed_loop.argtypes = [f64, i32, f64, f64, i64]
        lib.or_rank_closed_loop.restype = f64
        lib.or_update.argtypes = [P, ctypes.c_int, f64, f64, f64, f64, i32, P, P, P]
        lib.or_update.restype = ctypes.c_int
        lib.or_update_ex.argtypes = [P, ctypes.c_int, f64, f64, f64, f64, i32, ctypes.c_int, ctypes.c_int, P, P, P]
        lib.or_update_ex.restype = ctypes.c_int
        lib.or_graph_resize.argtypes = [P, i32]
        lib.or_graph_resize.restype = ctypes.c_int
        lib.or_resize_ranks.argtypes = [i32, P, i32, P]
        lib.or_threads.restype = ctypes.c_int
        lib.or_set_threads.argtypes = [ctypes.c_int]
        _libs[parallel] = lib
    return lib


class _Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("delta_R", ctypes.c_double), ("vertices_ever_affected", ctypes.c_int64),
                ("edges_processed", ctypes.c_int64), ("vertices_processed", ctypes.c_int64),
                ("tie_rel", ctypes.c_double)]


@dataclass
class Stats:
    iterations: int
    converged: bool
    delta_R: float
    vertices_ever_affected: int
    edges_processed: int
    vertices_processed: int
    # smallest |x / t - 1| between a compared quantity x and its threshold t
    # over every expand / prune / stop decision of the run (near-ties)
    tie_rel: float = float("inf")


class OracleError(RuntimeError):
    pass


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _ptr(a):
    return a.ctypes.data if a.size else None


def resize_ranks(r_old, n_new: int) -> np.ndarray:
    """Ranks carried over a resize: r * n / n_new for the kept vertices,
    1 / n_new for added ones (closed form from Eq. 1)."""
    r = np.ascontiguousarray(np.asarray(r_old, dtype=np.float64))
    out = np.zeros(int(n_new), np.float64)
    _load().or_resize_ranks(r.size, r.ctypes.data, int(n_new), out.ctypes.data)
    return out


def rank_plain(alpha: float, n: int, c: float) -> float:
    """Eq. 1 for one vertex: (1 - alpha)/n + alpha * c."""
    return _load().or_rank_plain(alpha, n, c)


def rank_closed_loop(alpha: float, n: int, c: float, Rv: float, d: int) -> float:
    """Eq. 2 for one vertex (closed-loop form of DF-P, appendix derivation)."""
    return _load().or_rank_closed_loop(alpha, n, c, Rv, d)


class Graph:
    """Edge set over [0, n) with one self-loop per vertex (Sec. 5.1.3).
    parallel=True runs it on the OpenMP build (same results, bit for bit)."""

    def __init__(self, n: int, src, dst, parallel: bool = False):
        self._lib = lib = _load(bool(parallel))
        s, d = _i32(src), _i32(dst)
        if s.shape != d.shape:
            raise ValueError("src and dst differ in length")
        h = ctypes.c_void_p()
        rc = lib.or_graph_create(int(n), int(s.size), _ptr(s), _ptr(d), ctypes.byref(h))
        if rc:
            raise OracleError(_ERR.get(rc, str(rc)))
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and getattr(self, "_lib", None) is not None:
            self._lib.or_graph_destroy(h)
            self._h = None

    @property
    def n(self) -> int:
        return self._lib.or_num_vertices(self._h)

    @property
    def m(self) -> int:
        return self._lib.or_num_edges(self._h)

    def apply_batch(self, del_src=(), del_dst=(), ins_src=(), ins_dst=()):
        """Deletions, then insertions, set semantics (Sec. 3.2)."""
        ds, dd, is_, id_ = _i32(del_src), _i32(del_dst), _i32(ins_src), _i32(ins_dst)
        if ds.shape != dd.shape or is_.shape != id_.shape:
            raise ValueError("endpoint arrays differ in length")
        rc = self._lib.or_apply_batch(self._h, _ptr(ds), _ptr(dd), ds.size, _ptr(is_), _ptr(id_), is_.size)
        if rc:
            raise OracleError(_ERR.get(rc, str(rc)))

    def resize(self, n_new: int):
        """Vertex insertion / deletion at the end of the id range: added
        vertices carry their self-loop only; removed ones must have no other
        edge.  Clears the last batch's effective change."""
        rc = self._lib.or_graph_resize(self._h, int(n_new))
        if rc:
            raise OracleError(_ERR.get(rc, str(rc)))

    def out_csr(self):
        off = np.zeros(self.n + 1, np.int64)
        adj = np.zeros(max(self.m, 1), np.int32)
        self._lib.or_get_out_csr(self._h, off.ctypes.data, adj.ctypes.data)
        return off, adj[: self.m]

    def in_csr(self):
        off = np.zeros(self.n + 1, np.int64)
        adj = np.zeros(max(self.m, 1), np.int32)
        self._lib.or_get_in_csr(self._h, off.ctypes.data, adj.ctypes.data)
        return off, adj[: self.m]

    def effective_delta(self):
        """(Delta-, Delta+) of the last batch as sorted (k, 2) int arrays of (src, dst)."""
        lib = self._lib
        nd, ni = lib.or_num_eff_del(self._h), lib.or_num_eff_ins(self._h)
        d = np.zeros(max(nd, 1), np.uint64)
        i = np.zeros(max(ni, 1), np.uint64)
        lib.or_get_eff_delta(self._h, d.ctypes.data, i.ctypes.data)

        def split(k):
            return np.stack([(k >> np.uint64(32)).astype(np.int64), (k & np.uint64(0xFFFFFFFF)).astype(np.int64)], 1)
        return split(d[:nd]), split(i[:ni])

    def initial_affected(self) -> np.ndarray:
        f = np.zeros(self.n, np.uint8)
        self._lib.or_initial_affected(self._h, f.ctypes.data)
        return f.astype(bool)

    def dt_affected(self) -> np.ndarray:
        f = np.zeros(self.n, np.uint8)
        if self._lib.or_dt_affected(self._h, f.ctypes.data):
            raise OracleError("out of memory")
        return f.astype(bool)

    def update(self, method, alpha=0.85, tau=1e-10, tau_f=1e-6, tau_p=1e-6, max_iter=500, r_prev=None,
               metric="relative", order="sync"):
        """Run one method; returns (ranks, Stats).  metric: the DF / DF-P
        measure of Sec. 4.3 ("relative", "absolute", "contrib"); order: "sync",
        "async" (Alg. 1 with one rank vector, ascending vertex id) or "ranges"
        (eight consecutive id ranges swept in order, each reading the ranks of
        the ranges before it as updated in this sweep)."""
        m = METHODS[method] if isinstance(method, str) else int(method)
        out = np.zeros(self.n, np.float64)
        prev = None if r_prev is None else np.ascontiguousarray(np.asarray(r_prev, dtype=np.float64))
        if prev is not None and prev.size != self.n:
            raise ValueError("r_prev has the wrong length")
        st = _Stats()
        rc = self._lib.or_update_ex(self._h, m, alpha, tau, tau_f, tau_p, int(max_iter), METRICS[metric],
                                  ORDERS[order], None if prev is None else prev.ctypes.data, out.ctypes.data,
                                  ctypes.byref(st))
        if rc:
            raise OracleError(_ERR.get(rc, str(rc)))
        return out, Stats(st.iterations, bool(st.converged), st.delta_R, st.vertices_ever_affected,
                          st.edges_processed, st.vertices_processed, st.tie_rel)
