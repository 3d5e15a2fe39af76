"""Seeded synthetic inputs shaped like the paper's workloads.

The one module that both the CPU oracle and the CUDA library are fed from.
It draws edge lists and update batches and holds none of the PageRank
arithmetic.  ``synth.c`` is the host implementation; ``synth_cuda.cu`` the
same definitions on the GPU for graphs too large to draw on the host (e.g.
R-MAT scale 25, 2^30 edges).  Both use the counter-based generator documented
in ``synth.c``, so for equal arguments they produce equal arrays.

Stand-ins (the paper's datasets are not available):
  * ``rmat``      -- R-MAT power-law graphs for the SuiteSparse graphs of Table 2
                     (random batches, Sec. 5.2.2);
  * ``batch``     -- 80 % uniform-pair insertions, 20 % deletions of existing
                     edges (Sec. 5.2.2);
  * ``temporal``  -- timestamped edge stream with repeats and heavy-tailed
                     degrees for the SNAP temporal graphs of Table 1
                     (Sec. 5.1.4).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")

RMAT_ABCD = (0.57, 0.19, 0.19, 0.05)


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, i32, i64, u32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
        lib.sy_draw.argtypes = [u64, u64, u64]
        lib.sy_draw.restype = u64
        lib.sy_perm.argtypes = [u32, u32, u64]
        lib.sy_perm.restype = u32
        lib.sy_rmat.argtypes = [ctypes.c_int, i64, u64, i32, i32, i32, P, P]
        lib.sy_batch.argtypes = [i32, P, P, i64, i64, i64, u64, P, P, P, P]
        lib.sy_temporal.argtypes = [i32, i64, u64, u32, u32, u32, P, P]
        _lib = lib
    return _lib


def _ppm(x: float) -> int:
    return int(round(x * 10000))


def rmat(scale: int, m: int, seed: int, abcd=RMAT_ABCD):
    """R-MAT edge list with 2^scale vertices and m drawn edges (repeats and
    self-loops included), ids relabelled by a seeded bijection."""
    if not (1 <= scale <= 31):
        raise ValueError("scale out of range")
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    a, b, c = (_ppm(x) for x in abcd[:3])
    _load().sy_rmat(scale, m, seed, a, b, c, src.ctypes.data, dst.ctypes.data)
    return src, dst


def unique_edges(src, dst):
    """Sorted distinct non-self-loop edges of an edge list (deletion candidates)."""
    s = np.asarray(src, np.int64)
    d = np.asarray(dst, np.int64)
    keep = s != d
    k = np.unique((s[keep] << 32) | d[keep])
    return (k >> 32).astype(np.int32), (k & 0xFFFFFFFF).astype(np.int32)


def batch(n: int, cand_src, cand_dst, size: int, seed: int, ins_frac: float = 0.8):
    """Random batch of ``size`` edges: round(ins_frac*size) uniform-pair
    insertions (u != v) and the rest deletions drawn uniformly (with
    replacement) from the candidate edges.  Returns (del_src, del_dst,
    ins_src, ins_dst)."""
    cs = np.ascontiguousarray(cand_src, np.int32)
    cd = np.ascontiguousarray(cand_dst, np.int32)
    n_ins = int(round(ins_frac * size))
    n_del = size - n_ins if cs.size else 0
    ds, dd = np.empty(n_del, np.int32), np.empty(n_del, np.int32)
    is_, id_ = np.empty(n_ins, np.int32), np.empty(n_ins, np.int32)
    _load().sy_batch(n, cs.ctypes.data if cs.size else None, cd.ctypes.data if cd.size else None, cs.size,
                     n_del, n_ins, seed, ds.ctypes.data if n_del else None, dd.ctypes.data if n_del else None,
                     is_.ctypes.data if n_ins else None, id_.ctypes.data if n_ins else None)
    return ds, dd, is_, id_


def temporal(n: int, m: int, seed: int, p_rep: float = 0.25, q_src: float = 0.2, q_dst: float = 0.2):
    """Temporal edge stream (in timestamp order) over n vertices."""
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    u32 = lambda x: min(int(x * 2**32), 2**32 - 1)
    _load().sy_temporal(n, m, seed, u32(p_rep), u32(q_src), u32(q_dst), src.ctypes.data, dst.ctypes.data)
    return src, dst


def perm(x: int, n: int, seed: int) -> int:
    return _load().sy_perm(x, n, seed)


def draw(seed: int, stream: int, ctr: int) -> int:
    return _load().sy_draw(seed, stream, ctr)
