"""GPU implementation of the synth generators (R-MAT and random batches) for
workloads too large to draw on the host.  Equal arguments give the same arrays
as the host generators in synth.c (tested on the GPU).  Outputs are torch CUDA
tensors; torch only provides the memory and the stream."""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth_cuda.cu")
_LIB = os.path.join(_HERE, "libsynth_cuda.so")


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-Xcompiler", "-fPIC",
                               "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB):
            raise RuntimeError("libsynth_cuda.so is not built (synth.gpu.build())")
        lib = ctypes.CDLL(_LIB)
        P, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        lib.sy_rmat_device.argtypes = [ctypes.c_int, i64, u64, i32, i32, i32, P, P, P]
        lib.sy_rmat_device.restype = ctypes.c_int
        lib.sy_batch_device.argtypes = [i32, P, P, i64, i64, i64, u64, P, P, P, P, P]
        lib.sy_batch_device.restype = ctypes.c_int
        _lib = lib
    return _lib


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def rmat(scale: int, m: int, seed: int, abcd=(0.57, 0.19, 0.19, 0.05)):
    """R-MAT edge list as two int32 CUDA tensors (same as synth.rmat)."""
    import torch
    src = torch.empty(m, dtype=torch.int32, device="cuda")
    dst = torch.empty(m, dtype=torch.int32, device="cuda")
    a, b, c = (int(round(x * 10000)) for x in abcd[:3])
    rc = _load().sy_rmat_device(scale, m, seed, a, b, c, src.data_ptr(), dst.data_ptr(), _stream())
    if rc:
        raise RuntimeError("sy_rmat_device failed (%d)" % rc)
    return src, dst


def batch(n: int, cand_src, cand_dst, size: int, seed: int, ins_frac: float = 0.8):
    """Random batch as four int32 CUDA tensors (same as synth.batch)."""
    import torch
    n_ins = int(round(ins_frac * size))
    n_cand = int(cand_src.numel())
    n_del = size - n_ins if n_cand else 0
    out = [torch.empty(k, dtype=torch.int32, device="cuda") for k in (n_del, n_del, n_ins, n_ins)]
    rc = _load().sy_batch_device(n, cand_src.data_ptr(), cand_dst.data_ptr(), n_cand, n_del, n_ins, seed,
                                 *[t.data_ptr() for t in out], _stream())
    if rc:
        raise RuntimeError("sy_batch_device failed (%d)" % rc)
    return tuple(out)
