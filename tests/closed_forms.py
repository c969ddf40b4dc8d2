"""ctypes loader of closed_forms.c (test-only closed-form counts, built with
gcc next to its source on first use; independent of the oracle and the
engine)."""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "closed_forms.c")
_SO = os.path.join(_HERE, "libclosed_forms.so")
_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            tmp = _SO + f".tmp{os.getpid()}"
            subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp], check=True,
                           capture_output=True)
            os.replace(tmp, _SO)
        L = ctypes.CDLL(_SO)
        for name in ("cf_triangles", "cf_trace_a4"):
            f = getattr(L, name)
            f.restype = ctypes.c_int64
            f.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
        _lib = L
    return _lib


def _args(rowptr, col):
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    c = np.ascontiguousarray(col, dtype=np.int32)
    return len(rp) - 1, rp, c


def triangles(rowptr, col) -> int:
    n, rp, c = _args(rowptr, col)
    r = _load().cf_triangles(n, rp.ctypes.data, c.ctypes.data)
    assert r >= 0
    return int(r)


def trace_a4(rowptr, col) -> int:
    n, rp, c = _args(rowptr, col)
    r = _load().cf_trace_a4(n, rp.ctypes.data, c.ctypes.data)
    assert r >= 0
    return int(r)


def c4_embeddings(rowptr, col) -> int:
    """tr(A^4) - 2 sum d^2 + 2|E| (2|E| = directed entries)."""
    d = np.diff(np.asarray(rowptr, dtype=np.int64))
    return trace_a4(rowptr, col) - 2 * int((d * d).sum()) + int(d.sum())
