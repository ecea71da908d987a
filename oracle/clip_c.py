"""Coupling matrix G by the C statement of half-space splitting (oracle).

Test infrastructure (oracle): never imported by the library.  Only tests,
the smoke check and bench.py's CPU baseline use it, to clip meshes of
millions of tets on the host cores in seconds (the convex-hull statement
takes milliseconds per tet).  `build()` compiles oracle/clip_split.c with
gcc (OpenMP when available) into oracle/_build/.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "clip_split.c")
_LIB = os.path.join(_HERE, "_build", "libclip_split.so")
_lib = None


def build():
    """Compile the C statement if its library is missing or older than the source."""
    if os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        raise RuntimeError("no C compiler for the oracle's clipping statement")
    base = [cc, "-O2", "-std=c99", "-shared", "-fPIC", _SRC, "-o", _LIB, "-lm"]
    r = subprocess.run(base[:2] + ["-fopenmp"] + base[2:], capture_output=True, text=True)
    if r.returncode != 0:  # no OpenMP: one thread
        r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle clipping build failed:\n" + r.stderr)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lb = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        lb.oracle_clip_candidates.argtypes = [ctypes.c_int64, P, P, P, P, ctypes.c_double, P, P, P]
        lb.oracle_clip_candidates.restype = ctypes.c_int
        _lib = lb
    return _lib


def coupling_csr(xyz, tets, n, lo=0.0, h=None):
    """CSR (row_ptr int64 [ntets+1], col int32, val float64) of G for the whole mesh.

    Grid conventions as clip.coupling_rows: n cells per axis (or (nx, ny, nz)),
    edge h (1 / nx when not given) from lo, cell index i + nx (j + ny k); a row
    holds the candidate cells with a nonzero volume, in index order."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    ext = np.ascontiguousarray(np.broadcast_to(np.asarray(n, dtype=np.int32), (3,)))
    h = (1.0 / ext[0]) if h is None else float(h)
    lo3 = np.ascontiguousarray(np.broadcast_to(np.asarray(lo, dtype=np.float64), (3,)))
    p = xyz[tets]
    a = np.clip(np.floor((p.min(axis=1) - lo3) / h).astype(np.int64), 0, ext - 1)
    b = np.clip(np.floor((p.max(axis=1) - lo3) / h).astype(np.int64), 0, ext - 1)
    cand = np.prod(b - a + 1, axis=1)
    off = np.zeros(len(tets) + 1, dtype=np.int64)
    np.cumsum(cand, out=off[1:])
    ccell = np.empty(int(off[-1]), dtype=np.int32)
    cvol = np.empty(int(off[-1]), dtype=np.float64)
    rc = _load().oracle_clip_candidates(len(tets), xyz.ctypes.data, tets.ctypes.data, ext.ctypes.data,
                                        lo3.ctypes.data, h, off.ctypes.data, ccell.ctypes.data, cvol.ctypes.data)
    if rc != 0:
        raise MemoryError("oracle clipping ran out of memory")
    keep = cvol > 0.0
    row = np.repeat(np.arange(len(tets)), cand)[keep]
    rowptr = np.zeros(len(tets) + 1, dtype=np.int64)
    np.cumsum(np.bincount(row, minlength=len(tets)), out=rowptr[1:])
    return rowptr, ccell[keep], cvol[keep]
