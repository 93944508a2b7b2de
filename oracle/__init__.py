"""CPU oracle for the g2 traversal path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never calls it and
shares no code with it.

``oracle.c`` holds the plain single-threaded definitions (see its header for
the passage each one follows); this module compiles it with gcc into
``liboracle.so`` on first use and wraps it with numpy in/out arrays.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
against brute force on tiny graphs, closed forms, library routines
(scipy.sparse.csgraph) or invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

INF32 = 2147483647


def build(force: bool = False) -> str:
    """Compile oracle.c (plain C, -O2, single thread) if stale."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            lib.oracle_bfs.argtypes = [ctypes.c_int32, P, P, ctypes.c_int32, P, P]
            lib.oracle_cc.argtypes = [ctypes.c_int32, P, P, P]
            lib.oracle_sssp.argtypes = [ctypes.c_int32, P, P, P, ctypes.c_int32, P]
            lib.oracle_pagerank.argtypes = [ctypes.c_int32, P, P, ctypes.c_double, ctypes.c_int32, P]
            lib.oracle_bc.argtypes = [ctypes.c_int32, P, P, P, ctypes.c_int32, P]
            lib.oracle_edgeblock.argtypes = [ctypes.c_int32, ctypes.c_int64, P, P, ctypes.c_int32,
                                             P, P, P]
            lib.oracle_edgeblock.restype = ctypes.c_int32
            lib.oracle_etwc_split.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                              ctypes.c_int32, P]
            lib.oracle_etwc_split.restype = None
            _lib = lib
    return _lib


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


def _check(rc, what):
    if rc == 1:
        raise MemoryError(f"oracle {what}: out of memory")
    if rc == 2:
        raise OverflowError(f"oracle {what}: distance overflows int32")
    if rc != 0:
        raise RuntimeError(f"oracle {what}: code {rc}")


def bfs(n, rowptr, col, src, want_parent=True):
    """(depth int32[n], parent int32[n] or None)."""
    lib = _load()
    rp, prp = _c(rowptr, np.int32)
    cl, pcl = _c(col, np.int32)
    depth = np.empty(n, np.int32)
    parent = np.empty(n, np.int32) if want_parent else None
    _check(lib.oracle_bfs(n, prp, pcl, int(src), depth.ctypes.data,
                          parent.ctypes.data if want_parent else None), "bfs")
    return depth, parent


def cc(n, rowptr, col):
    lib = _load()
    rp, prp = _c(rowptr, np.int32)
    cl, pcl = _c(col, np.int32)
    label = np.empty(n, np.int32)
    _check(lib.oracle_cc(n, prp, pcl, label.ctypes.data), "cc")
    return label


def sssp(n, rowptr, col, w, src):
    lib = _load()
    rp, prp = _c(rowptr, np.int32)
    cl, pcl = _c(col, np.int32)
    ww, pw = _c(w, np.int32)
    dist = np.empty(n, np.int32)
    _check(lib.oracle_sssp(n, prp, pcl, pw, int(src), dist.ctypes.data), "sssp")
    return dist


def pagerank(n, rowptr, col, damping=0.85, iters=20):
    lib = _load()
    rp, prp = _c(rowptr, np.int32)
    cl, pcl = _c(col, np.int32)
    x = np.empty(n, np.float64)
    _check(lib.oracle_pagerank(n, prp, pcl, float(damping), int(iters), x.ctypes.data), "pagerank")
    return x


def bc(n, rowptr, col, srcs):
    lib = _load()
    rp, prp = _c(rowptr, np.int32)
    cl, pcl = _c(col, np.int32)
    ss, pss = _c(srcs, np.int32)
    out = np.empty(n, np.float64)
    _check(lib.oracle_bc(n, prp, pcl, pss, int(ss.size), out.ctypes.data), "bc")
    return out


def edgeblock(n, src, dst, N):
    """Algorithm 1: (out_src, out_dst, seg_end[numSeg+1], numSeg)."""
    lib = _load()
    s, ps = _c(src, np.int32)
    d, pd = _c(dst, np.int32)
    m = s.size
    num_seg = (n + N - 1) // N
    os_ = np.empty(m, np.int32)
    od = np.empty(m, np.int32)
    seg_end = np.empty(num_seg + 1, np.int64)
    got = lib.oracle_edgeblock(n, m, ps, pd, int(N), os_.ctypes.data, od.ctypes.data,
                               seg_end.ctypes.data)
    if got < 0:
        raise MemoryError("oracle edgeblock: out of memory")
    return os_, od, seg_end, got


def etwc_split(start, end, warp=32, cta=256):
    """Algorithm 3 split: [(b0,e0) thread, (b1,e1) warp, (b2,e2) CTA]."""
    lib = _load()
    r = np.empty(6, np.int64)
    lib.oracle_etwc_split(int(start), int(end), int(warp), int(cta), r.ctypes.data)
    return [(int(r[0]), int(r[1])), (int(r[2]), int(r[3])), (int(r[4]), int(r[5]))]


def bfs_graph(g, src, want_parent=True):
    return bfs(g.n, g.rowptr, g.col, src, want_parent)


def cc_graph(g):
    return cc(g.n, g.rowptr, g.col)


def sssp_graph(g, w, src):
    return sssp(g.n, g.rowptr, g.col, w, src)


def pagerank_graph(g, damping=0.85, iters=20):
    return pagerank(g.n, g.rowptr, g.col, damping, iters)


def bc_graph(g, srcs):
    return bc(g.n, g.rowptr, g.col, srcs)
