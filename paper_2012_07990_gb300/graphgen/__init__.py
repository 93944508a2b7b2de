"""Seeded synthetic graph inputs shared by the CUDA path, the oracle and the bench.

This module prepares inputs only: CSR arrays (int32 row offsets ``rowptr[n+1]``
and adjacency ``col[m]``, lists sorted ascending, no self-loops or duplicate
arcs), integer edge weights, and source-vertex choices.  It holds none of the
traversal arithmetic.  Its C part (``graphgen.c``) is compiled on first use
with gcc into ``libg2gen.so`` next to this file.

Workload recipes (synthetic stand-ins for the paper's Table IV graphs, which
are real-world datasets not shipped here):

* ``rmat(scale, ef=16, a=.57, b=.19, c=.19, seed=1)`` -- power-law, symmetrised.
* ``road_grid(W, H, p_delete=.10, shortcut_frac=.01, reach=16, seed=1)`` --
  4-neighbour lattice with 10% of edges deleted and 1% local shortcuts.
* ``pair_weights(g, wmax, seed)`` -- symmetric integer weights in [1, wmax].
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libg2gen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile graphgen.c into libg2gen.so (gcc, OpenMP) if stale."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i64p = ctypes.POINTER(ctypes.c_int64)
            i32pp = ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))
            lib.g2gen_rmat.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_uint64, ctypes.c_int,
                                       i64p, i64p, i32pp, i32pp]
            lib.g2gen_grid.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int64,
                                       ctypes.c_int, ctypes.c_uint64, i64p, i64p, i32pp, i32pp]
            lib.g2gen_pair_weights.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p]
            lib.g2gen_csr_from_arcs.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                                ctypes.c_void_p, i64p, i32pp, i32pp]
            lib.g2gen_free.argtypes = [ctypes.c_void_p]
            lib.g2gen_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclass
class Graph:
    """Host CSR graph.  ``symmetric`` means every arc u->v has v->u."""
    n: int
    rowptr: np.ndarray  # int32[n+1]
    col: np.ndarray     # int32[m]
    symmetric: bool
    name: str = ""
    w: np.ndarray | None = None  # int32[m] or None

    @property
    def m(self) -> int:
        return int(self.col.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.rowptr.astype(np.int64))

    def max_degree_vertex(self) -> int:
        """Source rule of the workloads: max out-degree, ties -> lowest id."""
        d = self.degrees()
        return int(np.argmax(d)) if d.size else 0


def _take(n, m, rp, cl):
    lib = _load()
    rowptr = np.ctypeslib.as_array(rp, shape=(n + 1,)).copy()
    col = np.ctypeslib.as_array(cl, shape=(max(m, 1),))[:m].copy()
    lib.g2gen_free(ctypes.cast(rp, ctypes.c_void_p))
    lib.g2gen_free(ctypes.cast(cl, ctypes.c_void_p))
    return rowptr, col


def _call(fn, *args):
    n = ctypes.c_int64()
    m = ctypes.c_int64()
    rp = ctypes.POINTER(ctypes.c_int32)()
    cl = ctypes.POINTER(ctypes.c_int32)()
    rc = fn(*args, ctypes.byref(n), ctypes.byref(m), ctypes.byref(rp), ctypes.byref(cl))
    if rc != 0:
        raise RuntimeError(f"graph generator failed with code {rc}")
    return (n.value,) + _take(n.value, m.value, rp, cl)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, symmetric: bool = True) -> Graph:
    lib = _load()
    n, rowptr, col = _call(lib.g2gen_rmat, scale, edge_factor, a, b, c, seed, int(symmetric))
    return Graph(n, rowptr, col, symmetric, f"rmat{scale}_ef{edge_factor}_s{seed}")


def road_grid(W: int, H: int | None = None, p_delete: float = 0.10, shortcut_frac: float = 0.01,
              reach: int = 16, seed: int = 1) -> Graph:
    lib = _load()
    H = W if H is None else H
    nsc = int(round(shortcut_frac * W * H))
    n, rowptr, col = _call(lib.g2gen_grid, W, H, p_delete, nsc, reach, seed)
    return Graph(n, rowptr, col, True, f"grid{W}x{H}_s{seed}")


def from_arcs(n: int, src, dst, symmetric: bool = True, name: str = "") -> Graph:
    """CSR from an arc list; with ``symmetric`` the reverse arcs are added."""
    lib = _load()
    src = np.asarray(src, dtype=np.int32)
    dst = np.asarray(dst, dtype=np.int32)
    if src.size and (src.min() < 0 or dst.min() < 0 or src.max() >= n or dst.max() >= n):
        raise ValueError("arc endpoint out of range")
    if symmetric:
        src, dst = np.concatenate([src, dst]), np.concatenate([dst, src])
    src = np.ascontiguousarray(src)
    dst = np.ascontiguousarray(dst)
    m = ctypes.c_int64()
    rp = ctypes.POINTER(ctypes.c_int32)()
    cl = ctypes.POINTER(ctypes.c_int32)()
    rc = lib.g2gen_csr_from_arcs(n, src.size, src.ctypes.data, dst.ctypes.data, ctypes.byref(m),
                                 ctypes.byref(rp), ctypes.byref(cl))
    if rc != 0:
        raise RuntimeError(f"CSR assembly failed with code {rc}")
    rowptr, col = _take(n, m.value, rp, cl)
    return Graph(n, rowptr, col, symmetric, name)


def pair_weights(g: Graph, wmax: int, seed: int = 1) -> np.ndarray:
    """int32[m] weights in [1, wmax], equal on both arcs of an undirected edge."""
    lib = _load()
    w = np.empty(g.m, dtype=np.int32)
    lib.g2gen_pair_weights(g.n, g.rowptr.ctypes.data, g.col.ctypes.data, seed, wmax, w.ctypes.data)
    return w


# ----------------------------------------------------------------------------- small families
def path(n: int) -> Graph:
    i = np.arange(n - 1)
    return from_arcs(n, i, i + 1, name=f"path{n}")


def star(n: int) -> Graph:
    return from_arcs(n, np.zeros(n - 1, np.int32), np.arange(1, n), name=f"star{n}")


def cycle(n: int) -> Graph:
    i = np.arange(n)
    return from_arcs(n, i, (i + 1) % n, name=f"cycle{n}")


def complete(n: int) -> Graph:
    u, v = np.triu_indices(n, 1)
    return from_arcs(n, u, v, name=f"complete{n}")


def full_grid(W: int, H: int) -> Graph:
    return road_grid(W, H, p_delete=0.0, shortcut_frac=0.0, seed=0)


def gnp(n: int, p: float, seed: int, symmetric: bool = True) -> Graph:
    rng = np.random.default_rng(seed)
    a = rng.random((n, n)) < p
    if symmetric:
        a = np.triu(a, 1)
    else:
        np.fill_diagonal(a, False)
    u, v = np.nonzero(a)
    return from_arcs(n, u, v, symmetric=symmetric, name=f"gnp{n}_{p}_{seed}")


def disjoint_union(*gs: Graph) -> Graph:
    srcs, dsts, off = [], [], 0
    for g in gs:
        deg = g.degrees()
        srcs.append(np.repeat(np.arange(g.n), deg) + off)
        dsts.append(g.col.astype(np.int64) + off)
        off += g.n
    return from_arcs(off, np.concatenate(srcs), np.concatenate(dsts), symmetric=False,
                     name="union")._replace_sym(all(g.symmetric for g in gs))


def _replace_sym(self: Graph, sym: bool) -> Graph:
    self.symmetric = sym
    return self


Graph._replace_sym = _replace_sym  # type: ignore[attr-defined]


def random_sources(g: Graph, k: int, seed: int = 1) -> np.ndarray:
    """k sources uniform over non-isolated vertices (with replacement if needed)."""
    rng = np.random.default_rng(seed)
    cand = np.nonzero(g.degrees() > 0)[0]
    if cand.size == 0:
        return np.zeros(k, dtype=np.int32)
    return rng.choice(cand, size=k, replace=cand.size < k).astype(np.int32)
