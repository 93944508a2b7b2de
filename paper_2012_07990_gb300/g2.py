"""Python binding of libg2 (include/g2.h): argument marshalling only.

Every function named ``g2_*`` here calls the C entry point of the same name.
Device arrays are torch CUDA tensors (passed by data pointer); the stream is
torch's current CUDA stream unless one is given.  Every step of the traversal
runs in the CUDA library; there is no CPU fallback: importing this module
raises if ``libg2.so`` is missing or fails to load.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libg2.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libg2.so not built ({LIB_PATH}); run __graft_entry__.build() "
                      "or python -m paper_2012_07990_gb300.build_native")
_lib = ctypes.CDLL(LIB_PATH)

# ---------------------------------------------------------------- constants
G2_OK, G2_EINVAL, G2_ENOMEM, G2_ECUDA, G2_ETIMEOUT, G2_EUNSUPPORTED, G2_EOVERFLOW = range(7)
STATUS_NAMES = {0: "G2_OK", 1: "G2_EINVAL", 2: "G2_ENOMEM", 3: "G2_ECUDA", 4: "G2_ETIMEOUT",
                5: "G2_EUNSUPPORTED", 6: "G2_EOVERFLOW"}
G2_SYMMETRIC, G2_DEVICE_PTRS, G2_PREPARE_PAGERANK, G2_LOAD_OVERLAP = 0x1, 0x2, 0x4, 0x8
LB = {"VERTEX_BASED": 0, "CM": 1, "WM": 2, "STRICT": 3, "EDGE_ONLY": 4, "ETWC": 5, "TWC": 6}
G2_PUSH, G2_PULL = 0, 1
G2_BOOLMAP, G2_BITMAP = 0, 1
G2_FUSED, G2_UNFUSED_BOOLMAP, G2_UNFUSED_BITMAP = 0, 1, 2
G2_DEDUP_ENABLED, G2_DEDUP_DISABLED = 0, 1
G2_DEDUP_MONOTONIC_COUNTERS, G2_DEDUP_BITMAP, G2_DEDUP_BOOLMAP = 0, 1, 2
G2_CRITERIA_NONE, G2_INPUT_VERTEXSET_SIZE = 0, 1
G2_FRONTIER_SPARSE, G2_FRONTIER_BITMAP, G2_FRONTIER_BOOLMAP = 0, 1, 2
G2_OP_BFS, G2_OP_RELAX_MIN, G2_OP_LABEL_MIN, G2_OP_PR_ADD, G2_OP_BC_SIGMA, G2_OP_BC_DELTA = range(6)


class g2_schedule(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "load_balance", "edge_blocking", "blocking_size", "direction", "pull_frontier",
        "frontier_creation", "dedup", "dedup_type", "delta", "kernel_fusion")]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class g2_hybrid(ctypes.Structure):
    _fields_ = [("criteria", ctypes.c_int32), ("threshold", ctypes.c_float),
                ("s1", g2_schedule), ("s2", g2_schedule)]


class g2_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("push_rounds", ctypes.c_int32),
                ("pull_rounds", ctypes.c_int32), ("launches", ctypes.c_int32),
                ("arcs_examined", ctypes.c_int64), ("barriers", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class G2Error(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


# ---------------------------------------------------------------- signatures
P = ctypes.c_void_p
I32, I64, U32, F32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_float
_SIGS = {
    "g2_load_csr": [I32, I64, P, P, P, U32, P, ctypes.POINTER(P)],
    "g2_free_graph": [P],
    "g2_graph_view": [P, ctypes.POINTER(P)],
    "g2_graph_info": [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I32),
                      ctypes.POINTER(I64)],
    "g2_edge_block": [P, I32, ctypes.POINTER(I32), P],
    "g2_edge_block_export": [P, P, P, P, P],
    "g2_frontier_create": [P, I32, ctypes.POINTER(P)],
    "g2_frontier_free": [P],
    "g2_frontier_set": [P, P, I32, P],
    "g2_frontier_size": [P, ctypes.POINTER(I32), P],
    "g2_frontier_list": [P, P, I32, ctypes.POINTER(I32), P],
    "g2_edgeset_apply": [P, I32, P, P, P, ctypes.POINTER(g2_hybrid), P, ctypes.POINTER(I32), P],
    "g2_bfs": [P, I32, P, P, ctypes.POINTER(g2_hybrid), P],
    "g2_cc": [P, P, ctypes.POINTER(g2_hybrid), P],
    "g2_sssp_delta": [P, I32, I32, P, ctypes.POINTER(g2_hybrid), P],
    "g2_pagerank": [P, F32, I32, P, ctypes.POINTER(g2_hybrid), P],
    "g2_bc": [P, P, I32, P, ctypes.POINTER(g2_hybrid), P],
    "g2_bfs_batch": [P, P, I32, P, ctypes.POINTER(g2_hybrid), P],
    "g2_sssp_batch": [P, P, I32, I32, P, ctypes.POINTER(g2_hybrid), P],
    "g2_last_stats": [ctypes.POINTER(g2_stats)],
    "g2_set_count_arcs": [I32],
    "g2_last_error": [],
    "g2_selftest_wait_timeout": [I64, P],
    "g2_diag_gather": [P, I64, P, I32, I32, P, I32, ctypes.POINTER(F32), P],
    "g2_bfs_csr_static": [I32, I64, P, P, I32, P, P, P],
    "g2_sssp_async": [P, I32, I32, P, P],
    "g2_bfs_async": [P, I32, I32, P, P, P],
    "g2_set_kernel_timing": [I32],
    "g2_kernel_time": [ctypes.c_char_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64), I32],
    "g2_version": [],
}
_VOID = {"g2_free_graph", "g2_frontier_free", "g2_set_count_arcs", "g2_set_kernel_timing"}
_STR = {"g2_last_error", "g2_version"}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = None if _name in _VOID else (ctypes.c_char_p if _name in _STR else ctypes.c_int)


def exported_symbols():
    """Names of the C entry points this binding declares."""
    return list(_SIGS)


def last_error() -> str:
    return _lib.g2_last_error().decode()


def version() -> str:
    return _lib.g2_version().decode()


def _check(st: int, where: str):
    if st != G2_OK:
        raise G2Error(st, where, last_error())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return ctypes.c_void_p(t.ctypes.data)
    assert t.is_contiguous(), "arrays must be contiguous"
    return ctypes.c_void_p(t.data_ptr())


def _sched(s):
    if s is None:
        return None
    if isinstance(s, g2_hybrid):
        return ctypes.byref(s)
    if isinstance(s, g2_schedule):
        h = g2_hybrid()
        h.s1 = s
        return ctypes.byref(h)
    raise TypeError("schedule must be g2_schedule or g2_hybrid")


# ----------------------------------------------------------------- handles
class Graph:
    """Owner of a g2_graph handle (device CSR / CSC and workspace)."""

    def __init__(self, handle: ctypes.c_void_p, n: int, m: int, symmetric: bool, weighted: bool):
        self.handle = handle
        self.n, self.m, self.symmetric, self.weighted = n, m, symmetric, weighted

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "handle", None):
            _lib.g2_free_graph(self.handle)
            self.handle = None

    def view(self) -> "Graph":
        return g2_graph_view(self)

    def info(self):
        return g2_graph_info(self)


def g2_load_csr(n, rowptr, col, w=None, symmetric=True, stream=None,
                prepare_pagerank=False, overlap=False) -> Graph:
    """Copy a CSR graph to the device.  rowptr/col/w: numpy int32 (host) or
    torch int32 CUDA tensors (device).  prepare_pagerank: build PageRank's
    layouts in the background (G2_PREPARE_PAGERANK).  overlap: the load runs
    beside other GPU work (G2_LOAD_OVERLAP: the upload kernel on a quarter of
    the SMs, no copy engine for the arcs)."""
    dev = not isinstance(rowptr, np.ndarray)
    if not dev:
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        col = np.ascontiguousarray(col, dtype=np.int32)
        if w is not None:
            w = np.ascontiguousarray(w, dtype=np.int32)
    m = int(col.shape[0])
    flags = (G2_SYMMETRIC if symmetric else 0) | (G2_DEVICE_PTRS if dev else 0) | \
        (G2_PREPARE_PAGERANK if prepare_pagerank else 0) | (G2_LOAD_OVERLAP if overlap else 0)
    h = ctypes.c_void_p()
    _check(_lib.g2_load_csr(int(n), m, _ptr(rowptr), _ptr(col), _ptr(w), flags, _stream(stream),
                            ctypes.byref(h)), "g2_load_csr")
    return Graph(h, int(n), m, symmetric, w is not None)


def load_graph(g, weights=None, stream=None) -> Graph:
    """g2_load_csr of a graphgen.Graph (optionally with int32 weights)."""
    return g2_load_csr(g.n, g.rowptr, g.col, weights, g.symmetric, stream)


def g2_graph_view(g: Graph) -> Graph:
    h = ctypes.c_void_p()
    _check(_lib.g2_graph_view(g.handle, ctypes.byref(h)), "g2_graph_view")
    v = Graph(h, g.n, g.m, g.symmetric, g.weighted)
    v._parent = g  # keep the topology owner alive
    return v


def g2_graph_info(g: Graph):
    n, m, sm, l2 = I64(), I64(), I32(), I64()
    _check(_lib.g2_graph_info(g.handle, ctypes.byref(n), ctypes.byref(m), ctypes.byref(sm),
                              ctypes.byref(l2)), "g2_graph_info")
    return {"n": n.value, "m": m.value, "sm_count": sm.value, "l2_bytes": l2.value}


def g2_edge_block(g: Graph, N: int = 0, stream=None) -> int:
    ns = I32()
    _check(_lib.g2_edge_block(g.handle, int(N), ctypes.byref(ns), _stream(stream)), "g2_edge_block")
    return ns.value


def g2_edge_block_export(g: Graph, src, dst, seg_end, stream=None):
    _check(_lib.g2_edge_block_export(g.handle, _ptr(src), _ptr(dst), _ptr(seg_end), _stream(stream)),
           "g2_edge_block_export")


class Frontier:
    def __init__(self, g: Graph, fmt: int):
        self.g = g
        self.fmt = fmt
        h = ctypes.c_void_p()
        _check(_lib.g2_frontier_create(g.handle, int(fmt), ctypes.byref(h)), "g2_frontier_create")
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.g2_frontier_free(self.handle)
            self.handle = None

    def set(self, verts, stream=None):
        v = np.ascontiguousarray(verts, dtype=np.int32)
        _check(_lib.g2_frontier_set(self.handle, _ptr(v), int(v.size), _stream(stream)),
               "g2_frontier_set")

    def size(self, stream=None) -> int:
        s = I32()
        _check(_lib.g2_frontier_size(self.handle, ctypes.byref(s), _stream(stream)),
               "g2_frontier_size")
        return s.value

    def to_list(self, out, stream=None) -> int:
        k = I32()
        _check(_lib.g2_frontier_list(self.handle, _ptr(out), int(out.numel()), ctypes.byref(k),
                                     _stream(stream)), "g2_frontier_list")
        return k.value


def g2_frontier_create(g: Graph, fmt: int) -> Frontier:
    return Frontier(g, fmt)


def g2_edgeset_apply(g: Graph, op: int, fin, vdata, vdata2=None, sched=None, fout=None,
                     stream=None) -> int:
    size = I32(0)
    _check(_lib.g2_edgeset_apply(g.handle, int(op), fin.handle if fin is not None else None,
                                 _ptr(vdata), _ptr(vdata2), _sched(sched),
                                 fout.handle if fout is not None else None, ctypes.byref(size),
                                 _stream(stream)), "g2_edgeset_apply")
    return size.value


# -------------------------------------------------------------- algorithms
def g2_bfs(g: Graph, src: int, depth, parent=None, sched=None, stream=None):
    _check(_lib.g2_bfs(g.handle, int(src), _ptr(depth), _ptr(parent), _sched(sched),
                       _stream(stream)), "g2_bfs")


def g2_cc(g: Graph, label, sched=None, stream=None):
    _check(_lib.g2_cc(g.handle, _ptr(label), _sched(sched), _stream(stream)), "g2_cc")


def g2_sssp_delta(g: Graph, src: int, delta: int, dist, sched=None, stream=None):
    _check(_lib.g2_sssp_delta(g.handle, int(src), int(delta), _ptr(dist), _sched(sched),
                              _stream(stream)), "g2_sssp_delta")


def g2_sssp_async(g: Graph, src: int, delta: int, dist, stream=None):
    _check(_lib.g2_sssp_async(g.handle, int(src), int(delta), _ptr(dist), _stream(stream)),
           "g2_sssp_async")


def g2_bfs_async(g: Graph, src: int, delta: int, depth, parent=None, stream=None):
    _check(_lib.g2_bfs_async(g.handle, int(src), int(delta), _ptr(depth), _ptr(parent),
                             _stream(stream)), "g2_bfs_async")


def g2_pagerank(g: Graph, damping: float, iters: int, rank, sched=None, stream=None):
    _check(_lib.g2_pagerank(g.handle, float(damping), int(iters), _ptr(rank), _sched(sched),
                            _stream(stream)), "g2_pagerank")


def g2_bc(g: Graph, srcs, bc, sched=None, stream=None):
    s = np.ascontiguousarray(srcs, dtype=np.int32)
    _check(_lib.g2_bc(g.handle, _ptr(s), int(s.size), _ptr(bc), _sched(sched), _stream(stream)),
           "g2_bc")


def g2_bfs_batch(g: Graph, srcs, depth, sched=None, stream=None):
    s = np.ascontiguousarray(srcs, dtype=np.int32)
    _check(_lib.g2_bfs_batch(g.handle, _ptr(s), int(s.size), _ptr(depth), _sched(sched),
                             _stream(stream)), "g2_bfs_batch")


def g2_sssp_batch(g: Graph, srcs, delta: int, dist, sched=None, stream=None):
    s = np.ascontiguousarray(srcs, dtype=np.int32)
    _check(_lib.g2_sssp_batch(g.handle, _ptr(s), int(s.size), int(delta), _ptr(dist),
                              _sched(sched), _stream(stream)), "g2_sssp_batch")


def g2_bfs_csr_static(n: int, rowptr, col, src: int, depth, parent=None, stream=None):
    """BFS that allocates no device memory: rowptr/col are the caller's device
    CSR (torch int32 CUDA tensors), depth/parent the caller's outputs; the
    library's fixed scratch holds the frontiers (n <= 1,048,576)."""
    _check(_lib.g2_bfs_csr_static(int(n), int(col.numel()), _ptr(rowptr), _ptr(col), int(src),
                                  _ptr(depth), _ptr(parent), _stream(stream)), "g2_bfs_csr_static")


def g2_last_stats() -> dict:
    s = g2_stats()
    _check(_lib.g2_last_stats(ctypes.byref(s)), "g2_last_stats")
    return {f: getattr(s, f) for f, _ in s._fields_}


def g2_set_count_arcs(enable: bool):
    _lib.g2_set_count_arcs(1 if enable else 0)


def g2_set_kernel_timing(enable: bool):
    _lib.g2_set_kernel_timing(1 if enable else 0)


def g2_kernel_time(name: str, reset: bool = False):
    """(total ms, launches) recorded for the named kernel on this thread."""
    ms, k = ctypes.c_double(), I64()
    _check(_lib.g2_kernel_time(name.encode(), ctypes.byref(ms), ctypes.byref(k), 1 if reset else 0),
           "g2_kernel_time")
    return ms.value, k.value


def g2_selftest_wait_timeout(limit_ns: int, stream=None) -> int:
    """Returns the status code (G2_ETIMEOUT expected)."""
    return _lib.g2_selftest_wait_timeout(int(limit_ns), _stream(stream))


def g2_diag_gather(idx, x, mode, out, grid, stream=None) -> float:
    """Diagnostic gather pass (see include/g2.h); idx/x/out torch CUDA tensors.
    Returns the gather pass's device time in milliseconds."""
    n = 0 if x is None else int(x.numel())
    ms = F32()
    _check(_lib.g2_diag_gather(_ptr(idx), int(idx.numel()), _ptr(x), n, int(mode), _ptr(out),
                               int(grid), ctypes.byref(ms), _stream(stream)), "g2_diag_gather")
    return ms.value


# ------------------------------------------------------------- schedules
def schedule(lb="VERTEX_BASED", direction=G2_PUSH, pull_frontier=G2_BOOLMAP,
             frontier_creation=G2_FUSED, dedup=True, dedup_type=G2_DEDUP_MONOTONIC_COUNTERS,
             delta=0, kernel_fusion=False, edge_blocking=False, blocking_size=0) -> g2_schedule:
    s = g2_schedule()
    s.load_balance = LB[lb] if isinstance(lb, str) else int(lb)
    s.direction = direction
    s.pull_frontier = pull_frontier
    s.frontier_creation = frontier_creation
    s.dedup = G2_DEDUP_ENABLED if dedup else G2_DEDUP_DISABLED
    s.dedup_type = dedup_type
    s.delta = delta
    s.kernel_fusion = 1 if kernel_fusion else 0
    s.edge_blocking = 1 if edge_blocking else 0
    s.blocking_size = blocking_size
    return s


def hybrid(s1: g2_schedule, s2: g2_schedule, threshold: float) -> g2_hybrid:
    h = g2_hybrid()
    h.criteria = G2_INPUT_VERTEXSET_SIZE
    h.threshold = threshold
    h.s1 = s1
    h.s2 = s2
    return h


def simple(s: g2_schedule) -> g2_hybrid:
    h = g2_hybrid()
    h.criteria = G2_CRITERIA_NONE
    h.s1 = s
    return h
