"""Python binding of the C-ABI in ``include/tmotif.h`` (ctypes).

Argument marshalling only: every step of loading, tree building and
counting runs in ``libtmotif.so``.  The functions carry the C names.  Host
arrays are numpy; device arrays are torch CUDA tensors (their pointers are
passed with the matching TM_*_DEVICE flag).  There is no fallback: if the
library is missing or a call fails, a :class:`TMError` is raised.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtmotif.so")

TM_OK = 0
TM_EINVAL = -1
TM_ENOMEM = -2
TM_ECUDA = -3
TM_ETIMEOUT = -4
TM_EUNSUPPORTED = -5
TM_MAX_EDGES = 8
TM_MAX_VERTICES = 8

TM_INPUT_DEVICE = 0x1
TM_PRESORTED = 0x2

TM_COMINE = 0x0
TM_PERMOTIF = 0x1
TM_LEAF_SCAN = 0x10
TM_SCHED_DYNAMIC = 0x100

TM_ROOTS_DEVICE = 0x1
TM_COUNTS_DEVICE = 0x2

TM_WORK_FIELDS = 4
WORK_NAMES = ("candidates", "expansions", "probes", "leaf_evals")

ERRORS = {TM_EINVAL: "TM_EINVAL", TM_ENOMEM: "TM_ENOMEM", TM_ECUDA: "TM_ECUDA",
          TM_ETIMEOUT: "TM_ETIMEOUT", TM_EUNSUPPORTED: "TM_EUNSUPPORTED"}


class TMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "error"), code, msg))
        self.code = code


class tm_graph_info(ctypes.Structure):
    _fields_ = [("n_edges", ctypes.c_int64), ("n_nodes", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("n_pairs", ctypes.c_int64), ("max_out_degree", ctypes.c_int64),
                ("max_in_degree", ctypes.c_int64), ("device_bytes", ctypes.c_int64)]


class tm_tree_info(ctypes.Structure):
    _fields_ = [("n_motifs", ctypes.c_int32), ("n_nodes", ctypes.c_int32), ("n_leaves", ctypes.c_int32),
                ("depth", ctypes.c_int32), ("n_deltas", ctypes.c_int32), ("max_vertices", ctypes.c_int32),
                ("similarity", ctypes.c_double)]


class tm_tree_node(ctypes.Structure):
    _fields_ = [("parent", ctypes.c_int32), ("n_edges", ctypes.c_int32), ("n_children", ctypes.c_int32),
                ("n_refs", ctypes.c_int32), ("u", ctypes.c_int8 * TM_MAX_EDGES),
                ("v", ctypes.c_int8 * TM_MAX_EDGES)]


class tm_count_args(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("roots", ctypes.c_void_p),
                ("n_roots", ctypes.c_int64), ("root_lo", ctypes.c_int64), ("root_hi", ctypes.c_int64),
                ("per_root_counts", ctypes.c_void_p), ("per_root_work", ctypes.c_void_p),
                ("ctas_per_sm", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class tm_run_stats(ctypes.Structure):
    _fields_ = [("n_roots", ctypes.c_int64), ("candidates", ctypes.c_int64), ("expansions", ctypes.c_int64),
                ("probes", ctypes.c_int64), ("leaf_evals", ctypes.c_int64), ("algo_bytes", ctypes.c_int64),
                ("tasks_split", ctypes.c_int64), ("launches", ctypes.c_int64), ("kernel_ms", ctypes.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None

EXPORTS = ("tm_graph_load", "tm_graph_get_info", "tm_graph_edges", "tm_graph_free", "tm_tree_build",
           "tm_tree_get_info", "tm_tree_get_node", "tm_tree_free", "tm_count", "tm_count_noalloc",
           "tm_last_error", "tm_version")


def lib():
    """Load libtmotif.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise TMError(TM_ECUDA, "libtmotif.so not built (run paper_2507_14813_b300/build.py)")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        L.tm_graph_load.argtypes = [P, P, P, i64, i32, u32, P, ctypes.POINTER(P)]
        L.tm_graph_get_info.argtypes = [P, ctypes.POINTER(tm_graph_info)]
        L.tm_graph_edges.argtypes = [P, P, P, P]
        L.tm_graph_free.argtypes = [P]
        L.tm_tree_build.argtypes = [P, P, i32, P, ctypes.POINTER(P)]
        L.tm_tree_get_info.argtypes = [P, ctypes.POINTER(tm_tree_info)]
        L.tm_tree_get_node.argtypes = [P, i32, ctypes.POINTER(tm_tree_node)]
        L.tm_tree_free.argtypes = [P]
        L.tm_count.argtypes = [P, P, ctypes.POINTER(tm_count_args), P, ctypes.POINTER(tm_run_stats), P]
        L.tm_count_noalloc.argtypes = [P, P, P, i64, i64, i64, P, P]
        L.tm_last_error.restype = ctypes.c_char_p
        L.tm_version.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name not in ("tm_last_error", "tm_version"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc: int):
    if rc != TM_OK:
        raise TMError(rc, lib().tm_last_error().decode())


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, on_device, keepalive) for a numpy array or torch tensor."""
    if x is None:
        return None, False, None
    if _is_torch(x):
        import torch
        want = {np.int32: torch.int32, np.int64: torch.int64}[dtype]
        if x.dtype != want or not x.is_contiguous():
            raise TypeError("expected a contiguous %s tensor" % want)
        return ctypes.c_void_p(x.data_ptr()), x.is_cuda, x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data_as(ctypes.c_void_p), False, a


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def tm_last_error() -> str:
    return lib().tm_last_error().decode()


def tm_version() -> str:
    return lib().tm_version().decode()


def tm_graph_load(src, dst, t, n_nodes: int, flags: int = 0, stream=None) -> ctypes.c_void_p:
    ps, ds, ks = _ptr(src, np.int32)
    pd, dd, kd = _ptr(dst, np.int32)
    pt, dt, kt = _ptr(t, np.int64)
    if ds or dd or dt:
        if not (ds and dd and dt):
            raise TypeError("src, dst and t must all be host or all be device arrays")
        flags |= TM_INPUT_DEVICE
    n = len(ks) if ks is not None else 0
    out = ctypes.c_void_p()
    _check(lib().tm_graph_load(ps, pd, pt, n, int(n_nodes), flags, _stream(stream), ctypes.byref(out)))
    return out


def tm_graph_get_info(g) -> dict:
    info = tm_graph_info()
    _check(lib().tm_graph_get_info(g, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in info._fields_ if name != "reserved"}


def tm_graph_edges(g):
    n = tm_graph_get_info(g)["n_edges"]
    s = np.empty(n, np.int32)
    d = np.empty(n, np.int32)
    t = np.empty(n, np.int64)
    _check(lib().tm_graph_edges(g, s.ctypes.data_as(ctypes.c_void_p), d.ctypes.data_as(ctypes.c_void_p),
                                t.ctypes.data_as(ctypes.c_void_p)))
    return s, d, t


def tm_graph_free(g) -> None:
    _check(lib().tm_graph_free(g))


def motif_arrays(motifs: Sequence):
    off = np.zeros(len(motifs) + 1, np.int32)
    uv = []
    for i, m in enumerate(motifs):
        off[i + 1] = off[i] + len(m)
        for a, b in m:
            uv += [a, b]
    return np.asarray(uv if uv else [0], np.int8), off


def tm_tree_build(motifs: Sequence, deltas) -> ctypes.c_void_p:
    uv, off = motif_arrays(motifs)
    d = np.broadcast_to(np.asarray(deltas, np.int64), (len(motifs),)).copy()
    out = ctypes.c_void_p()
    _check(lib().tm_tree_build(uv.ctypes.data_as(ctypes.c_void_p), off.ctypes.data_as(ctypes.c_void_p),
                               len(motifs), d.ctypes.data_as(ctypes.c_void_p), ctypes.byref(out)))
    return out


def tm_tree_get_info(tr) -> dict:
    info = tm_tree_info()
    _check(lib().tm_tree_get_info(tr, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in info._fields_}


def tm_tree_get_node(tr, index: int) -> dict:
    n = tm_tree_node()
    _check(lib().tm_tree_get_node(tr, int(index), ctypes.byref(n)))
    C = tuple((n.u[k], n.v[k]) for k in range(n.n_edges))
    return {"parent": n.parent, "C": C, "n_children": n.n_children, "n_refs": n.n_refs}


def tm_tree_free(tr) -> None:
    _check(lib().tm_tree_free(tr))


def tm_count(g, tr, mode: int = TM_COMINE, roots=None, root_lo: int = 0, root_hi: int = 0,
             counts=None, per_root_counts=None, per_root_work=None, stats: bool = False,
             stream=None, ctas_per_sm: int = 0):
    """Counts of every motif (np.int64 array, or into the device tensor ``counts``).

    Returns ``counts`` or ``(counts, stats_dict)`` when ``stats``.
    """
    a = tm_count_args()
    a.mode = mode
    a.flags = 0
    keep = []
    if roots is not None:
        pr, on_dev, k = _ptr(roots, np.int32)
        keep.append(k)
        a.roots = pr
        a.n_roots = len(k)
        if on_dev:
            a.flags |= TM_ROOTS_DEVICE
    a.root_lo = root_lo
    a.root_hi = root_hi
    for name, arr in (("per_root_counts", per_root_counts), ("per_root_work", per_root_work)):
        if arr is not None:
            p, on_dev, k = _ptr(arr, np.int64)
            if not on_dev:
                raise TypeError(name + " must be a CUDA tensor")
            keep.append(k)
            setattr(a, name, p)
    a.ctas_per_sm = ctas_per_sm
    n_motifs = tm_tree_get_info(tr)["n_motifs"]
    if counts is None:
        out = np.zeros(n_motifs, np.int64)
        pc = out.ctypes.data_as(ctypes.c_void_p)
    else:
        pc, on_dev, out = _ptr(counts, np.int64)
        if on_dev:
            a.flags |= TM_COUNTS_DEVICE
    st = tm_run_stats()
    _check(lib().tm_count(g, tr, ctypes.byref(a), pc, ctypes.byref(st) if stats else None, _stream(stream)))
    return (out, st.as_dict()) if stats else out


def tm_count_noalloc(g, tr, counts, roots=None, root_lo: int = 0, root_hi: int = 0, stream=None):
    """Allocation-free count into the device tensor ``counts`` (int64, n_motifs).

    ``roots``: a CUDA int32 tensor of root edge ids, or None for the range.
    The call does not synchronise; it allocates no device memory (its
    scratch is a static array in the library, shared by all calls).
    """
    pc, on_dev, keep_c = _ptr(counts, np.int64)
    if not on_dev:
        raise TypeError("counts must be a CUDA tensor")
    pr, n = None, 0
    if roots is not None:
        pr, r_dev, keep_r = _ptr(roots, np.int32)
        if not r_dev:
            raise TypeError("roots must be a CUDA tensor")
        n = len(keep_r)
    _check(lib().tm_count_noalloc(g, tr, pr, n, root_lo, root_hi, pc, _stream(stream)))
    return counts


# ------------------------------------------------------------------ handles

class Graph:
    """Owning wrapper of a tm_graph handle."""

    def __init__(self, src, dst, t, n_nodes: int, presorted: bool = False, stream=None):
        self.h = tm_graph_load(src, dst, t, n_nodes, TM_PRESORTED if presorted else 0, stream)

    def info(self) -> dict:
        return tm_graph_get_info(self.h)

    def edges(self):
        return tm_graph_edges(self.h)

    def close(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            tm_graph_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Tree:
    """Owning wrapper of a tm_tree handle."""

    def __init__(self, motifs: Sequence, deltas):
        self.motifs = list(motifs)
        self.h = tm_tree_build(motifs, deltas)

    def info(self) -> dict:
        return tm_tree_get_info(self.h)

    def node(self, i: int) -> dict:
        return tm_tree_get_node(self.h, i)

    def nodes(self):
        return [self.node(i) for i in range(self.info()["n_nodes"])]

    def close(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            tm_tree_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def count(graph: Graph, tree: Tree, **kw):
    return tm_count(graph.h, tree.h, **kw)
