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
LIB_PATH = os.environ.get("TMOTIF_LIB") or os.path.join(HERE, "libtmotif.so")

TM_OK = 0
TM_EINVAL = -1
TM_ENOMEM = -2
TM_ECUDA = -3
TM_ETIMEOUT = -4
TM_EUNSUPPORTED = -5
TM_ECHECK = -6
TM_MAX_EDGES = 8
TM_MAX_VERTICES = 8

TM_INPUT_DEVICE = 0x1
TM_PRESORTED = 0x2

TM_COMINE = 0x0
TM_PERMOTIF = 0x1
TM_AUTO = 0x2
TM_COMINE_MIN_SM = 0.44
TM_LEAF_SCAN = 0x10
TM_SCHED_DYNAMIC = 0x100
TM_SCHED_PLANNED = 0x200
TM_GENERIC = 0x1000
TM_SCHED_SIBLINGS = 0x400
TM_SCHED_TIERS = 0x800
TM_COMPILE_CHAINS = 0x1
TM_COMPILE_CHECK = 0x2
TM_SPEC_MAX_NODES = 256
TM_FEATURES = 8
TM_MODEL_PARAMS = 4801

TM_ROOTS_DEVICE = 0x1
TM_COUNTS_DEVICE = 0x2

TM_WORK_CANDIDATES = 0
TM_WORK_EXPANSIONS = 1
TM_WORK_PROBES = 2
TM_WORK_LEAF_EVALS = 3
TM_WORK_FIELDS = 4
WORK_NAMES = ("candidates", "expansions", "probes", "leaf_evals")

ERRORS = {TM_EINVAL: "TM_EINVAL", TM_ENOMEM: "TM_ENOMEM", TM_ECUDA: "TM_ECUDA",
          TM_ETIMEOUT: "TM_ETIMEOUT", TM_EUNSUPPORTED: "TM_EUNSUPPORTED", TM_ECHECK: "TM_ECHECK"}


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
                ("similarity", ctypes.c_double), ("specialized", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class tm_tree_node(ctypes.Structure):
    _fields_ = [("parent", ctypes.c_int32), ("n_edges", ctypes.c_int32), ("n_children", ctypes.c_int32),
                ("n_refs", ctypes.c_int32), ("u", ctypes.c_int8 * TM_MAX_EDGES),
                ("v", ctypes.c_int8 * TM_MAX_EDGES)]


class tm_count_args(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("roots", ctypes.c_void_p),
                ("n_roots", ctypes.c_int64), ("root_lo", ctypes.c_int64), ("root_hi", ctypes.c_int64),
                ("per_root_counts", ctypes.c_void_p), ("per_root_work", ctypes.c_void_p),
                ("ctas_per_sm", ctypes.c_int32), ("offload_max", ctypes.c_int32), ("root_split", ctypes.c_void_p),
                ("poll_every", ctypes.c_int32), ("donate_seq", ctypes.c_int32), ("donate_leaf", ctypes.c_int32),
                ("sibling_always", ctypes.c_int32)]


class tm_server_config(ctypes.Structure):
    _fields_ = [("streams", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("mem_budget", ctypes.c_int64),
                ("mode", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class tm_request_stats(ctypes.Structure):
    _fields_ = [("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double), ("batch", ctypes.c_int32),
                ("batch_size", ctypes.c_int32)]


class tm_server_info(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_int64), ("requests_done", ctypes.c_int64), ("pending", ctypes.c_int64),
                ("in_flight", ctypes.c_int64), ("admitted_bytes", ctypes.c_int64),
                ("peak_admitted_bytes", ctypes.c_int64)]


class tm_tune(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int32), ("donate_seq", ctypes.c_int32), ("donate_leaf", ctypes.c_int32),
                ("poll_every", ctypes.c_int32), ("ms", ctypes.c_float)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class tm_compile_info(ctypes.Structure):
    _fields_ = [("kernels", ctypes.c_int32), ("compiled", ctypes.c_int32), ("wall_ms", ctypes.c_double),
                ("registers", ctypes.c_int32), ("local_bytes", ctypes.c_int32), ("static_smem", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("source_hash", ctypes.c_uint64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}


class tm_run_stats(ctypes.Structure):
    _fields_ = [("n_roots", ctypes.c_int64), ("candidates", ctypes.c_int64), ("expansions", ctypes.c_int64),
                ("probes", ctypes.c_int64), ("leaf_evals", ctypes.c_int64), ("algo_bytes", ctypes.c_int64),
                ("tasks_split", ctypes.c_int64), ("launches", ctypes.c_int64), ("kernel_ms", ctypes.c_double),
                ("warp_imbalance", ctypes.c_double), ("algo_bytes_lists", ctypes.c_int64),
                ("idle_expired", ctypes.c_int64), ("roots_thread_tier", ctypes.c_int64), ("roots_split", ctypes.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None

EXPORTS = ("tm_graph_load", "tm_graph_get_info", "tm_graph_edges", "tm_graph_free", "tm_tree_build",
           "tm_tree_get_info", "tm_tree_get_node", "tm_tree_free", "tm_tree_compile", "tm_count", "tm_count_noalloc",
           "tm_graph_bipartite", "tm_comine_advice", "tm_enumerate",
           "tm_features", "tm_model_create", "tm_model_free", "tm_model_get_params", "tm_model_set_params",
           "tm_model_fit_norm", "tm_model_predict", "tm_model_loss_grad", "tm_model_train", "tm_plan",
           "tm_plan_tiers",
           "tm_exec_create", "tm_exec_launch", "tm_exec_status", "tm_exec_free", "tm_autotune",
           "tm_server_open", "tm_server_submit", "tm_server_poll", "tm_server_get_info", "tm_server_close",
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
        L.tm_tree_compile.argtypes = [P, u32, ctypes.POINTER(tm_compile_info)]
        L.tm_count.argtypes = [P, P, ctypes.POINTER(tm_count_args), P, ctypes.POINTER(tm_run_stats), P]
        L.tm_count_noalloc.argtypes = [P, P, P, i64, i64, i64, P, P]
        F = ctypes.c_float
        L.tm_features.argtypes = [P, P, P, i64, P, P]
        L.tm_model_create.argtypes = [ctypes.c_uint64, ctypes.POINTER(P)]
        L.tm_model_free.argtypes = [P]
        L.tm_model_get_params.argtypes = [P, P, P]
        L.tm_model_set_params.argtypes = [P, P, P]
        L.tm_model_fit_norm.argtypes = [P, P, i64, P]
        L.tm_model_predict.argtypes = [P, P, i64, P, P]
        L.tm_model_loss_grad.argtypes = [P, P, P, i64, P, P, P]
        L.tm_model_train.argtypes = [P, P, P, i64, i32, i32, F, P, P]
        L.tm_plan.argtypes = [P, P, P, i64, ctypes.c_double, i32, P, P, P]
        L.tm_plan_tiers.argtypes = [P, P, P, i64, ctypes.c_double, i32, ctypes.c_double, P, P, P]
        L.tm_exec_create.argtypes = [P, P, ctypes.POINTER(tm_count_args), P, P, ctypes.POINTER(P)]
        L.tm_exec_launch.argtypes = [P, P]
        L.tm_exec_status.argtypes = [P, P]
        L.tm_exec_free.argtypes = [P]
        L.tm_autotune.argtypes = [P, P, ctypes.POINTER(tm_count_args), ctypes.POINTER(tm_tune), P]
        L.tm_server_open.argtypes = [P, ctypes.POINTER(tm_server_config), ctypes.POINTER(P)]
        L.tm_server_submit.argtypes = [P, P, P, i32, P, P, i64, ctypes.POINTER(i64)]
        L.tm_server_poll.argtypes = [P, i64, i32, P, ctypes.POINTER(tm_request_stats)]
        L.tm_server_get_info.argtypes = [P, ctypes.POINTER(tm_server_info)]
        L.tm_server_close.argtypes = [P]
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


def tm_graph_bipartite(g, stream=None) -> bool:
    out = ctypes.c_int32(-1)
    _check(lib().tm_graph_bipartite(g, ctypes.byref(out), _stream(stream)))
    return bool(out.value)


def tm_comine_advice(g, tr, stream=None) -> bool:
    """True: co-mine (TM_COMINE); False: mine each motif alone (TM_PERMOTIF)."""
    out = ctypes.c_int32(-1)
    _check(lib().tm_comine_advice(g, tr, ctypes.byref(out), _stream(stream)))
    return bool(out.value)


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
    return {name: getattr(info, name) for name, _ in info._fields_ if name != "reserved"}


def tm_tree_get_node(tr, index: int) -> dict:
    n = tm_tree_node()
    _check(lib().tm_tree_get_node(tr, int(index), ctypes.byref(n)))
    C = tuple((n.u[k], n.v[k]) for k in range(n.n_edges))
    return {"parent": n.parent, "C": C, "n_children": n.n_children, "n_refs": n.n_refs}


def tm_tree_free(tr) -> None:
    _check(lib().tm_tree_free(tr))


def tm_tree_compile(tr, flags: int = 0) -> dict:
    """Compile kernels specialised to the tree (runtime code generation);
    later counts on it use them unless mode has TM_GENERIC or TM_LEAF_SCAN."""
    info = tm_compile_info()
    _check(lib().tm_tree_compile(tr, int(flags), ctypes.byref(info)))
    return info.as_dict()


def _count_args(mode=TM_COMINE, roots=None, root_lo=0, root_hi=0, per_root_counts=None, per_root_work=None,
                ctas_per_sm=0, root_split=None, tune=None):
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
    if root_split is not None:
        p, on_dev, k = _ptr(root_split, np.int32)
        if not on_dev:
            raise TypeError("root_split must be a CUDA tensor")
        keep.append(k)
        a.root_split = p
    if tune is not None:
        a.ctas_per_sm = tune["ctas_per_sm"]
        a.donate_seq = tune["donate_seq"]
        a.donate_leaf = tune["donate_leaf"]
        a.poll_every = tune["poll_every"]
        a.offload_max = tune.get("offload_max", 0)
        a.sibling_always = tune.get("sibling_always", 0)
    return a, keep


def tm_count(g, tr, mode: int = TM_COMINE, roots=None, root_lo: int = 0, root_hi: int = 0,
             counts=None, per_root_counts=None, per_root_work=None, stats: bool = False,
             stream=None, ctas_per_sm: int = 0, root_split=None, tune=None):
    """Counts of every motif (np.int64 array, or into the device tensor ``counts``).

    Returns ``counts`` or ``(counts, stats_dict)`` when ``stats``.
    """
    a, keep = _count_args(mode, roots, root_lo, root_hi, per_root_counts, per_root_work, ctas_per_sm,
                          root_split, tune)
    n_motifs = tm_tree_get_info(tr)["n_motifs"]
    if counts is None:
        out = np.zeros(n_motifs, np.int64)
        pc = out.ctypes.data_as(ctypes.c_void_p)
    else:
        pc, on_dev, out = _ptr(counts, np.int64)
        if len(out.reshape(-1)) < n_motifs:
            raise ValueError("counts holds %d values; the tree has %d motifs" % (len(out.reshape(-1)), n_motifs))
        if on_dev:
            a.flags |= TM_COUNTS_DEVICE
    n_roots = a.n_roots if roots is not None else (
        (root_hi if root_hi > 0 else tm_graph_get_info(g)["n_edges"]) - root_lo)
    # the library writes [n_roots][fields] per-root outputs and reads n_roots
    # slices; it cannot see the tensors' lengths
    for name, arr, per in (("per_root_counts", per_root_counts, n_motifs),
                           ("per_root_work", per_root_work, TM_WORK_FIELDS), ("root_split", root_split, 1)):
        if arr is not None and arr.numel() < max(n_roots, 0) * per:
            raise ValueError("%s holds %d values; %d roots need %d" % (name, arr.numel(), n_roots, n_roots * per))
    st = tm_run_stats()
    _check(lib().tm_count(g, tr, ctypes.byref(a), pc, ctypes.byref(st) if stats else None, _stream(stream)))
    return (out, st.as_dict()) if stats else out


MATCH_FIELDS = 2 + TM_MAX_EDGES        # tm_match: motif, n_edges, eid[TM_MAX_EDGES] (int32 each)


def tm_enumerate(g, tr, cap: int, roots=None, root_lo: int = 0, root_hi: int = 0, mode: int = TM_COMINE,
                 stream=None):
    """Every match of every motif with its first edge among the roots.

    Returns ``(matches, n_found, counts)``: ``matches`` an int32 array of
    shape (min(n_found, cap), 2 + TM_MAX_EDGES) with rows (motif, n_edges,
    eid_1, ..., eid_8; -1 past n_edges), ``n_found`` the number of matches
    (> cap when records were dropped) and ``counts`` the matches per motif.
    """
    import torch
    a, keep = _count_args(mode, roots, root_lo, root_hi)
    n_motifs = tm_tree_get_info(tr)["n_motifs"]
    buf = torch.empty((max(cap, 0), MATCH_FIELDS), dtype=torch.int32, device="cuda") if cap > 0 else None
    out_p = ctypes.c_void_p(buf.data_ptr()) if buf is not None else None
    n_found = ctypes.c_int64(0)
    counts = np.zeros(n_motifs, np.int64)
    _check(lib().tm_enumerate(g, tr, ctypes.byref(a), out_p, ctypes.c_int64(cap), ctypes.byref(n_found),
                              counts.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    n = min(n_found.value, max(cap, 0))
    matches = buf[:n].cpu().numpy() if buf is not None else np.zeros((0, MATCH_FIELDS), np.int32)
    return matches, n_found.value, counts


def tm_count_noalloc(g, tr, counts, roots=None, root_lo: int = 0, root_hi: int = 0, stream=None):
    """Allocation-free count into the device tensor ``counts`` (int64, n_motifs).

    ``roots``: a CUDA int32 tensor of root edge ids, or None for the range.
    The call does not synchronise; it allocates no device memory (its
    scratch is a static array in the library, shared by all calls).
    """
    pc, on_dev, keep_c = _ptr(counts, np.int64)
    if not on_dev:
        raise TypeError("counts must be a CUDA tensor")
    n_motifs = tm_tree_get_info(tr)["n_motifs"]
    if counts.numel() < n_motifs:
        # the library writes n_motifs values and cannot see the tensor's length
        raise ValueError("counts holds %d values; the tree has %d motifs" % (counts.numel(), n_motifs))
    pr, n = None, 0
    if roots is not None:
        pr, r_dev, keep_r = _ptr(roots, np.int32)
        if not r_dev:
            raise TypeError("roots must be a CUDA tensor")
        n = len(keep_r)
    _check(lib().tm_count_noalloc(g, tr, pr, n, root_lo, root_hi, pc, _stream(stream)))
    return counts


class Exec:
    """A count captured once in a CUDA graph (tm_exec); counts land in ``counts``."""

    def __init__(self, g, tr, counts, stream=None, **kw):
        a, self._keep = _count_args(**kw)
        pc = _dev(counts, np.int64, "counts")
        self.counts = counts
        self.h = ctypes.c_void_p()
        _check(lib().tm_exec_create(g, tr, ctypes.byref(a), pc, _stream(stream), ctypes.byref(self.h)))

    def launch(self, stream=None):
        _check(lib().tm_exec_launch(self.h, _stream(stream)))

    def status(self, stream=None):
        _check(lib().tm_exec_status(self.h, _stream(stream)))

    def close(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _check(lib().tm_exec_free(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Owning wrapper of a tm_server (continuous batching over a resident graph)."""

    def __init__(self, graph, streams: int = 2, max_batch: int = 32, mem_budget: int = 4 << 30,
                 mode: int = TM_SCHED_DYNAMIC):
        self.graph = graph
        cfg = tm_server_config(streams, max_batch, mem_budget, mode, 0)
        self.h = ctypes.c_void_p()
        _check(lib().tm_server_open(graph.h, ctypes.byref(cfg), ctypes.byref(self.h)))
        self.n_motifs = {}

    def submit(self, motifs, deltas, roots) -> int:
        uv, off = motif_arrays(motifs)
        d = np.broadcast_to(np.asarray(deltas, np.int64), (len(motifs),)).copy()
        r = np.ascontiguousarray(roots, np.int32)
        tk = ctypes.c_int64(0)
        _check(lib().tm_server_submit(self.h, uv.ctypes.data_as(ctypes.c_void_p), off.ctypes.data_as(ctypes.c_void_p),
                                      len(motifs), d.ctypes.data_as(ctypes.c_void_p),
                                      r.ctypes.data_as(ctypes.c_void_p), len(r), ctypes.byref(tk)))
        self.n_motifs[tk.value] = len(motifs)
        return tk.value

    def poll(self, ticket: int, wait: bool = False):
        """None while pending, else (counts, stats dict)."""
        out = np.zeros(self.n_motifs[ticket], np.int64)
        st = tm_request_stats()
        rc = lib().tm_server_poll(self.h, ticket, 1 if wait else 0, out.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.byref(st))
        if rc == 0:
            return None
        if rc < 0:
            raise TMError(rc, tm_last_error())
        del self.n_motifs[ticket]
        return out, {name: getattr(st, name) for name, _ in st._fields_}

    def info(self) -> dict:
        i = tm_server_info()
        _check(lib().tm_server_get_info(self.h, ctypes.byref(i)))
        return {name: getattr(i, name) for name, _ in i._fields_}

    def close(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _check(lib().tm_server_close(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tm_autotune(g, tr, stream=None, **kw) -> dict:
    a, keep = _count_args(**kw)
    t = tm_tune()
    _check(lib().tm_autotune(g, tr, ctypes.byref(a), ctypes.byref(t), _stream(stream)))
    return t.as_dict()


# ------------------------------------------------------------------ learned scheduling

def _dev(x, dtype, name):
    p, on_dev, k = _ptr(x, dtype)
    if not on_dev:
        raise TypeError(name + " must be a CUDA tensor")
    return p


def _devf(x, name):
    import torch
    if not (_is_torch(x) and x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()):
        raise TypeError(name + " must be a contiguous CUDA float32 tensor")
    return ctypes.c_void_p(x.data_ptr())


def tm_features(g, tr, roots, feats, stream=None):
    n = len(roots)
    _check(lib().tm_features(g, tr, _dev(roots, np.int32, "roots"), n, _devf(feats, "feats"), _stream(stream)))
    return feats


class Model:
    """Owning wrapper of a tm_model (the scheduler's cost model)."""

    def __init__(self, seed: int = 1):
        self.h = ctypes.c_void_p()
        _check(lib().tm_model_create(int(seed), ctypes.byref(self.h)))

    def params(self):
        w = np.zeros(TM_MODEL_PARAMS, np.float32)
        nm = np.zeros(2 * TM_FEATURES, np.float32)
        _check(lib().tm_model_get_params(self.h, w.ctypes.data_as(ctypes.c_void_p), nm.ctypes.data_as(ctypes.c_void_p)))
        return w, nm

    def set_params(self, w=None, norm=None):
        pw = None if w is None else np.ascontiguousarray(w, np.float32)
        pn = None if norm is None else np.ascontiguousarray(norm, np.float32)
        _check(lib().tm_model_set_params(self.h, None if pw is None else pw.ctypes.data_as(ctypes.c_void_p),
                                         None if pn is None else pn.ctypes.data_as(ctypes.c_void_p)))

    def fit_norm(self, feats, stream=None):
        _check(lib().tm_model_fit_norm(self.h, _devf(feats, "feats"), feats.shape[0], _stream(stream)))

    def predict(self, feats, out, stream=None):
        _check(lib().tm_model_predict(self.h, _devf(feats, "feats"), feats.shape[0], _devf(out, "out"),
                                      _stream(stream)))
        return out

    def loss_grad(self, feats, labels, stream=None):
        loss = ctypes.c_float(0)
        g = np.zeros(TM_MODEL_PARAMS, np.float32)
        _check(lib().tm_model_loss_grad(self.h, _devf(feats, "feats"), _devf(labels, "labels"), feats.shape[0],
                                        ctypes.byref(loss), g.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
        return float(loss.value), g

    def train(self, feats, labels, epochs: int, batch: int = 256, lr: float = 1e-3, stream=None):
        hist = np.zeros(max(epochs, 1), np.float32)
        _check(lib().tm_model_train(self.h, _devf(feats, "feats"), _devf(labels, "labels"), feats.shape[0],
                                    int(epochs), int(batch), float(lr), hist.ctypes.data_as(ctypes.c_void_p),
                                    _stream(stream)))
        return hist[:epochs]

    def plan(self, feats, roots, roots_out, split_out, unit_work: float, max_split: int, stream=None,
             thread_work: float = 0.0):
        """Order and slices (tm_plan); with thread_work > 0, roots predicted
        below it get slice count 0: the thread tier of TM_SCHED_TIERS."""
        if thread_work > 0:
            _check(lib().tm_plan_tiers(self.h, _devf(feats, "feats"), _dev(roots, np.int32, "roots"), len(roots),
                                       float(unit_work), int(max_split), float(thread_work),
                                       _dev(roots_out, np.int32, "roots_out"), _dev(split_out, np.int32, "split_out"),
                                       _stream(stream)))
            return roots_out, split_out
        _check(lib().tm_plan(self.h, _devf(feats, "feats"), _dev(roots, np.int32, "roots"), len(roots),
                             float(unit_work), int(max_split), _dev(roots_out, np.int32, "roots_out"),
                             _dev(split_out, np.int32, "split_out"), _stream(stream)))
        return roots_out, split_out

    def close(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _check(lib().tm_model_free(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ handles

class Graph:
    """Owning wrapper of a tm_graph handle."""

    def __init__(self, src, dst, t, n_nodes: int, presorted: bool = False, stream=None):
        self.h = tm_graph_load(src, dst, t, n_nodes, TM_PRESORTED if presorted else 0, stream)

    def info(self) -> dict:
        return tm_graph_get_info(self.h)

    def edges(self):
        return tm_graph_edges(self.h)

    def bipartite(self) -> bool:
        return tm_graph_bipartite(self.h)

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

    def compile(self, flags: int = 0) -> dict:
        return tm_tree_compile(self.h, flags)

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
