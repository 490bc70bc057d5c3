"""CPU oracle for exact delta-temporal motif counting.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
path (the CUDA library and its binding) neither imports nor links it, and
this package imports nothing from the product.

* :func:`count_motif` -- Algorithm 1 (per motif), in ``tmotif_oracle.c``;
* :func:`comine` -- Algorithm 3 over an MG-Tree from :mod:`oracle.mgtree`
  (Algorithm 2);
* :func:`count_motif_timed` -- Algorithm 1 over roots with a time limit, for
  the timed CPU baseline.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

from . import mgtree

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tmotif_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

MAX_EDGES = 16


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, OpenMP for the timed baseline)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        lib.oracle_count_motif.argtypes = [P, P, P, i64, i32, P, P, ctypes.c_int, i64, P, i64, i64,
                                           ctypes.c_int, P, P, P]
        lib.oracle_count_motif.restype = ctypes.c_int
        lib.oracle_comine.argtypes = [P, P, P, i64, i32, ctypes.c_int, P, P, P, P, P, P, P,
                                      ctypes.c_int, i64, P, i64, i64, P, P, P]
        lib.oracle_comine.restype = ctypes.c_int
        lib.oracle_count_motif_mt.argtypes = [P, P, P, i64, i32, P, P, ctypes.c_int, i64, P, i64,
                                              ctypes.c_int, ctypes.c_double, P, P]
        lib.oracle_count_motif_mt.restype = ctypes.c_int
        lib.oracle_enumerate_motif.argtypes = [P, P, P, i64, i32, P, P, ctypes.c_int, i64, P, i64, P, i64, P]
        lib.oracle_enumerate_motif.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _graph(src, dst, t, n_nodes):
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    t = np.ascontiguousarray(t, np.int64)
    if n_nodes is None:
        n_nodes = int(max(src.max(initial=-1), dst.max(initial=-1))) + 1
    return src, dst, t, int(n_nodes)


def count_motif(src, dst, t, motif: Sequence, delta: int, roots=None, n_nodes=None,
                max_work: int = 0, per_root: bool = False, work: bool = False,
                root_budget: int = 0):
    """Algorithm 1: count one motif.  Returns total (and per-root / work arrays).

    ``max_work`` bounds the candidates examined; when it is exceeded the
    result is ``None`` (the count would be incomplete).  With ``root_budget``
    the bound applies per root instead: a root past it gets per-root count -1
    and is left out of the total.
    """
    if root_budget:
        max_work = int(root_budget)
    src, dst, t, V = _graph(src, dst, t, n_nodes)
    m = mgtree.canonical(motif)
    mu = np.array([e[0] for e in m], np.int8)
    mv = np.array([e[1] for e in m], np.int8)
    r = None if roots is None else np.ascontiguousarray(roots, np.int32)
    nr = len(src) if r is None else len(r)
    pr = np.zeros(nr, np.int64) if per_root else None
    wk = np.zeros(nr, np.int64) if work else None
    tot = ctypes.c_int64(0)
    rc = _load().oracle_count_motif(_p(src), _p(dst), _p(t), len(src), V, _p(mu), _p(mv), len(m),
                                    int(delta), _p(r), nr, int(max_work), 1 if root_budget else 0,
                                    ctypes.byref(tot), _p(pr), _p(wk))
    if rc < 0:
        raise ValueError("oracle rejected the motif or delta")
    total = None if rc == 1 else int(tot.value)
    if per_root or work:
        out = [total]
        if per_root:
            out.append(pr)
        if work:
            out.append(wk)
        return tuple(out)
    return total


def enumerate_motif(src, dst, t, motif: Sequence, delta: int, roots=None, n_nodes=None, cap: int = 1 << 22):
    """Algorithm 1, recording each match it completes.

    Returns ``(matches, total)``: an int32 array of shape (min(total, cap), m)
    with the edge ids of each match in motif edge order, and the number of
    matches.
    """
    src, dst, t, V = _graph(src, dst, t, n_nodes)
    m = mgtree.canonical(motif)
    mu = np.array([e[0] for e in m], np.int8)
    mv = np.array([e[1] for e in m], np.int8)
    r = None if roots is None else np.ascontiguousarray(roots, np.int32)
    nr = len(src) if r is None else len(r)
    out = np.zeros((max(cap, 1), len(m)), np.int32)
    n = ctypes.c_int64(0)
    rc = _load().oracle_enumerate_motif(_p(src), _p(dst), _p(t), len(src), V, _p(mu), _p(mv), len(m),
                                        int(delta), _p(r), nr, _p(out), int(cap), ctypes.byref(n))
    if rc < 0:
        raise ValueError("oracle rejected the motif or delta")
    return out[:min(n.value, cap)], int(n.value)


def count_motifs(src, dst, t, motifs, deltas, roots=None, n_nodes=None, per_root=False):
    """Algorithm 1 for each motif in turn (deltas: one per motif or a scalar)."""
    if np.isscalar(deltas):
        deltas = [deltas] * len(motifs)
    res = [count_motif(src, dst, t, m, d, roots=roots, n_nodes=n_nodes, per_root=per_root)
           for m, d in zip(motifs, deltas)]
    if per_root:
        return np.array([r[0] for r in res], np.int64), np.stack([r[1] for r in res], axis=1)
    return np.array(res, np.int64)


def comine(src, dst, t, motifs, delta: int, roots=None, n_nodes=None, per_root: bool = False,
           max_work: int = 0):
    """Algorithm 3 over the MG-Tree of ``motifs`` (Algorithm 2), one window delta."""
    src, dst, t, V = _graph(src, dst, t, n_nodes)
    tree = mgtree.construct_mg_tree(motifs)
    f = mgtree.flatten(tree, len(motifs), MAX_EDGES)
    r = None if roots is None else np.ascontiguousarray(roots, np.int32)
    nr = len(src) if r is None else len(r)
    counts = np.zeros(len(motifs), np.int64)
    pr = np.zeros((nr, len(motifs)), np.int64) if per_root else None
    rc = _load().oracle_comine(_p(src), _p(dst), _p(t), len(src), V, f["n_nodes"],
                               _p(f["node_len"]), _p(f["node_u"]), _p(f["node_v"]),
                               _p(f["child_off"]), _p(f["child_idx"]), _p(f["ref_off"]),
                               _p(f["ref_idx"]), len(motifs), int(delta), _p(r), nr,
                               int(max_work), _p(counts), _p(pr), None)
    if rc < 0:
        raise ValueError("oracle rejected the tree or delta")
    if rc == 1:
        return None
    return (counts, pr) if per_root else counts


def count_motif_timed(src, dst, t, motif, delta: int, roots, n_nodes=None, threads: int = 1,
                      time_limit: float = 20.0):
    """Algorithm 1 over ``roots`` on ``threads`` threads until ``time_limit`` seconds.

    Returns (per_root counts with -1 for roots not reached, roots finished).
    """
    src, dst, t, V = _graph(src, dst, t, n_nodes)
    m = mgtree.canonical(motif)
    mu = np.array([e[0] for e in m], np.int8)
    mv = np.array([e[1] for e in m], np.int8)
    r = np.ascontiguousarray(roots, np.int32)
    pr = np.zeros(len(r), np.int64)
    done = ctypes.c_int64(0)
    rc = _load().oracle_count_motif_mt(_p(src), _p(dst), _p(t), len(src), V, _p(mu), _p(mv),
                                       len(m), int(delta), _p(r), len(r), int(threads),
                                       float(time_limit), _p(pr), ctypes.byref(done))
    if rc < 0:
        raise ValueError("oracle rejected the motif or delta")
    return pr, int(done.value)
