"""Independent counting procedures used to pin the oracle.

None of these is the oracle's recursion: brute force walks every k-tuple of
edge ids, and the closed forms count 2-edge motifs with sorted index arrays.
"""
from __future__ import annotations

import itertools

import numpy as np


def brute_force(src, dst, t, motif, delta):
    """Count k-tuples e_1 < ... < e_k within the window with an injective map.

    Straight from the definition (Section 2): try every tuple, build the map
    edge by edge, reject a conflict or a non-injective map.
    """
    E = len(src)
    k = len(motif)
    cnt = 0
    for tup in itertools.combinations(range(E), k):
        if t[tup[-1]] - t[tup[0]] > delta:
            continue
        f = {}
        ok = True
        for (mu, mv), e in zip(motif, tup):
            for mx, gx in ((mu, int(src[e])), (mv, int(dst[e]))):
                if mx in f:
                    if f[mx] != gx:
                        ok = False
                        break
                else:
                    f[mx] = gx
            if not ok:
                break
        if ok and len(set(f.values())) == len(f):
            cnt += 1
    return cnt


def brute_force_matches(src, dst, t, motif, delta):
    """The matches themselves: every k-tuple of edge ids e_1 < ... < e_k within
    the window that has an injective map (the same test as brute_force)."""
    E = len(src)
    k = len(motif)
    out = []
    for tup in itertools.combinations(range(E), k):
        if t[tup[-1]] - t[tup[0]] > delta:
            continue
        f = {}
        ok = True
        for (mu, mv), e in zip(motif, tup):
            for mx, gx in ((mu, int(src[e])), (mv, int(dst[e]))):
                if f.setdefault(mx, gx) != gx:
                    ok = False
            if not ok:
                break
        if ok and len(set(f.values())) == len(f):
            out.append(tup)
    return out


def window_end(t, delta):
    """For each edge e: the last edge id with t <= t[e] + delta."""
    return np.searchsorted(t, t + delta, side="right") - 1


def _count_key_in_range(keys_sorted, eids_sorted, key, lo, hi):
    """#entries with keys == key and lo < eid <= hi (entries sorted by (key, eid))."""
    a = np.searchsorted(keys_sorted, key, side="left")
    b = np.searchsorted(keys_sorted, key, side="right")
    # within [a, b) eids ascend; locate eid bounds with a combined key
    comb = keys_sorted.astype(np.int64) * (1 << 32) + eids_sorted
    base = key.astype(np.int64) * (1 << 32)
    lo_pos = np.searchsorted(comb, base + lo, side="right")
    hi_pos = np.searchsorted(comb, base + hi, side="right")
    return np.clip(hi_pos, a, b) - np.clip(lo_pos, a, b)


def closed_form_2edge(src, dst, t, delta):
    """Exact totals of the four connected 2-edge motifs from sorted arrays.

    For each root e1 = (a -> b) with window (e1, w(e1)]:
      2-path  (0->1,1->2): out(b) in window with dst != a
      2-cycle (0->1,1->0): out(b) in window with dst == a
      out-star(0->1,0->2): out(a) in window with dst != b
      in-star (0->1,2->1): in(b) in window with src != a
    """
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    E = len(src)
    eid = np.arange(E, dtype=np.int64)
    w = window_end(np.asarray(t), delta)
    # vertex-keyed lists (key, eid) sorted
    o = np.lexsort((eid, src))
    out_k, out_e = src[o], eid[o]
    i = np.lexsort((eid, dst))
    in_k, in_e = dst[i], eid[i]
    # pair-keyed list: key = src * V + dst
    V = int(max(src.max(), dst.max())) + 1
    pk = src * V + dst
    p = np.lexsort((eid, pk))
    pr_k, pr_e = pk[p], eid[p]
    a, b = src, dst
    loop = a == b
    n_out_b = _count_key_in_range(out_k, out_e, b, eid, w)
    n_out_a = _count_key_in_range(out_k, out_e, a, eid, w)
    n_in_b = _count_key_in_range(in_k, in_e, b, eid, w)
    n_ba = _count_key_in_range(pr_k, pr_e, b * V + a, eid, w)
    n_ab = _count_key_in_range(pr_k, pr_e, a * V + b, eid, w)
    n_bb = _count_key_in_range(pr_k, pr_e, b * V + b, eid, w)
    n_aa = _count_key_in_range(pr_k, pr_e, a * V + a, eid, w)
    ok = ~loop
    path = n_out_b - n_ba - n_bb          # exclude dst == a and dst == b (self-loop at b)
    cycle = n_ba
    ostar = n_out_a - n_ab - n_aa
    istar = n_in_b - n_ab - n_bb
    return {
        "path": int(path[ok].sum()),
        "cycle": int(cycle[ok].sum()),
        "outstar": int(ostar[ok].sum()),
        "instar": int(istar[ok].sum()),
    }
