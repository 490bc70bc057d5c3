"""Independent counting procedures used to pin the oracle.

None of these is the oracle's recursion: brute force walks every k-tuple of
edge ids, and the closed forms count 2-edge motifs with sorted index arrays.
"""
from __future__ import annotations

import itertools
import math

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


# ---------------------------------------------------------------------------
# Per-root closed forms at full scale.
#
# For a root edge e_1 = (a -> b) with window (e_1, w], where w is the last
# edge id with t <= t(e_1) + delta (Section 2: the window is measured from
# the first edge and is inclusive; ties are ordered by edge id), the motifs
# below have counts that need at most one enumerated level and range counts
# over time-sorted lists.  Each is a restatement of the definition for one
# motif shape; none walks a search tree.

INT64_MAX = np.iinfo(np.int64).max


def window_end_sat(t, delta):
    """Last edge id with t <= t[e] + delta, the sum saturated at INT64_MAX."""
    t = np.asarray(t, np.int64)
    lim = np.where(t > INT64_MAX - np.int64(delta), INT64_MAX, t + np.int64(min(delta, INT64_MAX)))
    return np.searchsorted(t, lim, side="right").astype(np.int64) - 1


class ListIndex:
    """The out-, in- and (src, dst)-pair lists of an edge list as sorted
    int64 words key << 32 | eid, answering #{e in list(key) : lo < e <= hi}
    for arrays of queries with two binary searches each."""

    def __init__(self, src, dst):
        src = np.asarray(src, np.int64)
        dst = np.asarray(dst, np.int64)
        self.src, self.dst = src, dst
        eid = np.arange(len(src), dtype=np.int64)
        self.V = int(max(src.max(initial=0), dst.max(initial=0))) + 1
        self.out = np.sort((src << 32) | eid)
        self.inn = np.sort((dst << 32) | eid)
        self.pkeys, pid = np.unique(src * self.V + dst, return_inverse=True)
        self.pair = np.sort((pid.astype(np.int64) << 32) | eid)

    @staticmethod
    def _range(comb, key, lo, hi):
        base = np.asarray(key, np.int64) << 32
        a = np.searchsorted(comb, base + np.asarray(lo, np.int64), side="right")
        b = np.searchsorted(comb, base + np.asarray(hi, np.int64), side="right")
        return np.maximum(b - a, 0).astype(np.int64)

    def n_out(self, x, lo, hi):
        return self._range(self.out, x, lo, hi)

    def n_in(self, x, lo, hi):
        return self._range(self.inn, x, lo, hi)

    def _pid(self, x, y):
        k = np.asarray(x, np.int64) * self.V + np.asarray(y, np.int64)
        pos = np.minimum(np.searchsorted(self.pkeys, k), len(self.pkeys) - 1)
        found = (len(self.pkeys) > 0) & (self.pkeys[pos] == k) if len(self.pkeys) else np.zeros(k.shape, bool)
        return np.where(found, pos, 0), found

    def n_pair(self, x, y, lo, hi):
        pid, found = self._pid(x, y)
        return np.where(found, self._range(self.pair, pid, lo, hi), 0)

    def entries(self, which, key, lo, hi, key2=None):
        """Every entry of list(key_i) with lo_i < eid <= hi_i, for all i:
        (owner index i, eid) arrays in owner order, eids ascending per owner.
        which: "out", "in" or "pair" (key2 = the pair's destination)."""
        if which == "pair":
            k, found = self._pid(key, key2)
            comb = self.pair
        else:
            k = np.asarray(key, np.int64)
            found = np.ones(k.shape, bool)
            comb = self.out if which == "out" else self.inn
        base = k << 32
        a = np.searchsorted(comb, base + np.asarray(lo, np.int64), side="right")
        b = np.searchsorted(comb, base + np.asarray(hi, np.int64), side="right")
        n = np.where(found, np.maximum(b - a, 0), 0)
        owner = np.repeat(np.arange(len(n)), n)
        start = np.repeat(a - np.concatenate([[0], np.cumsum(n)[:-1]]), n)
        pos = start + np.arange(int(n.sum()))
        return owner, comb[pos] & 0xFFFFFFFF


def _esym(mult, k):
    """Elementary symmetric polynomial e_k of the multiplicities (exact
    integers, Newton's identities over power sums)."""
    p = [0] + [int(np.sum(np.asarray(mult, np.int64) ** i)) for i in range(1, k + 1)]
    e = [1]
    for j in range(1, k + 1):
        s = sum((-1) ** (i - 1) * e[j - i] * p[i] for i in range(1, j + 1))
        assert s % j == 0
        e.append(s // j)
    return e[k]


def _canon(m):
    lab = {}
    out = []
    for u, v in m:
        for x in (u, v):
            if x not in lab:
                lab[x] = len(lab)
        out.append((lab[u], lab[v]))
    return tuple(out)


def _star(idx, roots, a, b, w, k, out):
    """k-edge out-star (0->1, 0->2, ..., 0->k) or in-star (0->1, 2->1, ...,
    k->1): the later k-1 edges come from the root's centre list inside the
    window, with far ends pairwise distinct and outside {a, b}; per root that
    is e_{k-1} of the far ends' multiplicities."""
    centre = a if out else b
    owner, eids = idx.entries("out" if out else "in", centre, roots, w)
    far = (idx.dst if out else idx.src)[eids]
    res = np.zeros(len(roots), np.int64)
    bounds = np.searchsorted(owner, np.arange(len(roots) + 1))
    for i in range(len(roots)):
        if a[i] == b[i]:
            continue
        f = far[bounds[i]:bounds[i + 1]]
        f = f[(f != a[i]) & (f != b[i])]
        if len(f):
            _, mult = np.unique(f, return_counts=True)
            res[i] = _esym(mult, k - 1)
    return res


def closed_form_per_root(src, dst, t, motif, delta, roots, idx=None):
    """Per-root count of `motif` (any labelling; canonicalised here) for the
    given root edge ids, or KeyError when the shape has no closed form here.
    Supported: the four connected 2-edge motifs, k parallel edges, out- and
    in-stars of 3 and 4 edges, the 3-cycle, the 3-path, the feed-forward
    triangle (0->1, 0->2, 1->2), the ping-pongs (0->1, 1->0, 0->1[, 1->0]),
    (0->1, 1->0, 0->2) and (0->1, 2->1, 1->3)."""
    if idx is None:
        idx = ListIndex(src, dst)
    roots = np.asarray(roots, np.int64)
    W = window_end_sat(t, delta)
    a = idx.src[roots]
    b = idx.dst[roots]
    w = W[roots]
    r = roots
    m = _canon(motif)
    ok = a != b
    P = idx.n_pair
    if all(e == (0, 1) for e in m):                          # k parallel edges: C(n, k-1)
        n = P(a, b, r, w)
        res = np.array([math.comb(int(x), len(m) - 1) for x in n], np.int64)
    elif m == ((0, 1), (1, 2)):
        res = idx.n_out(b, r, w) - P(b, a, r, w) - P(b, b, r, w)
    elif m == ((0, 1), (1, 0)):
        res = P(b, a, r, w)
    elif m == ((0, 1), (0, 2)):
        res = idx.n_out(a, r, w) - P(a, b, r, w) - P(a, a, r, w)
    elif m == ((0, 1), (2, 1)):
        res = idx.n_in(b, r, w) - P(a, b, r, w) - P(b, b, r, w)
    elif m in (((0, 1), (0, 2), (0, 3)), ((0, 1), (0, 2), (0, 3), (0, 4))):
        return _star(idx, roots, a, b, w, len(m), True)
    elif m in (((0, 1), (2, 1), (3, 1)), ((0, 1), (2, 1), (3, 1), (4, 1))):
        return _star(idx, roots, a, b, w, len(m), False)
    else:
        res = np.zeros(len(roots), np.int64)
        if m in (((0, 1), (1, 2), (2, 0)), ((0, 1), (1, 2), (2, 3))):
            o, e2 = idx.entries("out", b, r, w)               # e2 = (b -> c), c outside {a, b}
            c = idx.dst[e2]
            keep = (c != a[o]) & (c != b[o])
            o, e2, c = o[keep], e2[keep], c[keep]
            if m[2] == (2, 0):                                # e3 = (c -> a)
                v = P(c, a[o], e2, w[o])
            else:                                             # e3 = (c -> d), d outside {a, b, c}
                v = idx.n_out(c, e2, w[o]) - P(c, a[o], e2, w[o]) - P(c, b[o], e2, w[o]) - P(c, c, e2, w[o])
        elif m == ((0, 1), (0, 2), (1, 2)):
            o, e2 = idx.entries("out", a, r, w)               # e2 = (a -> c), then e3 = (b -> c)
            c = idx.dst[e2]
            keep = (c != a[o]) & (c != b[o])
            o, e2, c = o[keep], e2[keep], c[keep]
            v = P(b[o], c, e2, w[o])
        elif m == ((0, 1), (2, 1), (1, 3)):
            o, e2 = idx.entries("in", b, r, w)                # e2 = (c -> b), then e3 = (b -> d)
            c = idx.src[e2]
            keep = (c != a[o]) & (c != b[o])
            o, e2, c = o[keep], e2[keep], c[keep]
            bo = b[o]
            v = idx.n_out(bo, e2, w[o]) - P(bo, a[o], e2, w[o]) - P(bo, bo, e2, w[o]) - P(bo, c, e2, w[o])
        elif m == ((0, 1), (1, 0), (0, 1)):
            o, e2 = idx.entries("pair", b, r, w, key2=a)      # e2 = (b -> a), then e3 = (a -> b)
            v = P(a[o], b[o], e2, w[o])
        elif m == ((0, 1), (1, 0), (0, 2)):
            o, e2 = idx.entries("pair", b, r, w, key2=a)      # e2 = (b -> a), then e3 = (a -> d)
            ao = a[o]
            v = idx.n_out(ao, e2, w[o]) - P(ao, b[o], e2, w[o]) - P(ao, ao, e2, w[o])
        elif m == ((0, 1), (1, 0), (0, 1), (1, 0)):
            # e3 = (a -> b) in the window: (b -> a) edges before it times after it
            o, e3 = idx.entries("pair", a, r, w, key2=b)
            v = P(b[o], a[o], r[o], e3) * P(b[o], a[o], e3, w[o])
        else:
            raise KeyError(m)
        np.add.at(res, o, v)
    return np.where(ok, res, 0).astype(np.int64)
