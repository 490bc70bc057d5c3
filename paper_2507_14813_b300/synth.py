"""Seeded synthetic inputs: temporal graphs, motif sets and root samples.

This module is the only code shared by the CUDA path and the CPU oracle. It
holds no step of the mining method: it draws edge lists, timestamps, motif
lists and root samples, nothing more.

Every random number comes from a counter-based splitmix64 stream: the value
at position ``i`` of stream ``s`` under seed ``k`` is ``mix64(base(k, s) +
(i + 1) * GOLDEN)``, so any element can be regenerated in isolation and the
output does not depend on chunking or thread count.

Stand-ins for the paper's datasets (the paper evaluates on five real temporal
graphs, Section 6 Table "Temporal graph datasets"; none is available here):

* endpoints: bounded rank-frequency Zipf(s), P(rank k) ~ k^-s for k in 1..V,
  node id k-1, src and dst independent, dst redrawn while dst == src;
* timestamps: uniform integers, or a two-state Markov-modulated Poisson
  process (calm rate 1/s, burst rate 100/s, exponential dwell times) from
  which exactly E seconds are drawn i.i.d. with probability proportional to
  the rate of their second;
* edges sorted by (t, generation index), which fixes the edge id (eid).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_U53 = 1.0 / float(1 << 53)


def _mix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 output function (Steele, Lea, Flood 2014), vectorised."""
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _base(seed: int, stream: int) -> np.uint64:
    k = np.array([(seed & 0xFFFFFFFF) << 32 | (stream & 0xFFFFFFFF)], dtype=np.uint64)
    return _mix64(k * GOLDEN)[0]


def rand_u64(seed: int, stream: int, start: int, n: int) -> np.ndarray:
    """n consecutive 64-bit draws of stream ``stream`` beginning at ``start``."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + 1 + n, dtype=np.uint64)
        return _mix64(_base(seed, stream) + idx * GOLDEN)


def rand_uniform(seed: int, stream: int, start: int, n: int) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (rand_u64(seed, stream, start, n) >> np.uint64(11)).astype(np.float64) * _U53


# ----------------------------------------------------------------------------
# endpoints
# ----------------------------------------------------------------------------

def zipf_cdf(n_nodes: int, s: float) -> np.ndarray:
    w = np.arange(1, n_nodes + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    c /= c[-1]
    c[-1] = 1.0
    return c


def zipf_draw(cdf: np.ndarray, u: np.ndarray) -> np.ndarray:
    idx = np.searchsorted(cdf, u, side="right")
    np.minimum(idx, cdf.size - 1, out=idx)
    return idx.astype(np.int32)


_CHUNK = 1 << 22


def zipf_endpoints(seed: int, n_nodes: int, n_edges: int, s: float) -> Tuple[np.ndarray, np.ndarray]:
    """Independent Zipf(s) src and dst, dst redrawn (fresh stream per attempt) while dst == src."""
    cdf = zipf_cdf(n_nodes, s)
    src = np.empty(n_edges, np.int32)
    dst = np.empty(n_edges, np.int32)
    for lo in range(0, n_edges, _CHUNK):
        n = min(_CHUNK, n_edges - lo)
        src[lo:lo + n] = zipf_draw(cdf, rand_uniform(seed, 1, lo, n))
        dst[lo:lo + n] = zipf_draw(cdf, rand_uniform(seed, 2, lo, n))
    if n_nodes < 2:
        raise ValueError("need at least two nodes for loop-free endpoints")
    attempt = 0
    bad = np.nonzero(src == dst)[0]
    while bad.size:
        attempt += 1
        # redraw only the colliding positions; the value for position i on
        # attempt j is element i of stream 2 + j, independent of the others
        u = _uniform_at(seed, 2 + attempt, bad)
        dst[bad] = zipf_draw(cdf, u)
        bad = bad[src[bad] == dst[bad]]
    return src, dst


def _uniform_at(seed: int, stream: int, positions: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        idx = positions.astype(np.uint64) + np.uint64(1)
        z = _mix64(_base(seed, stream) + idx * GOLDEN)
    return (z >> np.uint64(11)).astype(np.float64) * _U53


# ----------------------------------------------------------------------------
# timestamps
# ----------------------------------------------------------------------------

def uniform_times(seed: int, n_edges: int, t_max: int) -> np.ndarray:
    out = np.empty(n_edges, np.int64)
    for lo in range(0, n_edges, _CHUNK):
        n = min(_CHUNK, n_edges - lo)
        out[lo:lo + n] = (rand_uniform(seed, 3, lo, n) * t_max).astype(np.int64)
    return out


def bursty_rate(seed: int, span_s: int, rate_calm: float, rate_burst: float,
                mean_burst_s: float, mean_calm_s: float) -> np.ndarray:
    """Per-second rate of a two-state Markov-modulated Poisson process.

    The first state is drawn from the stationary distribution; dwell times are
    exponential, rounded up to whole seconds.
    """
    p_burst = mean_burst_s / (mean_burst_s + mean_calm_s)
    rate = np.empty(span_s, np.float64)
    k = 0
    u0 = rand_uniform(seed, 4, 0, 1)[0]
    burst = bool(u0 < p_burst)
    pos = 0
    while pos < span_s:
        blk = rand_uniform(seed, 5, k, 4096)
        for u in blk:
            mean = mean_burst_s if burst else mean_calm_s
            d = max(1, int(math.ceil(-mean * math.log1p(-u))))
            rate[pos:pos + d] = rate_burst if burst else rate_calm
            pos += d
            burst = not burst
            if pos >= span_s:
                break
        k += 4096
    return rate


def bursty_times(seed: int, n_edges: int, span_s: int = 30 * 86400, rate_calm: float = 1.0,
                 rate_burst: float = 100.0, mean_burst_s: float = 600.0) -> np.ndarray:
    """Exactly n_edges integer seconds drawn i.i.d. proportional to the rate.

    The burst time fraction p solves calm*(1-p) + burst*p = n_edges/span_s,
    which fixes the mean calm dwell as mean_burst_s*(1-p)/p.  Conditional on
    the number of events, an inhomogeneous Poisson process places them i.i.d.
    with density proportional to its rate.
    """
    mean_rate = n_edges / span_s
    p = (mean_rate - rate_calm) / (rate_burst - rate_calm)
    p = min(max(p, 1e-6), 1 - 1e-6)
    mean_calm_s = mean_burst_s * (1 - p) / p
    rate = bursty_rate(seed, span_s, rate_calm, rate_burst, mean_burst_s, mean_calm_s)
    cum = np.cumsum(rate)
    cum /= cum[-1]
    cum[-1] = 1.0
    out = np.empty(n_edges, np.int64)
    for lo in range(0, n_edges, _CHUNK):
        n = min(_CHUNK, n_edges - lo)
        s = np.searchsorted(cum, rand_uniform(seed, 3, lo, n), side="right")
        np.minimum(s, span_s - 1, out=s)
        out[lo:lo + n] = s
    return out


def sort_edges(src: np.ndarray, dst: np.ndarray, t: np.ndarray):
    """Order by (t, generation index): a stable sort on t."""
    order = np.argsort(t, kind="stable")
    return src[order].copy(), dst[order].copy(), t[order].copy()


# ----------------------------------------------------------------------------
# motif sets
# ----------------------------------------------------------------------------

Motif = Tuple[Tuple[int, int], ...]

CONFIG1_MOTIFS: List[Motif] = [
    ((0, 1), (1, 2)),
    ((0, 1), (1, 2), (2, 0)),
    ((0, 1), (1, 2), (2, 3)),
    ((0, 1), (1, 0)),
]

_C2_FAMILIES = [
    (((0, 1), (1, 2)), [((2, 0),), ((2, 3),), ((2, 3), (3, 0))]),
    (((0, 1), (0, 2)), [((0, 3),), ((1, 2),), ((0, 3), (0, 4))]),
    (((0, 1), (1, 0)), [((0, 1),), ((0, 2),), ((0, 1), (1, 0))]),
    (((0, 1), (2, 1)), [((3, 1),), ((1, 3),), ((3, 1), (4, 1))]),
]
CONFIG2_MOTIFS: List[Motif] = [pre + suf for pre, sufs in _C2_FAMILIES for suf in sufs]


def random_motif_tree(seed: int, max_edges: int = 6, max_motifs: int = 32,
                      p_internal_query: float = 0.25, min_edges: int = 2) -> List[Motif]:
    """A random prefix-sharing motif set, grown from the canonical edge 0->1.

    Each tree node draws a branching factor uniform in 1..4 and a fresh
    per-set depth limit D uniform in min_edges..max_edges; each child appends
    one edge with at least one endpoint already used (a new vertex takes the
    next label), with no two children of a node alike.  Leaves with at least
    min_edges edges are queries; internal nodes with at least min_edges edges
    are queries with probability p_internal_query.  Growth is breadth-first
    and stops at max_motifs queries.
    """
    ctr = [0]

    def u() -> float:
        v = rand_uniform(seed, 7, ctr[0], 1)[0]
        ctr[0] += 1
        return float(v)

    depth_limit = min_edges + int(u() * (max_edges - min_edges + 1))
    frontier: List[Motif] = [((0, 1),)]
    queries: List[Motif] = []
    while frontier and len(queries) < max_motifs:
        nxt: List[Motif] = []
        for m in frontier:
            nv = 1 + max(max(e) for e in m)
            if len(m) >= depth_limit:
                if len(m) >= min_edges and len(queries) < max_motifs:
                    queries.append(m)
                continue
            options = [(a, b) for a in range(nv + 1) for b in range(nv + 1)
                       if a != b and (a < nv or b < nv)]
            branch = 1 + int(u() * 4)
            kids = []
            for _ in range(branch):
                e = options[int(u() * len(options))]
                if e not in kids:
                    kids.append(e)
            if len(m) >= min_edges and u() < p_internal_query and len(queries) < max_motifs:
                queries.append(m)
            for e in kids:
                nxt.append(m + (e,))
        frontier = nxt
    return queries


def query_motifs(seed: int, lo_motifs: int = 1, hi_motifs: int = 16, lo_edges: int = 2,
                 hi_edges: int = 5) -> List[Motif]:
    """A serving query: 1..16 motifs of 2..5 edges from the random tree generator."""
    n = lo_motifs + int(rand_uniform(seed, 8, 0, 1)[0] * (hi_motifs - lo_motifs + 1))
    ms = random_motif_tree(seed, max_edges=hi_edges, max_motifs=n, min_edges=lo_edges)
    return ms[:n] if ms else [((0, 1), (1, 0))]


def motif_arrays(motifs: Sequence[Motif]):
    """Flatten motifs to (uv int8[2*sum m], off int32[n+1])."""
    off = np.zeros(len(motifs) + 1, np.int32)
    uv = []
    for i, m in enumerate(motifs):
        off[i + 1] = off[i] + len(m)
        for a, b in m:
            uv += [a, b]
    return np.asarray(uv, np.int8), off


# ----------------------------------------------------------------------------
# roots
# ----------------------------------------------------------------------------

def root_sample(seed: int, n_edges: int, n_roots: int) -> np.ndarray:
    """A seeded uniform sample of distinct root eids, ascending."""
    if n_roots >= n_edges:
        return np.arange(n_edges, dtype=np.int32)
    keys = rand_u64(seed, 9, 0, n_edges)
    pick = np.argpartition(keys, n_roots)[:n_roots]
    return np.sort(pick).astype(np.int32)


def root_sample_sparse(seed: int, n_edges: int, n_roots: int) -> np.ndarray:
    """A seeded uniform sample of distinct root eids for n_roots << n_edges,
    ascending: indices floor(u * n_edges) in draw order, duplicates skipped."""
    if n_roots * 64 > n_edges:
        return root_sample(seed, n_edges, n_roots)
    out, seen, pos = [], set(), 0
    while len(out) < n_roots:
        u = rand_uniform(seed, 15, pos, 2 * n_roots)
        pos += 2 * n_roots
        for x in (u * n_edges).astype(np.int64):
            if int(x) not in seen:
                seen.add(int(x))
                out.append(int(x))
                if len(out) == n_roots:
                    break
    return np.sort(np.array(out, np.int32))


# ----------------------------------------------------------------------------
# workload configurations
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class GraphSpec:
    name: str
    n_nodes: int
    n_edges: int
    zipf_s: float
    times: str            # "uniform" or "bursty"
    t_max: int = 0        # uniform: t in [0, t_max)
    span_s: int = 30 * 86400
    seed: int = 1


TINY = GraphSpec("tiny-2k-50k", 2000, 50_000, 1.8, "uniform", t_max=1_000_000, seed=2)
MID = GraphSpec("mid-1m-20m", 1_000_000, 20_000_000, 1.6, "bursty", seed=3)
BATCHED = GraphSpec("batched-5m-50m", 5_000_000, 50_000_000, 1.7, "bursty", seed=4)
SERVING = GraphSpec("serving-20m-200m", 20_000_000, 200_000_000, 1.7, "bursty", seed=6)

# The batched and serving sizes with milder endpoint skew.  Under
# rank-frequency Zipf(1.7) one vertex carries 49 % of all endpoints and the
# random motif sets' multi-edge and star motifs on hub pairs have more
# matches per root than can be enumerated at any of their windows; with
# Zipf(0.5) the top vertex carries 0.02 %.
BATCHED_MILD = GraphSpec("batched-5m-50m-zipf0.5", 5_000_000, 50_000_000, 0.5, "bursty", seed=4)
SERVING_MILD = GraphSpec("serving-20m-200m-zipf0.5", 20_000_000, 200_000_000, 0.5, "bursty", seed=6)

TINY_DELTA = 10_000
MID_DELTA = 3600


def make_graph(spec: GraphSpec, n_edges: int | None = None):
    """(src int32, dst int32, t int64), sorted by (t, generation index)."""
    e = spec.n_edges if n_edges is None else n_edges
    src, dst = zipf_endpoints(spec.seed, spec.n_nodes, e, spec.zipf_s)
    if spec.times == "uniform":
        t = uniform_times(spec.seed, e, spec.t_max)
    else:
        span = spec.span_s if n_edges is None else max(1, int(spec.span_s * e / spec.n_edges))
        t = bursty_times(spec.seed, e, span_s=span)
    return sort_edges(src, dst, t)


def serving_query(seed: int, n_edges: int, n_roots: int = 64):
    """A serving request: 1..16 motifs of 2..5 edges, a log-uniform integer
    window in [60, 86400] per request, and a seeded uniform root sample."""
    ms = query_motifs(seed, hi_edges=5)
    u = rand_uniform(seed, 14, 0, 1)[0]
    delta = int(math.exp(math.log(60) + u * (math.log(86400) - math.log(60))))
    return ms, delta, root_sample_sparse(seed, n_edges, n_roots)


def batched_sets(n_sets: int = 64, base_seed: int = 1000):
    """The batched workload's motif sets: (motifs, delta) per set."""
    deltas = (600, 3600, 86400)
    out = []
    for i in range(n_sets):
        s = base_seed + i
        d = deltas[int(rand_uniform(s, 10, 0, 1)[0] * 3)]
        out.append((random_motif_tree(s), d))
    return out


def tiny_graph(seed: int, n_nodes: int, n_edges: int, t_max: int, zipf_s: float = 1.2,
               self_loops: bool = False):
    """Small tie-heavy graphs for brute-force pins (optionally with self-loops)."""
    cdf = zipf_cdf(n_nodes, zipf_s)
    src = zipf_draw(cdf, rand_uniform(seed, 11, 0, n_edges))
    dst = zipf_draw(cdf, rand_uniform(seed, 12, 0, n_edges))
    if not self_loops:
        bad = np.nonzero(src == dst)[0]
        dst[bad] = (src[bad] + 1) % n_nodes
    t = (rand_uniform(seed, 13, 0, n_edges) * t_max).astype(np.int64)
    return sort_edges(src, dst, t)


def hub_graph(seed: int, n_nodes: int, n_edges: int, t_max: int, hub_out: float = 0.5, hub_in: float = 0.25,
              zipf_s: float = 0.8):
    """A graph with one hub (vertex 0): a fraction hub_out of the edges leave
    it and hub_in enter it; the other endpoints are Zipf(zipf_s) over
    vertices 1..n_nodes-1, so a hub window holds many distinct far ends with
    a few frequent ones; the remaining edges join two such vertices.
    Integer times uniform in [0, t_max) (tie-heavy when n_edges > t_max)."""
    u = rand_uniform(seed, 16, 0, n_edges)
    cdf = zipf_cdf(n_nodes - 1, zipf_s)
    a = (1 + zipf_draw(cdf, rand_uniform(seed, 17, 0, n_edges))).astype(np.int32)
    b = (1 + zipf_draw(cdf, rand_uniform(seed, 18, 0, n_edges))).astype(np.int32)
    src = a.copy()
    dst = b.copy()
    out_hub = u < hub_out
    in_hub = (u >= hub_out) & (u < hub_out + hub_in)
    src[out_hub] = 0
    dst[in_hub] = 0
    same = src == dst
    dst[same] = 1 + (dst[same] % (n_nodes - 1))
    t = (rand_uniform(seed, 19, 0, n_edges) * t_max).astype(np.int64)
    return sort_edges(src.astype(np.int32), dst.astype(np.int32), t)
