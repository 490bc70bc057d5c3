"""Pins for the CPU oracle: brute force, closed forms, invariants, tree shapes.

Each pin is a computation other than the oracle's recursion, chosen so that
a dropped term, a wrong sign or index, or a swapped endpoint in the oracle
fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import mgtree
from paper_2507_14813_b300 import synth
from tests import refimpl

# motifs exercising every candidate-list case of MatchEdge: out-list (u
# mapped), in-list (only v mapped, reading 4), both mapped, and both
# unmapped (a disconnected motif)
PIN_MOTIFS = [
    ((0, 1),),
    ((0, 1), (1, 2)),
    ((0, 1), (1, 0)),
    ((0, 1), (0, 2)),
    ((0, 1), (2, 1)),
    ((0, 1), (0, 1)),
    ((0, 1), (2, 3)),
    ((0, 1), (1, 2), (2, 0)),
    ((0, 1), (1, 2), (2, 3)),
    ((0, 1), (2, 1), (1, 0)),
    ((0, 1), (2, 0), (0, 2)),
    ((0, 1), (1, 0), (0, 1)),
    ((0, 1), (2, 3), (3, 0)),
    ((0, 1), (1, 2), (2, 3), (3, 0)),
    ((0, 1), (0, 2), (0, 3), (1, 2)),
    ((0, 1), (2, 1), (3, 1), (0, 1)),
]


def _tiny(seed, n_nodes, n_edges, t_max, self_loops=False):
    return synth.tiny_graph(seed, n_nodes, n_edges, t_max, zipf_s=0.9, self_loops=self_loops)


@pytest.mark.parametrize("seed", range(12))
def test_oracle_matches_brute_force(seed):
    # tie-heavy timestamps (t_max small), few vertices, some self-loops
    sizes = {1: 60, 2: 60, 3: 36, 4: 20}
    for motif in PIN_MOTIFS:
        k = len(motif)
        E = sizes[k]
        src, dst, t = _tiny(1000 + seed, 6 + seed % 5, E, 12 + 3 * seed, self_loops=seed % 3 == 0)
        for delta in (0, 3, 11):
            want = refimpl.brute_force(src, dst, t, motif, delta)
            got = oracle.count_motif(src, dst, t, motif, delta, n_nodes=12)
            assert got == want, (motif, delta, seed)


@pytest.mark.parametrize("seed", range(6))
def test_comine_matches_brute_force(seed):
    src, dst, t = _tiny(2000 + seed, 7, 22, 15, self_loops=seed % 2 == 0)
    motifs = [m for m in PIN_MOTIFS if len(m) <= 4]
    got = oracle.comine(src, dst, t, motifs, 7, n_nodes=7)
    want = [refimpl.brute_force(src, dst, t, m, 7) for m in motifs]
    assert list(got) == want


def test_closed_forms_2edge_full_tiny_config():
    src, dst, t = synth.make_graph(synth.TINY)
    cf = refimpl.closed_form_2edge(src, dst, t, synth.TINY_DELTA)
    motifs = {"path": ((0, 1), (1, 2)), "cycle": ((0, 1), (1, 0)),
              "outstar": ((0, 1), (0, 2)), "instar": ((0, 1), (2, 1))}
    for k, m in motifs.items():
        assert oracle.count_motif(src, dst, t, m, synth.TINY_DELTA) == cf[k], k


def test_closed_forms_2edge_with_self_loops():
    src, dst, t = _tiny(77, 9, 3000, 400, self_loops=True)
    assert (src == dst).any()
    cf = refimpl.closed_form_2edge(src, dst, t, 25)
    motifs = {"path": ((0, 1), (1, 2)), "cycle": ((0, 1), (1, 0)),
              "outstar": ((0, 1), (0, 2)), "instar": ((0, 1), (2, 1))}
    for k, m in motifs.items():
        assert oracle.count_motif(src, dst, t, m, 25) == cf[k], k


def test_parallel_edges_binomial():
    # n parallel edges a->b, all inside the window: k copies of (0->1) match C(n, k)
    n = 23
    src = np.zeros(n, np.int32)
    dst = np.ones(n, np.int32)
    t = np.arange(n, dtype=np.int64)
    for k in range(1, 5):
        m = tuple([(0, 1)] * k)
        assert oracle.count_motif(src, dst, t, m, 10**6) == math.comb(n, k)
    # window cuts: only tuples with span <= delta
    delta = 5
    want = sum(math.comb(min(delta, n - 1 - i), 2) for i in range(n))  # first edge i, 2 more in (i, i+delta]
    assert oracle.count_motif(src, dst, t, ((0, 1),) * 3, delta) == want


def test_alternating_pair_closed_form():
    # a->b, b->a, a->b, ... : (0->1, 1->0) counts ordered pairs of opposite direction
    n = 31
    src = np.array([i % 2 for i in range(n)], np.int32)
    dst = 1 - src
    t = np.arange(n, dtype=np.int64) * 10
    got = oracle.count_motif(src, dst, t, ((0, 1), (1, 0)), 10**9)
    assert got == sum(1 for i, j in itertools.combinations(range(n), 2) if src[i] != src[j])
    # 3-cycles are impossible on two vertices; a 2-path needs a third vertex
    assert oracle.count_motif(src, dst, t, ((0, 1), (1, 2), (2, 0)), 10**9) == 0
    assert oracle.count_motif(src, dst, t, ((0, 1), (1, 2)), 10**9) == 0


def test_strict_order_with_ties():
    # equal timestamps: order by edge id (reading 1), window inclusive (reading 2)
    src = np.array([0, 1, 2], np.int32)
    dst = np.array([1, 2, 0], np.int32)
    t = np.array([5, 5, 5], np.int64)
    assert oracle.count_motif(src, dst, t, ((0, 1), (1, 2), (2, 0)), 0) == 1
    t2 = np.array([5, 5, 6], np.int64)
    assert oracle.count_motif(src, dst, t2, ((0, 1), (1, 2), (2, 0)), 0) == 0
    assert oracle.count_motif(src, dst, t2, ((0, 1), (1, 2), (2, 0)), 1) == 1


def test_saturated_window():
    src = np.array([0, 1], np.int32)
    dst = np.array([1, 2], np.int32)
    t = np.array([2**62, 2**62 + 5], np.int64)
    assert oracle.count_motif(src, dst, t, ((0, 1), (1, 2)), 2**63 - 1) == 1


def _reverse(src, dst, t):
    # reverse edge direction and edge-id order; times negated keep the order valid
    return dst[::-1].copy(), src[::-1].copy(), (-t[::-1]).copy()


def _reverse_motif(m):
    return mgtree.canonical([(v, u) for (u, v) in reversed(m)])


@pytest.mark.parametrize("seed", range(3))
def test_time_reversal(seed):
    src, dst, t = _tiny(3000 + seed, 30, 1500, 3000)
    rs, rd, rt = _reverse(src, dst, t)
    # reversed ties keep reversed edge-id order because the reversed list is
    # sorted by (-t, reversed id)
    for m in PIN_MOTIFS[1:]:
        a = oracle.count_motif(src, dst, t, m, 60, n_nodes=30)
        b = oracle.count_motif(rs, rd, rt, _reverse_motif(m), 60, n_nodes=30)
        assert a == b, m


def test_relabel_invariance():
    src, dst, t = _tiny(4000, 40, 3000, 5000)
    rng_perm = np.argsort(synth.rand_u64(9, 1, 0, 40)).astype(np.int32)
    for m in PIN_MOTIFS:
        a = oracle.count_motif(src, dst, t, m, 90, n_nodes=40)
        b = oracle.count_motif(rng_perm[src], rng_perm[dst], t, m, 90, n_nodes=40)
        assert a == b


def test_delta_monotone_and_additive_over_roots():
    src, dst, t = synth.make_graph(synth.TINY)
    m = ((0, 1), (1, 2), (2, 0))
    prev = -1
    for d in (0, 100, 1000, 5000, 10000, 20000):
        c = oracle.count_motif(src, dst, t, m, d)
        assert c >= prev
        prev = c
    roots = np.arange(len(src), dtype=np.int32)
    parts = [roots[i::3] for i in range(3)]
    tot = sum(oracle.count_motif(src, dst, t, m, 10000, roots=p) for p in parts)
    assert tot == oracle.count_motif(src, dst, t, m, 10000)
    total, per_root = oracle.count_motif(src, dst, t, m, 10000, per_root=True)
    assert per_root.sum() == total


def test_comine_equals_permotif_tiny_config():
    src, dst, t = synth.make_graph(synth.TINY)
    a = oracle.comine(src, dst, t, synth.CONFIG1_MOTIFS, synth.TINY_DELTA)
    b = oracle.count_motifs(src, dst, t, synth.CONFIG1_MOTIFS, synth.TINY_DELTA)
    assert list(a) == list(b)


@pytest.mark.parametrize("seed", range(4))
def test_comine_equals_permotif_random_sets(seed):
    src, dst, t = _tiny(5000 + seed, 60, 4000, 20000)
    motifs = synth.random_motif_tree(100 + seed, max_edges=4, max_motifs=12)
    a = oracle.comine(src, dst, t, motifs, 300, n_nodes=60)
    b = oracle.count_motifs(src, dst, t, motifs, 300, n_nodes=60)
    assert list(a) == list(b)


def test_intermediate_visit_count_equals_motif_count():
    # the 2-path node of the tiny-config tree is visited once per 2-path match:
    # querying it as a motif on its own gives the same number as its count
    # inside the co-mined set
    src, dst, t = synth.make_graph(synth.TINY)
    alone = oracle.comine(src, dst, t, [((0, 1), (1, 2))], synth.TINY_DELTA)
    mixed = oracle.comine(src, dst, t, synth.CONFIG1_MOTIFS, synth.TINY_DELTA)
    assert alone[0] == mixed[0]


def test_duplicates_share_counts():
    src, dst, t = _tiny(6000, 20, 800, 2000)
    ms = [((0, 1), (1, 2)), ((5, 6), (6, 7)), ((0, 1), (1, 0))]
    c = oracle.comine(src, dst, t, ms, 100, n_nodes=20)
    assert c[0] == c[1]
    assert c[0] == oracle.count_motif(src, dst, t, ms[0], 100, n_nodes=20)


# ------------------------------------------------------------------- trees

def test_tree_walkthrough_shape():
    # Section 4.2 walkthrough: [M3, M4, M5]; M3 a 3-cycle, M4/M5 extend a->b->c->d
    M3 = ((0, 1), (1, 2), (2, 0))
    M4 = ((0, 1), (1, 2), (2, 3), (3, 0))
    M5 = ((0, 1), (1, 2), (2, 3), (3, 1))
    tr = mgtree.construct_mg_tree([M3, M4, M5])
    shape = tr.shape()
    assert shape[0] == ((0, 1), (1, 2)) and shape[1] is False           # I1
    kids = shape[2]
    assert [k[0] for k in kids] == [M3, ((0, 1), (1, 2), (2, 3))]       # M3 and I2
    assert kids[1][1] is False
    assert [g[0] for g in kids[1][2]] == [M4, M5]
    assert abs(tr.similarity() - 5 / 11) < 1e-12


def test_tree_tiny_config_shape():
    tr = mgtree.construct_mg_tree(synth.CONFIG1_MOTIFS)
    assert tr.shape() == (((0, 1),), False, [
        (((0, 1), (1, 0)), True, []),
        (((0, 1), (1, 2)), True, [(((0, 1), (1, 2), (2, 0)), True, []),
                                  (((0, 1), (1, 2), (2, 3)), True, [])]),
    ])
    assert tr.similarity() == 0.5


def test_tree_mid_config_similarity():
    tr = mgtree.construct_mg_tree(synth.CONFIG2_MOTIFS)
    assert abs(tr.similarity() - (1 - 17 / 40)) < 1e-12


def _prefixes(motifs):
    return {m[:i] for m in map(mgtree.canonical, motifs) for i in range(1, len(m) + 1)}


@pytest.mark.parametrize("seed", range(20))
def test_tree_is_radix_trie(seed):
    motifs = synth.random_motif_tree(300 + seed, max_edges=6, max_motifs=20)
    # add a few duplicates and relabelled copies
    motifs = motifs + [tuple((u + 3, v + 3) for u, v in motifs[0])]
    tr = mgtree.construct_mg_tree(motifs)
    canon = [mgtree.canonical(m) for m in motifs]
    pref = _prefixes(motifs)
    # SM numerator = number of distinct non-empty canonical prefixes
    num = (1 - tr.similarity()) * sum(len(m) for m in set(canon))
    assert round(num) == len(pref)
    # node set = root (longest common prefix) + motif ends + branch points
    ends = set(canon)
    kids = {}
    for p in pref:
        kids.setdefault(p[:-1], set()).add(p)
    branch = {p for p, ch in kids.items() if len(ch) >= 2 and p}
    lcp = canon[0]
    for m in canon[1:]:
        k = 0
        while k < min(len(lcp), len(m)) and lcp[k] == m[k]:
            k += 1
        lcp = lcp[:k]
    want = ends | branch | ({lcp} if lcp else set())
    got = {tr.nodes[g].C for g in tr.preorder()}
    assert got == want
    # every query has exactly one node with Q = it
    qs = [tr.nodes[g].Q for g in tr.preorder() if tr.nodes[g].Q is not None]
    assert sorted(qs) == sorted(set(canon))
    # children are longest-prefix extensions
    for g in tr.preorder():
        for c in tr.nodes[g].children:
            C, Cc = tr.nodes[g].C, tr.nodes[c].C
            assert Cc[:len(C)] == C and len(Cc) > len(C)


def test_canonical_labels():
    assert mgtree.canonical([(5, 3), (3, 9), (9, 5)]) == ((0, 1), (1, 2), (2, 0))
    assert mgtree.canonical([(2, 1), (0, 1)]) == ((0, 1), (2, 1))


def test_sparse_root_sample_is_distinct_sorted_and_seeded():
    a = synth.root_sample_sparse(5, 10**9, 500)
    b = synth.root_sample_sparse(5, 10**9, 500)
    assert np.array_equal(a, b) and len(set(a.tolist())) == 500
    assert np.all(np.diff(a) > 0) and a.min() >= 0 and a.max() < 10**9
    assert not np.array_equal(a, synth.root_sample_sparse(6, 10**9, 500))


@pytest.mark.parametrize("seed", range(8))
def test_oracle_enumeration_matches_brute_force(seed):
    """The recorded matches of Algorithm 1 are exactly the brute-force match list,
    on tie-heavy graphs with a self-loop, for every candidate-list case."""
    rng = np.random.default_rng(900 + seed)
    V, E = 6, 26
    src = rng.integers(0, V, E).astype(np.int32)
    dst = ((src + rng.integers(1, V, E)) % V).astype(np.int32)
    src[5] = dst[5]
    t = np.sort(rng.integers(0, 50, E)).astype(np.int64)
    for motif in [((0, 1), (1, 2)), ((0, 1), (1, 0), (0, 1)), ((0, 1), (0, 2), (0, 3)),
                  ((0, 1), (2, 1), (1, 3)), ((0, 1), (2, 3)), ((0, 1), (1, 2), (2, 0))]:
        for delta in (0, 12, 50):
            got, n = oracle.enumerate_motif(src, dst, t, motif, delta)
            want = refimpl.brute_force_matches(src, dst, t, motif, delta)
            assert n == len(want) == len(got)
            assert sorted(map(tuple, got.tolist())) == sorted(want)
    # a full buffer keeps the exact total
    got, n = oracle.enumerate_motif(src, dst, t, ((0, 1), (1, 2)), 50, cap=3)
    assert n == len(refimpl.brute_force_matches(src, dst, t, ((0, 1), (1, 2)), 50)) and len(got) == min(3, n)


@pytest.mark.parametrize("threads", [1, 3])
def test_multithreaded_oracle_per_root_equals_single(threads):
    """The timed CPU baseline's Algorithm 1 over roots (dynamic loop over
    threads, time limit) gives the per-root counts of the plain recursion
    when it finishes, and marks unreached roots -1 when it runs out of time."""
    src, dst, t = synth.make_graph(synth.TINY)
    roots = synth.root_sample(41, len(src), 2000)
    for m in synth.CONFIG1_MOTIFS + [((0, 1), (0, 2), (0, 3))]:
        _, want = oracle.count_motif(src, dst, t, m, synth.TINY_DELTA, roots=roots, per_root=True)
        got, done = oracle.count_motif_timed(src, dst, t, m, synth.TINY_DELTA, roots, threads=threads,
                                             time_limit=600.0)
        assert done == len(roots)
        assert np.array_equal(got, want), m
    # a limit that has passed before the first root: nothing is reached
    got, done = oracle.count_motif_timed(src, dst, t, synth.CONFIG1_MOTIFS[2], synth.TINY_DELTA, roots,
                                         threads=threads, time_limit=1e-9)
    assert done == int((got >= 0).sum()) and done < len(roots)
