"""Pins of the oracle's co-mining decision (Section 6, heuristic for co-mining).

The bipartite test is pinned by brute force over every 2-colouring of small
graphs, by networkx's own bipartite test on larger random graphs, and by
textbook cases; the decision rule by SM values the paper and the walkthrough
fix."""
import itertools

import networkx as nx
import numpy as np
import pytest

from oracle import heuristic
from oracle.mgtree import construct_mg_tree
from paper_2507_14813_b300 import synth


def _brute_bipartite(src, dst, n):
    for colours in itertools.product((0, 1), repeat=n):
        if all(colours[a] != colours[b] for a, b in zip(src, dst)):
            return True
    return False


@pytest.mark.parametrize("seed", range(200))
def test_bipartite_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 9))
    e = int(rng.integers(0, 13))
    src = rng.integers(0, n, e).tolist()
    dst = rng.integers(0, n, e).tolist()
    if seed % 3 == 0:          # mostly loop-free, so both answers occur often
        dst = [(d if d != s else (d + 1) % n) for s, d in zip(src, dst)] if n > 1 else dst
    assert heuristic.is_bipartite(src, dst, n) == _brute_bipartite(src, dst, n)


@pytest.mark.parametrize("seed", range(20))
def test_bipartite_matches_networkx(seed):
    rng = np.random.default_rng(100 + seed)
    n = 300
    if seed % 2:
        # two sides, random directions: bipartite by construction, maybe plus one edge inside a side
        a = rng.integers(0, n // 2, 400)
        b = rng.integers(n // 2, n, 400)
        flip = rng.random(400) < 0.5
        src, dst = np.where(flip, b, a), np.where(flip, a, b)
        if seed % 4 == 1:
            src = np.append(src, 0)
            dst = np.append(dst, 1)
    else:
        src = rng.integers(0, n, 150)
        dst = (src + rng.integers(1, n, 150)) % n
    G = nx.Graph()
    G.add_nodes_from(range(n))
    G.add_edges_from(zip(src.tolist(), dst.tolist()))
    assert heuristic.is_bipartite(src, dst, n) == nx.is_bipartite(G)


def test_bipartite_textbook_cases():
    cyc = lambda k: (list(range(k)), [(i + 1) % k for i in range(k)])
    assert heuristic.is_bipartite(*cyc(4), 4)
    assert heuristic.is_bipartite(*cyc(10), 10)
    assert not heuristic.is_bipartite(*cyc(3), 3)
    assert not heuristic.is_bipartite(*cyc(9), 9)
    assert heuristic.is_bipartite([], [], 5)                      # no edges
    assert not heuristic.is_bipartite([2], [2], 5)                # a self-loop
    # complete bipartite K(3,4), edges in both directions
    s = [a for a in range(3) for b in range(3, 7)] + [b for a in range(3) for b in range(3, 7)]
    d = [b for a in range(3) for b in range(3, 7)] + [a for a in range(3) for b in range(3, 7)]
    assert heuristic.is_bipartite(s, d, 7)
    # a tree, then the same tree plus a triangle in another component
    assert heuristic.is_bipartite([0, 0, 1, 1], [1, 2, 3, 4], 8)
    assert not heuristic.is_bipartite([0, 0, 1, 1, 5, 6, 7], [1, 2, 3, 4, 6, 7, 5], 8)
    # multi-edges and antiparallel pairs do not matter
    assert heuristic.is_bipartite([0, 0, 1], [1, 1, 0], 2)
    # the tiny workload's Zipf graph has triangles
    src, dst, _ = synth.tiny_graph(2, 2000, 50_000, 1_000_000, zipf_s=1.8)
    assert not heuristic.is_bipartite(src, dst, 2000)


WALKTHROUGH = [((0, 1), (1, 2), (2, 0)), ((0, 1), (1, 2), (2, 3)), ((0, 1), (1, 0))]


def test_advice_follows_sm_threshold():
    tri = ([0, 1, 2], [1, 2, 0], 3)          # not bipartite
    sq = ([0, 1, 2, 3], [1, 2, 3, 0], 4)     # bipartite
    # config-1 group: SM = 0.5 >= 0.44, co-mine
    assert construct_mg_tree(synth.CONFIG1_MOTIFS).similarity() == pytest.approx(0.5)
    assert heuristic.comine_advice(*tri, synth.CONFIG1_MOTIFS)
    # config-2 group: SM = 0.575
    assert heuristic.comine_advice(*tri, synth.CONFIG2_MOTIFS)
    # a 2-path and a 2-out-star share only their first edge: SM = 1 - 3/4 = 0.25 < 0.44
    low = [((0, 1), (1, 2)), ((0, 1), (0, 2))]
    assert construct_mg_tree(low).similarity() == pytest.approx(0.25)
    assert not heuristic.comine_advice(*tri, low)
    # ... but a bipartite graph co-mines whatever the SM
    assert heuristic.comine_advice(*sq, low)
    # one motif alone: SM = 0, a chain either way; advice per-motif off a bipartite graph
    assert not heuristic.comine_advice(*tri, [((0, 1), (1, 2))])
