"""The co-mining decision of Section 6 ("Heuristic for Co-Mining"), for the oracle.

TEST INFRASTRUCTURE ONLY: used by tests/; the product path never imports it.

Section 6 reports that co-mining always paid off on a bipartite data graph
(no match can join two vertices of one side), and that on the GPU it needs a
similarity metric of at least 0.44 to beat mining each motif alone.  The
decision is therefore: co-mine if the graph is bipartite, otherwise co-mine
iff SM >= 0.44.  (The paper's further advice, to prefer a smaller window, is
a choice of the caller's delta, not of the miner.)

Bipartite here is the textbook definition on the undirected view of the
edge list: the vertices can be split into two sides with every edge joining
the two sides.  Breadth-first search colours each component; an edge between
two vertices of one colour (a self-loop included) means no such split exists.
"""
from __future__ import annotations

from collections import deque
from typing import Sequence

import numpy as np

from .mgtree import construct_mg_tree

COMINE_MIN_SM = 0.44


def is_bipartite(src, dst, n_nodes: int) -> bool:
    """True iff the undirected graph of the edges (src[i], dst[i]) is 2-colourable."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    adj = [[] for _ in range(n_nodes)]
    for a, b in zip(src.tolist(), dst.tolist()):
        if a == b:
            return False                      # a self-loop joins a vertex to itself
        adj[a].append(b)
        adj[b].append(a)
    colour = [-1] * n_nodes
    for s in range(n_nodes):
        if colour[s] >= 0:
            continue
        colour[s] = 0
        q = deque([s])
        while q:
            x = q.popleft()
            for y in adj[x]:
                if colour[y] < 0:
                    colour[y] = 1 - colour[x]
                    q.append(y)
                elif colour[y] == colour[x]:
                    return False
    return True


def comine_advice(src, dst, n_nodes: int, motifs: Sequence) -> bool:
    """True: co-mine the motif group; False: mine each motif alone."""
    if is_bipartite(src, dst, n_nodes):
        return True
    return construct_mg_tree(motifs).similarity() >= COMINE_MIN_SM
