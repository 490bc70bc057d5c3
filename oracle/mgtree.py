"""Motif-Group Tree construction for the oracle (Algorithm 2).

TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the
benchmark's CPU baseline; the product path never imports it.

The procedure follows Algorithm 2 (ConstructMGTree, CreateTree, InsertMotif,
GraphToTMap, InsertChild) step by step, with these readings of garbled or
silent points:

* canonical labels (reading 6): before grouping, each motif's vertices are
  relabelled in order of first appearance (edge order, source before
  destination), so that "the same edge at position T" means the same
  canonical (u, v);
* duplicates (reading 10): motifs with equal canonical form share one entry
  and the entry keeps every input position as a reference;
* Q_N (reading 7): a motif whose length equals T inside a group of two or
  more is the query of the node created (or reused) for that group; it stays
  in the group passed down and is skipped there as too short; singleton
  groups become leaves with C = Q = the motif;
* the ``pass`` for too-short motifs means "skip" (a motif that ended at an
  earlier T);
* the first call groups the whole set under the root (the walkthrough
  example reuses the root at T = 1);
* sibling order (reading 9): groups are visited in lexicographic order of
  their canonical edge at T;
* a root left with an empty C and a single child is replaced by that child.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

Edge = Tuple[int, int]
Motif = Tuple[Edge, ...]


def canonical(motif: Sequence[Edge]) -> Motif:
    """Relabel vertices in order of first appearance (edge order, src first)."""
    lab: Dict[int, int] = {}
    out = []
    for u, v in motif:
        for x in (u, v):
            if x not in lab:
                lab[x] = len(lab)
        out.append((lab[u], lab[v]))
    return tuple(out)


@dataclass
class Node:
    gid: str
    C: Motif = ()
    children: List[str] = field(default_factory=list)
    Q: Optional[Motif] = None


@dataclass
class MGTree:
    nodes: Dict[str, Node]
    root: str
    parent: Dict[str, Optional[str]]
    refs: Dict[Motif, List[int]]         # canonical motif -> input positions
    unique: List[Motif]

    def preorder(self) -> List[str]:
        out, stack = [], [self.root]
        while stack:
            g = stack.pop()
            out.append(g)
            stack.extend(reversed(self.nodes[g].children))
        return out

    def similarity(self) -> float:
        """Similarity Metric SM (Section 6): 1 - sum_N (|E_N| - |E_parent(N)|) / sum_M |E_M|."""
        num = 0
        for g in self.preorder():
            p = self.parent[g]
            num += len(self.nodes[g].C) - (len(self.nodes[p].C) if p is not None else 0)
        den = sum(len(m) for m in self.unique)
        return 1.0 - num / den

    def shape(self):
        """Nested (C, Q is not None, [children...]) for comparisons."""
        def rec(g):
            n = self.nodes[g]
            return (n.C, n.Q is not None, [rec(c) for c in n.children])
        return rec(self.root)


def construct_mg_tree(motifs: Sequence[Sequence[Edge]]) -> MGTree:
    """ConstructMGTree: TMaps and leaf nodes first, then CreateTree from T = 1."""
    canon = [canonical(m) for m in motifs]
    refs: Dict[Motif, List[int]] = {}
    for i, m in enumerate(canon):
        if len(m) == 0:
            raise ValueError("empty motif")
        refs.setdefault(m, []).append(i)
    unique = list(refs.keys())

    tmap: Dict[Motif, Dict[int, Edge]] = {}
    nodes: Dict[str, Node] = {}
    counter = [0]

    def new_gid() -> str:
        g = str(counter[0])
        counter[0] += 1
        return g

    def graph_to_tmap(m: Motif) -> Dict[int, Edge]:
        return {t + 1: e for t, e in enumerate(m)}    # temporal order -> static edge

    def leaf_gid(m: Motif) -> str:
        return "M" + str(unique.index(m))

    def insert_motif(m: Motif) -> None:
        nodes[leaf_gid(m)] = Node(leaf_gid(m), C=m, children=[], Q=m)

    def insert_child(p_gid: str, child_id: str) -> None:
        if p_gid != child_id:
            nodes[p_gid].children.append(child_id)

    def create_tree(T: int, p_gid: str, motif_group: List[Motif]) -> None:
        edge_group: Dict[Edge, List[Motif]] = {}
        for m in motif_group:
            if len(tmap[m]) < T:
                continue
            edge_group.setdefault(tmap[m][T], []).append(m)
        for e in sorted(edge_group):
            child_group = edge_group[e]
            q = None
            for m in child_group:
                if len(m) == T:
                    q = m
                    break
            if len(child_group) == 1:
                insert_child(p_gid, leaf_gid(child_group[0]))
                continue
            c_gid = p_gid if len(child_group) == len(motif_group) else new_gid()
            rep = child_group[0]
            nodes.setdefault(c_gid, Node(c_gid))
            nodes[c_gid].C = tuple(tmap[rep][i] for i in range(1, T + 1))
            nodes[c_gid].Q = q
            insert_child(p_gid, c_gid)
            # q stays in the group: at T + 1 it is skipped as too short, so
            # the group then counts as split and a node carrying a query is
            # never extended by reuse
            create_tree(T + 1, c_gid, child_group)

    for m in unique:
        tmap[m] = graph_to_tmap(m)
        insert_motif(m)
    root_gid = new_gid()
    nodes[root_gid] = Node(root_gid, C=(), children=[], Q=None)
    create_tree(1, root_gid, list(unique))

    root = root_gid
    while not nodes[root].C and nodes[root].Q is None and len(nodes[root].children) == 1:
        root = nodes[root].children[0]

    parent: Dict[str, Optional[str]] = {root: None}
    stack = [root]
    while stack:
        g = stack.pop()
        for c in nodes[g].children:
            parent[c] = g
            stack.append(c)
    reach = {g: nodes[g] for g in parent}
    return MGTree(reach, root, parent, refs, unique)


def flatten(tree: MGTree, n_queries: int, max_edges: int = 16):
    """Node table for the C oracle: root first, then preorder."""
    import numpy as np
    order = tree.preorder()
    idx = {g: i for i, g in enumerate(order)}
    n = len(order)
    node_len = np.zeros(n, np.int32)
    node_u = np.zeros(n * max_edges, np.int8)
    node_v = np.zeros(n * max_edges, np.int8)
    child_off = np.zeros(n + 1, np.int32)
    child_idx = []
    ref_off = np.zeros(n + 1, np.int32)
    ref_idx = []
    for i, g in enumerate(order):
        nd = tree.nodes[g]
        node_len[i] = len(nd.C)
        for k, (u, v) in enumerate(nd.C):
            node_u[i * max_edges + k] = u
            node_v[i * max_edges + k] = v
        child_idx += [idx[c] for c in nd.children]
        child_off[i + 1] = len(child_idx)
        if nd.Q is not None:
            ref_idx += tree.refs[nd.Q]
        ref_off[i + 1] = len(ref_idx)
    return dict(n_nodes=n, node_len=node_len, node_u=node_u, node_v=node_v,
                child_off=child_off, child_idx=np.asarray(child_idx, np.int32),
                ref_off=ref_off, ref_idx=np.asarray(ref_idx, np.int32), n_queries=n_queries)
