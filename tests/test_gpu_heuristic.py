"""The device bipartite test and the co-mining decision against the oracle's
breadth-first colouring and decision rule (Section 6, heuristic for
co-mining), and TM_AUTO's choice of path."""
import numpy as np
import pytest

import oracle
from oracle import heuristic
from paper_2507_14813_b300 import build, synth, tmotif

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    tmotif.lib()


def _graph(src, dst, n):
    src = np.asarray(src, np.int32)
    dst = np.asarray(dst, np.int32)
    t = np.arange(len(src), dtype=np.int64)
    return tmotif.Graph(src, dst, t, n, presorted=True)


def _cases():
    rng = np.random.default_rng(7)
    out = {}
    out["tiny_zipf"] = synth.tiny_graph(2, 2000, 50_000, 1_000_000, zipf_s=1.8)[:2] + (2000,)
    n = 20_000
    a = rng.integers(0, n // 2, 60_000)
    b = rng.integers(n // 2, n, 60_000)
    flip = rng.random(60_000) < 0.5
    out["two_sides"] = (np.where(flip, b, a), np.where(flip, a, b), n)
    out["two_sides_plus_one"] = (np.append(out["two_sides"][0], 3), np.append(out["two_sides"][1], 4), n)
    # long paths and cycles need many labelling rounds; ids shuffled so chains are deep
    m = 200_000
    perm = rng.permutation(m)
    out["long_path"] = (perm[:-1], perm[1:], m)
    k = 100_001
    pk = rng.permutation(k)
    out["long_odd_cycle"] = (pk, np.roll(pk, -1), k)
    out["long_even_cycle"] = (pk[:-1], np.roll(pk[:-1], -1), k)
    out["self_loop"] = (np.array([0, 1, 5]), np.array([1, 2, 5]), 8)
    out["isolated_vertices"] = (np.array([0, 2]), np.array([1, 3]), 100_000)
    out["antiparallel"] = (np.array([0, 1, 0, 1]), np.array([1, 0, 1, 0]), 2)
    return out


CASES = _cases()


@pytest.mark.parametrize("name", sorted(CASES))
def test_bipartite_matches_oracle(name):
    src, dst, n = CASES[name]
    g = _graph(src, dst, n)
    want = heuristic.is_bipartite(src, dst, n)
    assert g.bipartite() == want
    assert g.bipartite() == want            # cached answer
    g.close()


def test_bipartite_empty_graph():
    g = _graph([], [], 10)
    assert g.bipartite() is True
    g.close()


LOW = [((0, 1), (1, 2)), ((0, 1), (0, 2))]          # SM 0.25


@pytest.mark.parametrize("which", ["tiny_zipf", "two_sides"])
@pytest.mark.parametrize("motifs", [LOW, synth.CONFIG1_MOTIFS], ids=["low_sm", "config1"])
def test_advice_and_auto_mode(which, motifs):
    src, dst, n = CASES[which]
    g = _graph(src, dst, n)
    tr = tmotif.Tree(motifs, 50)
    want = heuristic.comine_advice(src, dst, n, motifs)
    assert tmotif.tm_comine_advice(g.h, tr.h) == want
    roots = np.arange(0, len(src), max(1, len(src) // 3000), dtype=np.int32)
    auto, st = tmotif.tm_count(g.h, tr.h, mode=tmotif.TM_AUTO, roots=roots, stats=True)
    co = tmotif.tm_count(g.h, tr.h, mode=tmotif.TM_COMINE, roots=roots)
    assert auto.tolist() == co.tolist()
    # the path taken: one launch co-mined, one launch per distinct motif otherwise
    assert st["launches"] == (1 if want else len(motifs))
    s = np.asarray(src, np.int32)
    d = np.asarray(dst, np.int32)
    t = np.arange(len(s), dtype=np.int64)
    ref = [oracle.count_motif(s, d, t, m, 50, roots=roots, n_nodes=n) for m in motifs]
    assert auto.tolist() == ref
    tr.close()
    g.close()


def test_auto_with_permotif_is_rejected():
    src, dst, n = CASES["antiparallel"]
    g = _graph(src, dst, n)
    tr = tmotif.Tree(LOW, 5)
    with pytest.raises(tmotif.TMError) as e:
        tmotif.tm_count(g.h, tr.h, mode=tmotif.TM_AUTO | tmotif.TM_PERMOTIF)
    assert e.value.code == tmotif.TM_EINVAL
    tr.close()
    g.close()
