"""Match enumeration (tm_enumerate) against brute force on tiny graphs, and
against the oracle's recorded matches, the definition, the oracle's counts and
tm_count at larger sizes:
every written record must be a match, no two records equal, and as many
records per motif as the count, which makes the set exact."""
import numpy as np
import pytest

import oracle
from paper_2507_14813_b300 import build, synth, tmotif
from tests.refimpl import brute_force_matches

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    tmotif.lib()


def _is_match(src, dst, t, motif, delta, eids):
    if any(b <= a for a, b in zip(eids, eids[1:])) or t[eids[-1]] - t[eids[0]] > delta:
        return False
    f = {}
    for (mu, mv), e in zip(motif, eids):
        for mx, gx in ((mu, int(src[e])), (mv, int(dst[e]))):
            if f.setdefault(mx, gx) != gx:
                return False
    return len(set(f.values())) == len(f)


def _records(matches, motifs):
    out = []
    for row in matches.tolist():
        m, n = row[0], row[1]
        assert n == len(motifs[m])
        assert all(x == -1 for x in row[2 + n:])
        out.append((m, tuple(row[2:2 + n])))
    return out


def _check_exact(src, dst, t, motifs, deltas, matches, counts):
    recs = _records(matches, motifs)
    assert len(set(recs)) == len(recs), "a match was written twice"
    per = np.zeros(len(motifs), np.int64)
    for m, eids in recs:
        assert _is_match(src, dst, t, motifs[m], deltas[m], eids), (m, eids)
        per[m] += 1
    assert per.tolist() == list(counts)


@pytest.mark.parametrize("seed", range(4))
def test_enumeration_equals_brute_force(seed):
    rng = np.random.default_rng(500 + seed)
    V, E = 6, 28
    src = rng.integers(0, V, E).astype(np.int32)
    dst = ((src + rng.integers(1, V, E)) % V).astype(np.int32)
    if seed % 2:
        src[3] = dst[3]                         # one self-loop edge
    t = np.sort(rng.integers(0, 60, E)).astype(np.int64)   # many ties
    motifs = [((0, 1), (1, 2)), ((0, 1), (1, 0), (0, 1)), ((0, 1), (0, 2), (0, 3)), ((0, 1), (1, 2)),
              ((0, 1), (2, 1), (1, 3)), ((0, 1), (1, 2), (2, 0))]
    deltas = [20, 35, 50, 8, 50, 60]
    g = tmotif.Graph(src, dst, t, V, presorted=True)
    tr = tmotif.Tree(motifs, deltas)
    matches, n_found, counts = tmotif.tm_enumerate(g.h, tr.h, cap=100_000)
    recs = _records(matches, motifs)
    assert n_found == len(recs)
    for m, motif in enumerate(motifs):
        want = sorted(brute_force_matches(src, dst, t, motif, deltas[m]))
        got = sorted(e for mm, e in recs if mm == m)
        assert got == want, m
        assert counts[m] == len(want)
    tr.close()
    g.close()


@pytest.fixture(scope="module")
def tiny():
    src, dst, t = synth.tiny_graph(2, 2000, 50_000, 1_000_000, zipf_s=1.8)
    g = tmotif.Graph(src, dst, t, 2000, presorted=True)
    yield src, dst, t, g
    g.close()


def test_enumeration_tiny_workload_sample(tiny):
    src, dst, t, g = tiny
    motifs = synth.CONFIG1_MOTIFS
    deltas = [synth.TINY_DELTA] * len(motifs)
    tr = tmotif.Tree(motifs, deltas)
    roots = synth.root_sample(9, len(src), 400)
    matches, n_found, counts = tmotif.tm_enumerate(g.h, tr.h, cap=2_000_000, roots=roots)
    assert n_found == len(matches)
    want = tmotif.tm_count(g.h, tr.h, roots=roots)
    assert counts.tolist() == want.tolist()
    ref = [oracle.count_motif(src, dst, t, m, synth.TINY_DELTA, roots=roots, n_nodes=2000) for m in motifs]
    assert counts.tolist() == ref
    _check_exact(src, dst, t, motifs, deltas, matches, counts)
    # the oracle's own match lists (Algorithm 1 recording its matches)
    recs = _records(matches, motifs)
    for mi, motif in enumerate(motifs):
        want, n = oracle.enumerate_motif(src, dst, t, motif, synth.TINY_DELTA, roots=roots, n_nodes=2000)
        assert n == counts[mi]
        assert sorted(e for m, e in recs if m == mi) == sorted(map(tuple, want.tolist()))
    tr.close()


def test_enumeration_overflow_keeps_total(tiny):
    src, dst, t, g = tiny
    motifs = synth.CONFIG1_MOTIFS
    deltas = [synth.TINY_DELTA] * len(motifs)
    tr = tmotif.Tree(motifs, deltas)
    roots = synth.root_sample(9, len(src), 400)
    _, total, counts = tmotif.tm_enumerate(g.h, tr.h, cap=0, roots=roots)
    assert total == int(counts.sum()) > 10
    cap = total // 3
    matches, n_found, counts2 = tmotif.tm_enumerate(g.h, tr.h, cap=cap, roots=roots)
    assert n_found == total and len(matches) == cap and counts2.tolist() == counts.tolist()
    recs = _records(matches, motifs)
    assert len(set(recs)) == cap
    for m, eids in recs:
        assert _is_match(src, dst, t, motifs[m], deltas[m], eids)
    tr.close()


def test_enumeration_root_forms_agree(tiny):
    import torch
    src, dst, t, g = tiny
    motifs = [((0, 1), (1, 2), (2, 0)), ((0, 1), (1, 0))]
    tr = tmotif.Tree(motifs, [5000, 20000])
    lo, hi = 1000, 1600
    a, na, ca = tmotif.tm_enumerate(g.h, tr.h, cap=10_000_000, root_lo=lo, root_hi=hi)
    r = np.arange(lo, hi, dtype=np.int32)
    b, nb, cb = tmotif.tm_enumerate(g.h, tr.h, cap=10_000_000, roots=torch.from_numpy(r).cuda())
    assert na == nb and ca.tolist() == cb.tolist()
    assert sorted(map(tuple, a.tolist())) == sorted(map(tuple, b.tolist()))
    assert ca.tolist() == tmotif.tm_count(g.h, tr.h, root_lo=lo, root_hi=hi).tolist()
    tr.close()


def test_enumeration_rejects_bad_arguments(tiny):
    src, dst, t, g = tiny
    tr = tmotif.Tree(synth.CONFIG1_MOTIFS, 100)
    for kw in ({"mode": tmotif.TM_PERMOTIF}, {"mode": tmotif.TM_LEAF_SCAN}, {"mode": tmotif.TM_AUTO},
               {"roots": np.array([len(src)], np.int32)}, {"cap": -1}):
        args = {"cap": 10, **kw}
        with pytest.raises(tmotif.TMError) as e:
            tmotif.tm_enumerate(g.h, tr.h, **args)
        assert e.value.code == tmotif.TM_EINVAL
    tr.close()
