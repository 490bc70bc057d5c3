"""Batched counting: many motif sets merged into one tree (each motif with
its own window), one persistent launch, replayed from a CUDA graph, with
launch parameters from the autotuner.  Counts must equal each set counted
alone, and the oracle."""
import numpy as np
import pytest

import oracle
from paper_2507_14813_b300 import build, synth, tmotif

pytestmark = pytest.mark.gpu

D = tmotif.TM_SCHED_DYNAMIC


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    tmotif.lib()


@pytest.fixture(scope="module")
def small():
    src, dst, t = synth.tiny_graph(4242, 300, 20000, 200000, zipf_s=1.3)
    g = tmotif.Graph(src, dst, t, 300, presorted=True)
    sets = [(synth.random_motif_tree(1000 + i, max_edges=5, max_motifs=12), [300, 1500, 6000][i % 3])
            for i in range(16)]
    return src, dst, t, g, sets


def _merged(sets):
    motifs, deltas, owner = [], [], []
    for i, (ms, d) in enumerate(sets):
        motifs += ms
        deltas += [d] * len(ms)
        owner += [i] * len(ms)
    return motifs, deltas, np.array(owner)


def test_merged_tree_equals_each_set_alone(small):
    src, dst, t, g, sets = small
    motifs, deltas, owner = _merged(sets)
    tr = tmotif.Tree(motifs, deltas)
    assert tr.info()["n_deltas"] == 3
    got = tmotif.count(g, tr, mode=D)
    for i, (ms, d) in enumerate(sets):
        alone = tmotif.count(g, tmotif.Tree(ms, d))
        assert got[owner == i].tolist() == alone.tolist()
    # oracle on the first few sets
    for i, (ms, d) in enumerate(sets[:3]):
        want = [oracle.count_motif(src, dst, t, m, d, n_nodes=300) for m in ms]
        assert got[owner == i].tolist() == want


def test_exec_graph_replays_match(small):
    import torch
    src, dst, t, g, sets = small
    motifs, deltas, _ = _merged(sets)
    tr = tmotif.Tree(motifs, deltas)
    want = tmotif.count(g, tr)
    roots = torch.arange(len(src), dtype=torch.int32, device="cuda")
    out = torch.full((len(motifs),), -1, dtype=torch.int64, device="cuda")
    ex = tmotif.Exec(g.h, tr.h, out, mode=D, roots=roots)
    for _ in range(3):
        out.fill_(-1)
        ex.launch()
        ex.status()
        assert out.cpu().tolist() == want.tolist()
    # a range and the static mode too
    out2 = torch.zeros(len(motifs), dtype=torch.int64, device="cuda")
    ex2 = tmotif.Exec(g.h, tr.h, out2, root_lo=100, root_hi=15000)
    ex2.launch()
    ex2.status()
    assert out2.cpu().tolist() == tmotif.count(g, tr, root_lo=100, root_hi=15000).tolist()


def test_exec_rejects_host_roots(small):
    import torch
    src, dst, t, g, sets = small
    tr = tmotif.Tree(sets[0][0], sets[0][1])
    out = torch.zeros(len(sets[0][0]), dtype=torch.int64, device="cuda")
    with pytest.raises(tmotif.TMError) as e:
        tmotif.Exec(g.h, tr.h, out, roots=np.arange(10, dtype=np.int32))
    assert e.value.code == tmotif.TM_EINVAL


def test_autotune_picks_a_valid_shape_and_counts_stay_exact(small):
    import torch
    src, dst, t, g, sets = small
    motifs, deltas, _ = _merged(sets)
    tr = tmotif.Tree(motifs, deltas)
    roots = torch.from_numpy(synth.root_sample(5, len(src), 4000)).cuda()
    tune = tmotif.tm_autotune(g.h, tr.h, mode=D, roots=roots)
    assert tune["ctas_per_sm"] in (0, 2, 3, 4) and tune["donate_seq"] > 0 and tune["poll_every"] > 0
    assert tune["ms"] > 0
    a = tmotif.count(g, tr, mode=D, roots=roots, tune=tune)
    b = tmotif.count(g, tr, roots=roots)
    assert a.tolist() == b.tolist()
    # every grid point gives the same counts
    for c, s_, l_, p_ in [(2, 32, 256, 1), (3, 1024, 4096, 16)]:
        x = tmotif.count(g, tr, mode=D, roots=roots,
                         tune=dict(ctas_per_sm=c, donate_seq=s_, donate_leaf=l_, poll_every=p_))
        assert x.tolist() == b.tolist()
