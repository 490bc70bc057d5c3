"""Sibling splitting and multi-offload (the paper's GPU load-balancing
policies) against the oracle and the closed forms.

With TM_SCHED_SIBLINGS a warp about to descend into several children of a
node hands all but the first to the queue as tasks that carry the partial
match, and a donation hands over up to one piece per idle warp.  Here the
splitting is forced (sibling_always: every such descent splits, idle warps
or not) with the smallest donation thresholds, so every task path runs;
counts are int64 and must be bit-exact.
"""
import numpy as np
import pytest

import oracle
from paper_2507_14813_b300 import build, synth, tmotif
from tests import refimpl
from tests.test_gpu_closed_forms import HUB3, HUB_DELTA
from tests.test_oracle_pins import PIN_MOTIFS

pytestmark = pytest.mark.gpu

S = tmotif.TM_SCHED_SIBLINGS
P = tmotif.TM_SCHED_PLANNED
FORCED = {"ctas_per_sm": 0, "donate_seq": 32, "donate_leaf": 32, "poll_every": 1, "offload_max": 8,
          "sibling_always": 1}
NATURAL = {"ctas_per_sm": 0, "donate_seq": 0, "donate_leaf": 4096, "poll_every": 16, "offload_max": 8}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    tmotif.lib()


@pytest.mark.parametrize("mode", [S, S | tmotif.TM_LEAF_SCAN, S | tmotif.TM_PERMOTIF])
def test_tiny_config_forced_siblings(mode):
    src, dst, t = synth.make_graph(synth.TINY)
    g = tmotif.Graph(src, dst, t, synth.TINY.n_nodes, presorted=True)
    tr = tmotif.Tree(synth.CONFIG1_MOTIFS, synth.TINY_DELTA)
    want = oracle.count_motifs(src, dst, t, synth.CONFIG1_MOTIFS, synth.TINY_DELTA)
    got, st = tmotif.count(g, tr, mode=mode, tune=FORCED, stats=True)
    assert got.tolist() == want.tolist()
    assert st["tasks_split"] > 0


@pytest.mark.parametrize("seed", range(4))
def test_pin_motifs_forced_siblings(seed):
    """The pin motifs' tree has many siblings under its root; several windows."""
    src, dst, t = synth.tiny_graph(9700 + seed, 9 + seed, 400 + 50 * seed, 300, zipf_s=1.0, self_loops=seed % 2 == 0)
    deltas = [(i * 5 + seed) % 40 for i in range(len(PIN_MOTIFS))]
    g = tmotif.Graph(src, dst, t, 9 + seed, presorted=True)
    tr = tmotif.Tree(PIN_MOTIFS, deltas)
    want = [oracle.count_motif(src, dst, t, m, d, n_nodes=9 + seed) for m, d in zip(PIN_MOTIFS, deltas)]
    for mode in (S, S | tmotif.TM_LEAF_SCAN):
        assert tmotif.count(g, tr, mode=mode, tune=FORCED).tolist() == want


@pytest.mark.parametrize("seed", range(3))
def test_random_trees_forced_siblings(seed):
    src, dst, t = synth.tiny_graph(9800 + seed, 40, 3000, 60000, zipf_s=1.3)
    motifs = synth.random_motif_tree(600 + seed, max_edges=5, max_motifs=20)
    deltas = [[300, 1000, 2000][(i + seed) % 3] for i in range(len(motifs))]
    g = tmotif.Graph(src, dst, t, 40, presorted=True)
    tr = tmotif.Tree(motifs, deltas)
    want = [oracle.count_motif(src, dst, t, m, d, n_nodes=40) for m, d in zip(motifs, deltas)]
    assert tmotif.count(g, tr, mode=S, tune=FORCED).tolist() == want


@pytest.mark.parametrize("tune", [FORCED, NATURAL])
def test_mid_bench_sample_siblings_closed_forms(tune):
    """The benchmark's 64 hub roots of the mid workload, learned-plan style
    planned splits on top: per-root counts equal the closed forms."""
    import torch
    src, dst, t = synth.make_graph(synth.MID)
    g = tmotif.Graph(src, dst, t, synth.MID.n_nodes, presorted=True)
    idx = refimpl.ListIndex(src, dst)
    roots = synth.root_sample(100, len(src), 64)
    tr = tmotif.Tree(synth.CONFIG2_MOTIFS, synth.MID_DELTA)
    pr = torch.zeros((64, 12), dtype=torch.int64, device="cuda")
    sp = torch.full((64,), 64, dtype=torch.int32, device="cuda")
    tmotif.count(g, tr, roots=torch.from_numpy(roots).cuda(), per_root_counts=pr, mode=S | P, root_split=sp, tune=tune)
    pr = pr.cpu().numpy()
    for j, m in enumerate(synth.CONFIG2_MOTIFS):
        try:
            want = refimpl.closed_form_per_root(src, dst, t, m, synth.MID_DELTA, roots, idx=idx)
        except KeyError:
            continue
        assert np.array_equal(pr[:, j], want), m


def test_hub_graph_forced_siblings():
    import torch
    src, dst, t = synth.hub_graph(31, 4000, 40000, 40000)
    g = tmotif.Graph(src, dst, t, 4000, presorted=True)
    roots = np.unique(np.concatenate([np.nonzero(src == 0)[0][::100], synth.root_sample(3, len(src), 200)]))
    tr = tmotif.Tree(HUB3, HUB_DELTA)
    want = np.stack([oracle.count_motif(src, dst, t, m, HUB_DELTA, roots=roots, per_root=True)[1] for m in HUB3],
                    axis=1)
    pr = torch.zeros((len(roots), len(HUB3)), dtype=torch.int64, device="cuda")
    tmotif.count(g, tr, roots=torch.from_numpy(roots.astype(np.int32)).cuda(), per_root_counts=pr, mode=S,
                 tune=FORCED)
    assert np.array_equal(pr.cpu().numpy(), want)
