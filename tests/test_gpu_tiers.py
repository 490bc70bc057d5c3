"""The thread tier (TM_SCHED_TIERS): roots the plan marks light (slice
count 0, the tail of the planned order) run one per lane as a serial walk
of the MG-Tree; the rest run one per warp, those with slice counts above 1
cut across many warps.  Counts are int64 and must equal the oracle's, per
root, whatever the tier; the tier histogram must match the plan.
"""
import numpy as np
import pytest

import oracle
from paper_2507_14813_b300 import build, synth, tmotif
from tests import refimpl
from tests.test_gpu_closed_forms import HUB4, HUB_DELTA
from tests.test_oracle_pins import PIN_MOTIFS

pytestmark = pytest.mark.gpu

T = tmotif.TM_SCHED_TIERS | tmotif.TM_SCHED_PLANNED
D = tmotif.TM_SCHED_DYNAMIC


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    tmotif.lib()


def _plan(roots, n_lane, head_split=1):
    """A hand-made plan: the first roots one per warp (slice count head_split),
    the last n_lane in the thread tier (slice count 0)."""
    import torch
    r = torch.from_numpy(np.asarray(roots, np.int32)).cuda()
    sp = np.full(len(roots), head_split, np.int32)
    if n_lane:
        sp[len(roots) - n_lane:] = 0
    return r, torch.from_numpy(sp).cuda()


def _count(g, tr, roots, n_lane, mode, head_split=1, stats=False):
    import torch
    r, sp = _plan(roots, n_lane, head_split)
    pr = torch.zeros((len(roots), len(tr.motifs)), dtype=torch.int64, device="cuda")
    out = tmotif.count(g, tr, roots=r, per_root_counts=pr, mode=mode, root_split=sp, stats=stats)
    return (pr.cpu().numpy(), out[1]) if stats else pr.cpu().numpy()


@pytest.mark.parametrize("mode", [T, T | D, T | tmotif.TM_PERMOTIF, T | tmotif.TM_LEAF_SCAN | D])
@pytest.mark.parametrize("frac", [1.0, 0.5])
def test_tiny_config_thread_tier(mode, frac):
    src, dst, t = synth.make_graph(synth.TINY)
    g = tmotif.Graph(src, dst, t, synth.TINY.n_nodes, presorted=True)
    tr = tmotif.Tree(synth.CONFIG1_MOTIFS, synth.TINY_DELTA)
    roots = synth.root_sample(51, len(src), 6000)
    n_lane = int(frac * len(roots))
    got, st = _count(g, tr, roots, n_lane, mode, head_split=4, stats=True)
    _, want = oracle.count_motifs(src, dst, t, synth.CONFIG1_MOTIFS, synth.TINY_DELTA, roots=roots, per_root=True)
    assert np.array_equal(got, want)
    if not mode & tmotif.TM_PERMOTIF:
        assert st["roots_thread_tier"] == n_lane
        assert st["n_roots"] == len(roots)


@pytest.mark.parametrize("seed", range(4))
def test_pin_motifs_thread_tier(seed):
    """Every candidate-list case (global window, in-list, both mapped),
    several windows, tie-heavy graphs with self-loops, all in the thread tier."""
    src, dst, t = synth.tiny_graph(9900 + seed, 9 + seed, 400 + 50 * seed, 300, zipf_s=1.0, self_loops=seed % 2 == 0)
    deltas = [(i * 3 + seed) % 40 for i in range(len(PIN_MOTIFS))]
    g = tmotif.Graph(src, dst, t, 9 + seed, presorted=True)
    tr = tmotif.Tree(PIN_MOTIFS, deltas)
    roots = np.arange(len(src))
    want = np.stack([oracle.count_motif(src, dst, t, m, d, roots=roots, n_nodes=9 + seed, per_root=True)[1]
                     for m, d in zip(PIN_MOTIFS, deltas)], axis=1)
    for mode in (T, T | D):
        assert np.array_equal(_count(g, tr, roots, len(roots) // 2 + seed, mode), want)


@pytest.mark.parametrize("seed", range(3))
def test_random_trees_thread_tier(seed):
    src, dst, t = synth.tiny_graph(9950 + seed, 40, 3000, 60000, zipf_s=1.3)
    motifs = synth.random_motif_tree(650 + seed, max_edges=5, max_motifs=20)
    deltas = [[300, 1000, 2000][(i + seed) % 3] for i in range(len(motifs))]
    g = tmotif.Graph(src, dst, t, 40, presorted=True)
    tr = tmotif.Tree(motifs, deltas)
    roots = synth.root_sample(seed, len(src), 1500)
    want = np.stack([oracle.count_motif(src, dst, t, m, d, roots=roots, n_nodes=40, per_root=True)[1]
                     for m, d in zip(motifs, deltas)], axis=1)
    assert np.array_equal(_count(g, tr, roots, 1000, T | D), want)


def test_max_size_motifs_thread_tier():
    src, dst, t = synth.tiny_graph(9960, 8, 1500, 4000, zipf_s=0.3)
    motifs = [tuple((i, (i + 1) % 8) for i in range(8)), tuple((i, i + 1) for i in range(7)),
              tuple((0, i + 1) for i in range(7)) + ((1, 0),)]
    g = tmotif.Graph(src, dst, t, 8, presorted=True)
    tr = tmotif.Tree(motifs, 150)
    roots = np.arange(len(src))
    want = np.stack([oracle.count_motif(src, dst, t, m, 150, roots=roots, n_nodes=8, per_root=True)[1]
                     for m in motifs], axis=1)
    assert np.array_equal(_count(g, tr, roots, len(roots), T), want)


def test_hub_graph_thread_tier_closed_forms():
    """Hub roots counted lane by lane: 4-edge stars (window arithmetic leaves
    after a serial scan of long hub windows) against the closed forms."""
    src, dst, t = synth.hub_graph(31, 4000, 40000, 40000)
    g = tmotif.Graph(src, dst, t, 4000, presorted=True)
    roots = np.unique(np.concatenate([np.nonzero(src == 0)[0][::400], synth.root_sample(3, len(src), 100)]))
    tr = tmotif.Tree(HUB4, HUB_DELTA)
    idx = refimpl.ListIndex(src, dst)
    want = np.stack([refimpl.closed_form_per_root(src, dst, t, m, HUB_DELTA, roots, idx=idx) for m in HUB4], axis=1)
    assert np.array_equal(_count(g, tr, roots, len(roots) // 2, T | D), want)


def test_plan_tiers_from_the_cost_model():
    """tm_plan_tiers: a trained model's predictions order the roots, the
    predicted-light ones get slice count 0 at the tail, and counting with
    that plan equals the oracle."""
    import torch
    src, dst, t = synth.make_graph(synth.TINY)
    g = tmotif.Graph(src, dst, t, synth.TINY.n_nodes, presorted=True)
    tr = tmotif.Tree(synth.CONFIG1_MOTIFS, synth.TINY_DELTA)
    train = torch.from_numpy(synth.root_sample(61, len(src), 2048)).cuda()
    work = torch.zeros((2048, tmotif.TM_WORK_FIELDS), dtype=torch.int64, device="cuda")
    tmotif.count(g, tr, roots=train, per_root_work=work, stats=True)
    w = work.cpu().numpy()
    y = torch.from_numpy(np.log1p(w[:, 0] + w[:, 2]).astype(np.float32)).cuda()
    X = torch.zeros((2048, tmotif.TM_FEATURES), dtype=torch.float32, device="cuda")
    tmotif.tm_features(g.h, tr.h, train, X)
    model = tmotif.Model(seed=3)
    model.fit_norm(X)
    model.train(X, y, epochs=60, batch=256, lr=3e-3)
    roots = torch.from_numpy(synth.root_sample(62, len(src), 5000)).cuda()
    F = torch.zeros((5000, tmotif.TM_FEATURES), dtype=torch.float32, device="cuda")
    tmotif.tm_features(g.h, tr.h, roots, F)
    ro, sp = torch.zeros_like(roots), torch.zeros_like(roots)
    thr = float(np.median(w[:, 0] + w[:, 2]))
    model.plan(F, roots, ro, sp, unit_work=1e4, max_split=64, thread_work=thr)
    s = sp.cpu().numpy()
    assert (s == 0).any() and (s > 0).any()
    assert np.all(np.diff(s) <= 0)                      # non-increasing: the light tail last
    got, st = tmotif.count(g, tr, roots=ro, root_split=sp, mode=T | D, stats=True)
    assert st["roots_thread_tier"] == int((s == 0).sum())
    want = oracle.count_motifs(src, dst, t, synth.CONFIG1_MOTIFS, synth.TINY_DELTA, roots=ro.cpu().numpy())
    assert got.tolist() == want.tolist()
