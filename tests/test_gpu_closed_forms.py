"""Full-size parity: the CUDA path against closed forms and the oracle.

The mid workload (1M nodes, 20M edges, Zipf(1.6), bursty times, delta =
3600 s) has hub roots whose 4-edge star counts (10^14 per root) no
enumeration reaches.  Their counts are pinned here, per root and bit-exact,
by the closed forms of ``tests/refimpl.py`` (range counts over time-sorted
lists and elementary symmetric polynomials of far-end multiplicities; each
is itself pinned against brute force and the oracle on tiny graphs).  Every
scheduling mode is compared: static, reactive splitting, a planned split
and both together, co-mined and per-motif.

A second, smaller hub graph is sized so that the oracle finishes: its hub
windows span more than 30 chunks of 32 entries with more than 256 distinct
far ends, so the star frames' occurrence table fills, evicts and is taken
over, and donated top-down slices run.  It is compared with the oracle per
root in every mode.
"""
import numpy as np
import pytest

import oracle
from paper_2507_14813_b300 import build, synth, tmotif
from tests import refimpl

pytestmark = pytest.mark.gpu

D = tmotif.TM_SCHED_DYNAMIC
P = tmotif.TM_SCHED_PLANNED
# tiny thresholds: donations at every poll, of slices down to one chunk
EAGER = {"ctas_per_sm": 0, "donate_seq": 32, "donate_leaf": 32, "poll_every": 1}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    tmotif.lib()


@pytest.fixture(scope="module")
def mid():
    src, dst, t = synth.make_graph(synth.MID)
    g = tmotif.Graph(src, dst, t, synth.MID.n_nodes, presorted=True)
    idx = refimpl.ListIndex(src, dst)
    return src, dst, t, g, idx


def _per_root(g, tr, roots, n_motifs, mode, split=None, tune=None):
    import torch
    r = torch.from_numpy(np.asarray(roots, np.int32)).cuda()
    pr = torch.zeros((len(roots), n_motifs), dtype=torch.int64, device="cuda")
    sp = None
    if mode & P:
        sp = torch.full((len(roots),), split, dtype=torch.int32, device="cuda")
    tot = tmotif.count(g, tr, roots=r, per_root_counts=pr, mode=mode, root_split=sp, tune=tune)
    pr = pr.cpu().numpy()
    assert np.array_equal(pr.sum(axis=0), tot)
    return pr


def _closed_columns(src, dst, t, motifs, delta, roots, idx):
    cols = {}
    for j, m in enumerate(motifs):
        try:
            cols[j] = refimpl.closed_form_per_root(src, dst, t, m, delta, roots, idx=idx)
        except KeyError:
            pass
    return cols


def test_mid_all_roots_two_edge_motifs(mid):
    """The four connected 2-edge motifs over all 20M root edges of the mid
    graph: totals and a 4096-root per-root sample equal the closed forms."""
    src, dst, t, g, idx = mid
    ms = [((0, 1), (1, 2)), ((0, 1), (1, 0)), ((0, 1), (0, 2)), ((0, 1), (2, 1))]
    tr = tmotif.Tree(ms, synth.MID_DELTA)
    allr = np.arange(len(src))
    want = [int(refimpl.closed_form_per_root(src, dst, t, m, synth.MID_DELTA, allr, idx=idx).sum()) for m in ms]
    for mode in (0, D, tmotif.TM_PERMOTIF):
        assert tmotif.count(g, tr, mode=mode).tolist() == want, mode
    roots = synth.root_sample(31, len(src), 4096)
    pr = _per_root(g, tr, roots, 4, D)
    for j, m in enumerate(ms):
        assert np.array_equal(pr[:, j], refimpl.closed_form_per_root(src, dst, t, m, synth.MID_DELTA, roots, idx=idx))


MID_MODES = [("dyn", D, None), ("permotif-dyn", tmotif.TM_PERMOTIF | D, None), ("planned", P, 256),
             ("planned-dyn", P | D, 64), ("permotif-planned-dyn", tmotif.TM_PERMOTIF | P | D, 16)]


@pytest.mark.parametrize("name,mode,split", MID_MODES)
def test_mid_bench_sample_closed_forms(mid, name, mode, split):
    """The benchmark's 64-root sample of the mid workload, all 12 motifs in
    one tree: per-root counts of the 11 motifs with a closed form equal it,
    bit-exact, in each scheduling mode."""
    src, dst, t, g, idx = mid
    roots = synth.root_sample(100, len(src), 64)
    ms = synth.CONFIG2_MOTIFS
    tr = tmotif.Tree(ms, synth.MID_DELTA)
    cols = _closed_columns(src, dst, t, ms, synth.MID_DELTA, roots, idx)
    assert len(cols) == 11
    pr = _per_root(g, tr, roots, len(ms), mode, split=split)
    for j, want in cols.items():
        assert np.array_equal(pr[:, j], want), (name, ms[j])


@pytest.mark.parametrize("seed,n", [(23, 24), (24, 32), (25, 32)])
def test_mid_heavy_split_roots_closed_forms(mid, seed, n):
    """The heavy-root samples of the splitting tests, with eager donation
    (slices down to one chunk, a look for idle warps at every chunk)."""
    src, dst, t, g, idx = mid
    roots = synth.root_sample(seed, len(src), n)
    ms = synth.CONFIG2_MOTIFS
    tr = tmotif.Tree(ms, synth.MID_DELTA)
    cols = _closed_columns(src, dst, t, ms, synth.MID_DELTA, roots, idx)
    for mode, split, tune in ((D, None, EAGER), (P | D, 512, None)):
        pr = _per_root(g, tr, roots, len(ms), mode, split=split, tune=tune)
        for j, want in cols.items():
            assert np.array_equal(pr[:, j], want), (mode, ms[j])


# ---------------------------------------------------------------- hub graph

HUB_DELTA = 2000
HUB3 = [((0, 1), (1, 2), (2, 0)), ((0, 1), (1, 2), (2, 3)), ((0, 1), (0, 2), (0, 3)), ((0, 1), (0, 2), (1, 2)),
        ((0, 1), (1, 0), (0, 1)), ((0, 1), (1, 0), (0, 2)), ((0, 1), (2, 1), (3, 1)), ((0, 1), (2, 1), (1, 3)),
        ((0, 1), (1, 2), (2, 3), (3, 0)), ((0, 1), (0, 2))]
HUB4 = [((0, 1), (0, 2), (0, 3), (0, 4)), ((0, 1), (2, 1), (3, 1), (4, 1)), ((0, 1), (0, 2), (0, 3)),
        ((0, 1), (2, 1), (3, 1)), ((0, 1), (1, 0), (0, 1), (1, 0))]

HUB_MODES = [
    ("comine", 0, None, None), ("comine-scan", tmotif.TM_LEAF_SCAN, None, None),
    ("permotif", tmotif.TM_PERMOTIF, None, None), ("permotif-scan", tmotif.TM_PERMOTIF | tmotif.TM_LEAF_SCAN, None, None),
    ("dyn", D, None, None), ("dyn-eager", D, None, EAGER), ("scan-dyn-eager", tmotif.TM_LEAF_SCAN | D, None, EAGER),
    ("permotif-dyn-eager", tmotif.TM_PERMOTIF | D, None, EAGER),
    ("planned", P, 16, None), ("planned-dyn-eager", P | D, 8, EAGER), ("permotif-planned", tmotif.TM_PERMOTIF | P, 4, None),
]


@pytest.fixture(scope="module")
def hub():
    src, dst, t = synth.hub_graph(31, 4000, 40000, 40000)
    g = tmotif.Graph(src, dst, t, 4000, presorted=True)
    hub_out = np.nonzero(src == 0)[0]
    hub_in = np.nonzero(dst == 0)[0]
    roots = np.unique(np.concatenate([hub_out[::100], hub_in[::50], synth.root_sample(3, len(src), 200)]))
    idx = refimpl.ListIndex(src, dst)
    # the hub windows are what the test is for: many chunks, many far ends
    W = refimpl.window_end_sat(t, HUB_DELTA)
    o, e = idx.entries("out", src[roots], roots, W[roots])
    sizes = np.bincount(o, minlength=len(roots))
    far = [len(np.unique(dst[e][o == i])) for i in np.nonzero(sizes > 900)[0]]
    assert sizes.max() > 30 * 32 and min(far) > 256
    want3 = np.stack([oracle.count_motif(src, dst, t, m, HUB_DELTA, roots=roots, per_root=True)[1] for m in HUB3],
                     axis=1)
    return src, dst, t, g, roots, idx, want3


@pytest.mark.parametrize("name,mode,split,tune", HUB_MODES)
def test_hub_graph_oracle_per_root(hub, name, mode, split, tune):
    src, dst, t, g, roots, idx, want3 = hub
    tr = tmotif.Tree(HUB3, HUB_DELTA)
    pr = _per_root(g, tr, roots, len(HUB3), mode, split=split, tune=tune)
    assert np.array_equal(pr, want3), name


@pytest.mark.parametrize("name,mode,split,tune", [m for m in HUB_MODES if not m[1] & tmotif.TM_LEAF_SCAN])
def test_hub_graph_four_edge_stars_closed_forms(hub, name, mode, split, tune):
    src, dst, t, g, roots, idx, _ = hub
    tr = tmotif.Tree(HUB4, HUB_DELTA)
    pr = _per_root(g, tr, roots, len(HUB4), mode, split=split, tune=tune)
    for j, m in enumerate(HUB4):
        want = refimpl.closed_form_per_root(src, dst, t, m, HUB_DELTA, roots, idx=idx)
        assert np.array_equal(pr[:, j], want), (name, m)
