"""GPU parity: the CUDA path against the CPU oracle, element by element.

Counts are 64-bit integers, so the bar is bit-exact equality.  Every call
goes through the C-ABI (ctypes binding); the oracle is the plain recursion
of Algorithms 1 and 3.
"""
import numpy as np
import pytest

import oracle
from paper_2507_14813_b300 import build, synth, tmotif
from tests.test_oracle_pins import PIN_MOTIFS

pytestmark = pytest.mark.gpu

D = tmotif.TM_SCHED_DYNAMIC
P = tmotif.TM_SCHED_PLANNED
MODES = [
    ("comine", tmotif.TM_COMINE),
    ("comine-scan", tmotif.TM_COMINE | tmotif.TM_LEAF_SCAN),
    ("permotif", tmotif.TM_PERMOTIF),
    ("permotif-scan", tmotif.TM_PERMOTIF | tmotif.TM_LEAF_SCAN),
    ("comine-dyn", tmotif.TM_COMINE | D),
    ("comine-scan-dyn", tmotif.TM_COMINE | tmotif.TM_LEAF_SCAN | D),
    ("permotif-dyn", tmotif.TM_PERMOTIF | D),
    ("comine-planned", tmotif.TM_COMINE | P),
    ("comine-planned-dyn", tmotif.TM_COMINE | P | D),
    ("permotif-scan-planned", tmotif.TM_PERMOTIF | tmotif.TM_LEAF_SCAN | P),
]


def count_mode(g, tr, mode, n_edges, **kw):
    """tm_count over every root edge; a planned mode cuts each root's
    first-level lists into 4 slices."""
    if mode & P:
        import torch
        kw["root_split"] = torch.full((n_edges,), 4, dtype=torch.int32, device="cuda")
    return tmotif.count(g, tr, mode=mode, **kw)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    tmotif.lib()


@pytest.fixture(scope="module")
def tiny():
    src, dst, t = synth.make_graph(synth.TINY)
    g = tmotif.Graph(src, dst, t, synth.TINY.n_nodes, presorted=True)
    want = oracle.count_motifs(src, dst, t, synth.CONFIG1_MOTIFS, synth.TINY_DELTA)
    return src, dst, t, g, want


@pytest.mark.parametrize("name,mode", MODES)
def test_tiny_config_full(tiny, name, mode):
    src, dst, t, g, want = tiny
    tr = tmotif.Tree(synth.CONFIG1_MOTIFS, synth.TINY_DELTA)
    got = count_mode(g, tr, mode, len(src))
    assert got.tolist() == want.tolist(), name


@pytest.mark.parametrize("mode", [0, D])
def test_tiny_config_per_root(tiny, mode):
    import torch
    src, dst, t, g, want = tiny
    tr = tmotif.Tree(synth.CONFIG1_MOTIFS, synth.TINY_DELTA)
    roots = synth.root_sample(11, len(src), 4000)
    pr = torch.zeros((len(roots), len(synth.CONFIG1_MOTIFS)), dtype=torch.int64, device="cuda")
    got = tmotif.count(g, tr, roots=roots, per_root_counts=pr, mode=mode)
    _, want_pr = oracle.count_motifs(src, dst, t, synth.CONFIG1_MOTIFS, synth.TINY_DELTA, roots=roots,
                                     per_root=True)
    assert np.array_equal(pr.cpu().numpy(), want_pr)
    assert got.tolist() == want_pr.sum(axis=0).tolist()


def test_tiny_config_root_range_additivity(tiny):
    src, dst, t, g, want = tiny
    tr = tmotif.Tree(synth.CONFIG1_MOTIFS, synth.TINY_DELTA)
    E = len(src)
    cuts = [0, 1, 777, 20000, 31001, E]
    parts = [tmotif.count(g, tr, root_lo=a, root_hi=b) for a, b in zip(cuts[:-1], cuts[1:])]
    assert np.sum(parts, axis=0).tolist() == want.tolist()


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("name,mode", MODES)
def test_pin_motifs_small_graphs(seed, name, mode):
    # tie-heavy, self-loops on some seeds, several windows in one tree
    src, dst, t = synth.tiny_graph(9000 + seed, 9 + seed, 400 + 50 * seed, 300, zipf_s=1.0,
                                   self_loops=seed % 2 == 0)
    deltas = [(i * 7 + seed) % 40 for i in range(len(PIN_MOTIFS))]
    g = tmotif.Graph(src, dst, t, 9 + seed, presorted=True)
    tr = tmotif.Tree(PIN_MOTIFS, deltas)
    want = [oracle.count_motif(src, dst, t, m, d, n_nodes=9 + seed) for m, d in zip(PIN_MOTIFS, deltas)]
    got = count_mode(g, tr, mode, len(src))
    assert got.tolist() == want


@pytest.mark.parametrize("seed", range(6))
def test_random_trees_multi_delta(seed):
    src, dst, t = synth.tiny_graph(9100 + seed, 40, 3000, 60000, zipf_s=1.3)
    motifs = synth.random_motif_tree(500 + seed, max_edges=5, max_motifs=20)
    deltas = [[300, 1000, 2000][(i + seed) % 3] for i in range(len(motifs))]
    g = tmotif.Graph(src, dst, t, 40, presorted=True)
    tr = tmotif.Tree(motifs, deltas)
    want = [oracle.count_motif(src, dst, t, m, d, n_nodes=40) for m, d in zip(motifs, deltas)]
    for _, mode in MODES:
        assert count_mode(g, tr, mode, len(src)).tolist() == want


def test_max_size_motifs():
    # 8 edges and 8 vertices: a 7-edge path closed back, and an 8-cycle
    src, dst, t = synth.tiny_graph(9200, 8, 1500, 4000, zipf_s=0.3)
    cyc8 = tuple((i, (i + 1) % 8) for i in range(8))
    path7 = tuple((i, i + 1) for i in range(7))
    star = tuple((0, i + 1) for i in range(7)) + ((1, 0),)
    motifs = [cyc8, path7, star]
    g = tmotif.Graph(src, dst, t, 8, presorted=True)
    tr = tmotif.Tree(motifs, 150)
    want = [oracle.count_motif(src, dst, t, m, 150, n_nodes=8) for m in motifs]
    for _, mode in MODES:
        assert count_mode(g, tr, mode, len(src)).tolist() == want


def test_unsorted_and_device_input():
    import torch
    src, dst, t = synth.tiny_graph(9300, 30, 5000, 2000, zipf_s=1.1)
    # shuffle the input order; the library sorts by (t, input position)
    perm = np.argsort(synth.rand_u64(3, 3, 0, len(src)))
    s2, d2, t2 = src[perm], dst[perm], t[perm]
    order = np.argsort(t2, kind="stable")
    g = tmotif.Graph(s2, d2, t2, 30)
    es, ed, et = g.edges()
    assert np.array_equal(es, s2[order]) and np.array_equal(ed, d2[order]) and np.array_equal(et, t2[order])
    tr = tmotif.Tree(synth.CONFIG1_MOTIFS + PIN_MOTIFS[:6], 150)
    want = [oracle.count_motif(s2[order], d2[order], t2[order], m, 150, n_nodes=30)
            for m in synth.CONFIG1_MOTIFS + PIN_MOTIFS[:6]]
    assert tmotif.count(g, tr).tolist() == want
    # the same edges given as device tensors, presorted
    gd = tmotif.Graph(torch.from_numpy(es).cuda(), torch.from_numpy(ed).cuda(), torch.from_numpy(et).cuda(), 30,
                      presorted=True)
    assert tmotif.count(gd, tr).tolist() == want
    # counts into a device tensor, roots from a device tensor
    out = torch.zeros(len(want), dtype=torch.int64, device="cuda")
    roots = torch.arange(len(src), dtype=torch.int32, device="cuda")
    tmotif.count(gd, tr, counts=out, roots=roots)
    torch.cuda.synchronize()
    assert out.cpu().tolist() == want


def test_negative_times_and_large_window():
    src, dst, t = synth.tiny_graph(9400, 12, 2000, 1000, zipf_s=1.0)
    t = t - 500 - 2**40
    g = tmotif.Graph(src, dst, t, 12)
    ms = [((0, 1), (1, 2), (2, 0)), ((0, 1), (1, 0))]
    tr = tmotif.Tree(ms, [2**63 - 1, 37])
    want = [oracle.count_motif(src, dst, t, ms[0], 2**63 - 1, n_nodes=12),
            oracle.count_motif(src, dst, t, ms[1], 37, n_nodes=12)]
    assert tmotif.count(g, tr).tolist() == want


def test_empty_and_single_edge_graphs():
    e = np.zeros(0, np.int32)
    g0 = tmotif.Graph(e, e, np.zeros(0, np.int64), 5)
    tr = tmotif.Tree(synth.CONFIG1_MOTIFS + [((0, 1),)], 10)
    assert tmotif.count(g0, tr).tolist() == [0] * 5
    g1 = tmotif.Graph(np.array([1], np.int32), np.array([2], np.int32), np.array([7], np.int64), 5)
    assert tmotif.count(g1, tr).tolist() == [0, 0, 0, 0, 1]
    g2 = tmotif.Graph(np.array([3], np.int32), np.array([3], np.int32), np.array([7], np.int64), 5)
    assert tmotif.count(g2, tr).tolist() == [0] * 5


def test_errors():
    src, dst, t = synth.tiny_graph(9500, 10, 100, 1000)
    with pytest.raises(tmotif.TMError) as e:
        tmotif.Graph(src, dst + 100, t, 10)
    assert e.value.code == tmotif.TM_EINVAL
    with pytest.raises(tmotif.TMError) as e:
        tmotif.Graph(src, dst, t[::-1].copy(), 10, presorted=True)
    assert e.value.code == tmotif.TM_EINVAL
    g = tmotif.Graph(src, dst, t, 10)
    tr = tmotif.Tree(synth.CONFIG1_MOTIFS, 10)
    with pytest.raises(tmotif.TMError) as e:
        tmotif.count(g, tr, roots=np.array([0, 100], np.int32))
    assert e.value.code == tmotif.TM_EINVAL
    with pytest.raises(tmotif.TMError) as e:
        tmotif.count(g, tr, root_lo=5, root_hi=101)
    assert e.value.code == tmotif.TM_EINVAL


def test_device_roots_out_of_range(tiny):
    """A device root list is range-checked by the kernel: the call reports
    TM_EINVAL when it synchronises, and the binding rejects per-root outputs
    shorter than the root list."""
    import torch
    src, dst, t, g, _ = tiny
    tr = tmotif.Tree(synth.CONFIG1_MOTIFS, synth.TINY_DELTA)
    for bad in (len(src), -1):
        roots = torch.tensor([5, bad, 7], dtype=torch.int32, device="cuda")
        for mode in (0, D):
            with pytest.raises(tmotif.TMError) as e:
                tmotif.count(g, tr, roots=roots, mode=mode)
            assert e.value.code == tmotif.TM_EINVAL
    roots = torch.tensor([5, 6, 7], dtype=torch.int32, device="cuda")
    short = torch.zeros((2, 4), dtype=torch.int64, device="cuda")
    with pytest.raises(ValueError):
        tmotif.count(g, tr, roots=roots, per_root_counts=short)
    assert tmotif.count(g, tr, roots=roots).tolist() == oracle.count_motifs(
        src, dst, t, synth.CONFIG1_MOTIFS, synth.TINY_DELTA, roots=[5, 6, 7]).tolist()


def test_stats_and_work_counters(tiny):
    import torch
    src, dst, t, g, want = tiny
    tr = tmotif.Tree(synth.CONFIG1_MOTIFS, synth.TINY_DELTA)
    roots = synth.root_sample(12, len(src), 1000)
    work = torch.zeros((len(roots), tmotif.TM_WORK_FIELDS), dtype=torch.int64, device="cuda")
    got, st = tmotif.count(g, tr, roots=roots, per_root_work=work, stats=True)
    w = work.cpu().numpy()
    assert st["n_roots"] == len(roots)
    assert w[:, 0].sum() == st["candidates"] and w[:, 1].sum() == st["expansions"]
    assert w[:, 3].sum() == st["leaf_evals"]
    assert st["algo_bytes"] >= 16 * len(roots) + 8 * st["candidates"]
    assert st["kernel_ms"] > 0
    # scan mode visits every leaf candidate: its candidate count bounds the leaf totals
    _, st2 = tmotif.count(g, tr, roots=roots, mode=tmotif.TM_LEAF_SCAN, stats=True)
    assert st2["leaf_evals"] == 0 and st2["candidates"] >= got.sum()


# motifs whose every level has exactly one mapped endpoint, so the kernel and
# Algorithm 1 scan the same list at every level
ONE_LIST = [((0, 1), (1, 2), (2, 3)), ((0, 1), (0, 2), (0, 3)), ((0, 1), (2, 1), (3, 1)), ((0, 1), (2, 1), (1, 3)),
            ((0, 1), (1, 2), (1, 3), (3, 4))]


@pytest.mark.parametrize("motif", ONE_LIST)
def test_work_counters_equal_oracle_work(tiny, motif):
    """Per-root work (a10) against an independent count: scanning each level
    (TM_LEAF_SCAN, one warp per root) examines exactly the adjacency entries
    inside the window after the previous match, which is the number of
    candidates Algorithm 1 examines."""
    import torch
    src, dst, t, g, _ = tiny
    roots = synth.root_sample(13, len(src), 3000)
    tr = tmotif.Tree([motif], synth.TINY_DELTA)
    work = torch.zeros((len(roots), tmotif.TM_WORK_FIELDS), dtype=torch.int64, device="cuda")
    pr = torch.zeros((len(roots), 1), dtype=torch.int64, device="cuda")
    tmotif.count(g, tr, roots=roots, per_root_work=work, per_root_counts=pr, mode=tmotif.TM_LEAF_SCAN, stats=True)
    _, want_pr, want_work = oracle.count_motif(src, dst, t, motif, synth.TINY_DELTA, roots=roots, per_root=True,
                                               work=True)
    assert np.array_equal(pr.cpu().numpy()[:, 0], want_pr)
    assert np.array_equal(work.cpu().numpy()[:, tmotif.TM_WORK_CANDIDATES], want_work)


@pytest.fixture(scope="module")
def mid():
    src, dst, t = synth.make_graph(synth.MID)
    g = tmotif.Graph(src, dst, t, synth.MID.n_nodes, presorted=True)
    return src, dst, t, g


@pytest.mark.parametrize("leaf", [0, tmotif.TM_LEAF_SCAN])
def test_mid_config_sampled_roots(mid, leaf):
    """Mid workload (1M nodes, 20M edges, 12 motifs, delta 3600): per-root
    parity on 300 seeded roots, for every (root, motif) count the oracle
    finishes within a work budget of 10^6 candidates.  Each motif is counted
    on the GPU for the roots the oracle finished for it."""
    import torch
    src, dst, t, g = mid
    roots = synth.root_sample(21, len(src), 160)
    n_cmp = 0
    for m in synth.CONFIG2_MOTIFS:
        _, pr = oracle.count_motif(src, dst, t, m, synth.MID_DELTA, roots=roots, per_root=True,
                                   root_budget=300_000)
        done = pr >= 0
        assert done.sum() >= 8
        tr = tmotif.Tree([m], synth.MID_DELTA)
        got = torch.zeros((int(done.sum()), 1), dtype=torch.int64, device="cuda")
        tmotif.count(g, tr, roots=roots[done], per_root_counts=got, mode=leaf)
        assert np.array_equal(got.cpu().numpy()[:, 0], pr[done]), m
        n_cmp += int(done.sum())
    assert n_cmp >= 200


def test_mid_config_comine_modes_agree(mid):
    """Moderately heavy roots of the mid workload (oracle work up to 5*10^6
    candidates per root and motif): co-mined and per-motif, scan and window
    arithmetic, and the oracle all agree exactly."""
    src, dst, t, g = mid
    roots = synth.root_sample(22, len(src), 64)
    ms = [synth.CONFIG2_MOTIFS[i] for i in (0, 1, 3, 4, 6, 7, 9, 10)]
    keep = np.ones(len(roots), bool)
    cols = []
    for m in ms:
        _, pr = oracle.count_motif(src, dst, t, m, synth.MID_DELTA, roots=roots, per_root=True,
                                   root_budget=2_000_000)
        cols.append(pr)
        keep &= pr >= 0
    assert keep.sum() >= 5
    want = np.stack(cols, axis=1)[keep].sum(axis=0)
    tr = tmotif.Tree(ms, synth.MID_DELTA)
    sub = roots[keep]
    a = tmotif.count(g, tr, roots=sub)
    b = tmotif.count(g, tr, roots=sub, mode=tmotif.TM_LEAF_SCAN)
    c = tmotif.count(g, tr, roots=sub, mode=tmotif.TM_PERMOTIF)
    d = tmotif.count(g, tr, roots=sub, mode=D)
    assert a.tolist() == b.tolist() == c.tolist() == d.tolist() == want.tolist()


def test_mid_config_heavy_roots_split(mid):
    """Heavy roots of the mid workload, beyond the oracle: the dynamic launch
    (subtrees split across warps) must give the counts of the static one,
    and co-mined must equal per-motif, for all 12 motifs."""
    import torch
    src, dst, t, g = mid
    roots = synth.root_sample(23, len(src), 24)
    tr = tmotif.Tree(synth.CONFIG2_MOTIFS, synth.MID_DELTA)
    a, st = tmotif.count(g, tr, roots=roots, mode=D, stats=True)
    assert st["tasks_split"] > 0
    b = tmotif.count(g, tr, roots=roots, mode=D | tmotif.TM_PERMOTIF)
    assert a.tolist() == b.tolist()
    pr = torch.zeros((len(roots), 12), dtype=torch.int64, device="cuda")
    c = tmotif.count(g, tr, roots=roots, mode=D, per_root_counts=pr)
    assert c.tolist() == a.tolist()
    assert pr.sum(dim=0).cpu().tolist() == a.tolist()
    # the 3-edge motifs also through the static launch (one warp per root)
    tr3 = tmotif.Tree([m for m in synth.CONFIG2_MOTIFS if len(m) == 3], synth.MID_DELTA)
    s3 = tmotif.count(g, tr3, roots=roots)
    d3 = tmotif.count(g, tr3, roots=roots, mode=D)
    assert s3.tolist() == d3.tolist() == [a[i] for i, m in enumerate(synth.CONFIG2_MOTIFS) if len(m) == 3]


def test_mid_config_heavy_star_leaves_vs_scan(mid):
    """Star leaves (out- and in-stars) on heavy roots: counting from the
    level's survivor suffix and the edge's own pair run must equal the scan,
    with subtrees split across warps."""
    src, dst, t, g = mid
    roots = synth.root_sample(24, len(src), 32)
    ms = [((0, 1), (0, 2), (0, 3)), ((0, 1), (2, 1), (3, 1)), ((0, 1), (0, 2)), ((0, 1), (2, 1)),
          ((0, 1), (1, 2), (1, 3))]
    tr = tmotif.Tree(ms, [synth.MID_DELTA, synth.MID_DELTA, 1800, 3600, 900])
    a, st = tmotif.count(g, tr, roots=roots, mode=D, stats=True)
    b = tmotif.count(g, tr, roots=roots, mode=D | tmotif.TM_LEAF_SCAN)
    assert a.tolist() == b.tolist()
    assert st["tasks_split"] > 0


NESTED_STARS = [((0, 1), (0, 2), (0, 3)),
                ((0, 1), (0, 2), (1, 3), (1, 4)),
                ((0, 1), (0, 2), (1, 3), (3, 0)),
                ((0, 1), (2, 1), (3, 1)),
                ((0, 1), (2, 1), (0, 3), (4, 3))]


@pytest.mark.parametrize("mode", [0, D, tmotif.TM_PERMOTIF | D])
def test_nested_star_frames(tiny, mode):
    """A star frame owns the per-warp count table while a deeper star frame
    (nested under it) counts its stars from the pair index instead."""
    src, dst, t, g, _ = tiny
    tr = tmotif.Tree(NESTED_STARS, synth.TINY_DELTA)
    want = [oracle.count_motif(src, dst, t, m, synth.TINY_DELTA) for m in NESTED_STARS]
    assert tmotif.count(g, tr, mode=mode).tolist() == want


def test_nested_star_frames_mid_split(mid):
    import torch
    src, dst, t, g = mid
    # a short window keeps the scan mode (windows cubed per hub root) cheap
    roots = torch.from_numpy(synth.root_sample(25, len(src), 32)).cuda()
    tr = tmotif.Tree(NESTED_STARS, 120)
    a = tmotif.count(g, tr, roots=roots, mode=D)
    b = tmotif.count(g, tr, roots=roots, mode=D | tmotif.TM_LEAF_SCAN)
    split = torch.full((32,), 64, dtype=torch.int32, device="cuda")
    c = tmotif.count(g, tr, roots=roots, mode=tmotif.TM_SCHED_PLANNED, root_split=split)
    assert a.tolist() == b.tolist() == c.tolist()
