"""Tree-specialised kernels (the runtime code generation of Section 5.1)
against the oracle, the closed forms and the table-driven kernel.

Each tree here is compiled once for the module (independent programs on
parallel host threads, then served from the process cache).  Counts are
int64 and must be bit-exact: specialisation changes how the tree is read,
never what is counted.
"""
import threading

import numpy as np
import pytest

import oracle
from paper_2507_14813_b300 import build, synth, tmotif
from tests import refimpl
from tests.test_gpu_closed_forms import EAGER, HUB3, HUB4, HUB_DELTA
from tests.test_oracle_pins import PIN_MOTIFS

pytestmark = pytest.mark.gpu

D = tmotif.TM_SCHED_DYNAMIC
P = tmotif.TM_SCHED_PLANNED
G = tmotif.TM_GENERIC
PIN_DELTAS = [(i * 7 + 3) % 40 for i in range(len(PIN_MOTIFS))]


@pytest.fixture(scope="module")
def trees():
    build.build()
    tmotif.lib()
    spec = {
        "tiny": (synth.CONFIG1_MOTIFS, synth.TINY_DELTA, tmotif.TM_COMPILE_CHAINS),
        "pin": (PIN_MOTIFS, PIN_DELTAS, tmotif.TM_COMPILE_CHAINS),
        "mid": (synth.CONFIG2_MOTIFS, synth.MID_DELTA, 0),
        "hub3": (HUB3, HUB_DELTA, 0),
        "hub4": (HUB4, HUB_DELTA, 0),
    }
    out, info, err = {}, {}, []
    for name, (ms, d, _) in spec.items():
        out[name] = tmotif.Tree(ms, d)

    def run(name):
        try:
            info[name] = out[name].compile(spec[name][2])
        except Exception as e:          # reported below, on the main thread
            err.append((name, e))

    th = [threading.Thread(target=run, args=(n,)) for n in spec]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not err, err
    for name, tr in out.items():
        want = 1 + (len(tr.motifs) if spec[name][2] else 0)
        assert tr.info()["specialized"] >= 1 and info[name]["kernels"] <= want
    return out, info


def _split(n, s):
    import torch
    return torch.full((n,), s, dtype=torch.int32, device="cuda")


MODES = [("comine", 0, None), ("comine-dyn", D, None), ("planned-dyn", P | D, 4), ("permotif", tmotif.TM_PERMOTIF, None),
         ("permotif-dyn", tmotif.TM_PERMOTIF | D, None)]


@pytest.mark.parametrize("name,mode,split", MODES)
def test_tiny_config_full_specialised(trees, name, mode, split):
    tr = trees[0]["tiny"]
    src, dst, t = synth.make_graph(synth.TINY)
    g = tmotif.Graph(src, dst, t, synth.TINY.n_nodes, presorted=True)
    want = oracle.count_motifs(src, dst, t, synth.CONFIG1_MOTIFS, synth.TINY_DELTA)
    rs = _split(len(src), split) if split else None
    got = tmotif.count(g, tr, mode=mode, root_split=rs)
    assert got.tolist() == want.tolist()
    assert tmotif.count(g, tr, mode=mode | G, root_split=rs).tolist() == want.tolist()


@pytest.mark.parametrize("seed", range(4))
def test_pin_motifs_specialised(trees, seed):
    """Every candidate-list case (the disconnected motif scans the global
    window), several windows in one tree, tie-heavy graphs with self-loops."""
    tr = trees[0]["pin"]
    src, dst, t = synth.tiny_graph(9600 + seed, 9 + seed, 400 + 50 * seed, 300, zipf_s=1.0, self_loops=seed % 2 == 0)
    g = tmotif.Graph(src, dst, t, 9 + seed, presorted=True)
    want = [oracle.count_motif(src, dst, t, m, d, n_nodes=9 + seed) for m, d in zip(PIN_MOTIFS, PIN_DELTAS)]
    for _, mode, split in MODES:
        rs = _split(len(src), split) if split else None
        assert tmotif.count(g, tr, mode=mode, root_split=rs).tolist() == want


@pytest.fixture(scope="module")
def mid():
    src, dst, t = synth.make_graph(synth.MID)
    g = tmotif.Graph(src, dst, t, synth.MID.n_nodes, presorted=True)
    return src, dst, t, g, refimpl.ListIndex(src, dst)


@pytest.mark.parametrize("mode,split", [(D, None), (P | D, 64), (P, 256)])
def test_mid_bench_sample_specialised(trees, mid, mode, split):
    """The benchmark's 64 hub roots: per-root counts of the 11 motifs with a
    closed form equal it; all 12 equal the table-driven kernel's."""
    import torch
    tr = trees[0]["mid"]
    src, dst, t, g, idx = mid
    roots = synth.root_sample(100, len(src), 64)
    r = torch.from_numpy(roots).cuda()
    rs = _split(64, split) if split else None
    pr = torch.zeros((64, 12), dtype=torch.int64, device="cuda")
    tmotif.count(g, tr, roots=r, per_root_counts=pr, mode=mode, root_split=rs)
    pg = torch.zeros((64, 12), dtype=torch.int64, device="cuda")
    tmotif.count(g, tr, roots=r, per_root_counts=pg, mode=mode | G, root_split=rs)
    assert torch.equal(pr, pg)
    pr = pr.cpu().numpy()
    n = 0
    for j, m in enumerate(synth.CONFIG2_MOTIFS):
        try:
            want = refimpl.closed_form_per_root(src, dst, t, m, synth.MID_DELTA, roots, idx=idx)
        except KeyError:
            continue
        assert np.array_equal(pr[:, j], want), m
        n += 1
    assert n == 11


def test_mid_sampled_roots_oracle_specialised(trees, mid):
    """Mid-workload roots against the oracle, per root: each motif's column
    on the roots the oracle finishes for that motif within its budget."""
    import torch
    tr = trees[0]["mid"]
    src, dst, t, g, _ = mid
    roots = synth.root_sample(21, len(src), 160)
    got = torch.zeros((len(roots), 12), dtype=torch.int64, device="cuda")
    tmotif.count(g, tr, roots=torch.from_numpy(roots).cuda(), per_root_counts=got, mode=D)
    got = got.cpu().numpy()
    n_cmp = 0
    for j, m in enumerate(synth.CONFIG2_MOTIFS):
        _, pr = oracle.count_motif(src, dst, t, m, synth.MID_DELTA, roots=roots, per_root=True, root_budget=300_000)
        done = pr >= 0
        assert np.array_equal(got[done, j], pr[done]), m
        n_cmp += int(done.sum())
    assert n_cmp >= 200


def test_hub_graph_specialised(trees):
    """The hub graph's star frames (30+ chunks, > 256 distinct far ends) with
    eager donation, against the oracle and the closed forms."""
    import torch
    src, dst, t = synth.hub_graph(31, 4000, 40000, 40000)
    g = tmotif.Graph(src, dst, t, 4000, presorted=True)
    hub_out = np.nonzero(src == 0)[0]
    hub_in = np.nonzero(dst == 0)[0]
    roots = np.unique(np.concatenate([hub_out[::100], hub_in[::50], synth.root_sample(3, len(src), 200)]))
    r = torch.from_numpy(roots.astype(np.int32)).cuda()
    want3 = np.stack([oracle.count_motif(src, dst, t, m, HUB_DELTA, roots=roots, per_root=True)[1] for m in HUB3],
                     axis=1)
    idx = refimpl.ListIndex(src, dst)
    want4 = np.stack([refimpl.closed_form_per_root(src, dst, t, m, HUB_DELTA, roots, idx=idx) for m in HUB4], axis=1)
    for name, want in (("hub3", want3), ("hub4", want4)):
        tr = trees[0][name]
        for mode, tune in ((0, None), (D, EAGER), (P | D, EAGER)):
            pr = torch.zeros((len(roots), want.shape[1]), dtype=torch.int64, device="cuda")
            tmotif.count(g, tr, roots=r, per_root_counts=pr, mode=mode, tune=tune,
                         root_split=_split(len(roots), 8) if mode & P else None)
            assert np.array_equal(pr.cpu().numpy(), want), (name, mode)


def test_specialised_replay_and_device_counts(trees):
    """A graph-captured replay and device-resident counts use the
    specialised kernel like tm_count does."""
    import torch
    tr = trees[0]["tiny"]
    src, dst, t = synth.make_graph(synth.TINY)
    g = tmotif.Graph(src, dst, t, synth.TINY.n_nodes, presorted=True)
    want = oracle.count_motifs(src, dst, t, synth.CONFIG1_MOTIFS, synth.TINY_DELTA).tolist()
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    ex = tmotif.Exec(g.h, tr.h, out, mode=D)
    for _ in range(2):
        out.zero_()
        ex.launch()
        ex.status()
        assert out.cpu().tolist() == want
    tmotif.count(g, tr, counts=out, mode=D)
    torch.cuda.synchronize()
    assert out.cpu().tolist() == want
