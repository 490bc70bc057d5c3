"""Host-side checks of the tree-specialised kernels (runtime code
generation of Section 5.1): the generated program compiles for sm_103a
without a device, its arrays are sized to the tree (fewer spill bytes than
the table-driven kernel's), and bad requests are rejected."""
import threading

import pytest

from paper_2507_14813_b300 import build, synth, tmotif
from tests.test_oracle_pins import PIN_MOTIFS


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    tmotif.lib()


def test_generated_programs_compile_for_sm103a():
    # the mid workload's tree, and a multi-window tree whose disconnected
    # motif scans the global edge window; compiled side by side
    trees = [tmotif.Tree(synth.CONFIG2_MOTIFS, synth.MID_DELTA),
             tmotif.Tree(PIN_MOTIFS, [(i * 7) % 40 for i in range(len(PIN_MOTIFS))])]
    out = [None] * len(trees)

    def run(i):
        out[i] = trees[i].compile(tmotif.TM_COMPILE_CHECK)

    th = [threading.Thread(target=run, args=(i,)) for i in range(len(trees))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for info in out:
        assert info["kernels"] == 1 and info["compiled"] == 1
        assert 0 < info["registers"] <= 80          # __launch_bounds__(256, 3)
        assert info["static_smem"] > 0
    # the mid tree: depth 4 and 5 vertices size the per-warp state, and the
    # kernel spills at most a few words (the table-driven kernel: 36 B of
    # spill stores at the same 80 registers)
    assert out[0]["static_smem"] < 39488
    assert all(0 <= info["local_bytes"] <= 16 for info in out)
    # a check attaches nothing to the tree
    assert all(t.info()["specialized"] == 0 for t in trees)


def test_compile_rejects_bad_requests():
    tr = tmotif.Tree(synth.CONFIG1_MOTIFS, 10)
    with pytest.raises(tmotif.TMError) as e:
        tmotif.tm_tree_compile(tr.h, 0x80)
    assert e.value.code == tmotif.TM_EINVAL
    motifs = []
    for seed in range(20):
        motifs += synth.random_motif_tree(900 + seed, max_edges=6, max_motifs=32)
    big = tmotif.Tree(motifs, 10)
    assert big.info()["n_nodes"] > tmotif.TM_SPEC_MAX_NODES
    with pytest.raises(tmotif.TMError) as e:
        big.compile(tmotif.TM_COMPILE_CHECK)
    assert e.value.code == tmotif.TM_EUNSUPPORTED
